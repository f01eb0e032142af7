"""Compile the C part of the oracle (``kt_oracle.c``) into ``libkt_oracle.so``.

Test infrastructure: the oracle is built with the host C compiler, FP64, with
FMA contraction disabled (``-ffp-contract=off``) so that it gives the same
bits on every host architecture.  OpenMP is used when the compiler has it; the
row loop it parallelises has no cross-row dependence inside a step, so the
thread count never changes a result.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kt_oracle.c")
LIB = os.path.join(HERE, "libkt_oracle.so")


def _stale() -> bool:
    return not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC)


def build_oracle(force: bool = False) -> str:
    """Build ``libkt_oracle.so`` if it is missing or older than its source."""
    if not force and not _stale():
        return LIB
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=HERE)
    os.close(fd)
    base = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", tmp]
    try:
        r = subprocess.run(base[:-3] + ["-fopenmp"] + base[-3:] + ["-lm"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            r = subprocess.run(base + ["-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(tmp, LIB)
    finally:
        if os.path.exists(tmp):
            os.remove(tmp)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
