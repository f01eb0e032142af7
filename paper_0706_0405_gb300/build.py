"""Build ``liblbm.so`` (the CUDA library behind ``include/lbm.h``) in-tree.

Each translation unit under ``csrc/`` is compiled by nvcc for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``), in parallel, and linked into
``paper_0706_0405_gb300/liblbm.so`` with the CUDA runtime linked statically.
Objects go to ``paper_0706_0405_gb300/_build/``.  Nothing is compiled for the
host CPU beyond the C-ABI glue in the same library.
"""
from __future__ import annotations

import glob
import hashlib
import os
import shutil
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))


# Sources that define each profiled kernel's code: the kernel's own file and
# every header with device code it calls.
KERNEL_SOURCES = {
    "k_step_tile": ("lbm_step.cu", "lbm_device.cuh", "lbm_ptx.cuh"),
    "k_step_vec": ("lbm_step.cu", "lbm_device.cuh", "lbm_ptx.cuh"),
    "k_step_simple": ("lbm_step.cu", "lbm_device.cuh", "lbm_ptx.cuh"),
    "k_step_ring": ("lbm_step.cu", "lbm_device.cuh", "lbm_ptx.cuh"),
}


def source_hash(names=None) -> str:
    """Short hash of the sources the library is built from, or of the files
    with the given base names (used to tell whether a recorded profile still
    describes the current kernels)."""
    h = hashlib.sha1()
    for path in sorted(_deps()):
        if names is not None and os.path.basename(path) not in names:
            continue
        with open(path, "rb") as fh:
            h.update(os.path.basename(path).encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


def kernel_hash(kernel: str) -> str:
    """source_hash of the files that define ``kernel`` (all sources if the
    kernel is not listed)."""
    return source_hash(KERNEL_SOURCES.get(kernel))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build_library(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile and link ``liblbm.so`` if it is missing or older than a source."""
    if not force and not stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-I", INCLUDE, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=HERE)
    os.close(fd)
    try:
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("linking liblbm.so failed:\n" + r.stderr)
        os.replace(tmp, LIB)
    finally:
        if os.path.exists(tmp):
            os.remove(tmp)
    return LIB


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
