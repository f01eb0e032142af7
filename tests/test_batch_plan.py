"""Host logic of the batch kernel's step order, on the CPU: the neighbour
lists of csrc/lbm_batch_plan.h (which CTAs a CTA waits for before each step)
against a brute-force enumeration of bordering tile pairs, for contiguous and
strided tile walks, periodic and non-periodic sides, and tall problems."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0706_0405_gb300", "csrc")

HARNESS = r"""
#include "lbm_batch_plan.h"
extern "C" int plan(int ntiles, const int* tp, const int* tix, const int* tiy, const int* tx, const int* ty,
                    const int* base, const unsigned char* px, const unsigned char* py, int grid, int strided,
                    int max_nbr, int* out) {
    const int per = (ntiles + grid - 1) / grid;
    std::vector<int> v;
    const bool ok = lbm::batch_plan_neighbours(
        ntiles, tp, tix, tiy, tx, ty, base, px, py, grid,
        [&](int t) { return strided ? t % grid : t / per; }, max_nbr, v);
    for (size_t k = 0; k < v.size(); ++k) out[k] = v[k];
    return ok ? 1 : 0;
}
"""


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("plan")
    src, lib = d / "harness.cpp", d / "libplan.so"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(lib)],
                   check=True, capture_output=True)
    return ctypes.CDLL(str(lib)).plan


def _tiles(probs):
    """probs: (tiles_x, tiles_y, periodic_x, periodic_y); the tile list in the
    library's order (problem by problem, rows of tiles in order)."""
    tp, tix, tiy, base = [], [], [], []
    for p, (tx, ty, _, _) in enumerate(probs):
        base.append(len(tp))
        for iy in range(ty):
            for ix in range(tx):
                tp.append(p), tix.append(ix), tiy.append(iy)
    return np.array(tp), np.array(tix), np.array(tiy), np.array(base)


def _expected(probs, grid, strided):
    tp, tix, tiy, base = _tiles(probs)
    n = len(tp)
    per = (n + grid - 1) // grid
    owner = (lambda t: t % grid) if strided else (lambda t: t // per)
    want = [set() for _ in range(grid)]
    for t in range(n):
        tx, ty, px, py = probs[tp[t]]
        for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
            jx, jy = tix[t] + dx, tiy[t] + dy
            if not 0 <= jx < tx:
                if not px:
                    continue
                jx %= tx
            if not 0 <= jy < ty:
                if not py:
                    continue
                jy %= ty
            c, d = owner(t), owner(base[tp[t]] + jy * tx + jx)
            if c != d:
                want[c].add(d)
    return want


def _run(planner, probs, grid, strided, max_nbr=8):
    tp, tix, tiy, base = _tiles(probs)
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    tx = i32([p[0] for p in probs])
    ty = i32([p[1] for p in probs])
    px = np.ascontiguousarray([p[2] for p in probs], dtype=np.uint8)
    py = np.ascontiguousarray([p[3] for p in probs], dtype=np.uint8)
    out = np.full(grid * max_nbr, -7, dtype=np.int32)
    arrs = [i32(tp), i32(tix), i32(tiy), tx, ty, i32(base), px, py]
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    ok = planner(ctypes.c_int(len(tp)), *[ptr(a) for a in arrs], ctypes.c_int(grid), ctypes.c_int(int(strided)),
                 ctypes.c_int(max_nbr), ptr(out))
    return bool(ok), out.reshape(grid, max_nbr)


@pytest.mark.parametrize("strided", [False, True])
@pytest.mark.parametrize("seed", range(6))
def test_neighbour_lists_equal_brute_force(planner, strided, seed):
    rng = np.random.default_rng(seed)
    probs = [(int(rng.integers(1, 20)), int(rng.integers(1, 4)), bool(rng.random() < 0.3), bool(rng.random() < 0.6))
             for _ in range(int(rng.integers(1, 40)))]
    ntiles = sum(p[0] * p[1] for p in probs)
    for grid in sorted({1, 2, 7, max(1, ntiles // 3), ntiles, ntiles + 5}):
        want = _expected(probs, grid, strided)
        ok, out = _run(planner, probs, grid, strided, max_nbr=64)
        assert ok
        for c in range(grid):
            got = [v for v in out[c] if v >= 0]
            assert len(got) == len(set(got)) and set(got) == want[c], (grid, c)
            assert all(v == -1 for v in out[c][len(got):])
        # bordering is symmetric, so the lists are too
        for c in range(grid):
            for d in want[c]:
                assert c in want[d]


def test_thin_tubes_need_at_most_two_neighbours_and_overflow_is_reported(planner):
    """The batch workload's shape: one row of tiles per problem, periodic in y
    only, contiguous runs: each CTA borders at most its two neighbours in the
    walk.  A tall periodic problem walked with a stride borders many CTAs,
    and more than max_nbr is reported as a failure."""
    rng = np.random.default_rng(1)
    probs = [(int(rng.integers(4, 65)), 1, False, True) for _ in range(256)]
    ntiles = sum(p[0] for p in probs)
    for grid in (608, 912, 1064):
        ok, out = _run(planner, probs, grid, strided=False)
        assert ok and np.max(np.sum(out >= 0, axis=1)) <= 2
    tall = [(8, 40, True, True)]
    ok, _ = _run(planner, tall, 37, strided=True, max_nbr=4)
    assert not ok
    assert ntiles > 0
