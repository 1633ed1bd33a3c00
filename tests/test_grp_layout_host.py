"""csrc/grp_layout.cuh on the host: the row-group layout of the symmetric
kernels (which steps each block of the persistent grid takes, where its
partial sums go) checked against a plain enumeration of the units, for ragged
sizes, both group sizes, both kernels' shapes (FP64: single steps of equal
cost, particles reversed; mixed: whole phases of equal cost) and grids from one block to more blocks than the layout admits.

What is checked (tests/grp_layout_host.cpp): the closed forms of the phases
and tiles before each group and of the cost before each phase; that owners
ascend, cover every block and leave none empty; that each block's start
position is its first chunk; that the owners of a phase's chunks are the
range the apply kernel derives from the phase's first and last chunk; that
layout indices map one to one onto particles; Hmax; and the balance: a
block's range starts and ends within one chunk's cost of b C/B and
(b+1) C/B (whole phases: no block starts inside a phase)."""
import ctypes
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("grplayout") / "libgrplayout.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    os.path.join(HERE, "grp_layout_host.cpp"), "-o", str(out)], check=True)
    L = ctypes.CDLL(str(out))
    L.grp_layout_check.argtypes = [ctypes.c_long] + [ctypes.c_int] * 5 + [
        ctypes.c_long, ctypes.POINTER(ctypes.c_long)]
    L.grp_layout_check.restype = ctypes.c_int
    return L


SIZES = [1, 2, 31, 32, 33, 100, 255, 256, 257, 1000, 1023, 1024, 1025, 2049, 4096, 5000, 16384]
GRIDS = [1, 2, 3, 7, 152, 304, 608, 1_000_000]
# (G, S, wA, wB, rev): the FP64 kernel's shape, the mixed kernel's, the
# double-word kernel's, and others the arithmetic allows
SHAPES = [(4, 1, 1, 0, 1), (8, 32, 1, 0, 0), (12, 32, 2, 1, 1), (4, 1, 3, 1, 1), (4, 1, 2, 1, 1),
          (4, 1, 1, 1, 1), (4, 32, 1, 1, 0), (8, 1, 1, 0, 1), (8, 1, 2, 3, 0)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda sh: "G%d-S%d-w%d%d-r%d" % sh)
@pytest.mark.parametrize("n", SIZES)
def test_layout_against_enumeration(lib, n, shape):
    G, S, wA, wB, rev = shape
    for blocks in GRIDS:
        out = (ctypes.c_long * 7)()
        rc = lib.grp_layout_check(n, G, S, wA, wB, rev, blocks, out)
        assert rc == 0, f"n={n} shape={shape} blocks={blocks}: check {rc} failed"
        B, C, hmax, lo, hi, inside, chunk = list(out)
        assert 1 <= B <= max(1, C // (32 * (wA + wB * G)))
        # each end of a range within one chunk of b C / B
        assert C / B - chunk - 1 < lo and hi < C / B + chunk + 1, (n, shape, blocks, lo, hi)
        if S == 32:
            assert inside == 0


def test_headline_grid_is_balanced(lib):
    # 16384 bodies on 2 blocks of 4 warps per SM x 152 SMs: 33024 phases of
    # 32 steps, 132096 - 768 tiles
    out = (ctypes.c_long * 7)()
    assert lib.grp_layout_check(16384, 4, 1, 2, 1, 1, 304, out) == 0
    B, C, hmax, lo, hi, inside, chunk = list(out)
    assert B == 304 and C == 32 * (2 * 33024 + 4 * 33024 - 6 * 128)
    assert chunk == 6 and hi - lo <= 2 * chunk
