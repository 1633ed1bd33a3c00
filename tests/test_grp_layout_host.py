"""csrc/grp_layout.cuh on the host: the row-group layout of the symmetric
kernels (which phase-steps each block of the persistent grid takes, where its
partial sums go) checked against a plain enumeration of the units, for ragged
sizes, both group sizes, both chunk sizes (single steps for the FP64 kernel,
whole phases for the mixed one) and grids from one block to more blocks than
the layout admits.

What is checked (tests/grp_layout_host.cpp): the closed form of the phases
before each group; that owners ascend, cover every block and leave none
empty; at least one phase per block; that each block's start position is its
first unit; that the owners of a phase's units are the range the apply kernel
derives from the phase's first and last unit; that no chunk is split; that
layout indices map one to one onto particles (reversed for the FP64 kernel);
Hmax;
and the balance: every block holds U/B units to within one chunk (whole
phases: no block starts inside a phase)."""
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
    L.grp_layout_check.argtypes = [ctypes.c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_long, ctypes.POINTER(ctypes.c_long)]
    L.grp_layout_check.restype = ctypes.c_int
    return L


SIZES = [1, 2, 31, 32, 33, 100, 255, 256, 257, 1000, 1023, 1024, 1025, 2049, 4096, 5000, 16384]
GRIDS = [1, 2, 3, 7, 152, 304, 608, 1_000_000]


@pytest.mark.parametrize("S", [1, 32])
@pytest.mark.parametrize("G", [4, 8])
@pytest.mark.parametrize("n", SIZES)
def test_layout_against_enumeration(lib, n, G, S):
    for blocks in GRIDS:
        out = (ctypes.c_long * 6)()
        rc = lib.grp_layout_check(n, G, S, int(S == 1), blocks, out)
        assert rc == 0, f"n={n} G={G} S={S} blocks={blocks}: check {rc} failed"
        B, U, hmax, cmin, cmax, inside = list(out)
        assert 1 <= B <= max(1, U // 32)
        nc = U // S
        assert cmin == (nc // B) * S and cmax == -(-nc // B) * S, (n, G, S, blocks, cmin, cmax)
        if S == 32:
            assert inside == 0


def test_headline_grid_is_balanced(lib):
    # 16384 bodies on 2 blocks of 4 warps per SM x 152 SMs
    out = (ctypes.c_long * 6)()
    assert lib.grp_layout_check(16384, 4, 1, 1, 304, out) == 0
    B, U, hmax, cmin, cmax, inside = list(out)
    # 33024 phases of 32 steps; blocks of 3476 or 3477 steps
    assert B == 304 and U == 32 * 33024
    assert (cmin, cmax) == (3476, 3477)
