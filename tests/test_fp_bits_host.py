"""csrc/fp_bits.cuh on the host: the integer-pipe forms of x * 2^k (k = +-1)
and of the float-to-double conversion give exactly the bits of the FP64
operations they replace, for every class of operand (zero, subnormal, the
normal-range boundaries, infinity, NaN) and for random bit patterns."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("fpbits") / "libfpbits.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared",
                    "-fPIC", os.path.join(HERE, "fp_bits_host.cpp"), "-o", str(out)], check=True)
    L = ctypes.CDLL(str(out))
    P = ctypes.c_void_p
    L.scale2_many.argtypes = [P, ctypes.c_long, ctypes.c_int, P]
    L.f2d_many.argtypes = [P, ctypes.c_long, P]
    return L


def _edge_doubles():
    tiny = np.finfo(np.float64).tiny
    vals = [0.0, -0.0, tiny, -tiny, 2 * tiny, tiny / 2, 5e-324, -5e-324, 1.0, -1.5, 2.0 ** 1023,
            -(2.0 ** 1023), np.finfo(np.float64).max, -np.finfo(np.float64).max, np.inf, -np.inf,
            np.nan, 2.0 ** -1021, 2.0 ** 1022, 0.5, 3.0]
    return np.array(vals, dtype=np.float64)


def _random_doubles(n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2 ** 64, n, dtype=np.uint64).view(np.float64)


@pytest.mark.parametrize("k", [1, -1])
def test_scale2_matches_the_multiply(lib, k):
    x = np.concatenate([_edge_doubles(), _random_doubles(1_000_000, 7 + k)])
    out = np.empty_like(x)
    lib.scale2_many(x.ctypes.data, len(x), k, out.ctypes.data)
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        want = x * (2.0 if k > 0 else 0.5)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(out), nan)
    assert np.array_equal(out[~nan].view(np.int64), want[~nan].view(np.int64))


def test_f2d_matches_the_conversion(lib):
    rng = np.random.default_rng(3)
    fi = np.finfo(np.float32)
    edge = np.array([0.0, -0.0, fi.tiny, -fi.tiny, fi.tiny / 2, 1e-45, fi.max, -fi.max, np.inf,
                     -np.inf, np.nan, 1.0, -3.25], dtype=np.float32)
    rnd = rng.integers(0, 2 ** 32, 1_000_000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    f = np.concatenate([edge, rnd])
    out = np.empty(len(f), dtype=np.float64)
    lib.f2d_many(f.ctypes.data, len(f), out.ctypes.data)
    with np.errstate(invalid="ignore"):
        want = f.astype(np.float64)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(out), nan)
    assert np.array_equal(out[~nan].view(np.int64), want[~nan].view(np.int64))
