"""CPU check of the double-word primitives of the double-float Kepler path
(csrc/df64.cuh), built as host C++: every result is compared with the exact
value of the operation on the same float inputs (Python fractions), against
the published relative error bounds (u = 2^-24): add <= 3u^2, add_f <= 2u^2,
add without cancellation (like signs) <= 3u^2,
mul <= 5u^2, mul_f <= 2u^2, and <= 4u^2 for the Newton-corrected reciprocal
and reciprocal square root (exact value rounded to 60 bits).  The difference
of two doubles through their exact three-float form must be within 4u^2 of
the difference itself, also for coordinates that agree to 40 bits (a close
pair far from the origin)."""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
U2 = 2.0 ** -48


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("df64") / "libdf64host.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                    "-shared", "-fPIC", os.path.join(HERE, "df64_host.cpp"), "-o", out],
                   check=True)
    lib = ctypes.CDLL(out)
    P = ctypes.POINTER(ctypes.c_float)
    lib.dw_batch.argtypes = [ctypes.c_int, ctypes.c_long, P, P, P, P, P, P]
    D = ctypes.POINTER(ctypes.c_double)
    lib.tf_diff_batch.argtypes = [ctypes.c_long, D, D, P, P]
    return lib


def _split(d):
    h = d.astype(np.float32)
    l = (d - h.astype(np.float64)).astype(np.float32)
    return h, l


def _rand_dw(rng, n, lo=-30, hi=30, positive=False):
    d = rng.uniform(1.0, 2.0, n) * 2.0 ** rng.integers(lo, hi, n)
    if not positive:
        d *= rng.choice([-1.0, 1.0], n)
    return _split(d)


def _run(lib, op, xh, xl, yh, yl):
    n = xh.shape[0]
    zh = np.zeros(n, np.float32)
    zl = np.zeros(n, np.float32)
    f = lambda a: np.ascontiguousarray(a, np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    lib.dw_batch(op, n, f(xh), f(xl), f(yh), f(yl), f(zh), f(zl))
    return zh, zl


def _val(h, l):
    return Fraction(float(h)) + Fraction(float(l))


def _rel(got, exact):
    return abs(float((got - exact) / exact)) if exact != 0 else abs(float(got))


@pytest.mark.parametrize("op,bound", [(0, 3), (1, 3), (2, 2), (3, 5), (4, 2), (5, 5)])
def test_double_word_arithmetic_error_bounds(lib, op, bound):
    rng = np.random.default_rng(op)
    n = 4000
    xh, xl = _rand_dw(rng, n)
    yh, yl = _rand_dw(rng, n, -8, 8) if op in (0, 1, 2) else _rand_dw(rng, n)
    if op in (0, 1, 2):  # include near-cancelling pairs
        k = n // 4
        yh[:k] = -xh[:k] if op != 1 else xh[:k]
        yl[:k] = (rng.uniform(-1, 1, k) * np.abs(xh[:k]) * 2.0 ** -30).astype(np.float32)
    zh, zl = _run(lib, op, xh, xl, yh, yl)
    worst = 0.0
    for k in range(n):
        x = _val(xh[k], xl[k])
        y = _val(yh[k], 0.0) if op in (2, 4) else _val(yh[k], yl[k])
        exact = {0: x + y, 1: x - y, 2: x + y, 3: x * y, 4: x * y, 5: x * x}[op]
        worst = max(worst, _rel(_val(zh[k], zl[k]), exact))
        # normalised: |l| <= ulp(h) / 2
        assert abs(float(zl[k])) <= abs(float(zh[k])) * 2.0 ** -24 * 1.0000001
    assert worst <= bound * U2, worst / U2


def test_double_word_sum_without_cancellation(lib):
    # like-signed operands of any relative size
    rng = np.random.default_rng(8)
    n = 4000
    xh, xl = _rand_dw(rng, n, positive=True)
    yh, yl = _rand_dw(rng, n, -40, 40, positive=True)
    sign = rng.choice([-1.0, 1.0], n).astype(np.float32)
    xh, xl, yh, yl = xh * sign, xl * sign, yh * sign, yl * sign
    zh, zl = _run(lib, 8, xh, xl, yh, yl)
    worst = max(_rel(_val(zh[k], zl[k]), _val(xh[k], xl[k]) + _val(yh[k], yl[k]))
                for k in range(n))
    assert worst <= 3 * U2, worst / U2


@pytest.mark.parametrize("op", [6, 7])
def test_double_word_reciprocal_and_rsqrt(lib, op):
    import mpmath as mp
    rng = np.random.default_rng(10 + op)
    n = 4000
    xh, xl = _rand_dw(rng, n, -40, 40, positive=(op == 7))
    zh, zl = _run(lib, op, xh, xl, xh, xl)
    worst = 0.0
    with mp.workdps(40):
        for k in range(n):
            x = mp.mpf(float(xh[k])) + mp.mpf(float(xl[k]))
            exact = 1 / x if op == 6 else 1 / mp.sqrt(x)
            got = mp.mpf(float(zh[k])) + mp.mpf(float(zl[k]))
            worst = max(worst, float(abs((got - exact) / exact)))
    assert worst <= 4 * U2, worst / U2


def test_three_float_difference_is_relative_to_the_difference(lib):
    rng = np.random.default_rng(3)
    n = 6000
    a = rng.uniform(-1, 1, n) * 2.0 ** rng.integers(-20, 20, n)
    b = a.copy()
    # one third far apart, one third close (relative 2^-10..2^-40), one third
    # differing in the last few bits
    k = n // 3
    b[:k] = rng.uniform(-1, 1, k) * 2.0 ** rng.integers(-20, 20, k)
    b[k:2 * k] = a[k:2 * k] * (1 + rng.uniform(-1, 1, k) * 2.0 ** rng.integers(-40, -10, k))
    b[2 * k:] = np.nextafter(a[2 * k:], np.inf)
    b[2 * k:] = a[2 * k:] + (b[2 * k:] - a[2 * k:]) * rng.integers(1, 30, n - 2 * k)
    zh = np.zeros(n, np.float32)
    zl = np.zeros(n, np.float32)
    D = lambda x: np.ascontiguousarray(x).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    F = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    lib.tf_diff_batch(n, D(a), D(b), F(zh), F(zl))
    worst = 0.0
    for q in range(n):
        exact = Fraction(float(a[q])) - Fraction(float(b[q]))
        got = _val(zh[q], zl[q])
        if exact == 0:
            assert got == 0
            continue
        worst = max(worst, _rel(got, exact))
    assert worst <= 4 * U2, worst / U2


def _pair_lib(lib):
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    lib.dw_pair_batch.argtypes = [ctypes.c_long, D, D, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int, D, I, I]
    return lib


def _pair_cases(rng, n):
    """Relative states (r, v), masses and the step for a mix of the method's
    pair types: weak star-star flybys (Plummer-like), bound binaries with
    periods above the step, planet-star pairs, black-hole-star pairs and
    close hyperbolic encounters."""
    rv = np.zeros((n, 6))
    m = np.zeros(n)
    kind = rng.integers(0, 5, n)
    for k in range(n):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        w = rng.normal(size=3)
        if kind[k] == 0:    # star pair in a cluster
            m[k] = 2.0 / 1024
            rv[k, :3] = d * 10 ** rng.uniform(-2.5, 0.5)
            rv[k, 3:] = w * 0.5
        elif kind[k] == 1:  # binary
            m[k] = 2.0 / 16384
            a = 10 ** rng.uniform(-3, -2)
            rv[k, :3] = d * a
            rv[k, 3:] = np.cross(d, w / np.linalg.norm(w)) * np.sqrt(m[k] / a) * rng.uniform(0.5, 1.3)
        elif kind[k] == 2:  # planet
            m[k] = 1.0 + 10 ** rng.uniform(-5, -3)
            a = 10 ** rng.uniform(0, 1.4)
            rv[k, :3] = d * a
            t = np.cross(d, w)
            rv[k, 3:] = t / np.linalg.norm(t) * np.sqrt(m[k] / a) * rng.uniform(0.95, 1.05)
        elif kind[k] == 3:  # black hole and star
            m[k] = 1.0 + 1e-6
            r = 10 ** rng.uniform(-1, 0.5)
            rv[k, :3] = d * r
            t = np.cross(d, w)
            rv[k, 3:] = t / np.linalg.norm(t) * np.sqrt(m[k] / r) + w * 0.1
        else:               # close hyperbolic encounter
            m[k] = 2e-3
            rv[k, :3] = d * 10 ** rng.uniform(-3, -1.5)
            rv[k, 3:] = -d * rng.uniform(0.5, 3) + w * 0.3
    return rv, m, kind


@pytest.mark.parametrize("order", [2, 1, -1])
def test_double_word_pair_map_is_close_to_fp64_accuracy(lib, order):
    """The double-word pair map against the exact one (classical solver at
    40 digits): its error, relative to the pair's own |r| and |v|, is at
    most 2^10 times the FP64 oracle's error on the same pair, or 2^-44 where
    the FP64 error happens to vanish.  Double-word operations carry 3-5
    units of 2^-48 against FP64's half unit of 2^-52, and both are amplified
    alike by ill-conditioned encounters (a nearly head-on flyby that turns
    the relative velocity around)."""
    import mpmath as mp
    import oracle
    from classical_kepler import kepler_classical
    lib = _pair_lib(lib)
    rng = np.random.default_rng(20 + order)
    n = 1500
    rv, m, kind = _pair_cases(rng, n)
    tau = 2.0 ** -8
    pre = {2: 0.5, 1: 0.0, -1: 1.0}[order]
    post = 1.0 - pre
    out = np.zeros((n, 6))
    adm = np.zeros(n, np.int32)
    ev = np.zeros(n, np.int32)
    D = lambda x: np.ascontiguousarray(x).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    lib.dw_pair_batch(n, D(rv), D(m), tau, pre, post, 2, out.ctypes.data_as(
        ctypes.POINTER(ctypes.c_double)), adm.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    assert adm.mean() > 0.95, adm.mean()
    for kk in range(4):  # every cluster, binary, planet and black-hole pair
        assert adm[kind == kk].all()
    assert ev[adm == 1].max() <= 3
    pick = np.nonzero(adm)[0]
    pick = np.concatenate([pick[kind[pick] == 4], pick[kind[pick] != 4][:200]])
    worst = 0.0
    for k in pick:
        rr, vv = rv[k, :3], rv[k, 3:]
        with mp.workdps(40):
            R = [mp.mpf(float(x)) for x in rr]
            V = [mp.mpf(float(x)) for x in vv]
            T = mp.mpf(tau)
            R0 = [R[q] - mp.mpf(pre) * T * V[q] for q in range(3)]
            r1, v1 = kepler_classical(T, float(m[k]), R0, V)
            dr = np.array([float(r1[q] - mp.mpf(post) * T * v1[q] - R[q]) for q in range(3)])
            dv = np.array([float(v1[q] - V[q]) for q in range(3)])
        o1, o2, _, rc = oracle.kepler(tau, m[k], rr - pre * tau * vv, vv)
        assert rc == oracle.OK
        sr, sv = np.abs(rr).max(), np.abs(vv).max()
        e64 = max(np.abs((o1 - post * tau * o2) - rr - dr).max() / sr, np.abs(o2 - vv - dv).max() / sv)
        edw = max(np.abs(out[k, :3] * m[k] - dr).max() / sr, np.abs(out[k, 3:] * m[k] - dv).max() / sv)
        worst = max(worst, edw / max(1024 * e64, 2.0 ** -44))
    assert worst <= 1.0, worst


def test_bench_flop_counts_are_current(tmp_path):
    """bench.py's per-solve FP32 work of the double-word form must be the
    count of the current code (tests/df64_flop_count.py)."""
    import importlib.util
    import sys
    sys.path.insert(0, HERE)
    import df64_flop_count as dfc
    spec = importlib.util.spec_from_file_location("bench", os.path.join(os.path.dirname(HERE),
                                                                        "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    lib = dfc.build(str(tmp_path))
    for name, s in dfc.workloads().items():
        f, _, _ = dfc.count(lib, s)
        assert abs(f - bench.DF64_FLOPS_PER_SOLVE[name]) <= 0.5, (name, f)
