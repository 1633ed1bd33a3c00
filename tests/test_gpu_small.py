"""GPU parity of the single-block kernel for small systems (2 <= n <= 20,
FP64, each unordered pair once) against the CPU oracle.

The kernel keeps the system in shared memory, solves the pairs packed densely
over its lanes and runs every step of a call in one launch.  Tolerance as in
test_gpu_step (one step from identical input, per particle i):
    |dr_i| <= 1e-12 max(|r_i|, R_rms),   |dv_i| <= 1e-12 max(|v_i|, V_rms).
Several steps in one launch must equal the same steps one call at a time bit
for bit, and the multi-kernel step (SAKURA_FLAG_NO_SMALL) must agree to
within summation order.
"""
import contextlib
import os

import numpy as np
import pytest

import oracle
from paper_1402_3325_gb300 import ics
from paper_1402_3325_gb300 import sakura as sk

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_3325_gb300 import build
    build.build()
    sk.init(0, flags=sk.FLAG_STATS)
    yield
    sk.finalize()


@contextlib.contextmanager
def configured(**opts):
    sk.init(0, flags=opts.pop("flags", sk.FLAG_STATS), **opts)
    try:
        yield
    finally:
        sk.init(0, flags=sk.FLAG_STATS)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel_err(r, v, rr, vr):
    R = np.sqrt((rr ** 2).sum(1).mean())
    V = np.sqrt((vr ** 2).sum(1).mean())
    er = np.linalg.norm(r - rr, axis=1) / np.maximum(np.linalg.norm(rr, axis=1), R)
    ev = np.linalg.norm(v - vr, axis=1) / np.maximum(np.linalg.norm(vr, axis=1), V)
    return float(er.max()), float(ev.max())


def run(s, dt, order=2, nsteps=1):
    state = dev(s.soa())
    sk.evolve(state, dev(s.m), dt, order, nsteps)
    sk.check()
    return ics.from_soa(state.cpu().numpy())


def _systems():
    out = [("planetary9", ics.planetary(0)), ("planetary9b", ics.planetary(3)),
           ("double_binary4", ics.hierarchical_double_binary()),
           ("bh20", ics.plummer_bh(20, q=1e6, seed=1)),
           ("binaries20", ics.plummer_binaries(20, seed=2, f_bin=0.5))]
    for n in (2, 3, 4, 7, 16, 19, 20):
        out.append((f"random{n}", ics.random_cluster(n, seed=100 + n, mass_spread=2.0)))
    return out


SYSTEMS = _systems()
GUESSES = {"fp32": sk.GUESS_FP32, "standard": sk.GUESS_STANDARD, "taylor": sk.GUESS_TAYLOR}


@pytest.mark.parametrize("guess", list(GUESSES))
@pytest.mark.parametrize("order", [2, 1, -1])
@pytest.mark.parametrize("name,s", SYSTEMS, ids=[n for n, _ in SYSTEMS])
def test_small_step_matches_oracle(name, s, order, guess):
    with configured(guess=GUESSES[guess]):
        r, v = run(s, s.dt, order)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("guess", ["fp32", "standard"])
@pytest.mark.parametrize("order", [2, 1, -1])
@pytest.mark.parametrize("name,s", SYSTEMS, ids=[n for n, _ in SYSTEMS])
def test_small_double_word_step_matches_oracle(name, s, order, guess):
    # the double-word form: pair solves on the FP32 pipe, FP64 solves for the
    # pairs it does not admit, sums in FP64; the same 1e-12 bound
    with configured(guess=GUESSES[guess], precision=sk.PREC_DF64):
        sk.get_stats(reset=True)
        r, v = run(s, s.dt, order)
        st = sk.get_stats(reset=True)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)
    assert 0 <= st["fp32_pairs"] <= st["solves"] == s.n * (s.n - 1) // 2


def test_small_double_word_solves_most_pairs_and_repeats_bit_for_bit():
    s = ics.planetary(0)
    with configured(guess=sk.GUESS_FP32, precision=sk.PREC_DF64):
        sk.get_stats(reset=True)
        a = dev(s.soa())
        m = dev(s.m)
        sk.evolve(a, m, s.dt, 2, 40)
        st = sk.get_stats(reset=True)
        b = dev(s.soa())
        for _ in range(40):
            sk.step(b, m, s.dt, 2)
        sk.check()
    assert st["fp32_pairs"] >= 0.9 * st["solves"], st
    np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    rc, rr, vr = oracle.evolve(s.m, s.r, s.v, s.dt, 40)
    r, v = ics.from_soa(a.cpu().numpy())
    er, ev = rel_err(r, v, rr, vr)
    assert er <= 1e-11 and ev <= 1e-11, (er, ev)


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("name,s", SYSTEMS[:4], ids=[n for n, _ in SYSTEMS[:4]])
def test_small_composed_step_matches_oracle(name, s, order):
    with configured(guess=sk.GUESS_FP32):
        r, v = run(s, s.dt, order)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


def test_small_planetary_2000_steps_one_launch():
    # the 2000-step planetary run in one launch; as for the multi-kernel
    # step, the trajectories stay within 1e-9 of the oracle's (weak chaos)
    s = ics.planetary(0)
    with configured(guess=sk.GUESS_FP32):
        r, v = run(s, s.dt, 2, 2000)
    rc, rr, vr = oracle.evolve(s.m, s.r, s.v, s.dt, 2000)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= 1e-9 and ev <= 1e-9, (er, ev)


@pytest.mark.parametrize("order", [2, 4])
def test_small_evolve_equals_repeated_steps(order):
    s = ics.random_cluster(13, seed=7, mass_spread=2.0)
    with configured(guess=sk.GUESS_FP32):
        a = dev(s.soa())
        m = dev(s.m)
        sk.evolve(a, m, s.dt, order, 25)
        b = dev(s.soa())
        for _ in range(25):
            sk.step(b, m, s.dt, order)
        sk.check()
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        # host buffers, pageable and page-locked: the same launch
        host = np.ascontiguousarray(s.soa())
        sk.evolve_host(host, np.ascontiguousarray(s.m), s.dt, order, 25)
        np.testing.assert_array_equal(host, a.cpu().numpy())
        ps = torch.empty((6, s.n), dtype=torch.float64).pin_memory()
        pm = torch.empty((s.n,), dtype=torch.float64).pin_memory()
        ps.numpy()[...] = s.soa()
        pm.numpy()[...] = s.m
        sk.evolve_host(ps.numpy(), pm.numpy(), s.dt, order, 25)
        np.testing.assert_array_equal(ps.numpy(), a.cpu().numpy())


@pytest.mark.parametrize("form", ["fp64", "df64"])
@pytest.mark.parametrize("name,s", SYSTEMS, ids=[n for n, _ in SYSTEMS])
def test_small_agrees_with_multi_kernel_step(name, s, form):
    # one step from the same input: the same solves, a different summation
    # order, so rounding only, well inside the 1e-12 per-step bound that each
    # meets against the oracle.  (Over several steps the tight binaries, many
    # periods per step, amplify such differences: 7.6e-11 in v after three.)
    prec = sk.PREC_DF64 if form == "df64" else sk.PREC_FP64
    with configured(guess=sk.GUESS_FP32, precision=prec):
        r1, v1 = run(s, s.dt, 2)
    with configured(guess=sk.GUESS_FP32, precision=prec,
                    flags=sk.FLAG_STATS | sk.FLAG_NO_SMALL):
        r2, v2 = run(s, s.dt, 2)
    er, ev = rel_err(r1, v1, r2, v2)
    assert er <= 1e-13 and ev <= 1e-13, (er, ev)


def test_small_counts_pairs_and_solves():
    s = ics.random_cluster(20, seed=3)
    sk.get_stats(reset=True)
    run(s, s.dt, 4, 5)
    st = sk.get_stats(reset=True)
    assert st["steps"] == 15
    assert st["pairs"] == 15 * 20 * 19 and 2 * st["solves"] == st["pairs"]
    assert st["iters"] >= st["solves"] and 1 <= st["max_iters"] <= 50
    assert st["warp_slots"] >= st["iters"]


def test_small_limits_route_elsewhere():
    # n = 21 and the other forms take the multi-kernel paths; same results
    # as the oracle either way
    s = ics.random_cluster(21, seed=9, mass_spread=2.0)
    r, v = run(s, s.dt, 2)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)
    # (the mixed form's own parity bound is 1e-8, tests/test_gpu_mixed.py)
    s = ics.random_cluster(12, seed=9)
    for opts, tol in ((dict(pair_mode=sk.PAIRS_ORDERED), TOL),
                      (dict(precision=sk.PREC_MIXED), 1e-8)):
        with configured(**opts):
            r, v = run(s, s.dt, 2)
        rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
        er, ev = rel_err(r, v, rr, vr)
        assert er <= tol and ev <= tol, (opts, er, ev)


def test_small_zero_steps_is_a_no_op():
    s = ics.random_cluster(5, seed=1)
    state = dev(s.soa())
    sk.evolve(state, dev(s.m), s.dt, 2, 0)
    sk.check()
    np.testing.assert_array_equal(state.cpu().numpy(), s.soa())


@pytest.mark.parametrize("fault", ["coincident", "nonfinite", "mass"])
def test_small_faults_are_reported_once(fault):
    s = ics.random_cluster(10, seed=2)
    code = {"coincident": sk.E_COINCIDENT, "nonfinite": sk.E_NONFINITE, "mass": sk.E_MASS}
    if fault == "coincident":
        s.r[4] = s.r[7]
        s.v[4] = s.v[7]
    elif fault == "nonfinite":
        s.v[3, 2] = np.inf
    else:
        s.m[6] = 0.0
    state = dev(s.soa())
    sk.evolve(state, dev(s.m), 0.01, 2, 3)
    assert sk.check_code() == code[fault]
    assert sk.check_code() == sk.OK


def test_small_evolve_captured_in_a_graph():
    # no allocation and no synchronisation: capturable, and a replay equals
    # the direct call
    s = ics.planetary(1)
    stream = torch.cuda.Stream()
    with configured(guess=sk.GUESS_FP32, stream=stream.cuda_stream):
        m = dev(s.m)
        ref = dev(s.soa())
        with torch.cuda.stream(stream):
            sk.evolve(ref, m, s.dt, 2, 40)
        stream.synchronize()
        state = dev(s.soa())
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            sk.evolve(state, m, s.dt, 2, 20)
        state.copy_(dev(s.soa()))
        torch.cuda.synchronize()
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        sk.check()
        np.testing.assert_array_equal(state.cpu().numpy(), ref.cpu().numpy())
