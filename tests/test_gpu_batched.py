"""GPU tests of the batched ensemble path (sakura_step_batched): every
system is checked against the oracle run on that system alone."""
import contextlib
import os

import numpy as np
import pytest

import oracle
from paper_1402_3325_gb300 import ics
from paper_1402_3325_gb300 import sakura as sk

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1
TOL = 1e-12


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


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def run_batched(ens, order=2, nsteps=1, calls=1):
    st = dev(ens.state)
    m = dev(ens.m)
    off = dev(ens.offsets, torch.int64)
    dt = dev(ens.dt)
    for _ in range(calls):
        sk.step_batched(st, m, off, ens.offsets, dt, order, nsteps)
    sk.check()
    return st.cpu().numpy()


def small_ensemble(nsys=48, seed=3, n_lo=1, n_hi=64):
    e = ics.ensemble(nsys, seed=seed, n_lo=max(2, n_lo), n_hi=n_hi)
    return e


def rel_err(r, v, rr, vr):
    R = np.sqrt((rr ** 2).sum(1).mean())
    V = np.sqrt((vr ** 2).sum(1).mean())
    er = np.linalg.norm(r - rr, axis=1) / np.maximum(np.linalg.norm(rr, axis=1), R)
    ev = np.linalg.norm(v - vr, axis=1) / np.maximum(np.linalg.norm(vr, axis=1), V)
    return float(er.max()), float(ev.max())


def check_against_oracle(ens, got, order, nsteps, tol):
    worst = 0.0
    for k in range(ens.nsys):
        s = ens.system(k)
        a, b = int(ens.offsets[k]), int(ens.offsets[k + 1])
        rc, rr, vr = oracle.evolve(s.m, s.r, s.v, s.dt, nsteps, order)
        assert rc == oracle.OK
        r, v = ics.from_soa(got[:, a:b])
        er, ev = rel_err(r, v, rr, vr)
        worst = max(worst, er, ev)
    assert worst <= tol, worst
    return worst


@pytest.mark.parametrize("order", [2, 1, -1])
def test_batched_one_step_matches_oracle(order):
    ens = small_ensemble()
    got = run_batched(ens, order, 1)
    check_against_oracle(ens, got, order, 1, TOL)


@pytest.mark.parametrize("order", [2, 1, -1])
def test_batched_fp32_seed_matches_oracle(order):
    # the single-precision seed and the Taylor carry in the batched kernel
    ens = small_ensemble(seed=5)
    with configured(guess=sk.GUESS_FP32):
        sk.get_stats(reset=True)
        got = run_batched(ens, order, 3)
        st = sk.get_stats(reset=True)
    check_against_oracle(ens, got, order, 3, 1e-11)
    # each unordered pair is solved once
    assert 2 * st["solves"] == st["pairs"]
    assert st["carries"] > 0.5 * st["solves"]
    assert st["iters"] < 1.5 * st["solves"]


def test_batched_many_steps_matches_oracle():
    ens = small_ensemble(nsys=24, seed=8)
    got = run_batched(ens, 2, 20)
    check_against_oracle(ens, got, 2, 20, 1e-10)


def test_batched_includes_single_particle_and_pairs():
    # N = 1 systems only drift; N = 2 systems are exact Kepler orbits
    e = ics.ensemble(6, seed=1, n_lo=2, n_hi=3)
    one = ics.System(np.array([0.5]), np.array([[0.1, 0.2, 0.3]]), np.array([[0.3, -0.1, 0.2]]),
                     0.01)
    state = np.concatenate([one.soa(), e.state], 1)
    m = np.concatenate([one.m, e.m])
    off = np.concatenate([[0], 1 + e.offsets]).astype(np.int64)
    dt = np.concatenate([[0.01], e.dt])
    ens = ics.Ensemble(m, state, off, dt, np.zeros(7, dtype=np.int64))
    got = run_batched(ens, 2, 3)
    np.testing.assert_allclose(got[:3, 0], one.r[0] + 3 * 0.01 * one.v[0], rtol=0, atol=1e-15)
    check_against_oracle(ens, got, 2, 3, 1e-12)


def test_batched_shapes_and_autotune_are_bit_identical():
    ens = small_ensemble(nsys=96, seed=5)
    ref = run_batched(ens, 2, 2)
    w, b, times = sk.batched_tuning()
    assert w in (1, 2, 4, 8) and b > 0 and all(t > 0 for t in times.values())
    for warps in (1, 2, 8):
        with configured(block_warps=warps):
            got = run_batched(ens, 2, 2)
        np.testing.assert_array_equal(got, ref)


def test_batched_graph_replay_equals_one_call():
    ens = small_ensemble(nsys=40, seed=9)
    two_calls = run_batched(ens, 2, 3, calls=2)
    one_call = run_batched(ens, 2, 6, calls=1)
    np.testing.assert_array_equal(two_calls, one_call)


def test_batched_argument_errors():
    ens = small_ensemble(nsys=4, seed=2)
    lib = sk.load()
    st, m = dev(ens.state), dev(ens.m)
    off, dt = dev(ens.offsets, torch.int64), dev(ens.dt)
    bad = ens.offsets.copy()
    bad[0] = 1
    assert lib.sakura_step_batched(sk._ptr(st), sk._ptr(m), sk._ptr(off), bad.ctypes.data, 4,
                                   sk._ptr(dt), 2, 1) == sk.E_ARG
    big = np.array([0, 65], dtype=np.int64)
    assert lib.sakura_step_batched(sk._ptr(st), sk._ptr(m), sk._ptr(off), big.ctypes.data, 1,
                                   sk._ptr(dt), 2, 1) == sk.E_ARG
    assert lib.sakura_step_batched(sk._ptr(st), sk._ptr(m), sk._ptr(off),
                                   ens.offsets.ctypes.data, 4, sk._ptr(dt), 3, 1) == sk.E_ARG
