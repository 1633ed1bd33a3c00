"""sakura_step_noalloc: the step for callers that cannot allocate device memory.

Programs whose GPU memory belongs to another allocator, or loops that must not
call cudaMalloc/cudaFree, use this entry point: it keeps its scratch in a
fixed file-scope device array instead of allocating.  These tests call it
through the C ABI and compare it with sakura_step (same kernels, library
scratch) and with the CPU oracle, within the per-particle tolerance used by
the other GPU tests, on two consecutive calls.  The file is named so that
pytest collects it last; it passes alone in a fresh process and after the
other tests.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1402_3325_gb300 import ics
from paper_1402_3325_gb300 import sakura as sk

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_3325_gb300 import build
    build.build()
    sk.init(0, stream=torch.cuda.current_stream().cuda_stream)
    yield
    sk.finalize()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    """Largest per-particle position and velocity difference relative to
    max(|x_i|, rms) of the reference state b ([6, n])."""
    ra, va, rb, vb = a[:3].T, a[3:].T, b[:3].T, b[3:].T
    R = np.sqrt((rb ** 2).sum(1).mean())
    V = np.sqrt((vb ** 2).sum(1).mean())
    er = np.linalg.norm(ra - rb, axis=1) / np.maximum(np.linalg.norm(rb, axis=1), R)
    ev = np.linalg.norm(va - vb, axis=1) / np.maximum(np.linalg.norm(vb, axis=1), V)
    return float(er.max()), float(ev.max())


@pytest.mark.parametrize("name,s", [("plummer1024", ics.plummer(1024, seed=4)),
                                    ("random777", ics.random_cluster(777, seed=2)),
                                    ("planetary9", ics.planetary(3))])
def test_noalloc_matches_step_on_two_calls(name, s):
    stream = torch.cuda.current_stream().cuda_stream
    ref = _dev(s.soa())
    got = _dev(s.soa())
    mass = _dev(s.m)
    for call in range(2):
        sk.step(ref, mass, s.dt, 2)
        sk.step_noalloc(got, mass, s.dt, 2, stream=stream)
        sk.check()
        er, ev = _rel(got.cpu().numpy(), ref.cpu().numpy())
        assert er <= TOL and ev <= TOL, (name, call, er, ev)


@pytest.mark.parametrize("order", [2, 1, -1])
@pytest.mark.parametrize("name,s", [("random300", ics.random_cluster(300, seed=8, mass_spread=2.0)),
                                    ("planetary9", ics.planetary(5))])
def test_noalloc_matches_oracle_on_two_calls(name, s, order):
    # two consecutive calls against two oracle steps (the second call starts
    # from the first call's output, which also went through the shared array)
    got = _dev(s.soa())
    mass = _dev(s.m)
    r, v = s.r.copy(), s.v.copy()
    for call in range(2):
        sk.step_noalloc(got, mass, s.dt, order)
        rc, r, v = oracle.step(s.m, r, v, s.dt, order, nthreads=os.cpu_count() or 1)
        assert rc == oracle.OK
        ref = ics.to_soa(r, v)
        er, ev = _rel(got.cpu().numpy(), ref)
        assert er <= (call + 1) * TOL and ev <= (call + 1) * TOL, (name, order, call, er, ev)
        # continue both from the oracle's state so each call is one step
        got = _dev(ref)


def test_noalloc_single_particle_only_drifts():
    # one particle has no pairs: every order moves it by tau v
    got = _dev(np.array([[1.0], [2.0], [-3.0], [0.5], [-0.25], [2.0]]))
    mass = _dev(np.array([1.0]))
    for order, frac in ((2, 1.0), (1, 1.0), (-1, 1.0)):
        x0 = got.cpu().numpy().copy()
        sk.step_noalloc(got, mass, 0.125, order)
        x1 = got.cpu().numpy()
        np.testing.assert_allclose(x1[:3], x0[:3] + frac * 0.125 * x0[3:], rtol=0, atol=1e-15)
        np.testing.assert_array_equal(x1[3:], x0[3:])


def test_noalloc_near_its_size_limit_matches_ordered_step():
    # n close to the scratch limit, where the scratch layout is tightest;
    # against sakura_step in its ordered-pair mode (the same kernels)
    n = sk.NOALLOC_MAX_N - 5
    s = ics.random_cluster(n, seed=9)
    sk.init(0, stream=torch.cuda.current_stream().cuda_stream, pair_mode=sk.PAIRS_ORDERED)
    try:
        ref = _dev(s.soa())
        got = _dev(s.soa())
        mass = _dev(s.m)
        sk.step(ref, mass, s.dt, 2)
        sk.step_noalloc(got, mass, s.dt, 2)
        sk.check()
        er, ev = _rel(got.cpu().numpy(), ref.cpu().numpy())
        assert er <= TOL and ev <= TOL, (er, ev)
    finally:
        sk.init(0, stream=torch.cuda.current_stream().cuda_stream)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n = sk.NOALLOC_MAX_N + 1
    state = torch.zeros((6, n), dtype=torch.float64, device="cuda")
    mass = torch.ones(n, dtype=torch.float64, device="cuda")
    lib = sk.load()
    rc = lib.sakura_step_noalloc(sk._ptr(state), sk._ptr(mass), n, 0.01, 2, None)
    assert rc == sk.E_ARG


def test_noalloc_reports_a_fault_then_recovers():
    s = ics.random_cluster(64, seed=5)
    s.r[3] = s.r[4]
    s.v[3] = s.v[4]
    state = _dev(s.soa())
    lib = sk.load()
    rc = lib.sakura_step_noalloc(sk._ptr(state), sk._ptr(_dev(s.m)), s.n, s.dt, 2, None)
    assert rc == sk.E_COINCIDENT
    # the shared status word is cleared by the next call
    good = ics.random_cluster(64, seed=6)
    ref = _dev(good.soa())
    got = _dev(good.soa())
    mass = _dev(good.m)
    sk.step(ref, mass, good.dt, 2)
    sk.step_noalloc(got, mass, good.dt, 2)
    er, ev = _rel(got.cpu().numpy(), ref.cpu().numpy())
    assert er <= TOL and ev <= TOL
