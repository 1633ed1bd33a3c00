"""sakura_step_noalloc: the step for callers that cannot allocate device memory.

Programs whose GPU memory belongs to another allocator, or loops that must not
call cudaMalloc/cudaFree, use this entry point: it keeps its scratch in a
fixed file-scope device array instead of allocating.  These tests call it
through the C ABI and compare it with sakura_step (same kernels, library
scratch) within the per-particle tolerance used by the other GPU tests, on
two consecutive calls.  The file is named so that pytest collects it last;
it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

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
