"""GPU tests of the composed higher-order steps (orders 4, 6, 8: Yoshida's
triple jump of the second-order map, the composition route of Sec. 2.2).

Each composed step must equal the oracle's composed step within the per-step
parity bound (relative 1e-12 against max(|r_i|, R_rms), likewise for v), in
both pair modes, in the host-buffer entry point and in the batched path.  The
oracle's composition is pinned separately (tests/test_oracle_step.py): exact
for N = 2, fourth and sixth order in the symmetric Eq. 28 limit.
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


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel_err(r, v, rr, vr):
    R = np.sqrt((rr ** 2).sum(1).mean())
    V = np.sqrt((vr ** 2).sum(1).mean())
    er = np.linalg.norm(r - rr, axis=1) / np.maximum(np.linalg.norm(rr, axis=1), R)
    ev = np.linalg.norm(v - vr, axis=1) / np.maximum(np.linalg.norm(vr, axis=1), V)
    return float(er.max()), float(ev.max())


SYSTEMS = [("planetary9", ics.planetary(0)), ("binary", ics.random_cluster(2, seed=5)),
           ("random33", ics.random_cluster(33, seed=33, mass_spread=2.0)),
           ("random257", ics.random_cluster(257, seed=257, mass_spread=2.0))]


@pytest.mark.parametrize("pairs", [sk.PAIRS_SYMMETRIC, sk.PAIRS_ORDERED])
@pytest.mark.parametrize("order", [4, 6, 8])
@pytest.mark.parametrize("name,s", SYSTEMS, ids=[n for n, _ in SYSTEMS])
def test_composed_step_matches_oracle(name, s, order, pairs):
    with configured(pair_mode=pairs, guess=sk.GUESS_TAYLOR):
        state = dev(s.soa())
        sk.step(state, dev(s.m), s.dt, order)
        sk.check()
        r, v = ics.from_soa(state.cpu().numpy())
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


def test_composed_plummer_1024():
    s = ics.plummer(1024, seed=1)
    state = dev(s.soa())
    sk.step(state, dev(s.m), s.dt, 4)
    sk.check()
    r, v = ics.from_soa(state.cpu().numpy())
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 4, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


def test_composed_counts_maps():
    s = ics.random_cluster(40, seed=2)
    state = dev(s.soa())
    sk.get_stats(reset=True)
    sk.step(state, dev(s.m), s.dt, 6)
    st = sk.get_stats(reset=True)
    assert st["steps"] == 9 and st["pairs"] == 9 * 40 * 39


def test_composed_evolve_host_equals_device_steps():
    s = ics.random_cluster(70, seed=4)
    host = np.ascontiguousarray(s.soa())
    sk.evolve_host(host, np.ascontiguousarray(s.m), s.dt, 4, 3)
    state = dev(s.soa())
    mass = dev(s.m)
    for _ in range(3):
        sk.step(state, mass, s.dt, 4)
    sk.check()
    np.testing.assert_array_equal(host, state.cpu().numpy())


@pytest.mark.parametrize("order", [4, 6])
def test_composed_batched_matches_oracle(order):
    ens = ics.ensemble(24, seed=21)
    st = dev(ens.state)
    sk.step_batched(st, dev(ens.m), dev(ens.offsets, torch.int64), ens.offsets, dev(ens.dt),
                    order, 2)
    sk.check()
    got = st.cpu().numpy()
    for k in range(ens.nsys):
        s = ens.system(k)
        a, b = int(ens.offsets[k]), int(ens.offsets[k + 1])
        rc, rr, vr = oracle.evolve(s.m, s.r, s.v, s.dt, 2, order)
        r, v = ics.from_soa(got[:, a:b])
        er, ev = rel_err(r, v, rr, vr)
        assert er <= TOL and ev <= TOL, (k, er, ev)


def test_composed_orders_rejected_elsewhere():
    lib = sk.load()
    state = dev(np.zeros((6, 4)))
    mass = dev(np.ones(4))
    for order in (3, 5, 10):
        assert lib.sakura_step(sk._ptr(state), sk._ptr(mass), 4, 0.1, order) == sk.E_ARG
    # the allocation-free entry point keeps to the maps of orders 2, 1, -1
    assert lib.sakura_step_noalloc(sk._ptr(state), sk._ptr(mass), 4, 0.1, 4, None) == sk.E_ARG
