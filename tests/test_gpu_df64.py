"""GPU parity of the double-word form (SAKURA_PREC_DF64): every unordered
pair solved once, the Kepler solves in double-word arithmetic on the FP32
pipe, against the FP64 oracle at the same per-step bound as the FP64 form
(relative 1e-12 against max(|r_i|, R_rms), likewise for v).

Covers every order, N from 2 to 16384 (ragged tiles, diagonal tiles, a
single tile), grid shapes down to one block, the FP64 fallback queue (a
swarm of fast flybys whose pairs leave single-precision range, tight
binaries whose step exceeds the period), composed orders, determinism and
the statistics of the double-word solves; for both symmetric kernels, the
systolic tiles (the default below about 13400 bodies) and the row-group
phases (the default beyond, forced with SAKURA_FLAG_GROUPS on the small
cases).
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
    sk.init(0, flags=sk.FLAG_STATS, precision=sk.PREC_DF64, guess=sk.GUESS_TAYLOR)
    yield
    sk.finalize()


@contextlib.contextmanager
def configured(**opts):
    base = dict(flags=sk.FLAG_STATS, precision=sk.PREC_DF64, guess=sk.GUESS_TAYLOR)
    base.update(opts)
    sk.init(0, **base)
    try:
        yield
    finally:
        sk.init(0, flags=sk.FLAG_STATS, precision=sk.PREC_DF64, guess=sk.GUESS_TAYLOR)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_step(s, tau, order=2, nsteps=1):
    state = dev(s.soa())
    mass = dev(s.m)
    for _ in range(nsteps):
        sk.step(state, mass, tau, order)
    sk.check()
    return ics.from_soa(state.cpu().numpy())


def rel_err(r, v, rr, vr):
    R = np.sqrt((rr ** 2).sum(1).mean())
    V = np.sqrt((vr ** 2).sum(1).mean())
    er = np.linalg.norm(r - rr, axis=1) / np.maximum(np.linalg.norm(rr, axis=1), R)
    ev = np.linalg.norm(v - vr, axis=1) / np.maximum(np.linalg.norm(vr, axis=1), V)
    return float(er.max()), float(ev.max())


SMALL = [("planetary9", ics.planetary(0))] + [
    (f"random{n}", ics.random_cluster(n, seed=n, mass_spread=2.0))
    for n in (2, 3, 31, 32, 33, 255, 256, 257, 513)]


@pytest.mark.parametrize("order", [2, 1, -1])
@pytest.mark.parametrize("name,s", SMALL, ids=[n for n, _ in SMALL])
def test_df64_step_matches_oracle(name, s, order):
    r, v = gpu_step(s, s.dt, order)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("blocks", [0, 1, 7, 300])
def test_df64_plummer_1024_and_grid_shapes(blocks):
    s = ics.plummer(1024, seed=0)
    with configured(grid_blocks=blocks):
        r, v = gpu_step(s, s.dt, 2)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


KERNELS = [(sk.FLAG_TILES, 0), (sk.FLAG_GROUPS, 1)]


@pytest.mark.parametrize("order", [2, 1, -1])
@pytest.mark.parametrize("name,s", SMALL, ids=[n for n, _ in SMALL])
def test_df64_row_groups_match_oracle(name, s, order):
    # (systems of up to 20 bodies otherwise run in the single-block kernel)
    with configured(flags=sk.FLAG_STATS | sk.FLAG_GROUPS | sk.FLAG_NO_SMALL):
        sk.get_stats(reset=True)
        r, v = gpu_step(s, s.dt, order)
        st = sk.get_stats(reset=True)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)
    assert st["group_launches"] == 1


@pytest.mark.parametrize("blocks", [0, 1, 7, 143, 5000])
def test_df64_row_group_grid_shapes(blocks):
    # 1024 particles: 8 groups of 4 row blocks, 144 phases dealt whole; a
    # block's range may start or end inside a group (7 or 143 blocks), 5000
    # are clamped
    s = ics.plummer(1024, seed=0)
    with configured(grid_blocks=blocks, flags=sk.FLAG_STATS | sk.FLAG_GROUPS):
        r, v = gpu_step(s, s.dt, 2)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


def test_df64_tiles_and_row_groups_agree_and_are_deterministic():
    s = ics.random_cluster(3001, seed=4, mass_spread=2.0)
    out = {}
    for flag, _ in KERNELS:
        with configured(flags=sk.FLAG_STATS | flag):
            out[flag] = gpu_step(s, s.dt, 2)
            again = gpu_step(s, s.dt, 2)
        np.testing.assert_array_equal(out[flag][0], again[0])
        np.testing.assert_array_equal(out[flag][1], again[1])
    er, ev = rel_err(*out[sk.FLAG_GROUPS], *out[sk.FLAG_TILES])
    assert er <= TOL and ev <= TOL, (er, ev)


def _full_size_sample(s, k=48, seed=0):
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0, s.n - 1], rng.choice(s.n, k, replace=False)]))
    r, v = gpu_step(s, s.dt, 2)
    rc, rs, vs = oracle.step_sample(s.m, s.r, s.v, s.dt, idx, 2, nthreads=NCPU)
    assert rc == oracle.OK
    R = np.sqrt((r ** 2).sum(1).mean())
    V = np.sqrt((v ** 2).sum(1).mean())
    er = np.linalg.norm(r[idx] - rs, axis=1) / np.maximum(np.linalg.norm(rs, axis=1), R)
    ev = np.linalg.norm(v[idx] - vs, axis=1) / np.maximum(np.linalg.norm(vs, axis=1), V)
    return float(er.max()), float(ev.max())


@pytest.mark.parametrize("flag,groups", KERNELS, ids=["tiles", "groups"])
def test_df64_full_size_bh_cluster_sampled(flag, groups):
    with configured(flags=sk.FLAG_STATS | flag):
        sk.get_stats(reset=True)
        er, ev = _full_size_sample(ics.bh_cluster(16384, seed=0))
        assert (sk.get_stats(reset=True)["group_launches"] > 0) == bool(groups)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("flag,groups", KERNELS, ids=["tiles", "groups"])
def test_df64_full_size_binaries_sampled(flag, groups):
    # the binaries with periods below the step go to the FP64 queue
    s = ics.plummer_binaries(16384, seed=0)
    # sample the binary members as well as random particles
    with configured(flags=sk.FLAG_STATS | flag):
        er, ev = _full_size_sample(s, seed=3)
    assert er <= TOL and ev <= TOL, (er, ev)


def test_df64_default_kernel_at_16384_is_row_groups():
    s = ics.bh_cluster(16384, seed=0)
    sk.get_stats(reset=True)
    gpu_step(s, s.dt, 2)
    assert sk.get_stats(reset=True)["group_launches"] == 1


@pytest.mark.parametrize("flag,groups", KERNELS, ids=["tiles", "groups"])
def test_df64_fast_swarm_uses_the_fp64_queue(flag, groups):
    rng = np.random.default_rng(0)
    n = 64
    m = np.full(n, 1e-6)
    r = rng.uniform(-2.5e-4, 2.5e-4, (n, 3))
    v = rng.normal(0.0, 300.0, (n, 3))
    s = ics.System(m, r, v, 1e-3, "fast-swarm")
    with configured(flags=sk.FLAG_STATS | flag):
        sk.get_stats(reset=True)
        r1, v1 = gpu_step(s, s.dt, 2)
        st = sk.get_stats(reset=True)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r1, v1, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)
    assert st["fp32_pairs"] < st["solves"]  # some pairs went to FP64
    assert st["group_launches"] == groups


@pytest.mark.parametrize("order", [4, 6])
def test_df64_composed_orders(order):
    s = ics.random_cluster(97, seed=4, mass_spread=2.0)
    r, v = gpu_step(s, s.dt, order)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


def test_df64_is_deterministic():
    s = ics.plummer(777, seed=5)
    a = gpu_step(s, s.dt, 2)
    b = gpu_step(s, s.dt, 2)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("flag,groups", KERNELS, ids=["tiles", "groups"])
def test_df64_counts_double_word_solves(flag, groups):
    s = ics.plummer(1024, seed=2)
    with configured(flags=sk.FLAG_STATS | flag):
        sk.get_stats(reset=True)
        gpu_step(s, s.dt, 2)
        st = sk.get_stats(reset=True)
    # a Plummer sphere has no pair outside the double-word class
    assert st["fp32_pairs"] == st["solves"]
    assert st["fallbacks"] == 0


def test_df64_trajectory_planetary_200_steps():
    # 200 steps of the planetary system against the FP64 form of the library
    s = ics.planetary(0)
    r, v = gpu_step(s, s.dt, 2, nsteps=200)
    with configured(precision=sk.PREC_FP64):
        r64, v64 = gpu_step(s, s.dt, 2, nsteps=200)
    er, ev = rel_err(r, v, r64, v64)
    assert er <= 1e-10 and ev <= 1e-10, (er, ev)
