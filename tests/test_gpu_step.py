"""GPU parity of the FP64 step and the energy against the CPU oracle.

Every call goes through the C ABI (libsakura.so) via the ctypes binding.
Tolerance (one step from identical input, per particle i):
    |dr_i| <= 1e-12 max(|r_i|, R_rms),   |dv_i| <= 1e-12 max(|v_i|, V_rms)
with R_rms, V_rms the system's RMS position and speed (the floor covers
particles near the origin or at rest, e.g. a central black hole).
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


def systems_small():
    out = [("planetary9", ics.planetary(0))]
    for n in (2, 3, 31, 32, 33, 255, 256, 257, 513):
        out.append((f"random{n}", ics.random_cluster(n, seed=n, mass_spread=2.0)))
    return out


SMALL = systems_small()


@pytest.mark.parametrize("order", [2, 1, -1])
@pytest.mark.parametrize("name,s", SMALL, ids=[n for n, _ in SMALL])
def test_step_matches_oracle(name, s, order):
    with configured(pair_mode=sk.PAIRS_ORDERED):
        r, v = gpu_step(s, s.dt, order)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("guess", [sk.GUESS_STANDARD, sk.GUESS_TAYLOR])
def test_plummer_1024_step_matches_oracle(guess):
    s = ics.plummer(1024, seed=0)
    with configured(guess=guess, pair_mode=sk.PAIRS_ORDERED):
        r, v = gpu_step(s, s.dt, 2)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("order", [2, 1, -1])
def test_taylor_guess_small_systems(order):
    for name, s in SMALL[:6]:
        with configured(guess=sk.GUESS_TAYLOR, pair_mode=sk.PAIRS_ORDERED):
            r, v = gpu_step(s, s.dt, order)
        rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
        er, ev = rel_err(r, v, rr, vr)
        assert er <= TOL and ev <= TOL, (name, er, ev)


def test_taylor_guess_reduces_iterations():
    s = ics.plummer(1024, seed=0)
    its = {}
    for guess in (sk.GUESS_STANDARD, sk.GUESS_TAYLOR):
        with configured(guess=guess):
            sk.get_stats(reset=True)
            gpu_step(s, s.dt, 2)
            st = sk.get_stats(reset=True)
        its[guess] = st["iters"] / st["solves"]
    assert its[sk.GUESS_TAYLOR] < its[sk.GUESS_STANDARD] - 0.2


@pytest.mark.parametrize("warps,blocks", [(4, 1), (8, 3), (16, 7), (4, 77), (8, 5000)])
def test_launch_shapes_match_oracle(warps, blocks):
    s = ics.random_cluster(1000, seed=21, mass_spread=1.0)
    with configured(block_warps=warps, grid_blocks=blocks, pair_mode=sk.PAIRS_ORDERED):
        r, v = gpu_step(s, s.dt, 2)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


def test_single_particle_only_drifts():
    s = ics.System(np.array([1.0]), np.array([[0.1, 0.2, 0.3]]), np.array([[1.0, -2.0, 0.5]]),
                   0.25)
    r, v = gpu_step(s, s.dt, 2)
    np.testing.assert_allclose(r[0], s.r[0] + 0.25 * s.v[0], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(v, s.v)


def _full_size_sample(s, k=48, seed=0):
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0, s.n - 1], rng.choice(s.n, k, replace=False)]))
    r, v = gpu_step(s, s.dt, 2)
    rc, rs, vs = oracle.step_sample(s.m, s.r, s.v, s.dt, idx, 2, nthreads=NCPU)
    assert rc == oracle.OK
    # system-wide scales from the full GPU state
    R = np.sqrt((r ** 2).sum(1).mean())
    V = np.sqrt((v ** 2).sum(1).mean())
    er = np.linalg.norm(r[idx] - rs, axis=1) / np.maximum(np.linalg.norm(rs, axis=1), R)
    ev = np.linalg.norm(v[idx] - vs, axis=1) / np.maximum(np.linalg.norm(vs, axis=1), V)
    return float(er.max()), float(ev.max())


def test_full_size_bh_cluster_sampled():
    with configured(pair_mode=sk.PAIRS_ORDERED):
        er, ev = _full_size_sample(ics.bh_cluster(16384, seed=0))
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("guess", [sk.GUESS_STANDARD, sk.GUESS_TAYLOR])
def test_full_size_plummer_binaries_sampled(guess):
    s = ics.plummer_binaries(16384, seed=0)
    with configured(guess=guess, pair_mode=sk.PAIRS_ORDERED):
        er, ev = _full_size_sample(s, seed=1)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("n", [2, 9, 100, 1024, 3001])
def test_energy_matches_oracle(n):
    s = ics.planetary(0) if n == 9 else ics.random_cluster(n, seed=n)
    E = sk.energy(dev(s.soa()), dev(s.m))
    Eo = oracle.energy(s.m, s.r, s.v)[0]
    assert abs(E - Eo) <= 1e-14 * abs(Eo)


def test_planetary_trajectory_2000_steps():
    # the full 2000-step planetary run; chaos is weak here, so the two
    # trajectories stay within 1e-9 of each other (measured: 1.0e-10)
    s = ics.planetary(0)
    r, v = gpu_step(s, s.dt, 2, nsteps=2000)
    rc, rr, vr = oracle.evolve(s.m, s.r, s.v, s.dt, 2000)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= 1e-9 and ev <= 1e-9, (er, ev)
    E0 = oracle.energy(s.m, s.r, s.v)[0]
    E1 = sk.energy(dev(ics.to_soa(r, v)), dev(s.m))
    assert abs(E1 / E0 - 1) < 1e-6


def test_evolve_host_equals_device_steps():
    s = ics.random_cluster(300, seed=3)
    r, v = gpu_step(s, s.dt, 2, nsteps=3)
    host = s.soa().copy()
    sk.evolve_host(host, s.m.copy(), s.dt, 2, 3)
    np.testing.assert_array_equal(host, ics.to_soa(r, v))


def _pinned(a):
    t = torch.empty(a.shape, dtype=torch.float64).pin_memory()
    t.numpy()[...] = a
    return t


@pytest.mark.parametrize("order,nsteps", [(2, 1), (2, 3), (1, 2), (4, 1), (4, 2)])
def test_evolve_host_pinned_equals_device_steps(order, nsteps):
    # page-locked buffers: the kernels read and write the host state in
    # place (one sub-step, or the first and last of several)
    s = ics.random_cluster(300, seed=3)
    r, v = gpu_step(s, s.dt, order, nsteps=nsteps)
    hs, hm = _pinned(s.soa()), _pinned(s.m)
    sk.get_stats(reset=True)
    sk.evolve_host(hs.numpy(), hm.numpy(), s.dt, order, nsteps)
    sub = 3 if order == 4 else 1
    assert sk.get_stats(reset=True)["steps"] == sub * nsteps
    np.testing.assert_array_equal(hs.numpy(), ics.to_soa(r, v))
    np.testing.assert_array_equal(hm.numpy(), s.m)


@pytest.mark.parametrize("form", ["df64", "mixed", "ordered"])
def test_evolve_host_pinned_other_forms(form):
    opts = {"df64": dict(precision=sk.PREC_DF64), "mixed": dict(precision=sk.PREC_MIXED),
            "ordered": dict(pair_mode=sk.PAIRS_ORDERED)}[form]
    s = ics.random_cluster(200, seed=5)
    with configured(**opts):
        r, v = gpu_step(s, s.dt, 2, nsteps=2)
        hs, hm = _pinned(s.soa()), _pinned(s.m)
        sk.evolve_host(hs.numpy(), hm.numpy(), s.dt, 2, 2)
        np.testing.assert_array_equal(hs.numpy(), ics.to_soa(r, v))


def test_evolve_host_pinned_state_pageable_masses():
    # one page-locked buffer and one pageable one: the copy-engine path
    s = ics.random_cluster(100, seed=4)
    r, v = gpu_step(s, s.dt, 2, nsteps=2)
    hs = _pinned(s.soa())
    sk.evolve_host(hs.numpy(), s.m.copy(), s.dt, 2, 2)
    np.testing.assert_array_equal(hs.numpy(), ics.to_soa(r, v))


def test_evolve_host_pinned_zero_steps_and_single_particle():
    s = ics.random_cluster(50, seed=6)
    hs, hm = _pinned(s.soa()), _pinned(s.m)
    sk.evolve_host(hs.numpy(), hm.numpy(), s.dt, 2, 0)
    np.testing.assert_array_equal(hs.numpy(), s.soa())
    one = _pinned(s.soa()[:, :1].copy())
    m1 = _pinned(s.m[:1].copy())
    sk.evolve_host(one.numpy(), m1.numpy(), 0.25, 2, 2)
    x0 = s.soa()[:, 0]
    np.testing.assert_allclose(one.numpy()[:3, 0], x0[:3] + 0.5 * x0[3:], rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(one.numpy()[3:, 0], x0[3:])


def test_evolve_host_pinned_reports_faults_once():
    bad = ics.random_cluster(40, seed=2)
    bad.r[5] = bad.r[6]
    bad.v[5] = bad.v[6]
    good = ics.random_cluster(40, seed=2)
    hs, hm = _pinned(bad.soa()), _pinned(bad.m)
    for _ in range(2):
        hs.numpy()[...] = bad.soa()
        with pytest.raises(sk.SakuraError) as e:
            sk.evolve_host(hs.numpy(), hm.numpy(), 0.01, 2, 1)
        assert e.value.code == sk.E_COINCIDENT
    hs.numpy()[...] = good.soa()
    sk.evolve_host(hs.numpy(), hm.numpy(), 0.01, 2, 1)
    assert sk.check_code() == sk.OK
    r, v = gpu_step(good, 0.01, 2)
    np.testing.assert_array_equal(hs.numpy(), ics.to_soa(r, v))


def test_stats_count_pairs_and_iterations():
    s = ics.random_cluster(200, seed=9)
    with configured(pair_mode=sk.PAIRS_ORDERED):
        sk.get_stats(reset=True)
        gpu_step(s, s.dt, 2, nsteps=2)
        st = sk.get_stats(reset=True)
    assert st["steps"] == 2 and st["pairs"] == 2 * 200 * 199
    assert st["iters"] >= st["pairs"] and st["warp_slots"] >= st["iters"]
    assert 1 <= st["max_iters"] <= 50


def _expect_fault(s, code, **opts):
    with configured(**opts):
        state = dev(s.soa())
        mass = dev(s.m)
        sk.step(state, mass, 0.01, 2)
        assert sk.check_code() == code
        assert sk.check_code() == sk.OK  # the fault is reported once


def test_fault_coincident_pair():
    s = ics.random_cluster(40, seed=2)
    s.r[5] = s.r[6]
    s.v[5] = s.v[6]
    _expect_fault(s, sk.E_COINCIDENT)


def test_fault_nonfinite_state():
    s = ics.random_cluster(40, seed=2)
    s.v[3, 1] = np.nan
    _expect_fault(s, sk.E_NONFINITE)


def test_fault_bad_mass():
    s = ics.random_cluster(40, seed=2)
    s.m[7] = 0.0
    _expect_fault(s, sk.E_MASS)


def test_fault_kepler_not_converged():
    # one Laguerre step and no bisection cannot converge a strong flyby
    m = np.array([0.5, 0.5])
    r = np.array([[0.005, 0.001, 0.0], [-0.005, -0.001, 0.0]])
    v = np.array([[-0.5, 7.5, 0.25], [0.5, -7.5, -0.25]])
    s = ics.System(m, r, v, 0.05)
    with configured(kepler_max_iter=1, kepler_bisection=0):
        state = dev(s.soa())
        sk.step(state, dev(s.m), 0.05, 2)
        assert sk.check_code() == sk.E_KEPLER
    # the default solver recovers the same pair and the context still works
    r1, v1 = gpu_step(s, 0.05, 2)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, 0.05, 2)
    er, ev = rel_err(r1, v1, rr, vr)
    assert er <= TOL and ev <= TOL


def test_argument_errors():
    lib = sk.load()
    state = dev(np.zeros((6, 4)))
    mass = dev(np.ones(4))
    assert lib.sakura_step(sk._ptr(state), sk._ptr(mass), 0, 0.1, 2) == sk.E_ARG
    assert lib.sakura_step(sk._ptr(state), sk._ptr(mass), 4, 0.1, 3) == sk.E_ARG
    assert lib.sakura_step(None, sk._ptr(mass), 4, 0.1, 2) == sk.E_ARG
    assert lib.sakura_step(sk._ptr(state), sk._ptr(mass), 4, float("nan"), 2) == sk.E_ARG


def _fast_swarm(n=64, seed=0):
    # stars of mass 1e-6 in a cube of side 5e-4 at speeds ~300: for most pairs
    # the standard guess t / r0 lies so far past the root (sqrt(-beta) t / r0
    # ~ 10^3) that the G functions overflow there
    rng = np.random.default_rng(seed)
    m = np.full(n, 1e-6)
    r = rng.uniform(-2.5e-4, 2.5e-4, (n, 3))
    v = rng.normal(0.0, 300.0, (n, 3))
    return ics.System(m, r, v, 1e-3, "fast-swarm")


@pytest.mark.parametrize("pairs", [sk.PAIRS_ORDERED, sk.PAIRS_SYMMETRIC])
@pytest.mark.parametrize("guess", [sk.GUESS_STANDARD, sk.GUESS_TAYLOR, sk.GUESS_FP32])
def test_fast_hyperbolic_pairs_with_overflowing_guess(guess, pairs):
    s = _fast_swarm()
    with configured(guess=guess, pair_mode=pairs):
        r, v = gpu_step(s, s.dt, 2)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


# --- symmetric mode: every unordered pair solved once (Newton's third law) ---

@pytest.mark.parametrize("guess", [sk.GUESS_TAYLOR, sk.GUESS_FP32])
@pytest.mark.parametrize("order", [2, 1, -1])
@pytest.mark.parametrize("name,s", SMALL, ids=[n for n, _ in SMALL])
def test_symmetric_step_matches_oracle(name, s, order, guess):
    with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=guess):
        r, v = gpu_step(s, s.dt, order)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("blocks", [0, 1, 7, 300])
def test_symmetric_plummer_1024_and_grid_shapes(blocks):
    s = ics.plummer(1024, seed=0)
    with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=sk.GUESS_TAYLOR, grid_blocks=blocks):
        r, v = gpu_step(s, s.dt, 2)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("guess", [sk.GUESS_TAYLOR, sk.GUESS_FP32])
def test_symmetric_full_size_binaries_sampled(guess):
    s = ics.plummer_binaries(16384, seed=0)
    with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=guess):
        er, ev = _full_size_sample(s, seed=2)
    assert er <= TOL and ev <= TOL, (er, ev)


def test_symmetric_fp32_guess_full_size_bh_cluster_sampled():
    with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=sk.GUESS_FP32):
        er, ev = _full_size_sample(ics.bh_cluster(16384, seed=1), seed=4)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("blocks", [0, 1, 300])
def test_fp32_guess_plummer_1024_one_evaluation(blocks):
    # the single-precision root is within ~1e-7 of the FP64 root, so one
    # FP64 evaluation and the Taylor carry finish every pair
    s = ics.plummer(1024, seed=0)
    with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=sk.GUESS_FP32, grid_blocks=blocks):
        sk.get_stats(reset=True)
        r, v = gpu_step(s, s.dt, 2)
        st = sk.get_stats(reset=True)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)
    assert st["iters"] == st["solves"] and st["carries"] == st["solves"]


def test_fp32_guess_falls_back_for_reduced_periods():
    # tight binaries whose period is below the step: t is reduced modulo the
    # period in FP64, so those pairs use the second-order guess
    s = ics.plummer_binaries(2048, seed=5)
    s = ics.System(s.m, s.r, s.v, 2.0 ** -6, "binaries-long-step")
    with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=sk.GUESS_FP32):
        sk.get_stats(reset=True)
        r, v = gpu_step(s, s.dt, 2)
        st = sk.get_stats(reset=True)
    # the fallback lanes start from the second-order guess and need a second
    # FP64 evaluation before their carry
    assert st["iters"] > st["solves"]
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([[0, 1, 2, 3], rng.choice(s.n, 40, replace=False)]))
    rc, rs, vs = oracle.step_sample(s.m, s.r, s.v, s.dt, idx, 2, nthreads=NCPU)
    R = np.sqrt((r ** 2).sum(1).mean())
    V = np.sqrt((v ** 2).sum(1).mean())
    er = np.linalg.norm(r[idx] - rs, axis=1) / np.maximum(np.linalg.norm(rs, axis=1), R)
    ev = np.linalg.norm(v[idx] - vs, axis=1) / np.maximum(np.linalg.norm(vs, axis=1), V)
    assert er.max() <= TOL and ev.max() <= TOL, (er.max(), ev.max())


def test_symmetric_counts_solves():
    n = 100  # blocks of 32, 32, 32, 4
    s = ics.random_cluster(n, seed=9)
    with configured(pair_mode=sk.PAIRS_SYMMETRIC):
        sk.get_stats(reset=True)
        gpu_step(s, s.dt, 2)
        st = sk.get_stats(reset=True)
    diag = 3 * 32 * 31 + 4 * 3
    assert st["pairs"] == n * (n - 1)
    assert st["solves"] == (n * (n - 1) - diag) // 2 + diag


def test_headline_evolve_32_steps_matches_oracle_and_single_steps():
    # the call path the benchmark times: one sakura_evolve call of 32 steps
    # (symmetric tiles, single-precision seed; each apply kernel drifts for
    # the next step), against 32 oracle steps (held to 32 x the per-step
    # bound) and bit for bit against 32 separate sakura_step calls
    s = ics.plummer(1024, seed=0)
    with configured(guess=sk.GUESS_FP32, pair_mode=sk.PAIRS_SYMMETRIC):
        st = dev(s.soa())
        m = dev(s.m)
        sk.evolve(st, m, s.dt, 2, 32)
        sk.check()
        r, v = ics.from_soa(st.cpu().numpy())
        st1 = dev(s.soa())
        for _ in range(32):
            sk.step(st1, m, s.dt, 2)
        sk.check()
        r1, v1 = ics.from_soa(st1.cpu().numpy())
    rc, rr, vr = oracle.evolve(s.m, s.r, s.v, s.dt, 32, 2, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r, v, rr, vr)
    print(f"evolve(32) vs oracle: r {er:.2e} v {ev:.2e}")
    assert er <= 32 * TOL and ev <= 32 * TOL
    np.testing.assert_array_equal(r, r1)
    np.testing.assert_array_equal(v, v1)


# --- the row-group kernel (the FP64 default from 4096 particles), forced on
# small systems ---

@pytest.mark.parametrize("guess", [sk.GUESS_STANDARD, sk.GUESS_TAYLOR, sk.GUESS_FP32])
@pytest.mark.parametrize("order", [2, 1, -1])
@pytest.mark.parametrize("name,s", SMALL, ids=[n for n, _ in SMALL])
def test_row_group_step_matches_oracle(name, s, order, guess):
    with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=guess,
                    flags=sk.FLAG_STATS | sk.FLAG_GROUPS | sk.FLAG_NO_SMALL):
        r, v = gpu_step(s, s.dt, order)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("blocks", [0, 1, 3, 7, 143, 144, 5000])
def test_row_group_grid_shapes_agree_with_oracle(blocks):
    # any grid: a block's range of phase-steps may start or end inside a
    # group or inside a phase (7 or 143 blocks over 144 phases), a group's row
    # sums then come in several pieces and a split phase's column sums in two
    # or more slots (1024 particles: 8 groups, 144 phases; 5000 blocks are
    # clamped to one phase each)
    s = ics.plummer(1024, seed=0)
    with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=sk.GUESS_FP32, grid_blocks=blocks,
                    flags=sk.FLAG_STATS | sk.FLAG_GROUPS):
        sk.get_stats(reset=True)
        r, v = gpu_step(s, s.dt, 2)
        st = sk.get_stats(reset=True)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)
    assert st["carries"] == st["solves"]
    assert st["group_launches"] == 1


def test_row_group_and_tile_kernels_agree_and_are_deterministic():
    # the two symmetric kernels differ only in summation order; each repeats
    # its own result bit for bit
    s = ics.random_cluster(3001, seed=4, mass_spread=2.0)
    out = {}
    for name, flag in (("tiles", sk.FLAG_TILES), ("groups", sk.FLAG_GROUPS)):
        with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=sk.GUESS_FP32,
                        flags=sk.FLAG_STATS | flag):
            sk.get_stats(reset=True)
            out[name] = gpu_step(s, s.dt, 2)
            again = gpu_step(s, s.dt, 2)
            assert sk.get_stats(reset=True)["group_launches"] == (2 if name == "groups" else 0)
        np.testing.assert_array_equal(out[name][0], again[0])
        np.testing.assert_array_equal(out[name][1], again[1])
    er, ev = rel_err(*out["groups"], *out["tiles"])
    assert er <= TOL and ev <= TOL, (er, ev)


@pytest.mark.parametrize("n,groups", [(4095, False), (4096, True)])
def test_default_fp64_kernel_choice_by_size(n, groups):
    # without a flag the symmetric FP64 step runs on tiles below 4096 bodies
    # and in row groups from there; either way within the oracle's tolerance
    # on a sample of rows
    s = ics.plummer(n, seed=3)
    with configured(pair_mode=sk.PAIRS_SYMMETRIC, guess=sk.GUESS_FP32):
        sk.get_stats(reset=True)
        r, v = gpu_step(s, s.dt, 2)
        assert (sk.get_stats(reset=True)["group_launches"] == 1) == groups
    rows = np.arange(0, n, 97)
    rc, rr, vr = oracle.step_sample(s.m, s.r, s.v, s.dt, rows, 2, nthreads=NCPU)
    assert rc == oracle.OK
    er, ev = rel_err(r[rows], v[rows], rr, vr)
    assert er <= TOL and ev <= TOL, (er, ev)


def test_row_group_evolve_matches_single_steps():
    # calls of several steps: each apply kernel drifts for the next step, and
    # the next row-group pair kernel starts only after it completes
    s = ics.plummer(2048, seed=1)
    with configured(guess=sk.GUESS_FP32, pair_mode=sk.PAIRS_SYMMETRIC,
                    flags=sk.FLAG_STATS | sk.FLAG_GROUPS):
        st = dev(s.soa())
        m = dev(s.m)
        sk.evolve(st, m, s.dt, 2, 8)
        st1 = dev(s.soa())
        for _ in range(8):
            sk.step(st1, m, s.dt, 2)
        sk.check()
        np.testing.assert_array_equal(st.cpu().numpy(), st1.cpu().numpy())
    rc, rr, vr = oracle.evolve(s.m, s.r, s.v, s.dt, 8, 2, nthreads=NCPU)
    r, v = ics.from_soa(st.cpu().numpy())
    er, ev = rel_err(r, v, rr, vr)
    assert er <= 8 * TOL and ev <= 8 * TOL, (er, ev)
