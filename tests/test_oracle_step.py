"""Pins for the oracle's whole step (Eqs. 23-27, the paper's listing).

Expected values come from outside the oracle:
  * N = 2: the method reduces to the exact Kepler flow plus a centre-of-mass
    drift (Sec. 3.1: "accurate to machine precision"), compared with the
    classical-anomaly solution in mpmath;
  * the Eq. 28 limit: with a drift-kick-drift pair solver the step must equal
    an independently written DKD leapfrog;
  * momentum and centre-of-mass invariants (antisymmetry of the increments);
  * second-order convergence against scipy's DOP853 at tight tolerance;
  * time symmetry: exact for N = 2 and for the Eq. 28 limit, O(tau^4) for
    N > 2 (non-commuting pair maps, Eq. 21);
  * qualitative: planetary energy error far below leapfrog's (Sec. 3.1);
  * orders 4, 6, 8 (triple-jump compositions, Sec. 2.2): exact for N = 2;
    fourth and sixth order in the Eq. 28 limit, where the base map is an
    exactly symmetric leapfrog; third order with Kepler pair maps for N > 2,
    whose time-symmetry defect is O(tau^4).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1402_3325_gb300 import ics


def _binary():
    m = np.array([0.7, 0.3])
    r = np.array([[0.4, 0.1, 0.0], [-0.5, 0.2, 0.1]])
    v = np.array([[0.1, 0.6, 0.0], [-0.2, -0.9, 0.1]])
    return m, r, v


@pytest.mark.parametrize("order", [2, 1, -1])
@pytest.mark.parametrize("tau", [0.37, -0.2, 3.9])
def test_two_body_step_is_exact(order, tau):
    pytest.importorskip("mpmath")
    from classical_kepler import kepler_classical_f64
    m, r, v = _binary()
    rc, r1, v1 = oracle.step(m, r, v, tau, order)
    assert rc == oracle.OK
    M = m.sum()
    R = (m[:, None] * r).sum(0) / M
    V = (m[:, None] * v).sum(0) / M
    rr, vv = kepler_classical_f64(tau, M, r[0] - r[1], v[0] - v[1])
    rr, vv = np.array(rr), np.array(vv)
    exp_r = np.stack([R + tau * V + m[1] / M * rr, R + tau * V - m[0] / M * rr])
    exp_v = np.stack([V + m[1] / M * vv, V - m[0] / M * vv])
    assert np.abs(r1 - exp_r).max() <= 1e-14 * max(1.0, abs(tau))
    assert np.abs(v1 - exp_v).max() <= 1e-14


def test_circular_binary_returns_after_one_period():
    m = np.array([0.6, 0.4])
    a = 1.0
    vrel = math.sqrt(1.0 / a)
    r = np.array([[0.4 * a, 0, 0], [-0.6 * a, 0, 0]])
    v = np.array([[0, 0.4 * vrel, 0], [0, -0.6 * vrel, 0]])
    P = 2 * math.pi * math.sqrt(a ** 3 / 1.0)
    rc, r1, v1 = oracle.evolve(m, r, v, P / 50, 50)
    assert rc == oracle.OK
    np.testing.assert_allclose(r1, r, atol=1e-13)
    np.testing.assert_allclose(v1, v, atol=1e-13)


def _leapfrog_dkd(m, r, v, tau):
    """Independent drift-kick-drift leapfrog on the full system."""
    rh = r + 0.5 * tau * v
    d = rh[:, None, :] - rh[None, :, :]
    dist = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(dist, np.inf)
    a = -(m[None, :, None] * d / dist[:, :, None] ** 3).sum(1)
    vn = v + tau * a
    return rh + 0.5 * tau * vn, vn


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_eq28_dkd_limit_is_leapfrog(seed):
    s = ics.random_cluster(9, seed=seed, mass_spread=3.0)
    tau = 0.01
    rc, r1, v1 = oracle.step(s.m, s.r, s.v, tau, 2, pair_solver=oracle.PAIR_DKD)
    assert rc == oracle.OK
    rl, vl = _leapfrog_dkd(s.m, s.r, s.v, tau)
    vs = np.abs(s.v).max()
    assert np.abs(r1 - rl).max() <= 1e-14 * np.abs(s.r).max()
    assert np.abs(v1 - vl).max() <= 1e-13 * vs


def test_eq28_limit_is_exactly_time_reversible():
    s = ics.random_cluster(6, seed=11)
    rc, r1, v1 = oracle.step(s.m, s.r, s.v, 0.02, 2, pair_solver=oracle.PAIR_DKD)
    rc, r2, v2 = oracle.step(s.m, r1, v1, -0.02, 2, pair_solver=oracle.PAIR_DKD)
    assert np.abs(r2 - s.r).max() <= 1e-14 * np.abs(s.r).max()
    assert np.abs(v2 - s.v).max() <= 1e-13 * np.abs(s.v).max()


@pytest.mark.parametrize("order", [2, 1, -1])
def test_momentum_and_centre_of_mass(order):
    s = ics.random_cluster(12, seed=4, mass_spread=2.0)
    tau = 1.0 / 64
    P0 = (s.m[:, None] * s.v).sum(0)
    C0 = (s.m[:, None] * s.r).sum(0)
    rc, r, v = oracle.evolve(s.m, s.r, s.v, tau, 8, order)
    assert rc == oracle.OK
    P1 = (s.m[:, None] * v).sum(0)
    C1 = (s.m[:, None] * r).sum(0)
    pscale = (s.m[:, None] * np.abs(s.v)).sum()
    assert np.abs(P1 - P0).max() <= 1e-14 * pscale
    assert np.abs(C1 - (C0 + 8 * tau * P0)).max() <= 1e-13 * (s.m[:, None] * np.abs(s.r)).sum()


def test_time_symmetry_two_body_roundoff():
    m, r, v = _binary()
    rc, r1, v1 = oracle.step(m, r, v, 0.3, 2)
    rc, r2, v2 = oracle.step(m, r1, v1, -0.3, 2)
    assert np.abs(r2 - r).max() <= 1e-14
    assert np.abs(v2 - v).max() <= 1e-14


def test_time_symmetry_residual_shrinks_fast_for_many_bodies():
    # Psi(-tau) o Psi(tau) = id only up to the non-commutativity of the pair
    # maps; the residual must fall at least like tau^3 (measured: tau^4)
    s = ics.random_cluster(8, seed=5)
    res = []
    for tau in (1 / 32, 1 / 64, 1 / 128):
        rc, r1, v1 = oracle.step(s.m, s.r, s.v, tau, 2)
        rc, r2, v2 = oracle.step(s.m, r1, v1, -tau, 2)
        res.append(max(np.abs(r2 - s.r).max(), np.abs(v2 - s.v).max()))
    assert res[0] / res[1] > 12 and res[1] / res[2] > 12
    assert res[2] < 1e-9


def _rhs(t, y, m):
    n = len(m)
    r = y[:3 * n].reshape(n, 3)
    v = y[3 * n:].reshape(n, 3)
    d = r[:, None, :] - r[None, :, :]
    dist = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(dist, np.inf)
    a = -(m[None, :, None] * d / dist[:, :, None] ** 3).sum(1)
    return np.concatenate([v.ravel(), a.ravel()])


def _reference(m, r, v, T):
    from scipy.integrate import solve_ivp
    y0 = np.concatenate([r.ravel(), v.ravel()])
    sol = solve_ivp(_rhs, (0, T), y0, method="DOP853", rtol=3e-14, atol=1e-16, args=(m,))
    n = len(m)
    return sol.y[:3 * n, -1].reshape(n, 3)


def test_second_order_convergence_planetary():
    s = ics.planetary(0)
    T = s.dt * 400
    rref = _reference(s.m, s.r, s.v, T)
    errs = []
    for f in (2, 4, 8):
        tau = s.dt * 4 / f
        rc, r1, _ = oracle.evolve(s.m, s.r, s.v, tau, int(round(T / tau)))
        assert rc == oracle.OK
        errs.append(np.abs(r1 - rref).max())
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5


def test_second_order_convergence_hierarchical_triple():
    m = np.array([0.5, 0.4, 0.1])
    r = np.array([[0.05, 0, 0], [-0.0625, 0, 0], [1.5, 0.3, 0]])
    vin = math.sqrt(0.9 / 0.1125)
    v = np.array([[0, 0.4 * vin / 0.9, 0], [0, -0.5 * vin / 0.9, 0], [0, 0.75, 0.05]])
    rref = _reference(m, r, v, 1.0)
    errs = []
    for k in (6, 7, 8):
        tau = 2.0 ** -k
        rc, r1, _ = oracle.evolve(m, r, v, tau, 2 ** k)
        errs.append(np.abs(r1 - rref).max())
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 8.0


def test_planetary_energy_far_better_than_leapfrog():
    # Sec. 3.1: for a planetary system the method conserves energy far better
    # than leapfrog at the same step; compare the largest error over two inner
    # orbits (leapfrog's error is periodic, so a single sample can mislead)
    s = ics.planetary(1)
    E0 = oracle.energy(s.m, s.r, s.v)[0]
    r, v = s.r, s.v
    rl, vl = s.r.copy(), s.v.copy()
    worst_s = worst_l = 0.0
    for _ in range(400):
        rc, r, v = oracle.step(s.m, r, v, s.dt, 2)
        assert rc == oracle.OK
        rl, vl = _leapfrog_dkd(s.m, rl, vl, s.dt)
        worst_s = max(worst_s, abs(oracle.energy(s.m, r, v)[0] / E0 - 1))
        worst_l = max(worst_l, abs(oracle.energy(s.m, rl, vl)[0] / E0 - 1))
    assert worst_s < worst_l / 30


@pytest.mark.parametrize("order", [4, 6, 8])
@pytest.mark.parametrize("tau", [0.37, -0.2, 3.9])
def test_composed_two_body_step_is_exact(order, tau):
    # every second-order sub-step is the exact two-body flow for N = 2, so the
    # composition is exact too if and only if its time weights sum to one
    pytest.importorskip("mpmath")
    from classical_kepler import kepler_classical_f64
    m, r, v = _binary()
    rc, r1, v1 = oracle.step(m, r, v, tau, order)
    assert rc == oracle.OK
    M = m.sum()
    R = (m[:, None] * r).sum(0) / M
    V = (m[:, None] * v).sum(0) / M
    rr, vv = kepler_classical_f64(tau, M, r[0] - r[1], v[0] - v[1])
    rr, vv = np.array(rr), np.array(vv)
    exp_r = np.stack([R + tau * V + m[1] / M * rr, R + tau * V - m[0] / M * rr])
    exp_v = np.stack([V + m[1] / M * vv, V - m[0] / M * vv])
    assert np.abs(r1 - exp_r).max() <= 2e-14 * max(1.0, abs(tau)) * (order - 1)
    assert np.abs(v1 - exp_v).max() <= 2e-14 * (order - 1)


def _triple():
    m = np.array([0.5, 0.4, 0.1])
    r = np.array([[0.05, 0, 0], [-0.0625, 0, 0], [1.5, 0.3, 0]])
    vin = math.sqrt(0.9 / 0.1125)
    v = np.array([[0, 0.4 * vin / 0.9, 0], [0, -0.5 * vin / 0.9, 0], [0, 0.75, 0.05]])
    return m, r, v


def _convergence(order, ks, pair_solver=oracle.PAIR_KEPLER):
    m, r, v = _triple()
    rref = _reference(m, r, v, 1.0)
    errs = []
    for k in ks:
        rc, r1, _ = oracle.evolve(m, r, v, 2.0 ** -k, 2 ** k, order, pair_solver=pair_solver)
        assert rc == oracle.OK
        errs.append(np.abs(r1 - rref).max())
    return [a / b for a, b in zip(errs, errs[1:])]


def test_composition_orders_in_the_symmetric_dkd_limit():
    # in the Eq. 28 limit the second-order map is the DKD leapfrog, which is
    # exactly time-symmetric: the triple jump must then give order 4 and 6
    # (error ratios 16 and 64 per halving), which pins its weights
    q4 = _convergence(4, (6, 7, 8), oracle.PAIR_DKD)
    assert 11 < q4[0] < 20 and 13 < q4[1] < 19, q4
    q6 = _convergence(6, (6, 7, 8), oracle.PAIR_DKD)
    assert q6[0] > 30 and q6[1] > 45, q6


def test_composition_of_kepler_pair_maps_is_third_order():
    # with Kepler pair maps the second-order step is time-symmetric only up
    # to O(tau^4) for N > 2 (pair maps computed from one state do not
    # commute, Eq. 21), and the triple jump cancels odd-order terms only:
    # the composed step is third order (ratio 8), not fourth
    q4 = _convergence(4, (6, 7, 8))
    assert 7.0 < q4[0] < 9.0 and 7.0 < q4[1] < 9.0, q4


def test_fast_swarm_step_is_nearly_free_motion():
    # stars of mass 1e-6 within 5e-4 of each other at speeds ~400: every
    # pair is a fast flyby whose deflection is tiny (tan(theta/2) = m / (b v^2)),
    # and for most pairs the standard guess lies far past the root; the step
    # must stay close to straight-line motion and conserve momentum
    rng = np.random.default_rng(0)
    n = 64
    m = np.full(n, 1e-6)
    r = rng.uniform(-2.5e-4, 2.5e-4, (n, 3))
    v = rng.normal(0.0, 300.0, (n, 3))
    rc, r1, v1 = oracle.step(m, r, v, 1e-3, 2)
    assert rc == oracle.OK
    assert np.abs(r1 - (r + 1e-3 * v)).max() < 1e-5
    assert np.abs(v1 - v).max() < 1e-1
    assert np.abs((m[:, None] * (v1 - v)).sum(0)).max() < 1e-15


def test_step_argument_errors():
    m, r, v = _binary()
    assert oracle.step(m, r, v, 0.1, 3)[0] == oracle.E_ARG
    assert oracle.step(m, r, v, 0.1, 5)[0] == oracle.E_ARG
    assert oracle.step(m, r, v, 0.1, 10)[0] == oracle.E_ARG
    assert oracle.step(np.array([1.0, 0.0]), r, v, 0.1, 2)[0] == oracle.E_MASS
    rn = r.copy()
    rn[0, 0] = np.nan
    assert oracle.step(m, rn, v, 0.1, 2)[0] == oracle.E_NONFINITE
    rc = oracle.step(m, np.zeros((2, 3)), v, 0.1, 2)[0]
    assert rc == oracle.E_COINCIDENT


def test_threads_do_not_change_bits():
    s = ics.plummer(64, seed=2)
    _, r1, v1 = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=1)
    _, r4, v4 = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=4)
    np.testing.assert_array_equal(r1, r4)
    np.testing.assert_array_equal(v1, v4)


@pytest.mark.parametrize("order", [2, 1, -1])
def test_step_sample_equals_full_step(order):
    s = ics.random_cluster(40, seed=8, mass_spread=2.0)
    idx = np.array([0, 7, 39, 13])
    _, r1, v1 = oracle.step(s.m, s.r, s.v, 1 / 64, order)
    rc, rs, vs = oracle.step_sample(s.m, s.r, s.v, 1 / 64, idx, order)
    assert rc == oracle.OK
    np.testing.assert_array_equal(rs, r1[idx])
    np.testing.assert_array_equal(vs, v1[idx])
