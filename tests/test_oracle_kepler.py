"""Pins for the oracle's two-body Kepler flow (Eq. 18) and Stumpff functions.

Nothing here retypes the oracle's formulas: expected values come from the
classical-anomaly solution in mpmath (tests/golden/kepler_cases.json, written
by tests/golden/make_kepler_cases.py), closed forms (circular orbits, cos/sin),
conservation laws of the two-body problem, and time reversal.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kepler_cases.json")


def _load_cases():
    with open(GOLDEN) as fh:
        d = json.load(fh)
    out = []
    for c in d["cases"]:
        out.append(dict(name=c["name"], tau=float.fromhex(c["tau"]), m=float.fromhex(c["m"]),
                        r0=np.array([float.fromhex(x) for x in c["r0"]]),
                        v0=np.array([float.fromhex(x) for x in c["v0"]]),
                        r1=np.array([float(x) for x in c["r1"]]),
                        v1=np.array([float(x) for x in c["v1"]])))
    return out


CASES = _load_cases()


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_kepler_matches_classical_solution(case):
    r1, v1, it, rc = oracle.kepler(case["tau"], case["m"], case["r0"], case["v0"])
    assert rc == oracle.OK
    # multi-revolution cases lose a few ulp per revolution through the period
    tol = 1e-13 if "multirev" in case["name"] else 2e-14
    assert np.abs(r1 - case["r1"]).max() <= tol * np.abs(case["r1"]).max()
    assert np.abs(v1 - case["v1"]).max() <= tol * np.abs(case["v1"]).max()


@pytest.mark.parametrize("frac", [0.01, 0.25, 0.5, 0.9, 1.0, 2.75])
def test_circular_orbit_rotates_by_mean_motion(frac):
    m, a = 1.7, 0.6
    vc = math.sqrt(m / a)
    P = 2 * math.pi * math.sqrt(a ** 3 / m)
    t = frac * P
    th = 2 * math.pi * frac
    r1, v1, _, rc = oracle.kepler(t, m, [a, 0, 0], [0, vc, 0])
    assert rc == oracle.OK
    np.testing.assert_allclose(r1, [a * math.cos(th), a * math.sin(th), 0], atol=1e-14 * a)
    np.testing.assert_allclose(v1, [-vc * math.sin(th), vc * math.cos(th), 0], atol=1e-14 * vc)


def test_circular_orbit_returns_after_one_period_in_steps():
    # n steps with n*tau = P bring the orbit back to its start
    m, a = 1.0, 1.0
    P = 2 * math.pi
    r, v = np.array([a, 0, 0.0]), np.array([0, 1.0, 0])
    n = 64
    for _ in range(n):
        r, v, _, rc = oracle.kepler(P / n, m, r, v)
        assert rc == oracle.OK
    np.testing.assert_allclose(r, [a, 0, 0], atol=1e-13)
    np.testing.assert_allclose(v, [0, 1, 0], atol=1e-13)


def _invariants(m, r, v):
    rn = np.linalg.norm(r)
    en = 0.5 * v @ v - m / rn
    h = np.cross(r, v)
    lrl = np.cross(v, h) - m * r / rn
    return en, h, lrl


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_two_body_invariants_conserved(case):
    m = case["m"]
    r1, v1, _, rc = oracle.kepler(case["tau"], m, case["r0"], case["v0"])
    assert rc == oracle.OK
    e0, h0, a0 = _invariants(m, case["r0"], case["v0"])
    e1, h1, a1 = _invariants(m, r1, v1)
    # round-off of evaluating an invariant is relative to the magnitudes of
    # the state it is evaluated at: take the larger of the two states (a fast
    # flyby ends a thousand times farther out than it starts)
    r0n, v0n = np.linalg.norm(case["r0"]), np.linalg.norm(case["v0"])
    r1n, v1n = np.linalg.norm(r1), np.linalg.norm(v1)
    escale = max(0.5 * v0n ** 2 + m / r0n, 0.5 * v1n ** 2 + m / r1n)
    tol = 1e-12 if "multirev" in case["name"] or "parabolic" in case["name"] else 1e-13
    assert abs(e1 - e0) <= tol * escale
    hscale = max(r0n * v0n, r1n * v1n)
    assert np.abs(h1 - h0).max() <= tol * hscale
    assert np.abs(a1 - a0).max() <= tol * max(m, hscale * max(v0n, v1n))


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_time_reversal(case):
    m, t = case["m"], case["tau"]
    r1, v1, _, _ = oracle.kepler(t, m, case["r0"], case["v0"])
    r2, v2, _, rc = oracle.kepler(-t, m, r1, v1)
    assert rc == oracle.OK
    # the flyby passes through r = 0.01 at v = 15: its Jacobian amplifies
    # round-off by ~10^3 on the way back
    tol = 1e-12 if ("multirev" in case["name"] or "flyby" in case["name"]) else 1e-13
    # round-off is relative to the largest state the orbit passes through
    rs = max(np.abs(case["r0"]).max(), np.abs(r1).max())
    vs = max(np.abs(case["v0"]).max(), np.abs(v1).max())
    assert np.abs(r2 - case["r0"]).max() <= tol * rs
    assert np.abs(v2 - case["v0"]).max() <= tol * vs


def test_lagrange_determinant_is_one():
    # f gdot - fdot g = 1: recover f, g, fdot, gdot from two orthogonal-ish
    # solves of the same orbit with linearly independent (r0, v0) columns
    m, t = 1.3, 0.37
    r0, v0 = np.array([0.8, 0.1, 0.0]), np.array([-0.2, 1.1, 0.0])
    r1, v1, _, _ = oracle.kepler(t, m, r0, v0)
    A = np.stack([r0[:2], v0[:2]], 1)
    f, g = np.linalg.solve(A, r1[:2])
    fd, gd = np.linalg.solve(A, v1[:2])
    assert abs(f * gd - fd * g - 1.0) < 1e-13


@pytest.mark.parametrize("x", [-30.0, -1.5, -0.1000001, -0.09, -1e-3, 0.0, 1e-6, 0.05,
                               0.0999999, 0.1000001, 2.0, 9.5, 39.0])
def test_stumpff_against_closed_forms_and_identities(x):
    mp = pytest.importorskip("mpmath")
    c = oracle.stumpff(x)
    with mp.workdps(40):
        X = mp.mpf(x)
        if x > 0:
            z = mp.sqrt(X)
            ref = [mp.cos(z), mp.sin(z) / z, (1 - mp.cos(z)) / X, (z - mp.sin(z)) / (X * z)]
        elif x < 0:
            z = mp.sqrt(-X)
            ref = [mp.cosh(z), mp.sinh(z) / z, (mp.cosh(z) - 1) / -X,
                   (mp.sinh(z) - z) / (-X * z)]
        else:
            ref = [mp.mpf(1), mp.mpf(1), mp.mpf(1) / 2, mp.mpf(1) / 6]
        ref = [float(q) for q in ref]
    for k in range(4):
        assert abs(c[k] - ref[k]) <= 2e-14 * max(1.0, abs(ref[k])), (k, c[k], ref[k])
    # c0 = 1 - x c2 and c1 = 1 - x c3
    assert abs(c[0] - (1 - x * c[2])) <= 1e-14 * max(1.0, abs(c[0]))
    assert abs(c[1] - (1 - x * c[3])) <= 1e-14 * max(1.0, abs(c[1]))


def test_kepler_failure_reported_without_bisection():
    # a strong flyby needs many Laguerre steps from the standard guess
    rc = oracle.kepler(0.05, 1.0, [0.01, 0.002, 0.0], [-1.0, 15.0, 0.5], max_iter=1,
                       use_bisection=False)[3]
    assert rc == oracle.E_KEPLER
    # with bisection enabled the same budget still converges
    r1, v1, _, rc = oracle.kepler(0.05, 1.0, [0.01, 0.002, 0.0], [-1.0, 15.0, 0.5],
                                  max_iter=1, use_bisection=True)
    assert rc == oracle.OK
    ref = [c for c in CASES if c["name"] == "hyperbolic-flyby"][0]
    assert np.abs(r1 - ref["r1"]).max() <= 1e-13 * np.abs(ref["r1"]).max()


def test_kepler_rejects_coincident_and_massless():
    assert oracle.kepler(0.1, 1.0, [0, 0, 0], [1, 0, 0])[3] == oracle.E_COINCIDENT
    assert oracle.kepler(0.1, 0.0, [1, 0, 0], [0, 1, 0])[3] == oracle.E_MASS


def test_zero_time_is_identity():
    r1, v1, _, rc = oracle.kepler(0.0, 1.0, [0.3, 0.4, 0.5], [0.1, 0.2, 0.3])
    assert rc == oracle.OK
    np.testing.assert_array_equal(r1, [0.3, 0.4, 0.5])
    np.testing.assert_array_equal(v1, [0.1, 0.2, 0.3])
