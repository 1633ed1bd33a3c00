"""Pins for the oracle's energy (Eqs. 1-3) and mixed-precision pair classes."""
import math

import numpy as np
import pytest

import oracle
from paper_1402_3325_gb300 import ics


def test_energy_matches_high_precision_sum():
    mp = pytest.importorskip("mpmath")
    s = ics.random_cluster(25, seed=7, mass_spread=4.0)
    E, T, U, rc = oracle.energy(s.m, s.r, s.v)
    assert rc == oracle.OK
    with mp.workdps(50):
        Tm = sum(mp.mpf(s.m[i]) / 2 * sum(mp.mpf(x) ** 2 for x in s.v[i]) for i in range(s.n))
        Um = mp.mpf(0)
        for i in range(s.n):
            for j in range(i + 1, s.n):
                d = mp.sqrt(sum((mp.mpf(s.r[i, q]) - mp.mpf(s.r[j, q])) ** 2 for q in range(3)))
                Um -= mp.mpf(s.m[i]) * mp.mpf(s.m[j]) / d
        Em = float(Tm + Um)
        Tm, Um = float(Tm), float(Um)
    assert abs(T - Tm) <= 4e-16 * abs(Tm)
    assert abs(U - Um) <= 4e-16 * abs(Um)
    assert abs(E - Em) <= 1e-15 * (abs(Tm) + abs(Um))


def test_two_body_energy_closed_form():
    m = np.array([2.0, 3.0])
    r = np.array([[0.0, 0, 0], [4.0, 0, 0]])
    v = np.array([[1.0, 0, 0], [0, 2.0, 0]])
    E, T, U, rc = oracle.energy(m, r, v)
    assert T == pytest.approx(0.5 * 2 * 1 + 0.5 * 3 * 4, rel=1e-16)
    assert U == pytest.approx(-2.0 * 3.0 / 4.0, rel=1e-16)
    assert E == pytest.approx(7.0 - 1.5, rel=1e-16)


def test_plummer_generator_is_virial():
    s = ics.plummer(256, seed=3)
    E, T, U, _ = oracle.energy(s.m, s.r, s.v)
    assert T == pytest.approx(0.25, rel=1e-12)
    assert U == pytest.approx(-0.5, rel=1e-12)
    assert E == pytest.approx(-0.25, rel=1e-12)


def _pair_from_elements(m, a, e, r_sep_scale=1.0):
    # a single pair with known eccentricity; relative orbit about m
    if e < 1:
        rr, vv = ics.elements_to_cartesian(np.array([m]), np.array([a]), np.array([e]),
                                           np.array([0.3]), np.array([0.2]),
                                           np.array([0.1]), np.array([1.0]))
    else:
        # hyperbolic: pericentre q with speed sqrt(m (1+e)/q)
        q = a
        rr = np.array([[q, 0.0, 0.0]])
        vv = np.array([[0.0, math.sqrt(m * (1 + e) / q), 0.0]])
    masses = np.array([m / 2, m / 2])
    r = np.stack([0.5 * rr[0], -0.5 * rr[0]])
    v = np.stack([0.5 * vv[0], -0.5 * vv[0]])
    return masses, r, v


@pytest.mark.parametrize("a,e,rule,expect", [
    (1.0, 0.05, 0, 1),     # wide, near-circular: single precision
    (1.0, 0.95, 0, 0),     # high eccentricity: double
    (0.02, 0.1, 0, 0),     # close pair: double
    (0.5, 30.0, 0, 0),     # strong hyperbola, literal rule: double
    (0.5, 30.0, 1, 1),     # strong hyperbola, e_hyp rule: single
    (0.5, 3.0, 1, 0),      # moderate hyperbola: double under both
])
def test_pair_class_rule(a, e, rule, expect):
    m, r, v = _pair_from_elements(1.0, a, e)
    cnt, mat = oracle.pair_classes(m, r, v, 0.0, rule=rule, want_matrix=True)
    assert cnt == 2 * expect
    assert mat[0, 1] == expect and mat[1, 0] == expect and mat[0, 0] == 0


def test_pair_class_counts_bh_cluster_literal_rule():
    # with the literal rule only black-hole/star pairs beyond 0.1 qualify
    s = ics.bh_cluster(200, seed=1)
    cnt, mat = oracle.pair_classes(s.m, s.r, s.v, s.dt, rule=0, want_matrix=True)
    d = np.linalg.norm(s.r - s.r[0], axis=1)
    far = int((d[1:] > 0.1).sum())
    assert cnt == 2 * far
    assert mat[1:, 1:].sum() == 0


@pytest.mark.parametrize("a,e", [(1.0, 0.05), (1.0, 0.95), (0.5, 30.0), (0.02, 3.0)])
def test_pair_class_values_are_the_elements(a, e):
    # the pair's r^2 and e^2 as the rule defines them, for a pair built from
    # known elements (tau = 0: the Kepler input is the pair's separation)
    m, r, v = _pair_from_elements(1.0, a, e)
    cnt, mat, r2, e2 = oracle.pair_classes(m, r, v, 0.0, want_values=True)
    sep2 = float(((r[0] - r[1]) ** 2).sum())
    assert r2[0, 1] == pytest.approx(sep2, rel=1e-15) and r2[1, 0] == r2[0, 1]
    assert e2[0, 1] == pytest.approx(e * e, rel=1e-12)
    assert r2[0, 0] == 0.0 and e2[1, 1] == 0.0


@pytest.mark.parametrize("order", [2, 1, -1])
def test_pair_class_input_is_the_undrifted_separation(order):
    # the first drift (Eq. 27a) and the backward drift of Eq. 17 cancel in the
    # pair's Kepler input for every order: r0 = r_i - r_j, v0 = v_i - v_j of
    # the state before the step, so r^2 and e^2 do not depend on tau
    s = ics.random_cluster(40, seed=3, mass_spread=3.0)
    c0, m0, r20, e20 = oracle.pair_classes(s.m, s.r, s.v, 0.0, rule=1, want_values=True)
    c1, m1, r21, e21 = oracle.pair_classes(s.m, s.r, s.v, 0.37, rule=1, order=order,
                                           want_values=True)
    off = ~np.eye(s.n, dtype=bool)
    np.testing.assert_allclose(r21[off], r20[off], rtol=1e-13)
    np.testing.assert_allclose(e21[off], e20[off], rtol=1e-10, atol=1e-12)
    d = s.r[:, None, :] - s.r[None, :, :]
    np.testing.assert_allclose(r20[off], (d ** 2).sum(-1)[off], rtol=1e-15)
