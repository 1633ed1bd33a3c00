"""The seeded synthetic inputs (paper_1402_3325_gb300/ics.py) have the
properties that the input recipe states: determinism by seed, masses,
centre-of-mass frames, virial energies, orbital elements and step sizes.
Energies are checked against the oracle's own energy (a separate
implementation), orbits by recovering their elements from the positions and
velocities."""
import math

import numpy as np
import pytest

import oracle
from paper_1402_3325_gb300 import ics


def com(s):
    M = s.m.sum()
    return (s.m[:, None] * s.r).sum(0) / M, (s.m[:, None] * s.v).sum(0) / M


def two_body_elements(mu, r, v):
    """Semi-major axis and eccentricity of relative orbits r, v [k, 3]."""
    rn = np.linalg.norm(r, axis=1)
    v2 = (v * v).sum(1)
    a = 1.0 / (2.0 / rn - v2 / mu)
    h = np.cross(r, v)
    evec = np.cross(v, h) / mu[:, None] - r / rn[:, None]
    return a, np.linalg.norm(evec, axis=1)


GENS = [lambda seed: ics.plummer(256, seed), lambda seed: ics.planetary(seed),
        lambda seed: ics.bh_cluster(256, seed), lambda seed: ics.plummer_binaries(256, seed),
        lambda seed: ics.random_cluster(40, seed, mass_spread=2.0)]


@pytest.mark.parametrize("gen", GENS, ids=["plummer", "planetary", "bh", "binaries", "random"])
def test_generators_are_determined_by_their_seed(gen):
    a, b, c = gen(3), gen(3), gen(4)
    for x, y in ((a.m, b.m), (a.r, b.r), (a.v, b.v)):
        np.testing.assert_array_equal(x, y)
    assert a.dt == b.dt and not np.array_equal(a.r, c.r)


@pytest.mark.parametrize("gen", GENS, ids=["plummer", "planetary", "bh", "binaries", "random"])
def test_generators_are_in_their_centre_of_mass_frame(gen):
    s = gen(1)
    R = np.sqrt((s.r ** 2).sum(1).mean())
    V = np.sqrt((s.v ** 2).sum(1).mean())
    rc, vc = com(s)
    assert np.abs(rc).max() <= 1e-14 * R and np.abs(vc).max() <= 1e-14 * V


def test_plummer_is_equal_mass_and_virial_with_energy_minus_a_quarter():
    s = ics.plummer(1024, seed=0)
    assert s.n == 1024 and np.all(s.m == 1.0 / 1024) and s.dt == 2.0 ** -8
    E, T, U, rc = oracle.energy(s.m, s.r, s.v)
    assert rc == oracle.OK
    assert abs(T - 0.25) <= 1e-13 and abs(U + 0.5) <= 1e-13 and abs(E + 0.25) <= 1e-13


def test_planetary_masses_orbits_and_step():
    for seed in range(4):
        s = ics.planetary(seed)
        assert s.n == 9 and s.m[0] == 1.0
        assert np.all((s.m[1:] >= 1e-5) & (s.m[1:] <= 1e-3))
        mu = 1.0 + s.m[1:]
        a, e = two_body_elements(mu, s.r[1:] - s.r[0], s.v[1:] - s.v[0])
        assert np.all((a >= 1.0 - 1e-9) & (a <= 30.0 + 1e-9)) and np.all(e <= 0.1 + 1e-9)
        inc = np.degrees(np.arccos(np.cross(s.r[1:] - s.r[0], s.v[1:] - s.v[0])[:, 2] /
                                   np.linalg.norm(np.cross(s.r[1:] - s.r[0],
                                                           s.v[1:] - s.v[0]), axis=1)))
        assert np.all(inc <= 2.0 + 1e-9)
        q = int(np.argmin(a))
        P_in = 2 * math.pi * math.sqrt(a[q] ** 3 / mu[q])
        assert abs(s.dt * 200 / P_in - 1.0) <= 1e-9


def test_bh_cluster_stars_circle_the_black_hole():
    s = ics.bh_cluster(2048, seed=0)
    assert s.m[0] == 1.0 and abs(s.m[1:].sum() - 1e-2) <= 1e-15 and s.dt == 2.0 ** -10
    dr, dv = s.r[1:] - s.r[0], s.v[1:] - s.v[0]
    rn, vn = np.linalg.norm(dr, axis=1), np.linalg.norm(dv, axis=1)
    assert np.abs((dr * dv).sum(1) / (rn * vn)).max() <= 1e-12  # perpendicular
    Menc = 1.0 + 1e-2 * rn ** 3 / (rn ** 2 + 1.0) ** 1.5
    np.testing.assert_allclose(vn, np.sqrt(Menc / rn), rtol=1e-12)


def test_plummer_binaries_have_the_stated_fraction_and_orbits():
    n = 512
    s = ics.plummer_binaries(n, seed=0)
    nb = int(round(0.1 * n)) // 2
    assert np.all(s.m == 1.0 / n) and s.dt == 2.0 ** -10
    # the members of a binary are each other's nearest neighbour and bound,
    # with a in [1e-4, 1e-2] and e < 1
    d = np.linalg.norm(s.r[:, None] - s.r[None], axis=2)
    np.fill_diagonal(d, np.inf)
    nn = d.argmin(1)
    pairs = [(i, j) for i, j in enumerate(nn) if nn[j] == i and i < j]
    i, j = np.array(pairs).T
    a, e = two_body_elements(s.m[i] + s.m[j], s.r[i] - s.r[j], s.v[i] - s.v[j])
    bound = (a > 0) & (a >= 1e-4 * (1 - 1e-9)) & (a <= 1e-2 * (1 + 1e-9)) & (e < 1.0)
    assert int(bound.sum()) == nb


def test_hierarchical_double_binary_geometry_and_step():
    s = ics.hierarchical_double_binary(ratio=100.0)
    assert s.n == 4 and np.all(s.m == 0.25)
    a, e = two_body_elements(np.array([0.5, 0.5]), s.r[[0, 2]] - s.r[[1, 3]],
                             s.v[[0, 2]] - s.v[[1, 3]])
    np.testing.assert_allclose(a, 0.01, rtol=1e-12)
    assert np.all(e <= 1e-12)
    P_out = 2 * math.pi * math.sqrt(1.0 / 1.0)
    assert abs(s.dt * 1000 / P_out - 1.0) <= 1e-14


def test_ensemble_packs_planetary_systems_by_their_own_seeds():
    ens = ics.ensemble(64, seed=5)
    sizes = ens.offsets[1:] - ens.offsets[:-1]
    assert ens.nsys == 64 and np.all((sizes >= 3) & (sizes <= 64))
    assert ens.offsets[0] == 0 and ens.state.shape == (6, ens.offsets[-1])
    for k in (0, 17, 63):
        s = ens.system(k)
        ref = ics.planetary(int(ens.seeds[k]), int(sizes[k]) - 1)
        np.testing.assert_array_equal(s.m, ref.m)
        np.testing.assert_array_equal(s.r, ref.r)
        np.testing.assert_array_equal(s.v, ref.v)
        assert s.dt == ref.dt > 0


def test_random_cluster_masses():
    s = ics.random_cluster(40, seed=2, mass_spread=2.0)
    assert abs(s.m.sum() - 1.0) <= 1e-15 and s.m.max() / s.m.min() <= 100.0
