"""Seeded synthetic initial conditions for the Sakura workloads.

These generators build the inputs that both the CUDA library and the CPU
oracle consume; they contain none of the integrator's arithmetic.  Every
generator is deterministic for a given seed (numpy PCG64).  Units are N-body
units, G = 1.  Arrays are returned in the listing layout: ``m[n]``,
``r[n][3]``, ``v[n][3]`` (float64); ``to_soa`` packs them into the library's
structure-of-arrays state ``[6][n]`` = rows x, y, z, vx, vy, vz.

Workload classes follow the paper's tests (Sec. 3): a planetary system, a
Plummer sphere, a cluster dominated by a central black hole, a cluster with
primordial binaries, and (for the batched form) ensembles of small planetary
systems.  The published initial-condition files are not available, so these
seeded generators stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class System:
    m: np.ndarray          # [n] masses
    r: np.ndarray          # [n, 3] positions
    v: np.ndarray          # [n, 3] velocities
    dt: float              # suggested constant time step
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.m.shape[0])

    def soa(self) -> np.ndarray:
        return to_soa(self.r, self.v)


def to_soa(r: np.ndarray, v: np.ndarray) -> np.ndarray:
    """[n,3] + [n,3] -> contiguous [6, n] (x, y, z, vx, vy, vz rows)."""
    return np.ascontiguousarray(np.concatenate([np.asarray(r).T, np.asarray(v).T], 0),
                                dtype=np.float64)


def from_soa(state: np.ndarray):
    """[6, n] -> ([n,3] positions, [n,3] velocities)."""
    state = np.asarray(state, dtype=np.float64)
    return np.ascontiguousarray(state[:3].T), np.ascontiguousarray(state[3:].T)


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def _isotropic(rng: np.random.Generator, k: int) -> np.ndarray:
    z = rng.uniform(-1.0, 1.0, k)
    phi = rng.uniform(0.0, 2.0 * math.pi, k)
    s = np.sqrt(1.0 - z * z)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], 1)


def _com_frame(m, r, v):
    M = m.sum()
    r = r - (m[:, None] * r).sum(0) / M
    v = v - (m[:, None] * v).sum(0) / M
    return r, v


def _eccentric_anomaly(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Solve E - e sin E = M (elliptic) by safeguarded Newton iteration."""
    M = np.mod(M, 2.0 * math.pi)
    E = np.where(e < 0.8, M, math.pi * np.ones_like(M))
    for _ in range(100):
        f = E - e * np.sin(E) - M
        E = E - f / (1.0 - e * np.cos(E))
    return E


def elements_to_cartesian(mu, a, e, inc, Omega, omega, Mean):
    """Classical orbital elements of bound orbits about gravitational
    parameter mu -> relative position and velocity [k, 3]."""
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), np.shape(a))
    E = _eccentric_anomaly(np.asarray(Mean, dtype=np.float64), np.asarray(e))
    cE, sE = np.cos(E), np.sin(E)
    b = np.sqrt(1.0 - e * e)
    x = a * (cE - e)
    y = a * b * sE
    nmot = np.sqrt(mu / a ** 3)
    den = 1.0 - e * cE
    vx = -a * nmot * sE / den
    vy = a * nmot * b * cE / den
    cO, sO = np.cos(Omega), np.sin(Omega)
    co, so = np.cos(omega), np.sin(omega)
    ci, si = np.cos(inc), np.sin(inc)
    # rotation R3(Omega) R1(i) R3(omega) applied to the perifocal frame
    P = np.stack([cO * co - sO * so * ci, sO * co + cO * so * ci, so * si], 1)
    Q = np.stack([-cO * so - sO * co * ci, -sO * so + cO * co * ci, co * si], 1)
    r = x[:, None] * P + y[:, None] * Q
    v = vx[:, None] * P + vy[:, None] * Q
    return r, v


def potential_energy(m: np.ndarray, r: np.ndarray, chunk: int = 2048) -> float:
    """Direct-summation potential energy, used only to put a sampled cluster
    into exact virial units before it is handed to either implementation."""
    n = m.shape[0]
    W = 0.0
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        d = r[a:b, None, :] - r[None, :, :]
        dist = np.sqrt((d * d).sum(-1))
        idx = np.arange(a, b)
        dist[idx - a, idx] = np.inf
        W += -0.5 * float((m[a:b, None] * m[None, :] / dist).sum())
    return W


def _plummer_positions(rng, k, rmax_frac=0.999):
    X = rng.uniform(0.0, rmax_frac, k)
    X = np.maximum(X, 1e-12)
    rad = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    return rad[:, None] * _isotropic(rng, k), rad


def _plummer_speeds(rng, rad):
    k = rad.shape[0]
    q = np.empty(k)
    todo = np.arange(k)
    while todo.size:
        x = rng.uniform(0.0, 1.0, todo.size)
        y = rng.uniform(0.0, 0.1, todo.size)
        ok = y < x * x * (1.0 - x * x) ** 3.5
        q[todo[ok]] = x[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (1.0 + rad * rad) ** (-0.25)
    return q * vesc


def _virialise(m, r, v):
    """Scale r and v so that T = 1/4 and W = -1/2 exactly (E = -1/4)."""
    W = potential_energy(m, r)
    T = 0.5 * float((m * (v * v).sum(1)).sum())
    r = r * (W / -0.5)
    v = v * math.sqrt(0.25 / T)
    return r, v


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def planetary(seed: int = 0, n_planets: int = 8, *, m_lo=1e-5, m_hi=1e-3, a_lo=1.0,
              a_hi=30.0, e_hi=0.1, inc_max_deg=2.0, steps_per_period=200) -> System:
    """Central mass 1 plus n_planets planets on independent heliocentric Kepler
    orbits (masses and semi-major axes log-uniform, e uniform, small random
    inclinations, random angles), moved to the centre-of-mass frame.
    dt = P_inner / steps_per_period."""
    rng = np.random.default_rng(seed)
    k = n_planets
    mp = np.exp(rng.uniform(math.log(m_lo), math.log(m_hi), k))
    a = np.exp(rng.uniform(math.log(a_lo), math.log(a_hi), k))
    e = rng.uniform(0.0, e_hi, k)
    inc = rng.uniform(0.0, math.radians(inc_max_deg), k)
    Om = rng.uniform(0.0, 2 * math.pi, k)
    om = rng.uniform(0.0, 2 * math.pi, k)
    Mn = rng.uniform(0.0, 2 * math.pi, k)
    rp, vp = elements_to_cartesian(1.0 + mp, a, e, inc, Om, om, Mn)
    m = np.concatenate([[1.0], mp])
    r = np.concatenate([np.zeros((1, 3)), rp])
    v = np.concatenate([np.zeros((1, 3)), vp])
    r, v = _com_frame(m, r, v)
    q = int(np.argmin(a))
    P_in = 2 * math.pi * math.sqrt(a[q] ** 3 / (1.0 + mp[q]))
    return System(m, r, v, P_in / steps_per_period, f"planetary-N{k + 1}-seed{seed}")


def plummer(n: int = 1024, seed: int = 0, *, virial: bool = True) -> System:
    """Equal-mass Plummer sphere (total mass 1) in virial N-body units.
    dt defaults to 2^-8."""
    rng = np.random.default_rng(seed)
    m = np.full(n, 1.0 / n)
    r, rad = _plummer_positions(rng, n)
    v = _plummer_speeds(rng, rad)[:, None] * _isotropic(rng, n)
    r, v = _com_frame(m, r, v)
    if virial:
        r, v = _virialise(m, r, v)
    return System(m, r, v, 2.0 ** -8, f"plummer-N{n}-seed{seed}")


def bh_cluster(n: int = 16384, seed: int = 0, *, m_bh=1.0, m_cluster=1e-2) -> System:
    """Black hole of mass m_bh at rest at the origin plus n-1 stars of total
    mass m_cluster, Plummer-distributed with scale 1, each on a circular
    velocity v = sqrt(M(<r)/r), M(<r) = m_bh + m_cluster r^3/(r^2+1)^1.5,
    in a random direction perpendicular to its radius vector.  Then the
    whole system is moved to its centre-of-mass frame.  dt = 2^-10."""
    rng = np.random.default_rng(seed)
    k = n - 1
    ms = np.full(k, m_cluster / k)
    rs, rad = _plummer_positions(rng, k)
    Menc = m_bh + m_cluster * rad ** 3 / (rad ** 2 + 1.0) ** 1.5
    vc = np.sqrt(Menc / rad)
    rhat = rs / rad[:, None]
    t = _isotropic(rng, k)
    t = t - (t * rhat).sum(1)[:, None] * rhat
    t /= np.linalg.norm(t, axis=1)[:, None]
    vs = vc[:, None] * t
    m = np.concatenate([[m_bh], ms])
    r = np.concatenate([np.zeros((1, 3)), rs])
    v = np.concatenate([np.zeros((1, 3)), vs])
    r, v = _com_frame(m, r, v)
    return System(m, r, v, 2.0 ** -10, f"bh-cluster-N{n}-seed{seed}")


def plummer_bh(n: int = 128, q: float = 1e6, seed: int = 0) -> System:
    """The paper's large-N test (Sec. 3.2): a Plummer sphere of n - 1
    equal-mass stars with a black hole of q times a star's mass at rest at
    its centre, total mass 1, in virial equilibrium.  Star positions follow
    the Plummer profile at the N-body-unit scale 3 pi / 16; each star's speed
    is x v_esc(r), with x drawn from the Plummer speed distribution
    x^2 (1 - x^2)^(7/2) and v_esc the escape speed of the combined potential
    (stars plus black hole), in an isotropic direction.  The system is moved
    to its centre-of-mass frame and the velocities alone are scaled to
    2T = -W, so the stars orbit at radii of order one whatever q is.  q = 1
    makes the black hole an ordinary star.  dt = 1e-4."""
    rng = np.random.default_rng(seed)
    k = n - 1
    m_star = 1.0 / (k + q)
    m_bh = q * m_star
    a = 3.0 * math.pi / 16.0
    rs, rad = _plummer_positions(rng, k)
    x = _plummer_speeds(rng, rad) / (math.sqrt(2.0) * (1.0 + rad * rad) ** (-0.25))
    rs, rad = rs * a, rad * a
    vesc = np.sqrt(2.0 * (k * m_star / np.sqrt(rad * rad + a * a) + m_bh / rad))
    vs = (x * vesc)[:, None] * _isotropic(rng, k)
    m = np.concatenate([[m_bh], np.full(k, m_star)])
    r = np.concatenate([np.zeros((1, 3)), rs])
    v = np.concatenate([np.zeros((1, 3)), vs])
    r, v = _com_frame(m, r, v)
    W = potential_energy(m, r)
    T = 0.5 * float((m * (v * v).sum(1)).sum())
    v = v * math.sqrt(-0.5 * W / T)
    return System(m, r, v, 1e-4, f"plummer-bh-N{n}-q{q:g}-seed{seed}")


def plummer_binaries(n: int = 16384, seed: int = 0, *, f_bin: float = 0.1,
                     a_lo=1e-4, a_hi=1e-2) -> System:
    """Plummer cluster of n equal-mass (1/n) particles of which a fraction
    f_bin are members of primordial binaries.  Binary and single centres are
    Plummer-sampled and virialised together; binary orbits have log-uniform
    semi-major axes in [a_lo, a_hi], thermal eccentricities (e = sqrt(U)),
    isotropic orientation and uniform mean anomaly.  dt = 2^-10."""
    rng = np.random.default_rng(seed)
    nb = int(round(f_bin * n)) // 2           # number of binaries
    ns = n - 2 * nb                           # singles
    nc = nb + ns
    mc = np.concatenate([np.full(nb, 2.0 / n), np.full(ns, 1.0 / n)])
    rc, rad = _plummer_positions(rng, nc)
    vc = _plummer_speeds(rng, rad)[:, None] * _isotropic(rng, nc)
    rc, vc = _com_frame(mc, rc, vc)
    rc, vc = _virialise(mc, rc, vc)
    a = np.exp(rng.uniform(math.log(a_lo), math.log(a_hi), nb))
    e = np.sqrt(rng.uniform(0.0, 1.0, nb))
    e = np.minimum(e, 0.999)
    inc = np.arccos(rng.uniform(-1.0, 1.0, nb))
    Om = rng.uniform(0.0, 2 * math.pi, nb)
    om = rng.uniform(0.0, 2 * math.pi, nb)
    Mn = rng.uniform(0.0, 2 * math.pi, nb)
    mb = 1.0 / n
    rrel, vrel = elements_to_cartesian(2 * mb, a, e, inc, Om, om, Mn)
    r1 = rc[:nb] + 0.5 * rrel
    r2 = rc[:nb] - 0.5 * rrel
    v1 = vc[:nb] + 0.5 * vrel
    v2 = vc[:nb] - 0.5 * vrel
    r = np.concatenate([r1, r2, rc[nb:]])
    v = np.concatenate([v1, v2, vc[nb:]])
    m = np.full(n, 1.0 / n)
    perm = rng.permutation(n)
    return System(m[perm], r[perm], v[perm], 2.0 ** -10,
                  f"plummer-binaries-N{n}-seed{seed}")


def hierarchical_double_binary(ratio: float = 100.0, m_each: float = 0.25) -> System:
    """Two equal circular binaries (separation a_in = 1/ratio) on a circular
    outer orbit of separation 1 (the paper's N = 4 hierarchical test).
    dt = P_outer / 1000."""
    a_out, a_in = 1.0, 1.0 / ratio
    mb = 2 * m_each
    # outer orbit of the two binary centres
    vo = math.sqrt(2 * mb / a_out)
    cen_r = np.array([[0.5 * a_out, 0, 0], [-0.5 * a_out, 0, 0]])
    cen_v = np.array([[0, 0.5 * vo, 0], [0, -0.5 * vo, 0]])
    vi = math.sqrt(mb / a_in)
    r, v = [], []
    for c in range(2):
        r += [cen_r[c] + [0, 0.5 * a_in, 0], cen_r[c] - [0, 0.5 * a_in, 0]]
        v += [cen_v[c] + [0, 0, 0.5 * vi], cen_v[c] - [0, 0, 0.5 * vi]]
    m = np.full(4, m_each)
    P_out = 2 * math.pi * math.sqrt(a_out ** 3 / (2 * mb))
    r, v = _com_frame(m, np.array(r, float), np.array(v, float))
    return System(m, r, v, P_out / 1000.0, f"double-binary-ratio{ratio:g}")


@dataclasses.dataclass
class Ensemble:
    """Many independent systems packed end to end (CSR offsets)."""
    m: np.ndarray         # [total]
    state: np.ndarray     # [6, total] SoA
    offsets: np.ndarray   # [nsys + 1] int64
    dt: np.ndarray        # [nsys]
    seeds: np.ndarray     # [nsys]

    @property
    def nsys(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def system(self, k: int) -> System:
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        r, v = from_soa(self.state[:, a:b])
        return System(self.m[a:b].copy(), r, v, float(self.dt[k]), f"ensemble-{k}")


def ensemble(nsys: int = 4096, seed: int = 0, n_lo: int = 3, n_hi: int = 64) -> Ensemble:
    """nsys planetary systems, each with N uniform in [n_lo, n_hi] (a central
    mass plus N-1 planets) built like the single planetary system from its own
    seed; each keeps its own dt = P_inner / 200."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_lo, n_hi + 1, nsys)
    seeds = rng.integers(0, 2 ** 31 - 1, nsys)
    ms, states, dts = [], [], []
    for k in range(nsys):
        s = planetary(int(seeds[k]), int(sizes[k]) - 1)
        ms.append(s.m)
        states.append(s.soa())
        dts.append(s.dt)
    offsets = np.zeros(nsys + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return Ensemble(np.concatenate(ms), np.concatenate(states, 1), offsets,
                    np.array(dts), seeds)


def random_cluster(n: int, seed: int = 0, *, mass_spread: float = 1.0) -> System:
    """Small unequal-mass test cluster: Plummer positions and speeds with
    log-uniform masses spanning mass_spread decades (total mass 1)."""
    rng = np.random.default_rng(seed)
    r, rad = _plummer_positions(rng, n)
    v = _plummer_speeds(rng, rad)[:, None] * _isotropic(rng, n)
    m = np.exp(rng.uniform(0.0, mass_spread * math.log(10.0), n))
    m /= m.sum()
    r, v = _com_frame(m, r, v)
    return System(m, r, v, 2.0 ** -8, f"random-N{n}-seed{seed}")
