"""Independent two-body reference for pinning the oracle's Kepler flow (Eq. 18).

This solves the classical Kepler equation in *eccentric* (ellipse) or
*hyperbolic* anomaly differences, in mpmath at 40 significant digits, and maps
back with the classical Lagrange f and g functions written in those anomalies.
It shares nothing with the universal-variable / Stumpff / Laguerre formulation
that the oracle and the CUDA library use, so agreement pins both the
formulation and the root finding.

    ellipse   (1/a > 0):  n t = dE - (e cos E0) sin dE + (e sin E0)(1 - cos dE)
    hyperbola (1/a < 0):  n t = (e cosh H0) sinh dH + (e sinh H0)(cosh dH - 1) - dH

with e cos E0 = 1 - r0/a, e sin E0 = (r0.v0)/sqrt(m a) and the hyperbolic
analogues e cosh H0 = 1 + r0/|a|, e sinh H0 = (r0.v0)/sqrt(m |a|).
"""
from __future__ import annotations

import mpmath as mp


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _bisect(fun, lo, hi, iters=400):
    flo = fun(lo)
    for _ in range(iters):
        mid = (lo + hi) / 2
        fm = fun(mid)
        if (fm < 0) == (flo < 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return (lo + hi) / 2


def kepler_classical(tau, m, r0, v0, dps: int = 40):
    """Return (r1, v1) as lists of mpf after time tau."""
    with mp.workdps(dps):
        t = mp.mpf(tau)
        mu = mp.mpf(m)
        R = [mp.mpf(x) for x in r0]
        V = [mp.mpf(x) for x in v0]
        r = mp.sqrt(_dot(R, R))
        sig = _dot(R, V)
        v2 = _dot(V, V)
        alpha = 2 / r - v2 / mu
        if alpha > 0:
            a = 1 / alpha
            n = mp.sqrt(mu / a ** 3)
            ec = 1 - r / a
            es = sig / mp.sqrt(mu * a)
            M = n * t

            def kep(d):
                return d - ec * mp.sin(d) + es * (1 - mp.cos(d)) - M

            d = _bisect(kep, M - 3, M + 3)
            rr = a * (1 - ec * mp.cos(d) + es * mp.sin(d))
            f = 1 - a / r * (1 - mp.cos(d))
            g = t - (d - mp.sin(d)) / n
            fd = -mp.sqrt(mu * a) * mp.sin(d) / (r * rr)
            gd = 1 - a / rr * (1 - mp.cos(d))
        elif alpha < 0:
            ah = -1 / alpha
            n = mp.sqrt(mu / ah ** 3)
            ec = 1 + r / ah
            es = sig / mp.sqrt(mu * ah)
            M = n * t

            def kep(d):
                return ec * mp.sinh(d) + es * (mp.cosh(d) - 1) - d - M

            # kep is increasing; bracket by doubling
            lo, hi = mp.mpf(-1), mp.mpf(1)
            while kep(lo) > 0:
                lo *= 2
            while kep(hi) < 0:
                hi *= 2
            d = _bisect(kep, lo, hi)
            rr = ah * (ec * mp.cosh(d) + es * mp.sinh(d) - 1)
            f = 1 - ah / r * (mp.cosh(d) - 1)
            g = t - (mp.sinh(d) - d) / n
            fd = -mp.sqrt(mu * ah) * mp.sinh(d) / (r * rr)
            gd = 1 - ah / rr * (mp.cosh(d) - 1)
        else:  # pragma: no cover - exact parabola never occurs with random doubles
            raise ValueError("parabolic case not supported")
        r1 = [f * R[q] + g * V[q] for q in range(3)]
        v1 = [fd * R[q] + gd * V[q] for q in range(3)]
        return r1, v1


def kepler_classical_f64(tau, m, r0, v0):
    r1, v1 = kepler_classical(tau, m, r0, v0)
    return [float(x) for x in r1], [float(x) for x in v1]
