"""Rounding band of the mixed form's single-precision class decision.

The library decides each pair's class (single precision iff r > r_min and
e < e_max, or e > e_hyp) in FP32 on a float copy of the drifted state; the
oracle evaluates the same rule in FP64.  The two may disagree only where a
pair's r^2 or e^2 lies within the FP32 decision's rounding error of a
threshold.  This module bounds that error for one pair, from the pair's
double-precision Kepler input, by first-order propagation of the unit
roundoff u = 2^-24 through the kernel's operations (with a safety factor):

  inputs: positions as hi + lo floats (the separation to ~u of itself),
          velocities rounded to float (error u |v| each, so the relative
          velocity carries u (|v_i| + |v_j|)), masses rounded to float;
  r0 = dx - ptau dv, r^2, v^2, r0.v0 as sums of products;
  h^2 = r^2 v^2 - (r0.v0)^2, 2E = v^2 - 2m/r (hardware 1/sqrt(r^2));
  e < e_max  <=>  2E h^2 < (e_max^2 - 1) m^2, likewise for e_hyp.

Test helper only: it computes nothing that the tests compare against.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24
SAFETY = 4.0


def kepler_input(m, r, v, tau, order, i, j):
    """The pair's Kepler input (Eq. 26) in double precision."""
    drift = 0.5 * tau if order == 2 else (0.0 if order == 1 else tau)
    pre = 0.5 if order == 2 else (0.0 if order == 1 else 1.0)
    xi = r[i] + v[i] * drift
    xj = r[j] + v[j] * drift
    u0 = v[i] - v[j]
    x0 = (xi - xj) - u0 * (tau * pre)
    return x0, u0, m[i] + m[j], np.linalg.norm(v[i]) + np.linalg.norm(v[j]), abs(tau * pre)


def band(m, r, v, tau, order, i, j):
    """(band on r^2, band on e^2) of the pair (i, j): the single-precision
    decision may differ from the double-precision rule only when r^2 is
    within the first of r_min^2, or e^2 within the second of e_max^2 or
    e_hyp^2."""
    x0, u0, mm, V, ptau = kepler_input(m, r, v, tau, order, i, j)
    u = U32
    a = float(np.linalg.norm(x0))
    b = float(np.linalg.norm(u0))
    r2, v2 = a * a, b * b
    eta = float(x0 @ u0)
    h2 = r2 * v2 - eta * eta
    dx = 4 * u * a + 2 * ptau * u * V
    du = 2 * u * V
    dr2 = 2 * a * dx + 4 * u * r2
    dv2 = 2 * b * du + 4 * u * v2
    deta = a * du + b * dx + 4 * u * a * b
    dh2 = r2 * dv2 + v2 * dr2 + 2 * abs(eta) * deta + 4 * u * (r2 * v2 + eta * eta)
    twom_r = 2 * mm / a
    dtwom_r = twom_r * (dr2 / (2 * r2) + 6 * u)
    twoE = v2 - twom_r
    dtwoE = dv2 + dtwom_r + 2 * u * (v2 + twom_r)
    lhs = twoE * h2
    dlhs = abs(twoE) * dh2 + abs(h2) * dtwoE + 2 * u * abs(lhs)
    e2 = 1.0 + lhs / (mm * mm)
    de2 = dlhs / (mm * mm) + 8 * u * (abs(e2 - 1.0) + 1.0)
    return SAFETY * dr2, SAFETY * de2


def check_classes(gpu, orc, m, r, v, tau, order, rule, r_min=0.1, e_max=0.9, e_hyp=10.0):
    """Compare two class matrices pair by pair.  Every pair on which they
    differ must lie within the decision's rounding band of a threshold
    (its r^2 and e^2 from the oracle).  Returns the number of differing
    pairs; raises AssertionError for a difference outside the band."""
    import oracle
    diff = np.argwhere(gpu != orc)
    for i, j in diff:
        i, j = int(i), int(j)
        _, _, r2, e2 = oracle.pair_classes(m[[i, j]], r[[i, j]], v[[i, j]], tau, rule=rule,
                                           r_min=r_min, e_max=e_max, e_hyp=e_hyp,
                                           order=order, want_values=True)
        br, be = band(m, r, v, tau, order, i, j)
        near = (abs(r2[0, 1] - r_min * r_min) <= br or abs(e2[0, 1] - e_max * e_max) <= be or
                (rule == 1 and abs(e2[0, 1] - e_hyp * e_hyp) <= be))
        assert near, (f"pair ({i}, {j}) classed {int(gpu[i, j])} on the GPU and"
                      f" {int(orc[i, j])} by the oracle, away from every threshold:"
                      f" r^2 = {r2[0, 1]!r} (band {br:.2e}), e^2 = {e2[0, 1]!r}"
                      f" (band {be:.2e})")
    return int(diff.shape[0])
