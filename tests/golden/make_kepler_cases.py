"""Write tests/golden/kepler_cases.json: two-body Kepler-flow cases (Eq. 18)
with expected states from the classical anomaly solution at 40 digits
(tests/classical_kepler.py, mpmath).  No library or oracle code is used.

Inputs are stored as exact float64 hex strings, expected outputs as 25-digit
decimal strings.  Run from the repository root:

    python tests/golden/make_kepler_cases.py
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import mpmath as mp  # noqa: E402
from classical_kepler import kepler_classical  # noqa: E402


def _case(name, tau, m, r0, v0):
    return {"name": name, "tau": float(tau), "m": float(m), "r0": [float(x) for x in r0],
            "v0": [float(x) for x in v0]}


def cases():
    rng = np.random.default_rng(20140211)
    out = []
    # circular orbit, quarter period
    out.append(_case("circular-quarter", 0.25 * 2 * math.pi, 1.0, [1, 0, 0], [0, 1, 0]))
    # eccentric ellipse through pericentre
    out.append(_case("ellipse-e0.9-peri", 0.3, 1.0, [1.0, 0.0, 0.0], [0.0, 0.3, 0.05]))
    # several revolutions of a bound orbit (period reduction)
    out.append(_case("ellipse-multirev", 17.3, 2.0, [0.3, -0.1, 0.05], [0.4, 2.2, -0.3]))
    # backward in time
    out.append(_case("ellipse-backward", -0.71, 1.0, [0.5, 0.2, -0.1], [-0.3, 1.1, 0.2]))
    # weak hyperbolic encounter, Plummer-like star pair (m_ij = 2/1024, dt = 2^-8)
    out.append(_case("weak-hyperbolic", 2.0 ** -8, 2.0 / 1024, [0.31, -0.52, 0.2],
                     [0.41, 0.13, -0.62]))
    # strong hyperbolic flyby
    out.append(_case("hyperbolic-flyby", 0.05, 1.0, [0.01, 0.002, 0.0], [-1.0, 15.0, 0.5]))
    # near-parabolic, bound side and unbound side
    v_esc = math.sqrt(2.0)
    out.append(_case("near-parabolic-bound", 0.8, 1.0, [1, 0, 0], [0.1, v_esc * (1 - 1e-9), 0]))
    out.append(_case("near-parabolic-unbound", 0.8, 1.0, [1, 0, 0], [0.1, v_esc * (1 + 1e-9), 0]))
    # nearly radial infall (tiny angular momentum)
    out.append(_case("nearly-radial", 0.2, 1.0, [1.0, 0.0, 0.0], [-0.2, 1e-4, 0.0]))
    # tiny star-star mass around a black hole cluster (m_ij ~ 1.2e-6)
    out.append(_case("tiny-mass", 2.0 ** -10, 1.2e-6, [0.02, 0.01, -0.03], [0.9, -0.2, 0.1]))
    # tight binary over many periods (a ~ 1e-4, P < dt)
    out.append(_case("tight-binary", 2.0 ** -10, 2.0 / 16384, [1e-4, 2e-5, 0.0],
                     [0.0, 1.15, 0.1]))
    # fast, strongly hyperbolic star pairs whose standard guess t / r0 lies so
    # far past the root that the G-functions overflow there (sqrt(-beta) t / r0
    # > 710): approaching, receding, and backward in time
    out.append(_case("hyperbolic-guess-overflow-approach", 1e-3, 2e-6, [9e-5, 2e-5, -1e-5],
                     [-60.0, 25.0, 18.0]))
    out.append(_case("hyperbolic-guess-overflow-recede", 1e-3, 2e-6, [9e-5, 2e-5, -1e-5],
                     [120.0, -50.0, -36.0]))
    out.append(_case("hyperbolic-guess-overflow-backward", -1e-3, 2e-6, [9e-5, 2e-5, -1e-5],
                     [-60.0, 25.0, 18.0]))
    # close flyby (impact parameter 1.5e-5, ending 0.42 apart) whose guess
    # lies 2e4 / sqrt(-beta) past the root, where r(s) = F' is so large that
    # the Laguerre discriminant overflows
    out.append(_case("close-flyby-guess-far-past-root", 1e-3, 2e-6, [1.6e-5, -1.1e-5, 4e-6],
                     [-300.0, 180.0, 250.0]))
    # nearly head-on flyby (a pair of a fast star swarm) on which the Laguerre
    # step from far past the root once rounded to zero and was taken for
    # convergence
    out.append(_case("close-flyby-discriminant-overflow", 1e-3, 2e-6,
                     [-5.918864792495962e-06, 4.702523318676603e-05, 0.00044838192387707486],
                     [-34.92845080444039, -206.30318962125773, -252.43950821240344]))
    # random mix
    for k in range(12):
        m = float(10 ** rng.uniform(-6, 0.5))
        r = rng.normal(size=3) * 10 ** rng.uniform(-3, 0.5)
        rn = float(np.linalg.norm(r))
        vc = math.sqrt(m / rn)
        v = rng.normal(size=3) * vc * 10 ** rng.uniform(-0.5, 1.0)
        P = 2 * math.pi * math.sqrt(rn ** 3 / m)
        tau = float(P * 10 ** rng.uniform(-4, 0.3)) * (1 if rng.uniform() < 0.8 else -1)
        out.append(_case(f"random-{k}", tau, m, r, v))
    return out


def main():
    res = []
    mp.mp.dps = 40
    for c in cases():
        r1, v1 = kepler_classical(c["tau"], c["m"], c["r0"], c["v0"])
        c = dict(c)
        c["tau"] = float.hex(c["tau"])
        c["m"] = float.hex(c["m"])
        c["r0"] = [float.hex(x) for x in c["r0"]]
        c["v0"] = [float.hex(x) for x in c["v0"]]
        c["r1"] = [mp.nstr(x, 25, min_fixed=-1, max_fixed=-1) for x in r1]
        c["v1"] = [mp.nstr(x, 25, min_fixed=-1, max_fixed=-1) for x in v1]
        res.append(c)
    path = os.path.join(os.path.dirname(__file__), "kepler_cases.json")
    with open(path, "w") as fh:
        json.dump({"source": "classical anomaly Kepler solution, mpmath 40 digits "
                             "(tests/classical_kepler.py); flow of Eq. 18",
                   "cases": res}, fh, indent=1)
    print(f"wrote {len(res)} cases to {path}")


if __name__ == "__main__":
    main()
