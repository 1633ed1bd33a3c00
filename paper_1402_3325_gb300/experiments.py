"""The paper's accuracy experiments whose initial conditions its text fully
describes, run on the GPU through the library:

* the N = 4 hierarchical double binary (Sec. 3.1): two equal circular
  binaries of separation a_in = 1 / ratio on a circular outer orbit of
  separation 1, ratio = a_out / a_in = 10, 100, 1000, integrated for one outer
  period P_out at constant steps P_out / 2^k (all ratios share P_out, so each
  k is one batched call over the three systems);
* the 128-body Plummer sphere with a central black hole (Sec. 3.2): mass
  ratios q = M_bh / M_star from 1 to 1e12 (ics.plummer_bh), constant steps
  1e-3, 1e-4 or 1e-5, one N-body time unit.

Each row carries the relative energy error |E1 / E0 - 1|, with E from the
library's double-double energy kernel (Eqs. 1-3).  The paper compares these
with leapfrog and Hermite codes, which are not part of this library.

    python -m paper_1402_3325_gb300.experiments qsweep --taus 1e-3 1e-4 --seeds 0 1 2 3
    python -m paper_1402_3325_gb300.experiments double-binary --ks 8 10 12 14
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import ics
from . import sakura as sk

Q_VALUES = (1.0, 1e1, 1e2, 1e3, 1e4, 1e5, 1e6, 1e7, 1e8, 1e9, 1e10, 1e11, 1e12)
RATIOS = (10.0, 100.0, 1000.0)


def _dev(a, torch, device, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device=device)


def q_sweep(qs=Q_VALUES, taus=(1e-3,), seeds=(0,), n: int = 128, span: float = 1.0,
            order: int = 2, device: str = "cuda"):
    """Energy error of the Plummer sphere with a central black hole after
    `span` time units, for every (tau, q, seed).  The library must be
    initialised."""
    import torch
    rows = []
    for tau in taus:
        nsteps = int(round(span / tau))
        for q in qs:
            for seed in seeds:
                s = ics.plummer_bh(n, q, seed)
                state = _dev(s.soa(), torch, device)
                mass = _dev(s.m, torch, device)
                E0 = sk.energy(state, mass)
                for _ in range(nsteps):
                    sk.step(state, mass, tau, order)
                E1 = sk.energy(state, mass)
                rows.append({"q": float(q), "tau": float(tau), "seed": int(seed),
                             "steps": nsteps, "order": order, "E0": E0,
                             "dE_E": abs(E1 / E0 - 1.0)})
    return rows


def double_binary(ratios=RATIOS, ks=(8, 10, 12, 14), order: int = 2, device: str = "cuda"):
    """Energy error of the hierarchical double binaries after one outer
    period at steps P_out / 2^k, for every (k, ratio): one batched call per
    k over all ratios.  The library must be initialised."""
    import torch
    systems = [ics.hierarchical_double_binary(r) for r in ratios]
    offsets = np.arange(len(systems) + 1, dtype=np.int64) * 4
    state0 = np.concatenate([s.soa() for s in systems], axis=1)
    mass = _dev(np.concatenate([s.m for s in systems]), torch, device)
    offs = _dev(offsets, torch, device, torch.int64)
    P_out = np.array([s.dt * 1000.0 for s in systems])  # ics: dt = P_out / 1000

    def energies(state):
        return [sk.energy(state[:, a:b].contiguous(), mass[a:b].contiguous())
                for a, b in zip(offsets[:-1], offsets[1:])]

    rows = []
    for k in ks:
        state = _dev(state0, torch, device)
        E0 = energies(state)
        dt = _dev(P_out / 2.0 ** k, torch, device)
        sk.step_batched(state, mass, offs, offsets, dt, order, 2 ** k)
        E1 = energies(state)
        for r, P, e0, e1 in zip(ratios, P_out, E0, E1):
            rows.append({"ratio": float(r), "k": int(k), "tau": float(P / 2.0 ** k),
                         "steps": 2 ** k, "order": order, "E0": e0,
                         "dE_E": abs(e1 / e0 - 1.0)})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("experiment", choices=["qsweep", "double-binary"])
    ap.add_argument("--taus", type=float, nargs="+", default=[1e-3])
    ap.add_argument("--seeds", type=int, nargs="+", default=[0])
    ap.add_argument("--ks", type=int, nargs="+", default=[8, 10, 12, 14])
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--out", default=None, help="write the rows as JSON here")
    args = ap.parse_args()
    from . import build
    build.build()
    sk.init(0, guess=sk.GUESS_TAYLOR)
    if args.experiment == "qsweep":
        rows = q_sweep(taus=args.taus, seeds=args.seeds, order=args.order)
        for r in rows:
            print(f"tau {r['tau']:.0e} q {r['q']:8.0e} seed {r['seed']} dE/E {r['dE_E']:.3e}")
    else:
        rows = double_binary(ks=args.ks, order=args.order)
        for r in rows:
            print(f"ratio {r['ratio']:6.0f} tau P_out/2^{r['k']:<2d} dE/E {r['dE_E']:.3e}")
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(rows, fh, indent=1)
    sk.finalize()


if __name__ == "__main__":
    main()
