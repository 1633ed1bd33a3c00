"""Write tests/golden/bh16384_oracle_run.json: the oracle's own run of the
black-hole cluster (black hole of mass 1 plus 16383 stars of total mass 1e-2,
Plummer scale 1, circular velocities; seed 0), dt = 2^-10, 256 second-order
steps (Eqs. 27a-d), so that the mixed-precision form on the GPU can be checked
against the FP64 method over the whole run without repeating hours of CPU
work in every test.

Only the oracle (oracle/) and the seeded input generator are used.  Stored:
the initial energy and a SHA-256 of the initial state as this machine made
it, and after 32 and 256 steps the oracle's total energy (Eqs. 1-3,
compensated sums) and the positions and velocities of a fixed sample of
particles: the black hole, every 64th star and the 16 stars closest to the
black hole.  Floats are written with repr (exact round trip).

Run from the repository root (about 45 minutes on 8 cores):

    python tests/golden/make_bh16384_oracle_run.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "..")
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1402_3325_gb300 import ics  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bh16384_oracle_run.json")
N = 16384
SEED = 0
STEPS = 256
CHECKPOINTS = (32, 256)


def state_hash(s) -> str:
    h = hashlib.sha256()
    for a in (s.m, s.r, s.v):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return h.hexdigest()


def sample_indices(s) -> list[int]:
    rad = np.linalg.norm(s.r - s.r[0], axis=1)
    rad[0] = np.inf
    near = np.argsort(rad)[:16]
    idx = set([0]) | set(range(1, N, 64)) | set(int(k) for k in near)
    return sorted(int(k) for k in idx)


def main():
    s = ics.bh_cluster(N, seed=SEED)
    cores = os.cpu_count() or 1
    idx = sample_indices(s)
    E0 = oracle.energy(s.m, s.r, s.v)[0]
    out = {"workload": f"bh_cluster({N}, seed={SEED}), dt = 2^-10, order 2",
           "n": N, "seed": SEED, "dt": s.dt, "order": 2, "steps": STEPS,
           "initial_state_sha256": state_hash(s), "E0": E0, "sample": idx,
           "checkpoints": {}}
    r, v = s.r.copy(), s.v.copy()
    t0 = time.time()
    for k in range(1, STEPS + 1):
        rc, r, v = oracle.step(s.m, r, v, s.dt, 2, nthreads=cores)
        if rc != oracle.OK:
            raise SystemExit(f"oracle step {k} failed with {rc}")
        if k in CHECKPOINTS:
            E = oracle.energy(s.m, r, v)[0]
            out["checkpoints"][str(k)] = {
                "E": E, "r": [[float(x) for x in r[i]] for i in idx],
                "v": [[float(x) for x in v[i]] for i in idx]}
            print(f"step {k}: dE/E = {abs(E / E0 - 1):.3e} ({time.time() - t0:.0f} s)",
                  flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
