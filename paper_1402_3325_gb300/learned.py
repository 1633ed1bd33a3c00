"""Training pipeline of the learned initial guess.

Data come from the method's own runs: a cluster is integrated with the FP64
library path and, at a number of its steps, a sample of ordered pairs is
passed to ``sakura_sample_pairs``, which solves each pair's Kepler problem and
returns the network features and the target g = log(s / s_T2) / w
(include/sakura.h).  The sample is stratified: a fraction of close pairs
(found with a k-d tree, the pairs where the guess matters) and uniformly random
pairs.  The network is then trained on the GPU with ``sakura_mlp_train`` (the
library's own forward, backward and Adam kernels) and packed into the 4687-
float blob that ``sakura_load_mlp`` expects.

    python -m paper_1402_3325_gb300.learned --out weights.npy [--samples 10000000]
"""
from __future__ import annotations

import argparse
import math
import os

import numpy as np

from . import ics
from . import sakura as sk

PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(PKG, "data", "mlp_guess.npy")


def pair_sample(r: np.ndarray, rng: np.random.Generator, count: int, close_frac: float,
                close_radius: float) -> np.ndarray:
    """Ordered pair ids i*n+j: close_frac of them from the pairs closer than
    close_radius (both orders, drawn with replacement), the rest uniform."""
    from scipy.spatial import cKDTree
    n = r.shape[0]
    close = np.array(sorted(cKDTree(r).query_pairs(close_radius)), dtype=np.int64).reshape(-1, 2)
    n_close = int(count * close_frac) if close.shape[0] else 0
    ids = []
    if n_close:
        pick = close[rng.integers(0, close.shape[0], n_close)]
        flip = rng.integers(0, 2, n_close).astype(bool)
        i = np.where(flip, pick[:, 1], pick[:, 0])
        j = np.where(flip, pick[:, 0], pick[:, 1])
        ids.append(i * n + j)
    m = count - n_close
    i = rng.integers(0, n, m)
    j = (i + rng.integers(1, n, m)) % n
    ids.append(i * n + j)
    return np.concatenate(ids)


def generate(system: ics.System, samples: int, steps: int = 32, close_frac: float = 0.3,
             close_radius: float = 0.02, seed: int = 0, device: str = "cuda"):
    """(features, targets) CUDA tensors from `steps` steps of the system."""
    import torch
    rng = np.random.default_rng(seed)
    state = torch.tensor(system.soa(), device=device)
    mass = torch.tensor(system.m, device=device)
    per = int(math.ceil(samples / steps))
    feats, tgts = [], []
    for _ in range(steps):
        r = state[:3].T.cpu().numpy()
        ids = torch.tensor(pair_sample(r, rng, per, close_frac, close_radius), device=device)
        f, t = sk.sample_pairs(state, mass, system.dt, ids, 2)
        feats.append(f)
        tgts.append(t)
        sk.step(state, mass, system.dt, 2)
    sk.check()
    return torch.cat(feats)[:samples], torch.cat(tgts)[:samples]


def fit(features, targets, epochs: int = 3, batch: int = 8192, lr: float = 2e-3,
        seed: int = 0):
    """Train on the GPU; returns (blob float32[4687], minibatch losses)."""
    import torch
    dev = features.device
    f = features.cpu().numpy().astype(np.float64)
    t = np.clip(targets.cpu().numpy().astype(np.float64), -4.0, 4.0)
    mean = f.mean(0)
    scale = f.std(0)
    scale[scale < 1e-6] = 1.0
    oshift = float(t.mean())
    oscale = float(t.std()) or 1.0
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, 1 / math.sqrt(6), (64, 6))
    W2 = rng.normal(0, 1 / math.sqrt(64), (64, 64))
    W3 = rng.normal(0, 1 / math.sqrt(64), 64)
    params = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3,
                             np.zeros(1)]).astype(np.float32)
    perm = rng.permutation(f.shape[0])
    feat_d = torch.tensor(f[perm].astype(np.float32), device=dev)
    tgt_d = torch.tensor(((t[perm] - oshift) / oscale).astype(np.float32), device=dev)
    norm_d = torch.tensor(np.concatenate([mean, scale]).astype(np.float32), device=dev)
    p_d = torch.tensor(params, device=dev)
    losses = sk.mlp_train(p_d, norm_d, feat_d, tgt_d, batch, epochs, lr)
    blob = np.concatenate([p_d.cpu().numpy().astype(np.float64), mean, scale,
                           [oscale, oshift]]).astype(np.float32)
    return blob, losses.cpu().numpy()


def load_default():
    """Load the committed network into the library (it must be initialised)."""
    sk.load_mlp(np.load(DEFAULT_WEIGHTS))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--samples", type=int, default=10_000_000)
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args()
    from . import build
    build.build()
    sk.init(0)
    system = ics.plummer_binaries(args.n, seed=args.seed)
    feats, tgts = generate(system, args.samples, seed=args.seed)
    blob, losses = fit(feats, tgts, epochs=args.epochs, seed=args.seed)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, blob)
    k = max(1, len(losses) // 20)
    print(f"samples {feats.shape[0]} loss first {losses[:k].mean():.4e} last {losses[-k:].mean():.4e}"
          f" -> {args.out}")


if __name__ == "__main__":
    main()
