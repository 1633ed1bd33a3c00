"""GPU tests of the learned initial guess.

* Gradients of the project's FP32 training kernels equal the FP64 oracle's
  hand-written backward pass (oracle/mlp.py, itself pinned by finite
  differences) on the same batch.
* The BF16 warp inference used inside the pair kernels reproduces the
  oracle's forward pass to BF16 accuracy.
* A network trained on data from the method's own runs lowers the training
  loss, lowers the mean and the worst Kepler iteration counts against the
  standard guess, and leaves every result within the FP64 tolerance of the
  oracle (the guess only changes where the iteration starts).
"""
import contextlib
import os

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1402_3325_gb300 import ics
from paper_1402_3325_gb300 import learned
from paper_1402_3325_gb300 import sakura as sk

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_3325_gb300 import build
    build.build()
    sk.init(0, flags=sk.FLAG_STATS)
    yield
    sk.finalize()


@contextlib.contextmanager
def configured(**opts):
    sk.init(0, flags=opts.pop("flags", sk.FLAG_STATS), **opts)
    try:
        yield
    finally:
        sk.init(0, flags=sk.FLAG_STATS)


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_training_gradient_matches_oracle():
    rng = np.random.default_rng(4)
    theta = omlp.init_params(2) + rng.normal(0, 0.05, omlp.N_PARAMS)
    B = 1000
    x = rng.normal(size=(B, 6))
    t = rng.normal(size=B)
    L_ref, g_ref = omlp.loss_and_grad(theta, x, t)
    norm = dev(np.concatenate([np.zeros(6), np.ones(6)]), torch.float32)
    L, g = sk.mlp_grad(dev(theta, torch.float32), norm, dev(x, torch.float32),
                       dev(t, torch.float32))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(L - L_ref) <= 1e-5 * L_ref
    assert np.abs(g - g_ref).max() <= 2e-5 * np.abs(g_ref).max()


def _blob(theta, mean=None, scale=None, oscale=1.0, oshift=0.0):
    mean = np.zeros(6) if mean is None else mean
    scale = np.ones(6) if scale is None else scale
    return np.concatenate([theta, mean, scale, [oscale, oshift]]).astype(np.float32)


def test_bf16_inference_matches_oracle_forward():
    rng = np.random.default_rng(7)
    theta = omlp.init_params(5) + rng.normal(0, 0.02, omlp.N_PARAMS)
    mean = rng.normal(0, 0.5, 6)
    scale = rng.uniform(0.5, 2.0, 6)
    sk.load_mlp(_blob(theta, mean, scale, oscale=0.7, oshift=0.1))
    x = rng.normal(size=(3000, 6)) * scale + mean
    y_ref, _ = omlp.forward(theta, (x - mean) / scale)
    y_ref = np.clip(y_ref * 0.7 + 0.1, -4, 4)
    y = sk.mlp_eval(dev(x, torch.float32)).cpu().numpy()
    assert np.abs(y - y_ref).max() <= 0.05, np.abs(y - y_ref).max()
    assert np.abs(y - y_ref).mean() <= 0.01


@pytest.fixture(scope="module")
def trained():
    system = ics.plummer_binaries(4096, seed=3)
    f, t = learned.generate(system, 300_000, steps=6, seed=3)
    blob, losses = learned.fit(f, t, epochs=3, batch=4096, lr=3e-3, seed=3)
    return blob, losses


def test_training_lowers_the_loss(trained):
    blob, losses = trained
    k = max(1, len(losses) // 10)
    assert losses[-k:].mean() < 0.5 * losses[:k].mean()


def _stats_for(system, guess, blob=None):
    with configured(guess=guess):
        if blob is not None:
            sk.load_mlp(blob)
        st = dev(system.soa())
        sk.get_stats(reset=True)
        sk.step(st, dev(system.m), system.dt, 2)
        sk.check()
        out = sk.get_stats(reset=True)
        r, v = ics.from_soa(st.cpu().numpy())
    return out, r, v


def test_learned_guess_cuts_iterations_and_keeps_parity(trained):
    blob, _ = trained
    system = ics.plummer_binaries(4096, seed=11)
    std, _, _ = _stats_for(system, sk.GUESS_STANDARD)
    tay, _, _ = _stats_for(system, sk.GUESS_TAYLOR)
    lrn, r, v = _stats_for(system, sk.GUESS_LEARNED, blob)
    m_std = std["iters"] / std["solves"]
    m_lrn = lrn["iters"] / lrn["solves"]
    print(f"mean evaluations standard {m_std:.4f} taylor {tay['iters'] / tay['solves']:.4f}"
          f" learned {m_lrn:.4f}; max {std['max_iters']} / {tay['max_iters']} /"
          f" {lrn['max_iters']}")
    assert m_lrn < m_std - 0.01
    assert lrn["max_iters"] <= std["max_iters"]
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, system.n - 1], rng.choice(system.n, 40, replace=False)]))
    rc, rs, vs = oracle.step_sample(system.m, system.r, system.v, system.dt, idx, 2,
                                    nthreads=NCPU)
    R = np.sqrt((r ** 2).sum(1).mean())
    V = np.sqrt((v ** 2).sum(1).mean())
    er = np.linalg.norm(r[idx] - rs, axis=1) / np.maximum(np.linalg.norm(rs, axis=1), R)
    ev = np.linalg.norm(v[idx] - vs, axis=1) / np.maximum(np.linalg.norm(vs, axis=1), V)
    assert er.max() <= TOL and ev.max() <= TOL, (er.max(), ev.max())


@pytest.mark.parametrize("order", [2, 1, -1])
def test_learned_guess_parity_small_systems(trained, order):
    blob, _ = trained
    for s in (ics.planetary(2), ics.random_cluster(97, seed=1, mass_spread=2.0)):
        with configured(guess=sk.GUESS_LEARNED):
            sk.load_mlp(blob)
            st = dev(s.soa())
            sk.step(st, dev(s.m), s.dt, order)
            sk.check()
            r, v = ics.from_soa(st.cpu().numpy())
        rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
        R = np.sqrt((rr ** 2).sum(1).mean())
        V = np.sqrt((vr ** 2).sum(1).mean())
        er = np.linalg.norm(r - rr, axis=1) / np.maximum(np.linalg.norm(rr, axis=1), R)
        ev = np.linalg.norm(v - vr, axis=1) / np.maximum(np.linalg.norm(vr, axis=1), V)
        assert er.max() <= TOL and ev.max() <= TOL


def test_learned_guess_in_the_batched_path(trained):
    blob, _ = trained
    ens = ics.ensemble(40, seed=12)
    with configured(guess=sk.GUESS_LEARNED):
        sk.load_mlp(blob)
        st = dev(ens.state)
        sk.step_batched(st, dev(ens.m), dev(ens.offsets, torch.int64), ens.offsets,
                        dev(ens.dt), 2, 2)
        sk.check()
        got = st.cpu().numpy()
    for k in range(ens.nsys):
        s = ens.system(k)
        a, b = int(ens.offsets[k]), int(ens.offsets[k + 1])
        rc, rr, vr = oracle.evolve(s.m, s.r, s.v, s.dt, 2)
        r, v = ics.from_soa(got[:, a:b])
        R = np.sqrt((rr ** 2).sum(1).mean())
        V = np.sqrt((vr ** 2).sum(1).mean())
        er = np.linalg.norm(r - rr, axis=1) / np.maximum(np.linalg.norm(rr, axis=1), R)
        ev = np.linalg.norm(v - vr, axis=1) / np.maximum(np.linalg.norm(vr, axis=1), V)
        assert er.max() <= 1e-12 and ev.max() <= 1e-12


def test_load_rejects_bad_blobs():
    lib = sk.load()
    bad = np.zeros(4687, dtype=np.float32)  # input scales of zero
    assert lib.sakura_load_mlp(bad.ctypes.data, bad.nbytes) == sk.E_ARG
    short = np.ones(100, dtype=np.float32)
    assert lib.sakura_load_mlp(short.ctypes.data, short.nbytes) == sk.E_ARG


@pytest.mark.parametrize("order", [2, -1])
def test_learned_guess_in_the_row_group_kernel(trained, order):
    # the network inside the row-group kernel (the default from 8192
    # particles), forced on a small system
    blob, _ = trained
    s = ics.random_cluster(700, seed=3, mass_spread=2.0)
    with configured(guess=sk.GUESS_LEARNED, flags=sk.FLAG_STATS | sk.FLAG_GROUPS):
        sk.load_mlp(blob)
        st = dev(s.soa())
        sk.step(st, dev(s.m), s.dt, order)
        sk.check()
        r, v = ics.from_soa(st.cpu().numpy())
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    R = np.sqrt((rr ** 2).sum(1).mean())
    V = np.sqrt((vr ** 2).sum(1).mean())
    er = np.linalg.norm(r - rr, axis=1) / np.maximum(np.linalg.norm(rr, axis=1), R)
    ev = np.linalg.norm(v - vr, axis=1) / np.maximum(np.linalg.norm(vr, axis=1), V)
    assert er.max() <= TOL and ev.max() <= TOL


def test_learned_guess_against_the_single_precision_seed(trained):
    # The shipped FP64 default starts each FP64 iteration from the root of a
    # single-precision solve of the pair (within ~1e-7 of the FP64 root) and
    # finishes with one FP64 evaluation and the Taylor carry: one evaluation
    # is the least the convergence test allows.  The network's guess carries
    # its BF16 output error (~1e-3 of the correction), too far for the carry,
    # so every pair it guesses takes a second evaluation.  The network can
    # therefore beat the method without a seed (t / r0, asserted above) but
    # not the seeded form; this records the evaluation counts that say why.
    blob, _ = trained
    system = ics.plummer_binaries(4096, seed=11)
    seed, _, _ = _stats_for(system, sk.GUESS_FP32)
    lrn, _, _ = _stats_for(system, sk.GUESS_LEARNED, blob)
    std, _, _ = _stats_for(system, sk.GUESS_STANDARD)
    m_seed = seed["iters"] / seed["solves"]
    m_lrn = lrn["iters"] / lrn["solves"]
    m_std = std["iters"] / std["solves"]
    print(f"FP64 evaluations per solve: seed {m_seed:.4f} (carried"
          f" {seed['carries'] / seed['solves']:.4f}), learned {m_lrn:.4f}, standard {m_std:.4f}")
    assert m_seed < 1.01 and seed["carries"] >= 0.99 * seed["solves"]
    assert m_lrn > 1.99
    assert m_seed < m_lrn < m_std
