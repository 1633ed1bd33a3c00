"""GPU tests of the mixed-precision form (FP32 solves for distant, weakly
perturbing pairs; FP64 for the rest and for all accumulation).

* The pair classes the kernels use (exported by sakura_pair_classes) equal
  the oracle's double-precision rule on every pair except those within the
  single-precision decision's rounding band of a threshold
  (tests/mixed_band.py); the number of pairs the step solved in FP32 equals
  the exported class count, in both pair modes (the symmetric kernel decides
  once per unordered pair; the rule is symmetric in (i, j)).
* With a class rule that admits no pair, every pair goes through the per-warp
  FP64 queue and the step matches the FP64 oracle to 1e-12.
* Otherwise one step stays within the stated bound of the FP64 oracle
  (per-particle relative error, metric of the FP64 tests).
"""
import contextlib
import os

import numpy as np
import pytest

import oracle
from mixed_band import check_classes
from paper_1402_3325_gb300 import ics
from paper_1402_3325_gb300 import sakura as sk

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1
STEP_BOUND = 1e-8   # per-particle relative error of one mixed step vs the FP64 oracle


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_3325_gb300 import build
    build.build()
    sk.init(0, flags=sk.FLAG_STATS)
    yield
    sk.finalize()


@contextlib.contextmanager
def mixed(**opts):
    sk.init(0, flags=sk.FLAG_STATS, precision=sk.PREC_MIXED, **opts)
    try:
        yield
    finally:
        sk.init(0, flags=sk.FLAG_STATS)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def step_gpu(s, order=2, nsteps=1):
    st = dev(s.soa())
    m = dev(s.m)
    sk.get_stats(reset=True)
    for _ in range(nsteps):
        sk.step(st, m, s.dt, order)
    sk.check()
    stats = sk.get_stats(reset=True)
    r, v = ics.from_soa(st.cpu().numpy())
    return r, v, stats


def rel_err(r, v, rr, vr):
    R = np.sqrt((rr ** 2).sum(1).mean())
    V = np.sqrt((vr ** 2).sum(1).mean())
    er = np.linalg.norm(r - rr, axis=1) / np.maximum(np.linalg.norm(rr, axis=1), R)
    ev = np.linalg.norm(v - vr, axis=1) / np.maximum(np.linalg.norm(vr, axis=1), V)
    return float(er.max()), float(ev.max())


CASES = [
    ("bh2048-literal", lambda: ics.bh_cluster(2048, seed=3), 0),
    ("bh2048-hyp", lambda: ics.bh_cluster(2048, seed=3), 1),
    ("plummer1024-hyp", lambda: ics.plummer(1024, seed=5), 1),
    ("random300-hyp", lambda: ics.random_cluster(300, seed=7, mass_spread=2.0), 1),
]


PAIRS = [sk.PAIRS_SYMMETRIC, sk.PAIRS_ORDERED]


def classes_gpu(s, order):
    """The exported class matrix of the step from s (current configuration)."""
    return sk.pair_classes(dev(s.soa()), dev(s.m), s.dt, order).cpu().numpy()


def classes_checked(s, rule, order):
    """GPU class matrix, checked pair by pair against the oracle's rule."""
    got = classes_gpu(s, order)
    cnt, orc = oracle.pair_classes(s.m, s.r, s.v, s.dt, rule=rule, order=order,
                                   want_matrix=True)
    k = check_classes(got, orc, s.m, s.r, s.v, s.dt, order, rule)
    print(f"{s.name} rule {rule} order {order}: gpu {int(got.sum())} oracle {cnt} single-"
          f"precision pairs; {k} boundary pairs differ, all within the rounding band")
    return got


@pytest.mark.parametrize("pairs", PAIRS, ids=["symmetric", "ordered"])
@pytest.mark.parametrize("name,make,rule", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("order", [2, -1])
def test_mixed_class_count_and_accuracy(name, make, rule, order, pairs):
    s = make()
    with mixed(mixed_rule=rule, guess=sk.GUESS_TAYLOR, pair_mode=pairs):
        got = classes_checked(s, rule, order)
        r, v, st = step_gpu(s, order)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, order, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    print(f"{name} order {order}: fp32 pairs {st['fp32_pairs']} / {st['pairs']}"
          f" (classes {int(got.sum())}), err r {er:.2e} v {ev:.2e}")
    # every pair of the single-precision class converged in FP32 here
    assert st["fp32_pairs"] == int(got.sum())
    assert er <= STEP_BOUND and ev <= STEP_BOUND


@pytest.mark.parametrize("rule", [0, 1], ids=["literal", "hyp"])
def test_pair_classes_symmetric_and_zero_diagonal(rule):
    s = ics.random_cluster(500, seed=21, mass_spread=3.0)
    with mixed(mixed_rule=rule):
        got = classes_checked(s, rule, 2)
    assert (np.diag(got) == 0).all()
    np.testing.assert_array_equal(got, got.T)


@pytest.mark.parametrize("pairs", PAIRS, ids=["symmetric", "ordered"])
def test_mixed_without_fp32_pairs_is_fp64_exact(pairs):
    # r_min larger than the system: every pair takes the FP64 queue
    s = ics.random_cluster(700, seed=11, mass_spread=2.0)
    with mixed(mixed_r_min=1e6, pair_mode=pairs):
        r, v, st = step_gpu(s, 2)
    assert st["fp32_pairs"] == 0
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= 1e-12 and ev <= 1e-12, (er, ev)


@pytest.mark.parametrize("pairs", PAIRS, ids=["symmetric", "ordered"])
def test_mixed_energy_drift_bh_cluster(pairs):
    # BH cluster, hyperbolic rule: 16 steps of the mixed and the FP64 form
    # from the same start; energies from the oracle's compensated sum
    s = ics.bh_cluster(2048, seed=2)
    E0 = oracle.energy(s.m, s.r, s.v)[0]
    with mixed(mixed_rule=1, guess=sk.GUESS_TAYLOR, pair_mode=pairs):
        rm, vm, stm = step_gpu(s, 2, nsteps=16)
    rf, vf, _ = step_gpu(s, 2, nsteps=16)
    Em = oracle.energy(s.m, rm, vm)[0]
    Ef = oracle.energy(s.m, rf, vf)[0]
    print(f"dE/E fp64 {abs(Ef / E0 - 1):.3e} mixed {abs(Em / E0 - 1):.3e}"
          f" |Em-Ef|/|E| {abs(Em - Ef) / abs(E0):.3e} fp32 share"
          f" {stm['fp32_pairs'] / stm['pairs']:.3f}")
    assert abs(Em - Ef) <= 1e-9 * abs(E0)


@pytest.mark.parametrize("guess", [sk.GUESS_TAYLOR, sk.GUESS_FP32], ids=["taylor", "seed"])
@pytest.mark.parametrize("blocks", [1, 7])
@pytest.mark.parametrize("rule", [0, 1], ids=["literal", "hyp"])
def test_mixed_queue_across_segments(rule, blocks, guess):
    # few blocks, each over many windows and groups: FP64-class pairs queued
    # across the tiles of a window are solved together and added in queue
    # order; with the seed they start from a single-precision solve
    s = ics.bh_cluster(2048, seed=11)
    with mixed(mixed_rule=rule, guess=guess, pair_mode=sk.PAIRS_SYMMETRIC,
               grid_blocks=blocks):
        r, v, st = step_gpu(s, 2)
        r2, v2, _ = step_gpu(s, 2)
        got = classes_checked(s, rule, 2)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert st["fp32_pairs"] == int(got.sum())
    assert er <= STEP_BOUND and ev <= STEP_BOUND, (er, ev)
    np.testing.assert_array_equal(r, r2)
    np.testing.assert_array_equal(v, v2)


@pytest.mark.parametrize("guess", [sk.GUESS_STANDARD, sk.GUESS_FP32], ids=["standard", "seed"])
@pytest.mark.parametrize("blocks", [1, 5, 0])
def test_mixed_all_fp64_queue_across_segments_is_fp64_exact(blocks, guess):
    # every pair through the FP64 queue, whose entries span the tiles of a
    # window; the FP64 solves match the oracle to the FP64 bound
    s = ics.random_cluster(700, seed=12, mass_spread=2.0)
    with mixed(mixed_r_min=1e6, pair_mode=sk.PAIRS_SYMMETRIC, grid_blocks=blocks, guess=guess):
        r, v, st = step_gpu(s, 2)
    assert st["fp32_pairs"] == 0
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    assert er <= 1e-12 and ev <= 1e-12, (er, ev)


@pytest.mark.parametrize("guess", [sk.GUESS_TAYLOR, sk.GUESS_FP32], ids=["taylor", "seed"])
@pytest.mark.parametrize("kernel", [sk.FLAG_TILES, sk.FLAG_GROUPS], ids=["tiles", "groups"])
@pytest.mark.parametrize("rule", [0, 1], ids=["literal", "hyp"])
def test_mixed_tile_and_row_group_kernels(rule, kernel, guess):
    # the FP64 tile kernel with an inline class test (forced with
    # SAKURA_FLAG_TILES under either rule), and in row groups
    # (SAKURA_FLAG_GROUPS): the FP64 row-group kernel with the inline test
    # under the literal rule, the row-group mixed kernel under the
    # hyperbolic rule: same classes, oracle within the step bound, repeat
    # runs bit-identical
    s = ics.bh_cluster(2048, seed=3)
    sk.init(0, flags=sk.FLAG_STATS | kernel, precision=sk.PREC_MIXED, mixed_rule=rule,
            guess=guess)
    try:
        got = classes_checked(s, rule, 2)
        r, v, st = step_gpu(s, 2)
        r2, v2, _ = step_gpu(s, 2)
    finally:
        sk.init(0, flags=sk.FLAG_STATS)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    print(f"rule {rule} kernel {kernel}: fp32 pairs {st['fp32_pairs']}, err r {er:.2e} v {ev:.2e}")
    assert st["fp32_pairs"] == int(got.sum())
    assert st["group_launches"] == (1 if kernel == sk.FLAG_GROUPS else 0)
    assert er <= STEP_BOUND and ev <= STEP_BOUND
    np.testing.assert_array_equal(r, r2)
    np.testing.assert_array_equal(v, v2)


@pytest.mark.parametrize("guess", [sk.GUESS_TAYLOR, sk.GUESS_FP32], ids=["taylor", "seed"])
@pytest.mark.parametrize("kernel", [sk.FLAG_TILES, sk.FLAG_GROUPS], ids=["tiles", "groups"])
def test_literal_rule_inline_test_with_most_pairs_single_precision(kernel, guess):
    # a wide literal rule (e_max = 1e15: every pair beyond r_min) sends most
    # pairs through the inline FP32 solve of the FP64 kernels, on tiles and
    # in row groups, at a ragged size
    s = ics.random_cluster(1000, seed=17, mass_spread=2.0)
    emax = 1e15
    sk.init(0, flags=sk.FLAG_STATS | kernel, precision=sk.PREC_MIXED, mixed_rule=0,
            mixed_e_max=emax, guess=guess)
    try:
        got = classes_gpu(s, 2)
        r, v, st = step_gpu(s, 2)
        r2, v2, _ = step_gpu(s, 2)
    finally:
        sk.init(0, flags=sk.FLAG_STATS)
    cnt, orc = oracle.pair_classes(s.m, s.r, s.v, s.dt, rule=0, e_max=emax, want_matrix=True)
    k = check_classes(got, orc, s.m, s.r, s.v, s.dt, 2, 0, e_max=emax)
    rc, rr, vr = oracle.step(s.m, s.r, s.v, s.dt, 2, nthreads=NCPU)
    er, ev = rel_err(r, v, rr, vr)
    n = s.n
    print(f"kernel {kernel}: classes {int(got.sum())} of {n * (n - 1)} ({k} boundary pairs"
          f" differ), fp32 pairs {st['fp32_pairs']}, err r {er:.2e} v {ev:.2e}")
    assert got.sum() > 0.5 * n * (n - 1)
    assert st["fp32_pairs"] == int(got.sum())
    assert st["group_launches"] == (1 if kernel == sk.FLAG_GROUPS else 0)
    assert er <= STEP_BOUND and ev <= STEP_BOUND
    np.testing.assert_array_equal(r, r2)
    np.testing.assert_array_equal(v, v2)
