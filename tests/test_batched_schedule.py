"""The batched work schedule (csrc/step_batched.cu: build_batch_schedule),
through sakura_batched_schedule on the host, without a GPU: every system is
in exactly one task, a task holds at most 64 particles (its pairs then fit
the kernel's 2016 increment slots), tasks come longest first, and on the
4096-system ensemble the dense packing keeps at least 98 % of the lanes of
its 32-pair chunks busy."""
import numpy as np
import pytest

from paper_1402_3325_gb300 import build as sk_build
from paper_1402_3325_gb300 import ics
from paper_1402_3325_gb300 import sakura as sk


@pytest.fixture(scope="module", autouse=True)
def lib():
    sk_build.build()
    return sk.load()


def offsets_of(sizes):
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return off


def check(sizes):
    tasks = sk.batched_schedule(offsets_of(sizes))
    assert sorted(k for t in tasks for k in t) == list(range(len(sizes)))
    parts = [sum(sizes[k] for k in t) for t in tasks]
    pairs = [sum(sizes[k] * (sizes[k] - 1) // 2 for k in t) for t in tasks]
    assert max(parts) <= 64 and max(pairs) <= 2016
    assert pairs == sorted(pairs, reverse=True)
    return tasks, pairs


def test_ensemble_schedule_fills_the_lanes():
    ens = ics.ensemble(4096, seed=0)
    sizes = [int(x) for x in ens.offsets[1:] - ens.offsets[:-1]]
    tasks, pairs = check(sizes)
    fill = sum(pairs) / (32 * sum((p + 31) // 32 for p in pairs))
    assert fill >= 0.98, fill
    # best fit leaves little room: on average tasks are nearly full
    assert sum(sizes) / (64 * len(tasks)) >= 0.95


@pytest.mark.parametrize("lo,hi", [(1, 64), (1, 3), (64, 64), (30, 40)])
def test_random_mixes(lo, hi):
    sizes = [int(x) for x in np.random.default_rng(lo * 100 + hi).integers(lo, hi + 1, 500)]
    check(sizes)


def test_single_system_and_errors():
    assert sk.batched_schedule(np.array([0, 9])) == [[0]]
    lib = sk.load()
    import ctypes
    tb = np.zeros(3, dtype=np.int32)
    ts = np.zeros(2, dtype=np.int32)
    nt = ctypes.c_int()
    for off in ([0, 65], [0, 0], [1, 5]):
        o = np.array(off, dtype=np.int64)
        assert lib.sakura_batched_schedule(o.ctypes.data, 1, tb.ctypes.data, ts.ctypes.data,
                                           ctypes.byref(nt)) == sk.E_ARG
