"""The C ABI library builds, loads without a GPU and exports every function
that include/sakura.h declares.  No compute calls are made here."""
import ctypes

import pytest

from paper_1402_3325_gb300 import build as sk_build
from paper_1402_3325_gb300 import sakura as sk


@pytest.fixture(scope="module")
def lib():
    sk_build.build()
    return sk.load()


def test_header_declares_the_boundary():
    names = sk.header_functions()
    for required in ("sakura_init", "sakura_step", "sakura_energy", "sakura_finalize",
                     "sakura_step_batched", "sakura_load_mlp", "sakura_get_stats",
                     "sakura_strerror"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    raw = ctypes.CDLL(sk.LIB_PATH)
    missing = [n for n in sk.header_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_strerror_and_noinit_without_gpu(lib):
    assert sk.strerror(0) == "ok"
    assert "Kepler" in sk.strerror(sk.E_KEPLER)
    # before sakura_init every call reports E_NOINIT and touches no device
    assert lib.sakura_step(None, None, 4, 0.1, 2) == sk.E_NOINIT
    assert lib.sakura_check() == sk.E_NOINIT


def test_default_config_values(lib):
    c = sk.default_config()
    assert c.kepler_tol == 4.0 and c.kepler_max_iter == 50 and c.kepler_bisection == 1
    assert c.mixed_r_min == 0.1 and c.mixed_e_max == 0.9 and c.mixed_e_hyp == 10.0
    assert c.pair_mode == sk.PAIRS_SYMMETRIC
    assert ctypes.sizeof(sk.Config) >= 80


def test_mlp_size_constant_matches_header():
    with open(sk.HEADER) as fh:
        assert "4687" in fh.read()
    assert sk.MLP_FLOATS == 4687


def test_flag_and_small_limit_constants_match_the_sources():
    import os
    import re
    with open(sk.HEADER) as fh:
        hdr = fh.read()
    for name in ("SYNC_CHECK", "STATS", "TIMING", "NO_AUTOTUNE", "NO_SMALL"):
        m = re.search(r"#define SAKURA_FLAG_%s (\d+)u" % name, hdr)
        assert m and int(m.group(1)) == getattr(sk, "FLAG_" + name), name
    src = os.path.join(os.path.dirname(sk.LIB_PATH), "csrc", "step_small.cuh")
    with open(src) as fh:
        m = re.search(r"constexpr int kSmallMaxN = (\d+);", fh.read())
    assert m and int(m.group(1)) == sk.SMALL_MAX_N


def test_evolve_entry_points_without_gpu(lib):
    assert lib.sakura_evolve(None, None, 4, 0.1, 2, 3) == sk.E_NOINIT


def test_no_cpu_fallback(monkeypatch, tmp_path):
    # the binding takes CUDA tensors only, and a missing library is an error,
    # not a detour through host code
    torch = pytest.importorskip("torch")
    state = torch.zeros((6, 4), dtype=torch.float64)
    mass = torch.ones(4, dtype=torch.float64)
    for call in (lambda: sk.step(state, mass, 0.1, 2), lambda: sk.evolve(state, mass, 0.1, 2, 3),
                 lambda: sk.energy(state, mass)):
        with pytest.raises(ValueError, match="CUDA tensor"):
            call()
    monkeypatch.setattr(sk, "_lib", None)
    with pytest.raises(ImportError, match="no CPU fallback"):
        sk.load(str(tmp_path / "libsakura.so"))
