"""Python binding of the C ABI in include/sakura.h (ctypes, marshalling only).

Every step of the method runs in libsakura.so's CUDA kernels; this module
only converts arguments.  PyTorch supplies device memory and streams: device
arrays are passed as ``torch.Tensor`` objects on the CUDA device (float64,
contiguous), whose data pointers go straight to the library.

There is no CPU fallback: if libsakura.so is missing or cannot be loaded an
``ImportError``/``RuntimeError`` is raised.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsakura.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "sakura.h")

OK = 0
E_NOINIT = -1
E_ARG = -2
E_MASS = -3
E_COINCIDENT = -4
E_NONFINITE = -5
E_KEPLER = -6
E_CUDA = -7
E_TIMEOUT = -8
E_NOMEM = -9

PAIRS_ORDERED = 0
PAIRS_SYMMETRIC = 1
PREC_FP64 = 0
PREC_MIXED = 1
PREC_DF64 = 2
MIXED_RULE_LITERAL = 0
MIXED_RULE_HYP = 1
GUESS_STANDARD = 0
GUESS_LEARNED = 1
GUESS_TAYLOR = 2
GUESS_FP32 = 3
FLAG_SYNC_CHECK = 1
FLAG_STATS = 2
FLAG_TIMING = 4
FLAG_NO_AUTOTUNE = 8
FLAG_NO_SMALL = 16
FLAG_TILES = 32
FLAG_GROUPS = 64
# largest system of the single-block kernel (csrc/step_small.cuh)
SMALL_MAX_N = 20
BATCH_MAX_N = 64

MLP_FLOATS = 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1 + 6 + 6 + 2


class Config(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("precision", ctypes.c_int),
        ("mixed_rule", ctypes.c_int),
        ("mixed_r_min", ctypes.c_double),
        ("mixed_e_max", ctypes.c_double),
        ("mixed_e_hyp", ctypes.c_double),
        ("guess", ctypes.c_int),
        ("kepler_tol", ctypes.c_double),
        ("kepler_max_iter", ctypes.c_int),
        ("kepler_bisection", ctypes.c_int),
        ("flags", ctypes.c_uint),
        ("block_warps", ctypes.c_int),
        ("grid_blocks", ctypes.c_int),
        ("pair_mode", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in
                ("steps", "pairs", "iters", "max_iters", "warp_slots", "fp32_pairs",
                 "fallbacks", "solves", "timed_launches")] + [
                     ("pair_kernel_ms", ctypes.c_double), ("carries", ctypes.c_int64),
                     ("group_launches", ctypes.c_int64)]

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k, t in self._fields_ if t is ctypes.c_int64}
        d["pair_kernel_ms"] = float(self.pair_kernel_ms)
        return d


class SakuraError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


_lib = None


def load(path: str = LIB_PATH):
    """Load libsakura.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_1402_3325_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    D = ctypes.c_double
    I = ctypes.c_int
    lib.sakura_default_config.argtypes = [ctypes.POINTER(Config)]
    lib.sakura_default_config.restype = None
    lib.sakura_init.argtypes = [ctypes.POINTER(Config)]
    lib.sakura_finalize.argtypes = []
    lib.sakura_set_stream.argtypes = [P]
    lib.sakura_step.argtypes = [P, P, I64, D, I]
    lib.sakura_evolve.argtypes = [P, P, I64, D, I, I]
    lib.sakura_evolve_host.argtypes = [P, P, I64, D, I, I]
    lib.sakura_energy.argtypes = [P, P, I64, ctypes.POINTER(D)]
    lib.sakura_step_batched.argtypes = [P, P, P, P, I, P, I, I]
    lib.sakura_load_mlp.argtypes = [P, ctypes.c_size_t]
    lib.sakura_get_stats.argtypes = [ctypes.POINTER(Stats), I]
    lib.sakura_step_noalloc.argtypes = [P, P, I64, D, I, P]
    lib.sakura_sample_pairs.argtypes = [P, P, I64, D, I, P, I64, P, P, P]
    lib.sakura_pair_classes.argtypes = [P, P, I64, D, I, P]
    lib.sakura_mlp_grad.argtypes = [P, P, P, P, I64, P, P]
    lib.sakura_mlp_train.argtypes = [P, P, P, P, I64, I64, I, ctypes.c_float, P]
    lib.sakura_mlp_eval.argtypes = [P, I64, P]
    lib.sakura_batched_tuning.argtypes = [ctypes.POINTER(I), ctypes.POINTER(I),
                                          ctypes.POINTER(D)]
    lib.sakura_batched_schedule.argtypes = [P, I, P, P, ctypes.POINTER(I)]
    lib.sakura_check.argtypes = []
    lib.sakura_strerror.argtypes = [I]
    lib.sakura_strerror.restype = ctypes.c_char_p
    for name in ("sakura_init", "sakura_finalize", "sakura_set_stream", "sakura_step",
                 "sakura_evolve", "sakura_evolve_host", "sakura_energy", "sakura_step_batched",
                 "sakura_load_mlp", "sakura_get_stats", "sakura_check",
                 "sakura_step_noalloc", "sakura_batched_tuning", "sakura_batched_schedule",
                 "sakura_sample_pairs", "sakura_pair_classes",
                 "sakura_mlp_grad", "sakura_mlp_train", "sakura_mlp_eval"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def header_functions(header: str = HEADER):
    """Names of the functions include/sakura.h declares."""
    with open(header) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sakura_\w+)\s*\(", text)))


def strerror(code: int) -> str:
    return load().sakura_strerror(int(code)).decode()


def _check(code: int, where: str):
    if code != OK:
        raise SakuraError(code, where)


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (no copy)."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def default_config() -> Config:
    c = Config()
    load().sakura_default_config(ctypes.byref(c))
    return c


def init(device: int = 0, stream=None, **options) -> Config:
    """Create the library context.  options: any Config field by name."""
    c = default_config()
    c.device = int(device)
    if stream is not None:
        c.stream = ctypes.c_void_p(int(stream))
    for k, v in options.items():
        if not hasattr(c, k):
            raise TypeError(f"unknown option {k}")
        setattr(c, k, v)
    _check(load().sakura_init(ctypes.byref(c)), "sakura_init")
    return c


def finalize():
    _check(load().sakura_finalize(), "sakura_finalize")


def set_stream(stream):
    _check(load().sakura_set_stream(ctypes.c_void_p(int(stream))), "sakura_set_stream")


def step(state, masses, dt: float, order: int = 2):
    """One step in place on a CUDA float64 state [6, n] with masses [n]."""
    n = masses.shape[0]
    if tuple(state.shape) != (6, n):
        raise ValueError("state must have shape (6, n)")
    _check(load().sakura_step(_ptr(state), _ptr(masses), n, float(dt), int(order)),
           "sakura_step")


def evolve(state, masses, dt: float, order: int = 2, nsteps: int = 1):
    """nsteps steps in place on a CUDA float64 state [6, n] with masses [n]
    (one launch for the systems of the single-block kernel)."""
    n = masses.shape[0]
    if tuple(state.shape) != (6, n):
        raise ValueError("state must have shape (6, n)")
    _check(load().sakura_evolve(_ptr(state), _ptr(masses), n, float(dt), int(order),
                                int(nsteps)), "sakura_evolve")


NOALLOC_MAX_N = 65536


def step_noalloc(state, masses, dt: float, order: int = 2, stream=None):
    """sakura_step without any device allocation (file-scope scratch, n <=
    NOALLOC_MAX_N), for callers that cannot call cudaMalloc; synchronises."""
    n = masses.shape[0]
    if tuple(state.shape) != (6, n):
        raise ValueError("state must have shape (6, n)")
    s = ctypes.c_void_p(int(stream)) if stream is not None else None
    _check(load().sakura_step_noalloc(_ptr(state), _ptr(masses), n, float(dt), int(order), s),
           "sakura_step_noalloc")


def evolve_host(state, masses, dt: float, order: int = 2, nsteps: int = 1):
    """nsteps steps on host numpy arrays (float64, C-contiguous); state is
    updated in place."""
    import numpy as np
    assert state.dtype == np.float64 and state.flags.c_contiguous
    assert masses.dtype == np.float64 and masses.flags.c_contiguous
    n = masses.shape[0]
    assert state.shape == (6, n)
    _check(load().sakura_evolve_host(state.ctypes.data, masses.ctypes.data, n, float(dt),
                                     int(order), int(nsteps)), "sakura_evolve_host")


def energy(state, masses) -> float:
    n = masses.shape[0]
    out = ctypes.c_double()
    _check(load().sakura_energy(_ptr(state), _ptr(masses), n, ctypes.byref(out)),
           "sakura_energy")
    return out.value


def step_batched(state, masses, offsets, host_offsets, dt, order: int = 2, nsteps: int = 1):
    """Batched independent systems (CSR offsets); all device tensors except
    host_offsets (numpy int64)."""
    nsys = offsets.shape[0] - 1
    _check(load().sakura_step_batched(_ptr(state), _ptr(masses), _ptr(offsets),
                                      host_offsets.ctypes.data, nsys, _ptr(dt), int(order),
                                      int(nsteps)), "sakura_step_batched")


def batched_tuning():
    """(warps per block, blocks, {warps: ms}) chosen by the batched autotuner."""
    w = ctypes.c_int()
    b = ctypes.c_int()
    t = (ctypes.c_double * 4)()
    _check(load().sakura_batched_tuning(ctypes.byref(w), ctypes.byref(b), t),
           "sakura_batched_tuning")
    return w.value, b.value, {k: t[c] for c, k in enumerate((1, 2, 4, 8))}


def batched_schedule(host_offsets):
    """The batched work schedule for these systems (host only): a list of
    tasks, each a list of system indices, longest first."""
    import numpy as np
    off = np.ascontiguousarray(host_offsets, dtype=np.int64)
    nsys = off.shape[0] - 1
    tb = np.zeros(nsys + 1, dtype=np.int32)
    ts = np.zeros(max(nsys, 1), dtype=np.int32)
    nt = ctypes.c_int()
    _check(load().sakura_batched_schedule(off.ctypes.data, nsys, tb.ctypes.data, ts.ctypes.data,
                                          ctypes.byref(nt)), "sakura_batched_schedule")
    return [ts[tb[t]:tb[t + 1]].tolist() for t in range(nt.value)]


def pair_classes(state, masses, dt: float, order: int = 2):
    """The mixed form's precision class of every ordered pair of the step
    from state (CUDA uint8 [n, n], 1 = single precision), under the
    configured rule and thresholds."""
    import torch
    n = masses.shape[0]
    if tuple(state.shape) != (6, n):
        raise ValueError("state must have shape (6, n)")
    out = torch.empty((n, n), dtype=torch.uint8, device=state.device)
    _check(load().sakura_pair_classes(_ptr(state), _ptr(masses), n, float(dt), int(order),
                                      _ptr(out)), "sakura_pair_classes")
    return out


def load_mlp(weights):
    """weights: numpy float32 array of MLP_FLOATS values (see sakura.h)."""
    import numpy as np
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(load().sakura_load_mlp(w.ctypes.data, w.nbytes), "sakura_load_mlp")


MLP_PARAMS = 4673


def sample_pairs(state, masses, dt: float, pair_ids, order: int = 2, want_iters: bool = False):
    """Features [count, 6], targets [count] (and iterations) of the given
    ordered pairs (device int64 tensor of i * n + j), as CUDA tensors."""
    import torch
    n = masses.shape[0]
    count = int(pair_ids.shape[0])
    feat = torch.empty((count, 6), dtype=torch.float32, device=state.device)
    tgt = torch.empty((count,), dtype=torch.float32, device=state.device)
    its = torch.empty((count,), dtype=torch.int32, device=state.device) if want_iters else None
    _check(load().sakura_sample_pairs(_ptr(state), _ptr(masses), n, float(dt), int(order),
                                      _ptr(pair_ids), count, _ptr(feat), _ptr(tgt),
                                      _ptr(its) if its is not None else None),
           "sakura_sample_pairs")
    return (feat, tgt, its) if want_iters else (feat, tgt)


def mlp_grad(params, norm, features, targets):
    """(loss, gradient) of the network on one batch; all CUDA float32 tensors."""
    import torch
    grad = torch.empty_like(params)
    loss = torch.empty((1,), dtype=torch.float32, device=params.device)
    _check(load().sakura_mlp_grad(_ptr(params), _ptr(norm), _ptr(features), _ptr(targets),
                                  int(targets.shape[0]), _ptr(grad), _ptr(loss)),
           "sakura_mlp_grad")
    return float(loss.item()), grad


def mlp_train(params, norm, features, targets, batch: int, epochs: int, lr: float):
    """Adam training in place; returns the minibatch losses (CUDA tensor)."""
    import torch
    ns = int(targets.shape[0])
    steps = epochs * (ns // min(batch, ns))
    losses = torch.empty((max(1, steps),), dtype=torch.float32, device=params.device)
    _check(load().sakura_mlp_train(_ptr(params), _ptr(norm), _ptr(features), _ptr(targets), ns,
                                   int(batch), int(epochs), float(lr), _ptr(losses)),
           "sakura_mlp_train")
    return losses[:steps]


def mlp_eval(features):
    """Output of the loaded network for raw features (CUDA float32 [k, 6])."""
    import torch
    out = torch.empty((features.shape[0],), dtype=torch.float32, device=features.device)
    _check(load().sakura_mlp_eval(_ptr(features), int(features.shape[0]), _ptr(out)),
           "sakura_mlp_eval")
    return out


def get_stats(reset: bool = False) -> dict:
    s = Stats()
    _check(load().sakura_get_stats(ctypes.byref(s), int(bool(reset))), "sakura_get_stats")
    return s.as_dict()


def check():
    """Synchronise and raise on a pending device fault."""
    _check(load().sakura_check(), "sakura_check")


def check_code() -> int:
    return int(load().sakura_check())
