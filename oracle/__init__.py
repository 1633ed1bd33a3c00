"""CPU oracle for the Sakura integrator -- TEST INFRASTRUCTURE ONLY.

A plain FP64 statement of the method of Goncalves Ferrari, Boekholt &
Portegies Zwart (2014): the drift (Eq. 12), the W step with its per-pair maps
(Eqs. 19a/b, 26), the relative-to-absolute increment map (Eq. 23) and the
discrete second-order step (Eqs. 27a-d), with a universal-variable Kepler
solver (Eq. 18).  The arithmetic lives in ``sakura_oracle.c``; this module
compiles it with gcc and wraps it with ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package never imports the library.

Arrays here use the paper's listing layout: ``m[n]``, ``r[n][3]``, ``v[n][3]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sakura_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
E_ARG = -2
E_MASS = -3
E_COINCIDENT = -4
E_NONFINITE = -5
E_KEPLER = -6

PAIR_KEPLER = 0
PAIR_DKD = 1


class Stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("iters", ctypes.c_int64),
                ("max_iters", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (gcc, no contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            D = ctypes.c_double
            P = ctypes.POINTER(ctypes.c_double)
            I64 = ctypes.c_int64
            lib.oracle_stumpff.argtypes = [D, P]
            lib.oracle_stumpff.restype = None
            lib.oracle_kepler_opt.argtypes = [D, D, P, P, P, P,
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.c_int, ctypes.c_int, D]
            lib.oracle_kepler_opt.restype = ctypes.c_int
            lib.oracle_step.argtypes = [I64, P, P, P, D, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(Stats)]
            lib.oracle_step.restype = ctypes.c_int
            lib.oracle_step_sample.argtypes = [I64, P, P, P, D, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int64), I64, P, P,
                                               ctypes.c_int]
            lib.oracle_step_sample.restype = ctypes.c_int
            lib.oracle_energy.argtypes = [I64, P, P, P, P, P, P]
            lib.oracle_energy.restype = ctypes.c_int
            lib.oracle_pair_classes.argtypes = [I64, P, P, P, D, ctypes.c_int, ctypes.c_int,
                                                D, D, D,
                                                ctypes.POINTER(ctypes.c_uint8), P, P]
            lib.oracle_pair_classes.restype = I64
            lib.oracle_version.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec3(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3))


def stumpff(x: float) -> np.ndarray:
    """c_0..c_3 at x (series below |x| = 0.1, closed forms above)."""
    out = np.zeros(4)
    _load().oracle_stumpff(float(x), _dp(out))
    return out


def kepler(tau: float, m: float, r0, v0, *, max_iter: int = 50,
           use_bisection: bool = True, tol_eps: float = 4.0):
    """Exact two-body flow (Eq. 18) of the relative state (r0, v0) about total
    mass m over time tau.  Returns (r1, v1, iterations, status)."""
    r0 = _vec3(r0)
    v0 = _vec3(v0)
    r1 = np.zeros(3)
    v1 = np.zeros(3)
    it = ctypes.c_int(0)
    rc = _load().oracle_kepler_opt(float(tau), float(m), _dp(r0), _dp(v0), _dp(r1),
                                   _dp(v1), ctypes.byref(it), int(max_iter),
                                   int(bool(use_bisection)), float(tol_eps))
    return r1, v1, it.value, rc


def step(m, r, v, tau: float, order: int = 2, *, pair_solver: int = PAIR_KEPLER,
         nthreads: int = 1, stats: Stats | None = None):
    """One integrator step; returns (status, r_new, v_new) with copies of r, v."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    r = np.array(r, dtype=np.float64, order="C").reshape(-1, 3).copy()
    v = np.array(v, dtype=np.float64, order="C").reshape(-1, 3).copy()
    n = m.shape[0]
    assert r.shape == (n, 3) and v.shape == (n, 3)
    rc = _load().oracle_step(n, _dp(m), _dp(r), _dp(v), float(tau), int(order),
                             int(pair_solver), int(nthreads),
                             ctypes.byref(stats) if stats is not None else None)
    return rc, r, v


def step_sample(m, r, v, tau: float, idx, order: int = 2, *, nthreads: int = 1):
    """Post-step state of the particles listed in idx only (same values as
    ``step`` would give them).  Returns (status, r_idx [k,3], v_idx [k,3])."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    k = idx.shape[0]
    ro = np.zeros((k, 3))
    vo = np.zeros((k, 3))
    rc = _load().oracle_step_sample(m.shape[0], _dp(m), _dp(r), _dp(v), float(tau), int(order),
                                    idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), k,
                                    _dp(ro), _dp(vo), int(nthreads))
    return rc, ro, vo


def evolve(m, r, v, tau: float, nsteps: int, order: int = 2, **kw):
    """nsteps steps; returns (status, r, v)."""
    rc = OK
    for _ in range(nsteps):
        rc, r, v = step(m, r, v, tau, order, **kw)
        if rc != OK:
            break
    return rc, r, v


def energy(m, r, v):
    """(E, T, U, status) with compensated sums (Eqs. 1-3)."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    E = ctypes.c_double()
    T = ctypes.c_double()
    U = ctypes.c_double()
    rc = _load().oracle_energy(m.shape[0], _dp(m), _dp(r), _dp(v), ctypes.byref(E),
                               ctypes.byref(T), ctypes.byref(U))
    return E.value, T.value, U.value, rc


def pair_classes(m, r, v, tau: float, rule: int = 0, r_min: float = 0.1,
                 e_max: float = 0.9, e_hyp: float = 10.0, want_matrix: bool = False,
                 order: int = 2, want_values: bool = False):
    """Single-precision eligibility of every ordered pair of the step that
    starts from (r, v) (mixed-precision form): r = |r0| and e of the pair's
    Kepler input (Eq. 26), in double precision.  Returns (count, matrix or
    None), or (count, matrix, r2, e2) with the n x n squared separations and
    squared eccentricities when want_values."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    n = m.shape[0]
    want_matrix = want_matrix or want_values
    mat = np.zeros((n, n), dtype=np.uint8) if want_matrix else None
    ptr = mat.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if want_matrix else None
    r2 = np.zeros((n, n)) if want_values else None
    e2 = np.zeros((n, n)) if want_values else None
    cnt = _load().oracle_pair_classes(n, _dp(m), _dp(r), _dp(v), float(tau), int(order), int(rule),
                                      float(r_min), float(e_max), float(e_hyp), ptr,
                                      _dp(r2) if want_values else None,
                                      _dp(e2) if want_values else None)
    if want_values:
        return int(cnt), mat, r2, e2
    return int(cnt), mat


def version() -> str:
    return _load().oracle_version().decode()
