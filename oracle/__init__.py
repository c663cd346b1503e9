"""Plain FP64 CPU oracle for the worldline Wilson-loop path.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only users.  Nothing in the product
imports this package, and this package imports nothing from the product.

The per-loop arithmetic (Philox, Box-Muller, unit loops, segment integrals,
group sums) is plain C in ``wln_oracle.c``; the statistics (group means,
standard errors, jackknife, covariance) and the proper-time / radius
quadrature are plain numpy in ``stats.py``.  Every function states the
passage of Mazur & Heyl, arXiv:1407.7486, that it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wln_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libwln_oracle.so")

# The one command that builds the oracle (also issued by the package build step).
GCC_CMD = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           "-std=c11", "-o", _LIB, _SRC, "-lm"]

_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(GCC_CMD)
    return _LIB


class _Profile(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("F", ctypes.c_double), ("lam", ctypes.c_double), ("B", ctypes.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    lib.wln_oracle_loop_values.argtypes = [f64p, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.POINTER(_Profile), f64p, ctypes.c_int32, f64p,
                                           ctypes.c_int32, f64p, ctypes.c_int32]
    lib.wln_oracle_shuffle.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, i32p]
    lib.wln_oracle_philox4x32.argtypes = [u32p, u32p, ctypes.c_int, u32p]
    lib.wln_oracle_philox4x64.argtypes = [u64p, u64p, ctypes.c_int, u64p]
    lib.wln_oracle_philox_stream.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int32, u32p]
    lib.wln_oracle_raw_increments.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, f64p]
    lib.wln_oracle_gen_loops.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int32, f64p, ctypes.c_int32]
    lib.wln_oracle_gen_dloops.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int32, f64p, ctypes.c_int32]
    lib.wln_oracle_loop_phase_spin.argtypes = [f64p, ctypes.c_int32, ctypes.POINTER(_Profile),
                                               ctypes.c_double, ctypes.c_double,
                                               ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double)]
    lib.wln_oracle_phase_spin_many.argtypes = [f64p, ctypes.c_int64, ctypes.c_int32,
                                               ctypes.POINTER(_Profile), ctypes.c_double,
                                               ctypes.c_double, f64p, f64p, ctypes.c_int32]
    lib.wln_oracle_phase_abs_many.argtypes = [f64p, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.POINTER(_Profile), ctypes.c_double,
                                              ctypes.c_double, f64p, ctypes.c_int32]
    lib.wln_oracle_wilson_terms.argtypes = [ctypes.c_double, ctypes.c_double, f64p]
    lib.wln_oracle_group_sums.argtypes = [f64p, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.POINTER(_Profile), f64p, ctypes.c_int32,
                                          f64p, ctypes.c_int32, ctypes.c_int32, f64p,
                                          ctypes.c_int32]
    lib.wln_oracle_max_threads.restype = ctypes.c_int32
    _lib = lib
    return lib


def max_threads() -> int:
    return int(_load().wln_oracle_max_threads())


def _prof(profile) -> _Profile:
    return _Profile(int(profile.kind), 0, float(profile.F), float(profile.lam), float(profile.B))


# --------------------------------------------------------------------------
# Philox (Salmon et al., SC'11) -- the counter-based stream behind the loops.
# --------------------------------------------------------------------------
def philox4x32(ctr, key, rounds: int = 10) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    _load().wln_oracle_philox4x32(np.ascontiguousarray(ctr, np.uint32),
                                  np.ascontiguousarray(key, np.uint32), rounds, out)
    return out


def philox4x64(ctr, key, rounds: int = 10) -> np.ndarray:
    out = np.zeros(4, np.uint64)
    _load().wln_oracle_philox4x64(np.ascontiguousarray(ctr, np.uint64),
                                  np.ascontiguousarray(key, np.uint64), rounds, out)
    return out


def philox_stream(seed: int, n_loops: int, n_calls: int, loop0: int = 0) -> np.ndarray:
    """u32[n_loops][n_calls][4]: call j of loop l uses counter (j, l, 0, 0)."""
    out = np.zeros((n_loops, n_calls, 4), np.uint32)
    _load().wln_oracle_philox_stream(seed, loop0, n_loops, n_calls, out)
    return out


# --------------------------------------------------------------------------
# Unit loops (Sec. "Loop Generation").
# --------------------------------------------------------------------------
def raw_increments(seed: int, loop: int, ppl: int) -> np.ndarray:
    """Gaussian increments (variance 2/N per component) before closure: [2][N]."""
    xi = np.zeros((2, ppl), np.float64)
    _load().wln_oracle_raw_increments(seed, loop, ppl, xi)
    return xi


def gen_loops(seed: int, n_loops: int, ppl: int, loop0: int = 0, threads: int = 0) -> np.ndarray:
    """CM-centred closed unit loops y[l][c][k] (c = 0: x, 1: y)."""
    y = np.zeros((n_loops, 2, ppl), np.float64)
    _load().wln_oracle_gen_loops(seed, loop0, n_loops, ppl, y, threads or max_threads())
    return y


def gen_dloops(seed: int, n_loops: int, ppl: int, loop0: int = 0, threads: int = 0) -> np.ndarray:
    """d-loops (Eqs. yn2, ynk), CM-centred: y[l][c][k]."""
    y = np.zeros((n_loops, 2, ppl), np.float64)
    _load().wln_oracle_gen_dloops(seed, loop0, n_loops, ppl, y, threads or max_threads())
    return y


# --------------------------------------------------------------------------
# Wilson loops (Sec. "Wilson Loop", Eqs. wilsonloop, rhoi-Ci, Wfermfpl).
# --------------------------------------------------------------------------
def loop_phase_spin(y_loop: np.ndarray, profile, rho_cm: float, T: float):
    """(e * closed line integral of A, e * int_0^T B dtau) for one loop y[2][N]."""
    y_loop = np.ascontiguousarray(y_loop, np.float64)
    ph, sp = ctypes.c_double(), ctypes.c_double()
    _load().wln_oracle_loop_phase_spin(y_loop, y_loop.shape[-1], ctypes.byref(_prof(profile)),
                                       float(rho_cm), float(T), ctypes.byref(ph), ctypes.byref(sp))
    return ph.value, sp.value


def phase_spin(y: np.ndarray, profile, rho_cm: float, T: float, threads: int = 0):
    """Per-loop phase and spin arrays for loops y[l][2][N] at one point."""
    y = np.ascontiguousarray(y, np.float64)
    n = y.shape[0]
    ph = np.zeros(n, np.float64)
    sp = np.zeros(n, np.float64)
    _load().wln_oracle_phase_spin_many(y, n, y.shape[-1], ctypes.byref(_prof(profile)),
                                       float(rho_cm), float(T), ph, sp, threads or max_threads())
    return ph, sp


def phase_abs(y: np.ndarray, profile, rho_cm: float, T: float, threads: int = 0) -> np.ndarray:
    """Per loop, the sum over segments of |segment phase| (condition number of
    the phase sum, used to size rounding-error bars)."""
    y = np.ascontiguousarray(y, np.float64)
    out = np.zeros(y.shape[0], np.float64)
    _load().wln_oracle_phase_abs_many(y, y.shape[0], y.shape[-1], ctypes.byref(_prof(profile)),
                                      float(rho_cm), float(T), out, threads or max_threads())
    return out


def wilson_terms(phase: float, spin: float) -> np.ndarray:
    """[W_scal - 1, W_ferm - 1, sin phase, (W_scal - 1)^2, (W_ferm - 1)^2] of one loop."""
    w = np.zeros(5, np.float64)
    _load().wln_oracle_wilson_terms(float(phase), float(spin), w)
    return w


def group_sums(y: np.ndarray, profile, rho, T, n_groups: int, threads: int = 0) -> np.ndarray:
    """Group sums [n_T * n_rho][G][5] of one profile (rho fastest), Sec. "Grouping Worldlines"."""
    y = np.ascontiguousarray(y, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    n_loops, _, ppl = y.shape
    if n_loops % n_groups:
        raise ValueError("each group must hold the same number of loops")
    out = np.zeros((len(T) * len(rho), n_groups, 5), np.float64)
    _load().wln_oracle_group_sums(y, n_loops, ppl, ctypes.byref(_prof(profile)), rho, len(rho),
                                  T, len(T), n_groups, out, threads or max_threads())
    return out


def loop_values(y: np.ndarray, profile, rho, T, threads: int = 0) -> np.ndarray:
    """W - 1 of every loop at every point [n_T * n_rho][n_loops][2] (scalar,
    spinor; rho fastest)."""
    y = np.ascontiguousarray(y, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    n_loops, _, ppl = y.shape
    out = np.zeros((len(T) * len(rho), n_loops, 2), np.float64)
    _load().wln_oracle_loop_values(y, n_loops, ppl, ctypes.byref(_prof(profile)), rho, len(rho),
                                   T, len(T), out, threads or max_threads())
    return out


def shuffle(seed: int, point: int, n: int) -> np.ndarray:
    """The loop permutation of the random grouping of evaluation `point`."""
    a = np.zeros(n, np.int32)
    _load().wln_oracle_shuffle(seed, point, n, a)
    return a


from . import stats  # noqa: E402,F401  (numpy statistics and quadrature)
