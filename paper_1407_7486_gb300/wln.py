"""Python binding of libwln (ctypes): argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module turns
numpy arrays and torch tensors into pointers and sizes, and turns status
codes into exceptions.  There is no fallback: if ``libwln.so`` is missing or
no GPU is present, the calls raise.

The method names are the C entry points without the ``wln_`` prefix.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from .inputs import Profile

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwln.so")

WLN_K = 5
WLN_KL = 6
C_SCAL, C_FERM, C_SIN, C_SCAL_SQ, C_FERM_SQ = range(5)
PREC = {"fp64": 0, "fp32": 1, "fp32_comp": 1, "fp32_naive": 2}
STATUS = {0: "WLN_OK", 1: "WLN_EINVAL", 2: "WLN_ENOMEM", 3: "WLN_ECUDA",
          4: "WLN_ETIMEOUT", 5: "WLN_EBUSY"}
WLN_OK, WLN_EINVAL, WLN_ENOMEM, WLN_ECUDA, WLN_ETIMEOUT, WLN_EBUSY = range(6)

# Every entry point declared in include/wln.h, with its ctypes signature.
_P, _I32, _I64, _U64, _D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                            ctypes.c_double)
SIGNATURES = {
    "wln_create": ([ctypes.POINTER(_P), ctypes.c_int, _P], ctypes.c_int),
    "wln_destroy": ([_P], ctypes.c_int),
    "wln_set_stream": ([_P, _P], ctypes.c_int),
    "wln_synchronize": ([_P], ctypes.c_int),
    "wln_last_error": ([_P], ctypes.c_char_p),
    "wln_launch_count": ([_P], _I64),
    "wln_selftest_wait": ([_P, _I32], ctypes.c_int),
    "wln_gen_loops": ([_P, _U64, _I64, _I32, _I32, _I32, ctypes.POINTER(_P)], ctypes.c_int),
    "wln_gen_dloops": ([_P, _U64, _I64, _I32, _I32, _I32, ctypes.POINTER(_P)], ctypes.c_int),
    "wln_ensemble_from_host": ([_P, _P, _I32, _I32, ctypes.POINTER(_P)], ctypes.c_int),
    "wln_free_ensemble": ([_P, _P], ctypes.c_int),
    "wln_ensemble_info": ([_P, _P, _P, _P], ctypes.c_int),
    "wln_loops_copy": ([_P, _P, _P, _P], ctypes.c_int),
    "wln_set_low_angle": ([_P, ctypes.c_int32], ctypes.c_int),
    "wln_set_precision_guard": ([_P, _I32], ctypes.c_int),
    "wln_precision_guard_stats": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                   ctypes.POINTER(_I64), ctypes.POINTER(_I64), _I32], ctypes.c_int),
    "wln_philox_stream": ([_P, _U64, _I64, _I32, _I32, _P], ctypes.c_int),
    "wln_wilson_avg": ([_P, _P, _P, _I32, _P, _P, _P, _P, _I32, ctypes.c_int, _P], ctypes.c_int),
    "wln_wilson_avg_noalloc": ([_P, _P, _P, _I32, _P, _P, _P, _P, _I32, ctypes.c_int, _P],
                               ctypes.c_int),
    "wln_wilson_levels": ([_P, _P, _P, _I32, _P, _P, _P, _P, _I32, ctypes.c_int, _P],
                          ctypes.c_int),
    "wln_wilson_levels_nested": ([_P, _P, _P, _I32, _P, _P, _P, _P, _I32, ctypes.c_int, _P],
                                 ctypes.c_int),
    "wln_extrapolate": ([_P, _P, _I32, _I32, _I32, _P], ctypes.c_int),
    "wln_mapped_grid": ([_I32, ctypes.c_double, ctypes.c_double, _P], ctypes.c_int),
    "wln_effective_action_full": ([_P, _P, _I32, _P, _P, _P, _P, _P, _P, _I32, _I32, _I32, _P,
                                   _P, _P, _P], ctypes.c_int),
    "wln_wilson_loops": ([_P, _P, _P, _I32, _P, _P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "wln_group_sums_loops": ([_P, _P, _I64, _I32, _I32, _I32, ctypes.c_uint64, _P, _P],
                             ctypes.c_int),
    "wln_corrcoef": ([_P, _P, _I32, _I32, _I32, _I32, _I32, _P], ctypes.c_int),
    "wln_jackknife": ([_P, _P, _I32, _I32, _I32, _I32, _P, _P, _P, _P], ctypes.c_int),
    "wln_jackknife_packed": ([_P, _P, _I32, _I32, _I32, _I32, _P, _P, _P, _P], ctypes.c_int),
    "wln_loop_sem": ([_P, _P, _I32, _I32, _I32, _I32, _I32, _P], ctypes.c_int),
    "wln_effective_action": ([_P, _P, _I32, _P, _P, _P, _P, _P, _I32, _I32, _I32, _P, _P],
                             ctypes.c_int),
    "wln_set_tuning": ([_P, _I32, _I32, _I32, _I32, _I32], ctypes.c_int),
    "wln_batch_create": ([_P, _P, _P, _I32, _P, _P, _P, _P, _I32, ctypes.c_int,
                          ctypes.POINTER(_P)], ctypes.c_int),
    "wln_batch_run": ([_P, _P, _I32], ctypes.c_int),
    "wln_batch_results": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "wln_batch_info": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "wln_batch_free": ([_P, _P], ctypes.c_int),
    "wln_server_create": ([_P, _P, _I32, ctypes.c_int, _I64, _I32, ctypes.POINTER(_P)],
                          ctypes.c_int),
    "wln_server_submit": ([_P, _P, _P, _I32, _P, _I32, ctypes.POINTER(_I64)], ctypes.c_int),
    "wln_server_step": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)], ctypes.c_int),
    "wln_server_poll": ([_P, _I64, ctypes.POINTER(_I32), _P, _P, _P], ctypes.c_int),
    "wln_server_cancel": ([_P, _I64], ctypes.c_int),
    "wln_server_release": ([_P, _I64], ctypes.c_int),
    "wln_server_info": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I32),
                         ctypes.POINTER(_I32)], ctypes.c_int),
    "wln_server_free": ([_P], ctypes.c_int),
}


class WlnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _CProfile(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("F", ctypes.c_double),
                ("lam", ctypes.c_double), ("B", ctypes.c_double)]


class _CQuad(ctypes.Structure):
    _fields_ = [("rho_kind", ctypes.c_int32), ("T_kind", ctypes.c_int32),
                ("rho_scale", ctypes.c_double), ("T_scale", ctypes.c_double),
                ("small_T", ctypes.c_int32), ("reserved", ctypes.c_int32)]


GRID_LINEAR, GRID_LOG, GRID_MAPPED = 0, 1, 2


class Quad:
    """Quadrature grids of one profile for effective_action_full (wln_quad)."""

    def __init__(self, rho_kind: int = GRID_LINEAR, T_kind: int = GRID_LOG,
                 rho_scale: float = 0.0, T_scale: float = 0.0, small_T: bool = False):
        self.rho_kind, self.T_kind = rho_kind, T_kind
        self.rho_scale, self.T_scale, self.small_T = rho_scale, T_scale, small_T


def mapped_grid(n: int, scale: float, start: float = 0.0) -> np.ndarray:
    """Ascending nodes of [start, inf) under x = 1/(1 + v/scale) (wln_mapped_grid)."""
    out = np.empty(n, np.float64)
    st = load().wln_mapped_grid(n, float(scale), float(start), _ptr(out))
    if st != 0:
        raise WlnError(st, "wln_mapped_grid: needs n >= 1, scale > 0, start >= 0")
    return out


_lib = None


def load(path: str = LIB_PATH):
    """Load libwln.so (built by ``paper_1407_7486_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1407_7486_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(x) -> Optional[int]:
    """Raw address of a torch tensor or numpy array (None for None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _profiles(profiles: Sequence[Profile]):
    arr = (_CProfile * len(profiles))()
    for i, p in enumerate(profiles):
        arr[i] = _CProfile(int(p.kind), 0, float(p.F), float(p.lam), float(p.B))
    return arr


def _csr(grids: Sequence[Sequence[float]]):
    parts = [np.asarray(g, np.float64).reshape(-1) for g in grids]
    flat = np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros(0))
    off = np.zeros(len(grids) + 1, np.int32)
    off[1:] = np.cumsum([len(g) for g in grids])
    return flat, off


class Ensemble:
    """Device-resident loop ensemble owned by the library."""

    def __init__(self, ctx: "Context", handle: int):
        self._ctx = ctx
        self.handle = handle
        n, ppl, f64 = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ctx._check(load().wln_ensemble_info(handle, ctypes.byref(n), ctypes.byref(ppl),
                                            ctypes.byref(f64)))
        self.n_loops, self.ppl, self.has_fp64 = n.value, ppl.value, bool(f64.value)

    def free(self):
        if self.handle:
            load().wln_free_ensemble(self._ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            if self.handle and self._ctx.handle:
                self.free()
        except Exception:
            pass


class Context:
    """One device and one CUDA stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        h = ctypes.c_void_p()
        st = lib.wln_create(ctypes.byref(h), device, raw)
        if st != 0:
            raise WlnError(st, "wln_create failed (is a CUDA device present?)")
        self.handle = h.value

    # ----------------------------------------------------------- plumbing
    def _check(self, st: int):
        if st != 0:
            msg = load().wln_last_error(self.handle)
            raise WlnError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "handle", None):
            load().wln_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def selftest_wait(self, timeout_ms: int = 50) -> int:
        """Run the bounded-wait self-test; returns the status (WLN_ETIMEOUT = 4)."""
        return int(load().wln_selftest_wait(self.handle, timeout_ms))

    def synchronize(self):
        self._check(load().wln_synchronize(self.handle))

    def set_stream(self, stream):
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.stream = stream
        self._check(load().wln_set_stream(self.handle, raw))

    def set_tuning(self, points_per_lane: int = 0, warps: int = 0, rows: int = 0,
                   stages: int = 0, chain_blocks: int = 0):
        self._check(load().wln_set_tuning(self.handle, points_per_lane, warps, rows, stages,
                                          chain_blocks))

    def set_precision_guard(self, enabled=True):
        """The precision guard of the FP32-compensated group sums (on by
        default): loops whose float rounding would move a spinor group mean by
        more than half of 1e-6 max(1, <cosh spin>) are recomputed in
        double-float.  enabled="all" recomputes every recorded loop (a check
        of the double-float walk)."""
        mode = 2 if enabled == "all" else int(bool(enabled))
        self._check(load().wln_set_precision_guard(self.handle, mode))

    def precision_guard_stats(self, reset: bool = False) -> dict:
        """Running totals of the guard: loops recomputed, launches, queue
        overflows, selections that stopped at 64 loops."""
        v = [ctypes.c_int64() for _ in range(4)]
        self._check(load().wln_precision_guard_stats(self.handle, *[ctypes.byref(x) for x in v],
                                                     int(bool(reset))))
        return dict(zip(("escalated_loops", "launches", "overflows", "saturated"),
                        (x.value for x in v)))

    def set_low_angle(self, level: int = 2):
        """The cheaper forms of theta later float walks may take on blocks
        whose segments all subtend small angles: 0 none, 1 without the
        octant unfolding (same bits), 2 also the short series (default)."""
        self._check(load().wln_set_low_angle(self.handle, int(level)))

    @property
    def launch_count(self) -> int:
        return int(load().wln_launch_count(self.handle))

    def _empty(self, shape, dtype, where: str):
        """Output buffer: "host" (numpy), "pinned" (numpy over page-locked
        host memory, the fast path for device-to-host copies) or "device"
        (a torch tensor on this context's GPU)."""
        import torch
        if where == "host":
            return np.empty(shape, dtype)
        if where == "pinned":
            tdt = {np.float64: torch.float64, np.float32: torch.float32,
                   np.uint32: torch.int32}[dtype]
            return torch.empty(shape, dtype=tdt, pin_memory=True).numpy().view(dtype)
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.uint32: torch.int32}[dtype]
        return torch.empty(shape, dtype=tdt, device=f"cuda:{self.device}")

    # ---------------------------------------------------------- ensembles
    def gen_loops(self, seed: int, n_loops: int, ppl: int, keep_fp64: bool = False,
                  loop0: int = 0) -> Ensemble:
        h = ctypes.c_void_p()
        self._check(load().wln_gen_loops(self.handle, seed, loop0, n_loops, ppl, int(keep_fp64),
                                         ctypes.byref(h)))
        return Ensemble(self, h.value)

    def gen_dloops(self, seed: int, n_loops: int, ppl: int, keep_fp64: bool = False,
                   loop0: int = 0) -> Ensemble:
        """The paper's d-loop construction (same law, other draws)."""
        h = ctypes.c_void_p()
        self._check(load().wln_gen_dloops(self.handle, seed, loop0, n_loops, ppl, int(keep_fp64),
                                          ctypes.byref(h)))
        return Ensemble(self, h.value)

    def ensemble_from_host(self, xy) -> Ensemble:
        """xy: float32 [n_loops][2][ppl] (numpy or torch, host or device)."""
        if isinstance(xy, np.ndarray):
            xy = np.ascontiguousarray(xy, np.float32)
        n_loops, _, ppl = xy.shape
        h = ctypes.c_void_p()
        self._check(load().wln_ensemble_from_host(self.handle, _ptr(xy), n_loops, ppl,
                                                  ctypes.byref(h)))
        return Ensemble(self, h.value)

    def loops_copy(self, ens: Ensemble, f32=True, f64=False, where: str = "host",
                   out32=None, out64=None):
        """The loops as float (and/or double) [n_loops][2][ppl]; out32 / out64
        are caller-owned destinations (C-contiguous, that shape and type)."""
        shape = (ens.n_loops, 2, ens.ppl)
        for o, t in ((out32, np.float32), (out64, np.float64)):
            if o is not None and (tuple(o.shape) != shape or o.dtype != t
                                  or not o.flags["C_CONTIGUOUS"]):
                raise ValueError(f"output must be C-contiguous {t.__name__} of shape {shape}")
        a = out32 if out32 is not None else (self._empty(shape, np.float32, where) if f32 else None)
        b = out64 if out64 is not None else (self._empty(shape, np.float64, where) if f64 else None)
        self._check(load().wln_loops_copy(self.handle, ens.handle, _ptr(a), _ptr(b)))
        return a, b

    def philox_stream(self, seed: int, loop0: int, n_loops: int, n_calls: int,
                      where: str = "host"):
        out = self._empty((n_loops, n_calls, 4), np.uint32, where)
        self._check(load().wln_philox_stream(self.handle, seed, loop0, n_loops, n_calls,
                                             _ptr(out)))
        return out

    # ------------------------------------------------------- Wilson loops
    def wilson_avg(self, ens: Ensemble, profiles: Sequence[Profile], rho: Sequence, T: Sequence,
                   n_groups: int, prec: str = "fp32", out=None, where: str = "device"):
        """Group sums [n_points][n_groups][5]; points ordered profile, T, rho."""
        rho_f, rho_off = _csr(rho)
        T_f, T_off = _csr(T)
        n_points = int(sum(len(r) * len(t) for r, t in zip(rho, T)))
        if out is None:
            out = self._empty((n_points, n_groups, WLN_K), np.float64, where)
        profs = _profiles(profiles)
        self._check(load().wln_wilson_avg(self.handle, ens.handle, profs, len(profiles),
                                          _ptr(rho_f), _ptr(rho_off), _ptr(T_f), _ptr(T_off),
                                          n_groups, PREC[prec], _ptr(out)))
        return out

    def wilson_avg_noalloc(self, ens: Ensemble, profiles: Sequence[Profile], rho: Sequence,
                           T: Sequence, n_groups: int, prec: str = "fp32", out=None,
                           where: str = "device"):
        """wilson_avg through the entry point that allocates no device memory
        (working memory from the library's fixed 64 MiB array)."""
        rho_f, rho_off = _csr(rho)
        T_f, T_off = _csr(T)
        n_points = int(sum(len(r) * len(t) for r, t in zip(rho, T)))
        if out is None:
            out = self._empty((n_points, n_groups, WLN_K), np.float64, where)
        profs = _profiles(profiles)
        self._check(load().wln_wilson_avg_noalloc(self.handle, ens.handle, profs, len(profiles),
                                                  _ptr(rho_f), _ptr(rho_off), _ptr(T_f),
                                                  _ptr(T_off), n_groups, PREC[prec], _ptr(out)))
        return out

    def wilson_levels(self, ens: Ensemble, profiles: Sequence[Profile], rho: Sequence,
                      T: Sequence, n_groups: int, prec: str = "fp32", out=None,
                      where: str = "device", nested: bool = False):
        """Discretisation-level group sums [n_points][n_groups][6]: W - 1
        (scalar, spinor) at N, N/2 and N/4 points per loop, from the
        interleaved sub-loops of every loop as the paper combines them, or
        (nested=True) from the nested loops through all, even and 0 mod 4
        points."""
        rho_f, rho_off = _csr(rho)
        T_f, T_off = _csr(T)
        n_points = int(sum(len(r) * len(t) for r, t in zip(rho, T)))
        if out is None:
            out = self._empty((n_points, n_groups, WLN_KL), np.float64, where)
        profs = _profiles(profiles)
        fn = load().wln_wilson_levels_nested if nested else load().wln_wilson_levels
        self._check(fn(self.handle, ens.handle, profs, len(profiles), _ptr(rho_f), _ptr(rho_off),
                       _ptr(T_f), _ptr(T_off), n_groups, PREC[prec], _ptr(out)))
        return out

    def extrapolate(self, level_sums, n_groups: int, loops_per_group: int,
                    where: str = "device"):
        """[n_points][2][6]: for the scalar then the spinor loop, the level
        means (N, N/2, N/4), the extrapolation W_inf - 1, its group standard
        error, and the discretisation uncertainty |m_N - (W_inf - 1)|."""
        n_points = level_sums.shape[0]
        out = self._empty((n_points, 2, 6), np.float64, where)
        self._check(load().wln_extrapolate(self.handle, _ptr(level_sums), n_points, n_groups,
                                           loops_per_group, _ptr(out)))
        return out

    def wilson_loops(self, ens: Ensemble, profiles: Sequence[Profile], rho: Sequence, T: Sequence,
                     prec: str = "fp32", out=None, where: str = "device"):
        """Every loop's W - 1 at every point: [n_points][n_loops][2] (scalar, spinor)."""
        rho_f, rho_off = _csr(rho)
        T_f, T_off = _csr(T)
        n_points = int(sum(len(r) * len(t) for r, t in zip(rho, T)))
        if out is None:
            out = self._empty((n_points, ens.n_loops, 2), np.float64, where)
        profs = _profiles(profiles)
        self._check(load().wln_wilson_loops(self.handle, ens.handle, profs, len(profiles),
                                            _ptr(rho_f), _ptr(rho_off), _ptr(T_f), _ptr(T_off),
                                            PREC[prec], _ptr(out)))
        return out

    def group_sums_loops(self, loop_values, n_groups: int, shuffle: bool = False, seed: int = 0,
                         with_perm: bool = False, where: str = "device"):
        """Group sums [n_points][G][5] of per-loop values, contiguous groups or a
        random grouping per point; returns (sums, order or None)."""
        n_points, n_loops = int(loop_values.shape[0]), int(loop_values.shape[1])
        S = self._empty((n_points, n_groups, WLN_K), np.float64, where)
        perm = None
        if shuffle and with_perm:
            if where == "host":
                perm = np.empty((n_points, n_loops), np.int32)
            else:
                import torch
                perm = torch.empty((n_points, n_loops), dtype=torch.int32,
                                   device=f"cuda:{self.device}")
        self._check(load().wln_group_sums_loops(self.handle, _ptr(loop_values), n_points, n_loops,
                                                n_groups, int(bool(shuffle)), seed, _ptr(S),
                                                _ptr(perm)))
        return S, perm

    def corrcoef(self, x, ref: int, comp: int = 0, where: str = "device"):
        """Eq. corrcoef of every row of x ([rows][samples][stride]) with row ref."""
        n_rows, n_samples, stride = (int(v) for v in x.shape)
        out = self._empty((n_rows,), np.float64, where)
        self._check(load().wln_corrcoef(self.handle, _ptr(x), n_rows, n_samples, stride, comp,
                                        ref, _ptr(out)))
        return out

    # --------------------------------------------------------- statistics
    def jackknife(self, group_sums, n_groups: int, loops_per_group: int, comp: int,
                  jk_var: bool = True, cov=False, where: str = "device", out=None):
        """Group mean, SEM, jackknife variance and covariance; `out` may hold
        caller-owned buffers under the same keys (reused across calls).
        cov="packed": the covariance as its upper triangle, row by row
        (wln_jackknife_packed)."""
        n_points = group_sums.shape[0]
        packed = cov == "packed"
        out = out or {}
        mean = out.get("mean")
        mean = self._empty((n_points,), np.float64, where) if mean is None else mean
        sem = out.get("sem")
        sem = self._empty((n_points,), np.float64, where) if sem is None else sem
        jv = out.get("jk_var") if jk_var else None
        if jk_var and jv is None:
            jv = self._empty((n_points,), np.float64, where)
        cv = out.get("cov") if cov else None
        if cov and cv is None:
            shape = (n_points * (n_points + 1) // 2,) if packed else (n_points, n_points)
            cv = self._empty(shape, np.float64, where)
        fn = load().wln_jackknife_packed if packed else load().wln_jackknife
        self._check(fn(self.handle, _ptr(group_sums), n_points, n_groups, loops_per_group, comp,
                       _ptr(mean), _ptr(sem), _ptr(jv), _ptr(cv)))
        return {"mean": mean, "sem": sem, "jk_var": jv, "cov": cv}

    def loop_sem(self, group_sums, n_groups: int, n_loops: int, comp_sum: int, comp_sq: int,
                 where: str = "device"):
        n_points = group_sums.shape[0]
        out = self._empty((n_points,), np.float64, where)
        self._check(load().wln_loop_sem(self.handle, _ptr(group_sums), n_points, n_groups,
                                        n_loops, comp_sum, comp_sq, _ptr(out)))
        return out

    def effective_action(self, profiles: Sequence[Profile], rho: Sequence, T: Sequence,
                         group_sums, n_groups: int, loops_per_group: int, spinor: bool = True,
                         where: str = "device", out=None):
        """(per-group action [n_profiles][G], (mean, SEM) [n_profiles][2]);
        `out` may be a caller-owned pair of buffers."""
        rho_f, rho_off = _csr(rho)
        T_f, T_off = _csr(T)
        if out is not None:
            gg, ms = out
        else:
            gg = self._empty((len(profiles), n_groups), np.float64, where)
            ms = self._empty((len(profiles), 2), np.float64, where)
        profs = _profiles(profiles)
        self._check(load().wln_effective_action(self.handle, profs, len(profiles), _ptr(rho_f),
                                                _ptr(rho_off), _ptr(T_f), _ptr(T_off),
                                                _ptr(group_sums), n_groups, loops_per_group,
                                                int(spinor), _ptr(gg), _ptr(ms)))
        return gg, ms

    def effective_action_full(self, profiles: Sequence[Profile], rho: Sequence, T: Sequence,
                              group_sums, n_groups: int, loops_per_group: int,
                              quad: Optional[Sequence[Quad]] = None, spinor: bool = True,
                              where: str = "device"):
        """Full effective action: {"gamma_groups": [n_profiles][G], "gamma":
        [n_profiles][3] (mean, SEM, LCF), "density": [n_rho_total][3] (T
        integral at each radius: mean, SEM, LCF), "integrand": [n_points][3]}."""
        rho_f, rho_off = _csr(rho)
        T_f, T_off = _csr(T)
        n_points = int(sum(len(r) * len(t) for r, t in zip(rho, T)))
        out = {"gamma_groups": self._empty((len(profiles), n_groups), np.float64, where),
               "gamma": self._empty((len(profiles), 3), np.float64, where),
               "density": self._empty((len(rho_f), 3), np.float64, where),
               "integrand": self._empty((n_points, 3), np.float64, where)}
        cq = None
        if quad is not None:
            cq = (_CQuad * len(profiles))()
            for i, q in enumerate(quad):
                cq[i] = _CQuad(int(q.rho_kind), int(q.T_kind), float(q.rho_scale),
                               float(q.T_scale), int(bool(q.small_T)), 0)
        profs = _profiles(profiles)
        self._check(load().wln_effective_action_full(
            self.handle, profs, len(profiles), _ptr(rho_f), _ptr(rho_off), _ptr(T_f),
            _ptr(T_off), cq, _ptr(group_sums), n_groups, loops_per_group, int(spinor),
            _ptr(out["gamma_groups"]), _ptr(out["gamma"]), _ptr(out["density"]),
            _ptr(out["integrand"])))
        return out


class Batch:
    """A fixed set of profiles and grids whose runs can be replayed from a CUDA
    graph (wln_batch_*)."""

    def __init__(self, ctx: "Context", ens: Ensemble, profiles: Sequence[Profile], rho: Sequence,
                 T: Sequence, n_groups: int, prec: str = "fp32"):
        self._ctx = ctx
        self.ens = ens
        rho_f, rho_off = _csr(rho)
        T_f, T_off = _csr(T)
        h = ctypes.c_void_p()
        ctx._check(load().wln_batch_create(ctx.handle, ens.handle, _profiles(profiles),
                                           len(profiles), _ptr(rho_f), _ptr(rho_off), _ptr(T_f),
                                           _ptr(T_off), n_groups, PREC[prec], ctypes.byref(h)))
        self.handle = h.value
        self.n_groups = n_groups
        self.n_profiles = len(profiles)
        npts, nt, P, ch, kpr = (ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(),
                                ctypes.c_int32(), ctypes.c_int64())
        load().wln_batch_info(self.handle, ctypes.byref(npts), ctypes.byref(nt), ctypes.byref(P),
                              ctypes.byref(ch), ctypes.byref(kpr))
        self.n_points, self.n_tiles, self.P, self.chain = npts.value, nt.value, P.value, ch.value

    @property
    def kernels_per_run(self) -> int:
        k = ctypes.c_int64()
        load().wln_batch_info(self.handle, None, None, None, None, ctypes.byref(k))
        return k.value

    def run(self, graph: bool = True):
        self._ctx._check(load().wln_batch_run(self._ctx.handle, self.handle, int(graph)))

    def results(self, sums: bool = True, stats: bool = True, gamma: bool = True,
                where: str = "host"):
        S = self._ctx._empty((self.n_points, self.n_groups, WLN_K), np.float64, where) if sums else None
        st = self._ctx._empty((4, self.n_points), np.float64, where) if stats else None
        g = self._ctx._empty((2, self.n_profiles, 2), np.float64, where) if gamma else None
        self._ctx._check(load().wln_batch_results(self._ctx.handle, self.handle, _ptr(S), _ptr(st),
                                                  _ptr(g)))
        return S, st, g

    def free(self):
        if self.handle:
            load().wln_batch_free(self._ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (wln_server_*)."""

    QUEUED, RUNNING, FINISHING, DONE, CANCELLED = range(5)

    def __init__(self, ctx: "Context", ens: Ensemble, n_groups: int, prec: str = "fp32",
                 arena_bytes: int = 4 << 30, tile_groups_per_step: int = 64):
        self._ctx = ctx
        self.ens = ens
        self.n_groups = n_groups
        h = ctypes.c_void_p()
        ctx._check(load().wln_server_create(ctx.handle, ens.handle, n_groups, PREC[prec],
                                            arena_bytes, tile_groups_per_step, ctypes.byref(h)))
        self.handle = h.value
        self._npts = {}

    def submit(self, profile: Profile, rho, T) -> int:
        rho = np.ascontiguousarray(rho, np.float64)
        T = np.ascontiguousarray(T, np.float64)
        rid = ctypes.c_int64()
        self._ctx._check(load().wln_server_submit(self.handle, _profiles([profile]), _ptr(rho),
                                                  len(rho), _ptr(T), len(T), ctypes.byref(rid)))
        self._npts[rid.value] = len(rho) * len(T)
        return rid.value

    def step(self):
        a, q = ctypes.c_int32(), ctypes.c_int32()
        self._ctx._check(load().wln_server_step(self.handle, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def poll(self, rid: int, results: bool = True):
        st = ctypes.c_int32()
        n = self._npts[rid]
        S = np.empty((n, self.n_groups, WLN_K)) if results else None
        stats = np.empty((4, n)) if results else None
        gamma = np.empty((2, 1, 2)) if results else None
        self._ctx._check(load().wln_server_poll(self.handle, rid, ctypes.byref(st), _ptr(S),
                                                _ptr(stats), _ptr(gamma)))
        if st.value != self.DONE:
            return st.value, None
        return st.value, (S, stats, gamma)

    def cancel(self, rid: int):
        self._ctx._check(load().wln_server_cancel(self.handle, rid))

    def release(self, rid: int):
        self._ctx._check(load().wln_server_release(self.handle, rid))
        self._npts.pop(rid, None)

    def info(self):
        steps, free_b, a, q = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        load().wln_server_info(self.handle, ctypes.byref(steps), ctypes.byref(free_b),
                               ctypes.byref(a), ctypes.byref(q))
        return {"steps": steps.value, "arena_free_bytes": free_b.value, "active": a.value,
                "queued": q.value}

    def free(self):
        if self.handle:
            load().wln_server_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def header_symbols(header: Optional[str] = None) -> List[str]:
    """Names of the functions declared in include/wln.h."""
    import re
    if header is None:
        header = os.path.join(os.path.dirname(_HERE), "include", "wln.h")
    text = open(header).read()
    return sorted(set(re.findall(r"\b(wln_[a-z_0-9]+)\s*\(", text)))
