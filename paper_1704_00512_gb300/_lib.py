"""ctypes binding of libcheb.so: argument marshalling only.

Every function here has the name of the C entry point it calls (without the
``cheb_`` prefix), takes torch CUDA tensors for device memory, allocates the
workspace the call asks for with torch, and raises ``ChebError`` on a non-zero
status.  No computation happens in Python: a missing or unloadable library is
an error, never a fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcheb.so")

OK, ERR_INVALID, ERR_CUDA, ERR_NOT_SPD, ERR_BOUNDS, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_NOSPACE = range(8)
F64, F32, BF16, F64X = 0, 1, 2, 3  # F64X: FP64-accurate double-float products on the FP32 pipe
FERMI, ERFC, POWER, INTERVAL, PENALTY = 0, 1, 2, 3, 4

# Every symbol declared in include/cheb.h.
EXPORTS = [
    "cheb_last_error", "cheb_launch_count", "cheb_pattern_build", "cheb_tile_count", "cheb_tile_info", "cheb_plan_create", "cheb_plan_bind", "cheb_plan_info",
    "cheb_plan_destroy", "cheb_plan_attach_operator", "cheb_plan_bind_operator", "cheb_scale", "cheb_bounds_workspace_size", "cheb_bounds",
    "cheb_coeffs_workspace_size", "cheb_coeffs", "cheb_expand_workspace_size", "cheb_expand",
    "cheb_expand_stepwise_workspace_size", "cheb_expand_stepwise", "cheb_plan_create_batched",
    "cheb_plan_resident_info", "cheb_expand_batched", "cheb_block_diag", "cheb_lincomb", "cheb_mlp_param_count",
    "cheb_mlp_init", "cheb_mlp_forward", "cheb_mlp_loss", "cheb_mlp_backward", "cheb_mlp_adam", "cheb_mlp_features",
    "cheb_masked_product", "cheb_transpose", "cheb_restrict", "cheb_trace_workspace_size", "cheb_trace",
    "cheb_penalty_trace", "cheb_mu_search", "cheb_mu_search_noalloc", "cheb_newton_schulz", "cheb_newton_schulz_isqrt",
    "cheb_plan_col_info", "cheb_penalty_check", "cheb_mu_nodes", "cheb_lagrange_weights", "cheb_bounds_spd",
    "cheb_widen_bounds", "cheb_mlp_bracket", "cheb_locality_order_ws", "cheb_locality_order", "cheb_position_map",
    "cheb_gather_rows", "cheb_scatter_rows",
    "cheb_series_value", "cheb_bounds_warm", "cheb_plan_set_gather_builder", "cheb_plan_lists_copy", "cheb_set_plan_builder",
    "cheb_ssf_export_size", "cheb_ssf_export", "cheb_ssf_import_pattern", "cheb_ssf_import_values",
]


class ChebError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libcheb error {code}: {msg}")
        self.code = code


class CBsr(ctypes.Structure):
    _fields_ = [("nbr", ctypes.c_int64), ("nnzb", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("dtype", ctypes.c_int32)]


class CFunc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("mu", ctypes.c_double), ("kT", ctypes.c_double),
                ("a", ctypes.c_double), ("lo", ctypes.c_double), ("hi", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH, build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libcheb.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ChebError(ERR_INVALID, f"libcheb.so not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    p, i32, i64, dbl, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "cheb_last_error": ([], ctypes.c_char_p),
        "cheb_launch_count": ([], ctypes.c_uint64),
        "cheb_pattern_build": ([p, i64, dbl, dbl, p, p, P(i64), p], i32),
        "cheb_tile_count": ([i32], i32),
        "cheb_tile_info": ([i32, i32, P(i32), P(i32), P(i32)], i32),
        "cheb_plan_create": ([P(CBsr), i32, i32, P(p), P(sz), p], i32),
        "cheb_plan_bind": ([p, p, sz, p], i32),
        "cheb_plan_info": ([p, P(i64), P(i32), P(i32)], i32),
        "cheb_plan_destroy": ([p], i32),
        "cheb_plan_attach_operator": ([p, P(CBsr), P(sz), p], i32),
        "cheb_plan_bind_operator": ([p, p, sz, p], i32),
        "cheb_scale": ([P(CBsr), dbl, dbl, p, p], i32),
        "cheb_bounds_workspace_size": ([i64, i32, P(sz)], i32),
        "cheb_bounds": ([P(CBsr), i32, p, dbl, P(dbl), P(dbl), P(dbl), p, sz, p], i32),
        "cheb_coeffs_workspace_size": ([i32, i32, P(sz)], i32),
        "cheb_coeffs": ([P(CFunc), i32, dbl, dbl, dbl, i32, i32, P(i32), p, p, sz, p], i32),
        "cheb_expand_workspace_size": ([p, P(CBsr), i32, i32, P(sz)], i32),
        "cheb_expand": ([p, P(CBsr), i32, p, i32, i32, P(p), p, p, p, i32, p, sz, p], i32),
        "cheb_expand_stepwise_workspace_size": ([p, P(CBsr), i32, P(sz)], i32),
        "cheb_expand_stepwise": ([p, P(CBsr), i32, p, i32, i32, P(p), p, p, p, i32, p, sz, p], i32),
        "cheb_plan_create_batched": ([P(CBsr), i32, i32, i32, P(i64), P(p), P(sz), p], i32),
        "cheb_plan_resident_info": ([p, P(i64), P(i32), P(i32)], i32),
        "cheb_plan_col_info": ([p, P(i64), P(i32), P(i64)], i32),
        "cheb_penalty_check": ([p, i32, dbl, dbl, P(dbl), P(i32), p, sz, p], i32),
        "cheb_mu_nodes": ([dbl, dbl, i32, P(dbl)], i32),
        "cheb_widen_bounds": ([P(dbl), i32, dbl], i32),
        "cheb_locality_order_ws": ([i64], sz),
        "cheb_locality_order": ([p, i64, dbl, p, p, sz, p], i32),
        "cheb_position_map": ([P(CBsr), P(CBsr), p, p, p, sz, p], i32),
        "cheb_gather_rows": ([p, i64, p, i64, i32, p, p], i32),
        "cheb_scatter_rows": ([p, p, i64, i32, p, i64, p], i32),
        "cheb_mlp_bracket": ([P(ctypes.c_float), dbl, dbl, dbl, dbl, dbl, P(dbl), P(dbl)], i32),
        "cheb_series_value": ([p, p, i32, p, p], i32),
        "cheb_plan_set_gather_builder": ([p, i32], i32),
        "cheb_ssf_export_size": ([P(CBsr), P(i64), P(i64), p], i32),
        "cheb_ssf_export": ([P(CBsr), i64, p, p, p, p], i32),
        "cheb_ssf_import_pattern": ([i64, i64, p, P(i64), p, p, p], i32),
        "cheb_ssf_import_values": ([P(CBsr), i64, p, p, p, i64, p], i32),
        "cheb_plan_lists_copy": ([p, i32, p, ctypes.c_size_t, P(ctypes.c_size_t), p], i32),
        "cheb_set_plan_builder": ([i32], i32),
        "cheb_bounds_warm": ([P(CBsr), i32, p, dbl, P(dbl), P(dbl), P(dbl), P(dbl), p, ctypes.c_size_t, p], i32),
        "cheb_lagrange_weights": ([P(dbl), i32, dbl, P(dbl)], i32),
        "cheb_bounds_spd": ([P(CBsr), i32, p, dbl, P(dbl), P(dbl), p, sz, p], i32),
        "cheb_expand_batched": ([p, P(CBsr), i32, p, p, p, i32, i32, P(p), p, p, p, i32, i32, p, sz, p], i32),
        "cheb_block_diag": ([i32, P(CBsr), p, p, p, i32, p], i32),
        "cheb_lincomb": ([i32, P(dbl), P(p), i64, p, p], i32),
        "cheb_mlp_param_count": ([], i32),
        "cheb_mlp_init": ([p, ctypes.c_uint64, p], i32),
        "cheb_mlp_forward": ([p, p, i32, p, p, p], i32),
        "cheb_mlp_loss": ([p, p, p, i32, p, p, p], i32),
        "cheb_mlp_backward": ([p, p, i32, p, p, p, p, p], i32),
        "cheb_mlp_adam": ([p, p, p, p, i32, ctypes.c_float, p], i32),
        "cheb_mlp_features": ([p, i64, dbl, dbl, dbl, p, p], i32),
        "cheb_masked_product": ([p, P(CBsr), p, dbl, p, dbl, p, p], i32),
        "cheb_transpose": ([p, p, p, p], i32),
        "cheb_restrict": ([P(CBsr), P(CBsr), p, p], i32),
        "cheb_trace_workspace_size": ([P(CBsr), P(sz)], i32),
        "cheb_trace": ([P(CBsr), P(CBsr), p, p, sz, p], i32),
        "cheb_penalty_trace": ([p, i32, dbl, p, p, sz, p], i32),
        "cheb_mu_search": ([p, i32, dbl, dbl, i32, dbl, dbl, dbl, i32, p, p, p, sz, p], i32),
        "cheb_mu_search_noalloc": ([p, i32, dbl, dbl, i32, dbl, dbl, dbl, i32, p, p, p], i32),
        "cheb_newton_schulz": ([p, P(CBsr), p, p, p, p], i32),
        "cheb_newton_schulz_isqrt": ([p, P(CBsr), p, p, p, p, p], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int):
    if rc != OK:
        msg = _lib.cheb_last_error().decode()
        raise ChebError(rc, msg)


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256) + 256, dtype=torch.uint8, device=device)


def _aligned(t: torch.Tensor) -> int:
    p = t.data_ptr()
    return (p + 255) // 256 * 256


class Bsr:
    """4x4 block-CSR matrix on the GPU: row_ptr int64, col_idx int32, vals [nnzb, 4, 4]."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor | None = None):
        self.row_ptr = row_ptr
        self.col_idx = col_idx
        self.vals = vals

    @property
    def nbr(self) -> int:
        return self.row_ptr.numel() - 1

    @property
    def nnzb(self) -> int:
        return self.col_idx.numel()

    def with_vals(self, vals: torch.Tensor) -> "Bsr":
        return Bsr(self.row_ptr, self.col_idx, vals)

    def c(self) -> CBsr:
        dt = F64
        if self.vals is not None:
            dt = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[self.vals.dtype]
        return CBsr(self.nbr, self.nnzb, _ptr(self.row_ptr), _ptr(self.col_idx),
                    _ptr(self.vals) if self.vals is not None else None, dt)


def tile_shapes(precision: int) -> list[tuple[int, int, int]]:
    """cheb_tile_count / cheb_tile_info: (panel width, warps, blocks per SM) per tile index."""
    lib = load()
    out = []
    for t in range(lib.cheb_tile_count(precision)):
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib.cheb_tile_info(precision, t, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        out.append((a.value, b.value, c.value))
    return out


def launch_count() -> int:
    """cheb_launch_count: kernel launches made through the library so far."""
    return int(load().cheb_launch_count())


def pattern_build(xyz: torch.Tensor, box_L: float, r_cut: float, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
    """cheb_pattern_build (both calls)."""
    lib = load()
    n = xyz.shape[0]
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=xyz.device)
    nnzb = ctypes.c_int64(0)
    s = _stream(stream)
    _check(lib.cheb_pattern_build(_ptr(xyz), n, box_L, r_cut, _ptr(row_ptr), None, ctypes.byref(nnzb), s))
    col_idx = torch.empty(nnzb.value, dtype=torch.int32, device=xyz.device)
    _check(lib.cheb_pattern_build(_ptr(xyz), n, box_L, r_cut, _ptr(row_ptr), _ptr(col_idx), None, s))
    return row_ptr, col_idx


class Plan:
    """cheb_plan_create + cheb_plan_bind; keeps the pattern and workspace alive."""

    def __init__(self, P_out: Bsr, precision: int = F64, tile: int = -1, stream=None):
        lib = load()
        self.P_out = P_out
        self.precision = precision
        self.tile = tile
        h = ctypes.c_void_p()
        nbytes = ctypes.c_size_t(0)
        s = _stream(stream)
        cb = P_out.c()
        _check(lib.cheb_plan_create(ctypes.byref(cb), precision, tile, ctypes.byref(h), ctypes.byref(nbytes), s))
        self.handle = h
        self._ws = _ws(nbytes.value, P_out.row_ptr.device)
        _check(lib.cheb_plan_bind(h, ctypes.c_void_p(_aligned(self._ws)), nbytes.value, s))

    def attach_operator(self, L: Bsr, stream=None, gather: str | None = None) -> "Plan":
        """cheb_plan_attach_operator + cheb_plan_bind_operator: row lists for operator pattern L.

        gather: "device" (the gather-plan kernels) or "host" (the reference host
        builders) for the lists; None keeps the builder the plan was made with."""
        lib = load()
        nbytes = ctypes.c_size_t(0)
        s = _stream(stream)
        if gather is not None:
            if gather not in ("device", "host"):
                raise ValueError(f"attach_operator: gather must be 'device' or 'host', not {gather!r}")
            _check(lib.cheb_plan_set_gather_builder(self.handle, 1 if gather == "host" else 0))
        cb = L.c()
        _check(lib.cheb_plan_attach_operator(self.handle, ctypes.byref(cb), ctypes.byref(nbytes), s))
        self._op_ws = _ws(nbytes.value, L.row_ptr.device)
        self._op_pattern = (L.row_ptr, L.col_idx)  # the lists are used for operators with these pointers
        _check(lib.cheb_plan_bind_operator(self.handle, ctypes.c_void_p(_aligned(self._op_ws)), nbytes.value, s))
        return self

    def info(self) -> tuple[int, int, int]:
        a, b, c = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.cheb_plan_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.cheb_plan_destroy(self.handle)
            self.handle = None


def scale(M: Bsr, emin: float, emax: float, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    lib = load()
    out = torch.empty_like(M.vals) if out is None else out
    cb = M.c()
    _check(lib.cheb_scale(ctypes.byref(cb), emin, emax, _ptr(out), _stream(stream)))
    return out


def bounds(M: Bsr, k: int = 40, v0: torch.Tensor | None = None, margin_frac: float = 0.01,
           stream=None) -> tuple[float, float, tuple[float, float]]:
    """cheb_bounds: returns (emin, emax, (theta_min, theta_max))."""
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.cheb_bounds_workspace_size(M.nbr, k, ctypes.byref(nb)))
    ws = _ws(nb.value, M.vals.device)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    th = (ctypes.c_double * 2)()
    cb = M.c()
    _check(lib.cheb_bounds(ctypes.byref(cb), k, _ptr(v0), margin_frac, ctypes.byref(lo), ctypes.byref(hi), th,
                           ctypes.c_void_p(_aligned(ws)), nb.value, _stream(stream)))
    return lo.value, hi.value, (th[0], th[1])


def bounds_warm(M: Bsr, warm: tuple[float, float], k: int = 8, v0: torch.Tensor | None = None,
                margin_frac: float = 0.01, stream=None) -> tuple[float, float, tuple[float, float]]:
    """cheb_bounds_warm: the hull of the warm interval and k Lanczos steps' interval."""
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.cheb_bounds_workspace_size(M.nbr, k, ctypes.byref(nb)))
    ws = _ws(nb.value, M.vals.device)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    th = (ctypes.c_double * 2)()
    w = (ctypes.c_double * 2)(float(warm[0]), float(warm[1]))
    cb = M.c()
    _check(lib.cheb_bounds_warm(ctypes.byref(cb), k, _ptr(v0), margin_frac, w, ctypes.byref(lo), ctypes.byref(hi),
                                th, ctypes.c_void_p(_aligned(ws)), nb.value, _stream(stream)))
    return lo.value, hi.value, (th[0], th[1])


def make_funcs(funcs) -> ctypes.Array:
    arr = (CFunc * len(funcs))()
    for i, f in enumerate(funcs):
        arr[i] = CFunc(int(f["kind"]), float(f.get("mu", 0.0)), float(f.get("kT", 0.0)), float(f.get("a", 0.0)),
                       float(f.get("lo", 0.0)), float(f.get("hi", 0.0)))
    return arr


def coeffs(funcs, emin: float, emax: float, tol: float, n_max: int, rel: bool = False, device="cuda",
           stream=None, out: torch.Tensor | None = None) -> tuple[int, torch.Tensor]:
    """cheb_coeffs: returns (n, device tensor [n_f, n_max] with zeros beyond n).

    out: optional contiguous FP64 device tensor of n_f * n_max values to write into."""
    lib = load()
    nf = len(funcs)
    nb = ctypes.c_size_t(0)
    _check(lib.cheb_coeffs_workspace_size(nf, n_max, ctypes.byref(nb)))
    ws = _ws(nb.value, device)
    if out is None:
        out = torch.empty((nf, n_max), dtype=torch.float64, device=device)
    elif out.numel() != nf * n_max or out.dtype != torch.float64:
        raise ValueError("coeffs: out must hold n_f * n_max float64 values")
    n = ctypes.c_int32(0)
    _check(lib.cheb_coeffs(make_funcs(funcs), nf, emin, emax, tol, int(rel), n_max, ctypes.byref(n), _ptr(out),
                           ctypes.c_void_p(_aligned(ws)), nb.value, _stream(stream)))
    return n.value, out


def expand_workspace_size(plan: Plan, Mt: Bsr, precision: int, max_terms: int) -> int:
    nb = ctypes.c_size_t(0)
    cb = Mt.c()
    _check(load().cheb_expand_workspace_size(plan.handle, ctypes.byref(cb), precision, max_terms, ctypes.byref(nb)))
    return nb.value


def expand(plan: Plan, Mt: Bsr, n_terms: int, coeffs: torch.Tensor | None, acc: list[torch.Tensor],
           moments: torch.Tensor | None = None, G: torch.Tensor | None = None, gmoments: torch.Tensor | None = None,
           precision: int = F64, ws: torch.Tensor | None = None, stream=None, stepwise: bool = False):
    """cheb_expand (one launch, resident panels) or cheb_expand_stepwise.  acc: FP64 tensors on P_out."""
    lib = load()
    cb = Mt.c()
    nb = ctypes.c_size_t(0)
    if stepwise:
        _check(lib.cheb_expand_stepwise_workspace_size(plan.handle, ctypes.byref(cb), precision, ctypes.byref(nb)))
    else:
        _check(lib.cheb_expand_workspace_size(plan.handle, ctypes.byref(cb), precision, n_terms, ctypes.byref(nb)))
    need = nb.value
    if ws is None or ws.numel() < need + 256:
        ws = _ws(need, Mt.vals.device)
    nf = len(acc)
    arr = (ctypes.c_void_p * max(nf, 1))(*[t.data_ptr() for t in acc])
    stride = coeffs.shape[1] if coeffs is not None else n_terms
    fn = lib.cheb_expand_stepwise if stepwise else lib.cheb_expand
    _check(fn(plan.handle, ctypes.byref(cb), n_terms, _ptr(coeffs), stride, nf, arr, _ptr(moments), _ptr(G),
              _ptr(gmoments), precision, ctypes.c_void_p(_aligned(ws)), need, _stream(stream)))
    return ws


class BatchedPlan(Plan):
    """cheb_plan_create_batched: block-diagonal systems, panels never straddle two systems."""

    def __init__(self, P_out: Bsr, sys_row_start, precision: int = F32, tile: int = -1, stream=None):
        lib = load()
        self.P_out = P_out
        self.precision = precision
        self.tile = tile
        starts = (ctypes.c_int64 * len(sys_row_start))(*[int(x) for x in sys_row_start])
        self.nsys = len(sys_row_start) - 1
        h = ctypes.c_void_p()
        nbytes = ctypes.c_size_t(0)
        s = _stream(stream)
        cb = P_out.c()
        _check(lib.cheb_plan_create_batched(ctypes.byref(cb), precision, tile, self.nsys, starts, ctypes.byref(h),
                                            ctypes.byref(nbytes), s))
        self.handle = h
        self._ws = _ws(nbytes.value, P_out.row_ptr.device)
        _check(lib.cheb_plan_bind(h, ctypes.c_void_p(_aligned(self._ws)), nbytes.value, s))


def plan_col_info(plan: Plan) -> tuple[int, int, int]:
    """cheb_plan_col_info: (panels, largest union, operator entries) of the column-order step kernel (0 panels: not built)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().cheb_plan_col_info(plan.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def plan_lists(plan: Plan, which, stream=None) -> list[torch.Tensor]:
    """cheb_plan_lists_copy of the tables `which`, as device byte tensors."""
    lib = load()
    out = []
    for w in which:
        nb = ctypes.c_size_t(0)
        _check(lib.cheb_plan_lists_copy(plan.handle, w, None, 0, ctypes.byref(nb), _stream(stream)))
        t = torch.empty(max(nb.value, 1), dtype=torch.uint8, device=plan.P_out.row_ptr.device)
        _check(lib.cheb_plan_lists_copy(plan.handle, w, _ptr(t), t.numel(), ctypes.byref(nb), _stream(stream)))
        out.append(t[:nb.value])
    return out


def plan_col_lists(plan: Plan, stream=None) -> list[torch.Tensor]:
    """The six column-kernel lists (cheb_plan_lists_copy 0-5)."""
    return plan_lists(plan, range(6), stream)


def set_plan_builder(builder: str):
    """cheb_set_plan_builder: "device" (the default) or "host" (the reference builders) for later plans."""
    if builder not in ("device", "host"):
        raise ValueError(f"set_plan_builder: 'device' or 'host', not {builder!r}")
    _check(load().cheb_set_plan_builder(1 if builder == "host" else 0))


def ssf_export(A: Bsr, stream=None):
    """cheb_ssf_export: (keyg int32 [nseg, 4] as (c_s, c_e, r_s, r_e), keyv int64 [nseg], vals) on the device."""
    lib = load()
    cb = A.c()
    nseg, nnz = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.cheb_ssf_export_size(ctypes.byref(cb), ctypes.byref(nseg), ctypes.byref(nnz), _stream(stream)))
    dev = A.vals.device
    keyg = torch.empty((max(nseg.value, 1), 4), dtype=torch.int32, device=dev)
    keyv = torch.empty(max(nseg.value, 1), dtype=torch.int64, device=dev)
    vals = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=dev)
    _check(lib.cheb_ssf_export(ctypes.byref(cb), nseg.value, _ptr(keyg), _ptr(keyv), _ptr(vals), _stream(stream)))
    return keyg[:nseg.value], keyv[:nseg.value], vals[:nnz.value]


def ssf_import(n: int, keyg, keyv: torch.Tensor, vals: torch.Tensor, stream=None) -> Bsr:
    """cheb_ssf_import_pattern + cheb_ssf_import_values: the 4x4 block-CSR matrix of SSF descriptors.
    keyg: host or device int32 [nseg, 4]; keyv, vals: device tensors."""
    lib = load()
    kg_host = np.ascontiguousarray(torch.as_tensor(keyg).cpu().numpy().astype(np.int32)).reshape(-1)
    nseg = kg_host.size // 4
    nnzb = ctypes.c_int64(0)
    kgp = kg_host.ctypes.data_as(ctypes.c_void_p)
    _check(lib.cheb_ssf_import_pattern(n, nseg, kgp, ctypes.byref(nnzb), None, None, _stream(stream)))
    dev = vals.device
    rp = torch.empty(n // 4 + 1, dtype=torch.int64, device=dev)
    ci = torch.empty(max(nnzb.value, 1), dtype=torch.int32, device=dev)
    _check(lib.cheb_ssf_import_pattern(n, nseg, kgp, ctypes.byref(nnzb), _ptr(rp), _ptr(ci), _stream(stream)))
    A = Bsr(rp, ci[:nnzb.value], torch.empty((nnzb.value, 4, 4), dtype=torch.float64, device=dev))
    kg_dev = torch.as_tensor(kg_host, device=dev)
    kv = keyv.to(device=dev, dtype=torch.int64).contiguous()
    vv = vals.to(device=dev, dtype=torch.float64).contiguous()
    cb = A.c()
    _check(lib.cheb_ssf_import_values(ctypes.byref(cb), nseg, _ptr(kg_dev), _ptr(kv), _ptr(vv), vv.numel(),
                                      _stream(stream)))
    return A


def plan_resident_info(plan: Plan) -> tuple[int, int, int]:
    a, b, c = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().cheb_plan_resident_info(plan.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def expand_batched(plan: BatchedPlan, Mt: Bsr, max_terms: int, n_terms: torch.Tensor, coeffs: torch.Tensor | None,
                   coeff_offset: torch.Tensor | None, coeff_stride: int, acc: list[torch.Tensor],
                   moments: torch.Tensor | None = None, G: torch.Tensor | None = None,
                   gmoments: torch.Tensor | None = None, moment_stride: int = 0, precision: int = F32,
                   ws: torch.Tensor | None = None, stream=None):
    """cheb_expand_batched: every system of the block-diagonal batch in one launch."""
    lib = load()
    cb = Mt.c()
    nb = ctypes.c_size_t(0)
    _check(lib.cheb_expand_workspace_size(plan.handle, ctypes.byref(cb), precision, max_terms, ctypes.byref(nb)))
    need = nb.value
    if ws is None or ws.numel() < need + 256:
        ws = _ws(need, Mt.vals.device)
    nf = len(acc)
    arr = (ctypes.c_void_p * max(nf, 1))(*[t.data_ptr() for t in acc])
    _check(lib.cheb_expand_batched(plan.handle, ctypes.byref(cb), max_terms, _ptr(n_terms), _ptr(coeffs),
                                   _ptr(coeff_offset), coeff_stride, nf, arr, _ptr(moments), _ptr(G), _ptr(gmoments),
                                   moment_stride or max_terms, precision, ctypes.c_void_p(_aligned(ws)), need,
                                   _stream(stream)))
    return ws


def block_diag(parts: list[Bsr], with_vals: bool = True, stream=None) -> Bsr:
    """cheb_block_diag: the block-diagonal concatenation of parts (FP64 values if with_vals)."""
    dev = parts[0].row_ptr.device
    nbr = sum(p.nbr for p in parts)
    nnzb = sum(p.nnzb for p in parts)
    rp = torch.empty(nbr + 1, dtype=torch.int64, device=dev)
    ci = torch.empty(max(nnzb, 1), dtype=torch.int32, device=dev)[:nnzb]
    vals = torch.empty((nnzb, 4, 4), dtype=torch.float64, device=dev) if with_vals else None
    arr = (CBsr * len(parts))(*[p.c() for p in parts])
    _check(load().cheb_block_diag(len(parts), arr, _ptr(rp), ctypes.c_void_p(ci.data_ptr()), _ptr(vals), 8,
                                  _stream(stream)))
    return Bsr(rp, ci, vals)


def masked_product(plan: Plan, L: Bsr, R: torch.Tensor, C: torch.Tensor, alpha: float = 1.0,
                   D: torch.Tensor | None = None, beta: float = 0.0, stream=None) -> torch.Tensor:
    cb = L.c()
    _check(load().cheb_masked_product(plan.handle, ctypes.byref(cb), _ptr(R), alpha, _ptr(D), beta, _ptr(C),
                                      _stream(stream)))
    return C


def transpose(plan: Plan, A: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    out = torch.empty_like(A) if out is None else out
    _check(load().cheb_transpose(plan.handle, _ptr(A), _ptr(out), _stream(stream)))
    return out


def locality_order(xyz: torch.Tensor, box_L: float, stream=None) -> torch.Tensor:
    """cheb_locality_order: device int64 permutation (new atom -> old atom) along a Hilbert curve."""
    n = xyz.shape[0]
    lib = load()
    nb = int(lib.cheb_locality_order_ws(n))
    ws = _ws(nb, xyz.device)
    perm = torch.empty(n, dtype=torch.int64, device=xyz.device)
    _check(lib.cheb_locality_order(_ptr(xyz), n, float(box_L), _ptr(perm), ctypes.c_void_p(_aligned(ws)), nb,
                                   _stream(stream)))
    return perm


def position_map(P_new: Bsr, P_old: Bsr, perm: torch.Tensor, stream=None) -> torch.Tensor:
    """cheb_position_map: device int64 position in P_old of every block of P_new."""
    m = torch.empty(P_new.nnzb, dtype=torch.int64, device=perm.device)
    ws = _ws(4, perm.device)
    cn, co = P_new.c(), P_old.c()
    _check(load().cheb_position_map(ctypes.byref(cn), ctypes.byref(co), _ptr(perm), _ptr(m),
                                    ctypes.c_void_p(_aligned(ws)), 4, _stream(stream)))
    return m


def gather_rows(src: torch.Tensor, mapping: torch.Tensor, width: int, out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """cheb_gather_rows: out row i = src row mapping[i] (rows of width doubles)."""
    n = mapping.shape[0]
    if out is None:
        out = torch.empty(n * width, dtype=torch.float64, device=src.device)
    _check(load().cheb_gather_rows(_ptr(src), src.numel() // width, _ptr(mapping), n, width, _ptr(out),
                                   _stream(stream)))
    return out


def scatter_rows(src: torch.Tensor, mapping: torch.Tensor, width: int, out: torch.Tensor, stream=None) -> torch.Tensor:
    """cheb_scatter_rows: out row mapping[i] = src row i (rows of width doubles)."""
    _check(load().cheb_scatter_rows(_ptr(src), _ptr(mapping), mapping.shape[0], width, _ptr(out),
                                    out.numel() // width, _stream(stream)))
    return out


def restrict(A: Bsr, P: Bsr, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    out = torch.empty((P.nnzb, 4, 4), dtype=torch.float64, device=A.vals.device) if out is None else out
    ca, cp = A.c(), P.c()
    _check(load().cheb_restrict(ctypes.byref(ca), ctypes.byref(cp), _ptr(out), _stream(stream)))
    return out


def _trace_ws_bytes(B: Bsr) -> int:
    nb = ctypes.c_size_t(0)
    cbb = B.c()
    _check(load().cheb_trace_workspace_size(ctypes.byref(cbb), ctypes.byref(nb)))
    return nb.value


def trace(A: Bsr, B: Bsr, out: torch.Tensor | None = None, stream=None, ws: torch.Tensor | None = None) -> torch.Tensor:
    """cheb_trace: device scalar sum over B's pattern of A_ij B_ij (ws: optional preallocated workspace)."""
    lib = load()
    ca, cbb = A.c(), B.c()
    nb = ctypes.c_size_t(0)
    _check(lib.cheb_trace_workspace_size(ctypes.byref(cbb), ctypes.byref(nb)))
    if ws is None:
        ws = _ws(nb.value, A.vals.device)
    elif ws.numel() < nb.value + 256:
        raise ValueError("trace: workspace too small")
    out = torch.empty(1, dtype=torch.float64, device=A.vals.device) if out is None else out
    _check(lib.cheb_trace(ctypes.byref(ca), ctypes.byref(cbb), _ptr(out), ctypes.c_void_p(_aligned(ws)), nb.value,
                          _stream(stream)))
    return out


def penalty_check(moments: torch.Tensor, n_terms: int, alpha: float, threshold: float, stream=None):
    """cheb_penalty_check: (verdict, value); verdict 0 ok, -1 lower bound, +1 upper bound, 2 not finite."""
    ws = _ws(8 * n_terms + 8, moments.device)
    v, d = ctypes.c_double(0.0), ctypes.c_int32(0)
    _check(load().cheb_penalty_check(_ptr(moments), n_terms, alpha, threshold, ctypes.byref(v), ctypes.byref(d),
                                     ctypes.c_void_p(_aligned(ws)), 8 * n_terms + 8, _stream(stream)))
    return d.value, v.value


def series_value(coeffs: torch.Tensor, moments: torch.Tensor, n_terms: int, stream=None) -> torch.Tensor:
    """cheb_series_value: device scalar c_0/2 t_0 + sum_k c_k t_k."""
    out = torch.empty(1, dtype=torch.float64, device=moments.device)
    _check(load().cheb_series_value(_ptr(coeffs), _ptr(moments), n_terms, _ptr(out), _stream(stream)))
    return out


def mu_nodes(center: float, half: float, n: int) -> list[float]:
    """cheb_mu_nodes: Chebyshev points of the bracket [center - half, center + half]."""
    out = (ctypes.c_double * n)()
    _check(load().cheb_mu_nodes(center, half, n, out))
    return list(out)


def widen_bounds(bounds, verdict: int, frac: float) -> tuple[float, float]:
    """cheb_widen_bounds: the bounds with the side a penalty verdict names moved out."""
    b = (ctypes.c_double * 2)(float(bounds[0]), float(bounds[1]))
    _check(load().cheb_widen_bounds(b, int(verdict), float(frac)))
    return b[0], b[1]


def mlp_bracket(out, emin: float, emax: float, kT: float, min_half_kT: float, max_half_kT: float):
    """cheb_mlp_bracket: (mu_hat, half) in Ha from one network output (2 floats)."""
    o = (ctypes.c_float * 2)(float(out[0]), float(out[1]))
    mu, half = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().cheb_mlp_bracket(o, emin, emax, kT, min_half_kT, max_half_kT, ctypes.byref(mu),
                                   ctypes.byref(half)))
    return mu.value, half.value


def lagrange_weights(nodes, x: float) -> list[float]:
    """cheb_lagrange_weights."""
    n = len(nodes)
    a = (ctypes.c_double * n)(*[float(v) for v in nodes])
    out = (ctypes.c_double * n)()
    _check(load().cheb_lagrange_weights(a, n, x, out))
    return list(out)


def bounds_spd(S: Bsr, k: int = 40, v0: torch.Tensor | None = None, margin_frac: float = 0.01,
               stream=None) -> tuple[float, float]:
    """cheb_bounds_spd: Lanczos bounds with the SPD check and the lower-bound clamp."""
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.cheb_bounds_workspace_size(S.nbr, k, ctypes.byref(nb)))
    ws = _ws(nb.value, S.vals.device)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    cb = S.c()
    _check(lib.cheb_bounds_spd(ctypes.byref(cb), k, _ptr(v0), margin_frac, ctypes.byref(lo), ctypes.byref(hi),
                               ctypes.c_void_p(_aligned(ws)), nb.value, _stream(stream)))
    return lo.value, hi.value


def penalty_trace(moments: torch.Tensor, n_terms: int, alpha: float, stream=None) -> torch.Tensor:
    out = torch.empty(1, dtype=torch.float64, device=moments.device)
    ws = _ws(8 * n_terms, moments.device)
    _check(load().cheb_penalty_trace(_ptr(moments), n_terms, alpha, _ptr(out), ctypes.c_void_p(_aligned(ws)),
                                     8 * n_terms, _stream(stream)))
    return out


def mu_search(gmoments: torch.Tensor, n_terms: int, emin: float, emax: float, kind: int, kT: float, N_e: float,
              tol_N: float, max_iter: int = 100, bracket: tuple[float, float] | None = None,
              stream=None, result: torch.Tensor | None = None, ws: torch.Tensor | None = None) -> torch.Tensor:
    """cheb_mu_search: returns the 48-byte device result as a uint8 tensor.

    result / ws: optional preallocated result (48 bytes) and workspace (>= 8*n_terms + 256 bytes)."""
    res = torch.zeros(48, dtype=torch.uint8, device=gmoments.device) if result is None else result
    if ws is None:
        ws = _ws(8 * n_terms, gmoments.device)
    elif ws.numel() < 8 * n_terms + 256:
        raise ValueError("mu_search: workspace too small")
    br = None if bracket is None else (ctypes.c_double * 2)(*bracket)
    _check(load().cheb_mu_search(_ptr(gmoments), n_terms, emin, emax, kind, kT, N_e, tol_N, max_iter, br,
                                 _ptr(res), ctypes.c_void_p(_aligned(ws)), 8 * n_terms, _stream(stream)))
    return res


MU_SEARCH_NOALLOC_MAX_TERMS = 16384  # CHEB_MU_SEARCH_NOALLOC_MAX_TERMS


def mu_search_noalloc(gmoments: torch.Tensor, n_terms: int, emin: float, emax: float, kind: int, kT: float,
                      N_e: float, tol_N: float, max_iter: int = 100, bracket: tuple[float, float] | None = None,
                      result: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """cheb_mu_search_noalloc: the library's static scratch instead of a workspace.

    Calls on one device share that scratch: do not overlap two of them (see
    include/cheb.h).  result: optional 48-byte device uint8 tensor to reuse.
    """
    res = torch.zeros(48, dtype=torch.uint8, device=gmoments.device) if result is None else result
    br = None if bracket is None else (ctypes.c_double * 2)(*bracket)
    _check(load().cheb_mu_search_noalloc(_ptr(gmoments), n_terms, emin, emax, kind, kT, N_e, tol_N, max_iter, br,
                                         _ptr(res), _stream(stream)))
    return res


def decode_mu_batch(res: torch.Tensor) -> list[dict]:
    """Unpack a [n, 48] batch of mu-search results with one host copy."""
    host = res.cpu()
    return [decode_mu_result(host[i]) for i in range(host.shape[0])]


def decode_mu_result(res: torch.Tensor) -> dict:
    """Unpack the mu-search result (host copy)."""
    b = res.cpu()
    d = b[:32].view(torch.float64).tolist()
    bits = b[32:48].view(torch.int64).tolist()
    it = int(d[2])
    word = [x & ((1 << 64) - 1) for x in bits]
    seq = [(word[i >> 6] >> (i & 63)) & 1 for i in range(it - (1 if d[3] else 0))] if it else []
    return {"mu": d[0], "N": d[1], "iters": it, "converged": bool(d[3]), "bits": seq}


def newton_schulz(plan: Plan, S: Bsr, X0: torch.Tensor, X1: torch.Tensor, tmp: torch.Tensor,
                  stream=None) -> torch.Tensor:
    cb = S.c()
    _check(load().cheb_newton_schulz(plan.handle, ctypes.byref(cb), _ptr(X0), _ptr(X1), _ptr(tmp),
                                     _stream(stream)))
    return X1


def lincomb(weights, xs: list[torch.Tensor], out: torch.Tensor, stream=None) -> torch.Tensor:
    """cheb_lincomb: out = sum_i weights[i] * xs[i]."""
    n = len(xs)
    w = (ctypes.c_double * n)(*[float(v) for v in weights])
    arr = (ctypes.c_void_p * n)(*[t.data_ptr() for t in xs])
    _check(load().cheb_lincomb(n, w, arr, out.numel(), _ptr(out), _stream(stream)))
    return out


def mlp_param_count() -> int:
    return int(load().cheb_mlp_param_count())


def mlp_forward(theta: torch.Tensor, X: torch.Tensor, act: torch.Tensor, out: torch.Tensor, stream=None):
    _check(load().cheb_mlp_forward(_ptr(theta), _ptr(X), X.shape[0], _ptr(act), _ptr(out), _stream(stream)))
    return out


def mlp_loss(out: torch.Tensor, xstar: torch.Tensor, scale: torch.Tensor, dout: torch.Tensor,
             loss: torch.Tensor | None = None, stream=None):
    _check(load().cheb_mlp_loss(_ptr(out), _ptr(xstar), _ptr(scale), out.shape[0], _ptr(dout), _ptr(loss),
                                _stream(stream)))
    return dout


def mlp_backward(theta, X, act, dout, grad, ws, stream=None):
    _check(load().cheb_mlp_backward(_ptr(theta), _ptr(X), X.shape[0], _ptr(act), _ptr(dout), _ptr(grad), _ptr(ws),
                                    _stream(stream)))
    return grad


def mlp_init(seed: int, device, stream=None) -> torch.Tensor:
    """cheb_mlp_init: Xavier-uniform parameters (zero biases) from a seeded counter-based stream."""
    theta = torch.empty(mlp_param_count(), dtype=torch.float32, device=device)
    _check(load().cheb_mlp_init(_ptr(theta), ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _stream(stream)))
    return theta


def mlp_adam(theta, grad, m, v, t: int, lr: float, stream=None):
    _check(load().cheb_mlp_adam(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), t, lr, _stream(stream)))
    return theta


def mlp_features(moments: torch.Tensor, n_rows: int, emin: float, emax: float, N_e: float, out: torch.Tensor,
                 stream=None):
    _check(load().cheb_mlp_features(_ptr(moments), n_rows, emin, emax, N_e, _ptr(out), _stream(stream)))
    return out


def newton_schulz_isqrt(plan: Plan, S: Bsr, Z0: torch.Tensor, Z1: torch.Tensor, tmp1: torch.Tensor,
                        tmp2: torch.Tensor, stream=None) -> torch.Tensor:
    """cheb_newton_schulz_isqrt: Z1 = 1.5 Z0 - 0.5 P(Z0 P(S P(Z0 Z0)))."""
    cb = S.c()
    _check(load().cheb_newton_schulz_isqrt(plan.handle, ctypes.byref(cb), _ptr(Z0), _ptr(Z1), _ptr(tmp1), _ptr(tmp2),
                                           _stream(stream)))
    return Z1
