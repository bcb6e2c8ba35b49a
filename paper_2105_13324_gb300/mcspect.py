"""Thin ctypes binding of libmcspect.so (include/mcspect.h).

Argument marshalling only: every step runs in the CUDA library.  Device
buffers are torch CUDA tensors (PyTorch provides device memory and streams);
host buffers are NumPy arrays.  Function names follow the C entry points.

The library is loaded from paper_2105_13324_gb300/_build/libmcspect.so; if
it is missing, every call raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import phantoms as _ph

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmcspect.so")

MC_OK, MC_EINVAL, MC_ENOMEM, MC_ECUDA = 0, -1, -2, -3
MC_FP32, MC_FP64 = 0, 1
MC_VAL_F32, MC_VAL_F16, MC_VAL_BF16, MC_VAL_F16_A, MC_VAL_BF16_A = 0, 1, 2, 3, 4
VALUE_TYPES = {"f32": MC_VAL_F32, "f16": MC_VAL_F16, "bf16": MC_VAL_BF16, "f16_a": MC_VAL_F16_A,
               "bf16_a": MC_VAL_BF16_A}
MC_TALLY_ALL, MC_TALLY_PRIMARY, MC_TALLY_FORCED, MC_TALLY_FORCED_DIRECTION = 0, 1, 2, 4
FD_SCALE = 2.0 ** 48  # forced-detection weights are tallied as rint(w * 2^48)
FATE_NAMES = ("absorbed", "below_window", "escape", "cap")

# every symbol include/mcspect.h declares
EXPORTED = (
    "mc_plan_create", "mc_plan_build", "mc_plan_free", "mc_plan_tally", "mc_events_route", "mc_system_from_keys",
    "mc_vector_sum", "mc_mlem_start", "mc_build_system", "mc_build_system_range", "mc_system_from_events",
    "mc_system_from_weighted_events", "mc_system_export_values", "mc_system_free",
    "mc_system_info_get", "mc_system_export_csc", "mc_system_export_csr", "mc_system_set_value_type", "mc_system_set_spmv_layout",
    "mc_project", "mc_backproject", "mc_sensitivity", "mc_mlem_init", "mlem_iterate", "mlem_iterate_noalloc",
    "mc_system_subset", "osem_iterate", "mc_project_ratio", "mc_loglik", "mc_project_f64", "mc_backproject_f64", "mc_prior_quadratic",
    "mc_prior_quadratic_f64", "mc_pgd_step", "mc_system_autotune", "mc_batch_create", "mc_batch_mlem",
    "mc_batch_free", "mc_batch_mlem_persistent",
    "mc_trace_histories", "mc_debug_kn", "mc_debug_beam", "mc_debug_distance_map", "mc_kernel_launches",
    "mc_last_error",
)

RECORD_DTYPE = np.dtype([
    ("fate", np.uint8), ("n_events", np.uint8), ("pad", np.uint16),
    ("n_virtual", np.uint32), ("n_real", np.uint32), ("n_compton", np.uint32),
    ("n_draws", np.uint32), ("pad2", np.uint32), ("e_final_kev", np.float64),
    ("event_row", np.int32, (4,)),
])


class McError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mcspect error {code}: {msg}")
        self.code = code


class MCPhantom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("voxel_mm", ctypes.c_double), ("material_host", ctypes.c_void_p),
                ("n_materials", ctypes.c_int32), ("rho_host", ctypes.c_void_p),
                ("z_over_a_host", ctypes.c_void_p), ("z_eff_host", ctypes.c_void_p)]


class MCGeometry(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int32), ("start_deg", ctypes.c_double), ("arc_deg", ctypes.c_double),
                ("n_bins_u", ctypes.c_int32), ("n_bins_v", ctypes.c_int32), ("bin_mm", ctypes.c_double),
                ("radius_mm", ctypes.c_double), ("hole_len_mm", ctypes.c_double),
                ("hole_diam_mm", ctypes.c_double), ("fwhm_mm", ctypes.c_double), ("e0_kev", ctypes.c_double),
                ("window_frac", ctypes.c_double), ("photo_k", ctypes.c_double), ("precision", ctypes.c_int32),
                ("tally", ctypes.c_int32)]


class MCSystemInfo(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_events", ctypes.c_int64), ("first_history", ctypes.c_uint64),
                ("n_histories", ctypes.c_uint64), ("fates", ctypes.c_uint64 * 4), ("max_count", ctypes.c_uint32),
                ("value_type", ctypes.c_int32), ("build_ms_transport", ctypes.c_double),
                ("build_ms_assembly", ctypes.c_double), ("build_ms_detect", ctypes.c_double),
                ("spmv_fwd", ctypes.c_int32), ("spmv_bwd", ctypes.c_int32), ("weighted", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libmcspect.so (build it first with paper_2105_13324_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"libmcspect.so not found at {p}: run paper_2105_13324_gb300.build.build()")
        L = ctypes.CDLL(p)
        vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "mc_plan_create": [vp, vp, vp, vp],
            "mc_plan_build": [vp, u64, u64, u64, vp, vp],
            "mc_plan_free": [vp],
            "mc_plan_tally": [vp, u64, u64, u64, vp, i64, vp, vp, vp],
            "mc_events_route": [vp, i64, i64, i64, i32, vp, vp, vp],
            "mc_system_from_keys": [i64, i64, vp, i64, u64, u64, vp, vp],
            "mc_vector_sum": [i64, vp, vp, vp],
            "mc_mlem_start": [i64, vp, dbl, vp, vp],
            "mc_build_system": [vp, vp, u64, u64, vp, vp],
            "mc_build_system_range": [vp, vp, u64, u64, u64, vp, vp],
            "mc_system_from_events": [i64, i64, vp, vp, i64, u64, u64, vp, vp],
            "mc_system_from_weighted_events": [i64, i64, vp, vp, vp, i64, u64, u64, vp, vp],
            "mc_system_export_values": [vp, vp, vp, vp],
            "mc_system_free": [vp],
            "mc_system_info_get": [vp, vp],
            "mc_system_export_csc": [vp, vp, vp, vp, vp, vp],
            "mc_system_export_csr": [vp, vp, vp, vp, vp],
            "mc_system_set_value_type": [vp, i32, i32],
            "mc_project": [vp, vp, vp, vp],
            "mc_backproject": [vp, vp, vp, vp],
            "mc_sensitivity": [vp, vp, vp],
            "mc_mlem_init": [vp, vp, vp, vp],
            "mlem_iterate": [vp, vp, vp, i32, vp, vp],
            "mlem_iterate_noalloc": [vp, vp, vp, i32, vp, vp],
            "mc_system_subset": [vp, i64, i32, i32, vp, vp],
            "osem_iterate": [vp, vp, i32, vp, vp, vp, i32, vp],
            "mc_project_ratio": [vp, vp, vp, vp, vp],
            "mc_loglik": [vp, vp, vp, vp, vp],
            "mc_project_f64": [vp, vp, vp, vp],
            "mc_backproject_f64": [vp, vp, vp, vp],
            "mc_prior_quadratic": [i32, i32, i32, dbl, vp, vp, vp, vp],
            "mc_prior_quadratic_f64": [i32, i32, i32, dbl, vp, vp, vp, vp],
            "mc_pgd_step": [i64, dbl, vp, vp, vp, vp, vp],
            "mc_system_autotune": [vp, vp],
            "mc_system_set_spmv_layout": [vp, i32, i32, vp],
            "mc_batch_create": [vp, i32, vp, vp, vp],
            "mc_batch_mlem": [vp, i32, vp],
            "mc_batch_mlem_persistent": [vp, i32, vp],
            "mc_batch_free": [vp],
            "mc_trace_histories": [vp, vp, u64, u64, u64, vp],
            "mc_debug_kn": [dbl, i32, u64, u64, vp, vp],
            "mc_debug_beam": [vp, vp, u64, u64, vp, vp, dbl, vp],
            "mc_debug_distance_map": [vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.mc_kernel_launches.argtypes = []
        L.mc_kernel_launches.restype = ctypes.c_uint64
        L.mc_last_error.argtypes = []
        L.mc_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(rc):
    if rc != MC_OK:
        raise McError(rc, load().mc_last_error().decode(errors="replace"))


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


class _Inputs:
    """C structs for a Phantom + Geometry, keeping NumPy buffers alive."""

    def __init__(self, phantom: _ph.Phantom, geometry: _ph.Geometry, precision: int, primary_only: bool = False,
                 forced: bool = False, forced_direction: bool = False):
        self.material = np.ascontiguousarray(phantom.material, dtype=np.uint8)
        self.rho = np.ascontiguousarray(phantom.rho, dtype=np.float64)
        self.zoa = np.ascontiguousarray(phantom.z_over_a, dtype=np.float64)
        self.zeff = np.ascontiguousarray(phantom.z_eff, dtype=np.float64)
        nz, ny, nx = self.material.shape
        self.ph = MCPhantom(nx, ny, nz, float(phantom.voxel_mm), self.material.ctypes.data, len(self.rho),
                            self.rho.ctypes.data, self.zoa.ctypes.data, self.zeff.ctypes.data)
        g = geometry
        self.geo = MCGeometry(g.n_views, float(g.start_deg), float(g.arc_deg), g.n_bins_u, g.n_bins_v,
                              float(g.bin_mm), float(g.radius_mm), float(g.hole_len_mm), float(g.hole_diam_mm),
                              float(g.fwhm_mm), float(g.e0_kev), float(g.window_frac), float(g.photo_k),
                              int(precision),
                              (MC_TALLY_PRIMARY if primary_only else 0) | (MC_TALLY_FORCED if forced else 0)
                              | (MC_TALLY_FORCED_DIRECTION if forced_direction else 0))


def _precision(p):
    if p in ("fp32", MC_FP32):
        return MC_FP32
    if p in ("fp64", MC_FP64):
        return MC_FP64
    raise ValueError(f"precision must be 'fp32' or 'fp64', got {p!r}")


class System:
    """Owner of an mc_system handle (device-resident system matrix)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self):
        if not self._h:
            raise ValueError("system was freed")
        return self._h

    def info(self) -> dict:
        inf = MCSystemInfo()
        _check(load().mc_system_info_get(self.handle, ctypes.byref(inf)))
        return {"n_rows": inf.n_rows, "n_cols": inf.n_cols, "nnz": inf.nnz, "n_events": inf.n_events,
                "first_history": inf.first_history, "n_histories": inf.n_histories,
                "fates": [int(v) for v in inf.fates], "max_count": inf.max_count,
                "value_type": inf.value_type, "build_ms_transport": inf.build_ms_transport,
                "build_ms_assembly": inf.build_ms_assembly, "build_ms_detect": inf.build_ms_detect,
                "spmv_fwd": inf.spmv_fwd, "spmv_bwd": inf.spmv_bwd, "weighted": bool(inf.weighted)}

    @property
    def shape(self):
        i = self.info()
        return i["n_rows"], i["n_cols"]

    def export_csc(self, stream=None):
        i = self.info()
        cp = np.zeros(i["n_cols"] + 1, np.int64)
        ri = np.zeros(max(i["nnz"], 1), np.int32)
        cnt = np.zeros(max(i["nnz"], 1), np.uint32)
        nv = np.zeros(i["n_cols"], np.uint32)
        _check(load().mc_system_export_csc(self.handle, cp.ctypes.data, ri.ctypes.data, cnt.ctypes.data,
                                           nv.ctypes.data, _stream_ptr(stream)))
        return cp, ri[:i["nnz"]], cnt[:i["nnz"]], nv

    def export_csr(self, stream=None):
        i = self.info()
        rp = np.zeros(i["n_rows"] + 1, np.int64)
        ci = np.zeros(max(i["nnz"], 1), np.int32)
        cnt = np.zeros(max(i["nnz"], 1), np.uint32)
        _check(load().mc_system_export_csr(self.handle, rp.ctypes.data, ci.ctypes.data, cnt.ctypes.data,
                                           _stream_ptr(stream)))
        return rp, ci[:i["nnz"]], cnt[:i["nnz"]]

    def export_values(self, stream=None):
        """Entries as float64 in the CSC and CSR orders of export_csc /
        export_csr: counts, or the weight sums of a weighted system."""
        n = self.info()["nnz"]
        a = np.zeros(max(n, 1), np.float64)
        b = np.zeros(max(n, 1), np.float64)
        _check(load().mc_system_export_values(self.handle, a.ctypes.data, b.ctypes.data, _stream_ptr(stream)))
        return a[:n], b[:n]

    def set_value_type(self, value_type, allow_rounding=False):
        vt = VALUE_TYPES.get(value_type, value_type)
        _check(load().mc_system_set_value_type(self.handle, int(vt), int(bool(allow_rounding))))

    def free(self):
        if self._h:
            _check(load().mc_system_free(self._h))
            self._h = None

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.mc_system_free(self._h)
                self._h = None
        except Exception:
            pass


class Plan:
    """Owner of an mc_plan handle: phantom + geometry resident on the device."""

    def __init__(self, phantom, geometry, precision="fp32", stream=None, primary_only=False, forced=False,
                 forced_direction=False):
        inp = _Inputs(phantom, geometry, _precision(precision), primary_only, forced, forced_direction)
        h = ctypes.c_void_p()
        _check(load().mc_plan_create(ctypes.byref(inp.ph), ctypes.byref(inp.geo), _stream_ptr(stream),
                                     ctypes.byref(h)))
        self._h = h

    def build(self, first: int, count: int, seed: int, stream=None) -> System:
        return mc_plan_build(self, first, count, seed, stream)

    def free(self):
        if self._h:
            _check(load().mc_plan_free(self._h))
            self._h = None

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.mc_plan_free(self._h)
                self._h = None
        except Exception:
            pass


def mc_plan_create(phantom, geometry, precision="fp32", stream=None, primary_only=False, forced=False,
                   forced_direction=False) -> Plan:
    return Plan(phantom, geometry, precision, stream, primary_only, forced, forced_direction)


def mc_plan_build(plan: Plan, first: int, count: int, seed: int, stream=None) -> System:
    if not plan._h:
        raise ValueError("plan was freed")
    h = ctypes.c_void_p()
    _check(load().mc_plan_build(plan._h, int(first), int(count), int(seed), _stream_ptr(stream), ctypes.byref(h)))
    return System(h)


def mc_plan_free(plan: Plan):
    plan.free()


def mc_plan_tally(plan: Plan, first: int, count: int, seed: int, stream=None):
    """Event keys v*M + j (int64 CUDA tensor holding the unsigned keys) and
    fates of histories first..first+count-1; the buffer is resized and the
    deterministic tally repeated if the first estimate is too small."""
    import torch
    if not plan._h:
        raise ValueError("plan was freed")
    n = ctypes.c_int64(0)
    fates = (ctypes.c_uint64 * 4)()
    cap = max(1024, int(count) // 64)
    for _ in range(2):
        keys = torch.empty(cap, dtype=torch.int64, device="cuda")
        rc = load().mc_plan_tally(plan._h, int(first), int(count), int(seed), _dev_ptr(keys), cap, ctypes.byref(n),
                                  fates, _stream_ptr(stream))
        if rc == MC_OK:
            return keys[:n.value], [int(f) for f in fates]
        if n.value <= cap:
            _check(rc)
        cap = int(n.value)
    _check(rc)


def mc_events_route(keys, n_rows: int, rows_per_view: int, n_parts: int, stream=None):
    """Events grouped by the part owning their view, rows renumbered per
    part: (int64 CUDA tensor, list of per-part counts)."""
    import torch
    out = torch.empty_like(keys)
    counts = (ctypes.c_int64 * int(n_parts))()
    n = int(keys.numel())
    _check(load().mc_events_route(_dev_ptr(keys, torch.int64) if n else None, n, int(n_rows), int(rows_per_view),
                                  int(n_parts), _dev_ptr(out, torch.int64) if n else None, counts,
                                  _stream_ptr(stream)))
    return out, [int(c) for c in counts]


def mc_system_from_keys(n_rows: int, n_cols: int, keys, first: int, count: int, stream=None) -> System:
    import torch
    n = int(keys.numel())
    h = ctypes.c_void_p()
    _check(load().mc_system_from_keys(int(n_rows), int(n_cols), _dev_ptr(keys, torch.int64) if n else None, n,
                                      int(first), int(count), _stream_ptr(stream), ctypes.byref(h)))
    return System(h)


def mc_vector_sum(v, out, stream=None):
    import torch
    _check(load().mc_vector_sum(int(v.numel()), _dev_ptr(v, torch.float32), _dev_ptr(out, torch.float64),
                                _stream_ptr(stream)))
    return out


def mc_mlem_start(sens, sum_y: float, x, stream=None):
    import torch
    _check(load().mc_mlem_start(int(x.numel()), _dev_ptr(sens, torch.float64), float(sum_y),
                                _dev_ptr(x, torch.float32), _stream_ptr(stream)))
    return x


def mc_kernel_launches() -> int:
    return int(load().mc_kernel_launches())


def mc_build_system(phantom, geometry, n_histories: int, seed: int, precision="fp32", stream=None,
                    primary_only=False, forced=False, forced_direction=False) -> System:
    inp = _Inputs(phantom, geometry, _precision(precision), primary_only, forced, forced_direction)
    h = ctypes.c_void_p()
    _check(load().mc_build_system(ctypes.byref(inp.ph), ctypes.byref(inp.geo), int(n_histories), int(seed),
                                  _stream_ptr(stream), ctypes.byref(h)))
    return System(h)


def mc_build_system_range(phantom, geometry, first: int, count: int, seed: int, precision="fp32",
                          stream=None, primary_only=False, forced=False, forced_direction=False) -> System:
    inp = _Inputs(phantom, geometry, _precision(precision), primary_only, forced, forced_direction)
    h = ctypes.c_void_p()
    _check(load().mc_build_system_range(ctypes.byref(inp.ph), ctypes.byref(inp.geo), int(first), int(count),
                                        int(seed), _stream_ptr(stream), ctypes.byref(h)))
    return System(h)


def mc_system_from_events(n_rows: int, n_cols: int, rows, cols, first: int, count: int, stream=None) -> System:
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    if r.shape != c.shape:
        raise ValueError("rows and cols differ in length")
    h = ctypes.c_void_p()
    _check(load().mc_system_from_events(int(n_rows), int(n_cols), r.ctypes.data, c.ctypes.data, int(r.size),
                                        int(first), int(count), _stream_ptr(stream), ctypes.byref(h)))
    return System(h)


def mc_system_from_weighted_events(n_rows: int, n_cols: int, rows, cols, weights, first: int, count: int,
                                   stream=None) -> System:
    """weights: fixed-point event weights (uint64, w * 2^48 rounded)."""
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    w = np.ascontiguousarray(weights, dtype=np.uint64)
    if r.shape != c.shape or r.shape != w.shape:
        raise ValueError("rows, cols and weights differ in length")
    h = ctypes.c_void_p()
    _check(load().mc_system_from_weighted_events(int(n_rows), int(n_cols), r.ctypes.data, c.ctypes.data,
                                                 w.ctypes.data, int(r.size), int(first), int(count),
                                                 _stream_ptr(stream), ctypes.byref(h)))
    return System(h)


def mc_project(sys: System, x, q, stream=None):
    import torch
    _check(load().mc_project(sys.handle, _dev_ptr(x, torch.float32), _dev_ptr(q, torch.float32),
                             _stream_ptr(stream)))
    return q


def mc_backproject(sys: System, r, b, stream=None):
    import torch
    _check(load().mc_backproject(sys.handle, _dev_ptr(r, torch.float32), _dev_ptr(b, torch.float32),
                                 _stream_ptr(stream)))
    return b


def mc_sensitivity(sys: System, s, stream=None):
    import torch
    _check(load().mc_sensitivity(sys.handle, _dev_ptr(s, torch.float64), _stream_ptr(stream)))
    return s


def mc_mlem_init(sys: System, y, x, stream=None):
    import torch
    _check(load().mc_mlem_init(sys.handle, _dev_ptr(y, torch.float32), _dev_ptr(x, torch.float32),
                               _stream_ptr(stream)))
    return x


def mlem_iterate(sys: System, y, x, n_iter: int, loglik: bool = False, stream=None):
    """n_iter ML-EM updates of x in place; returns the log-likelihoods of the
    iterates before each update when loglik is set (else None)."""
    import torch
    ll = np.zeros(max(n_iter, 1), np.float64) if loglik else None
    _check(load().mlem_iterate(sys.handle, _dev_ptr(y, torch.float32), _dev_ptr(x, torch.float32), int(n_iter),
                               ll.ctypes.data if loglik else None, _stream_ptr(stream)))
    return ll[:n_iter] if loglik else None


def mlem_iterate_noalloc(sys: System, y, x, n_iter: int, loglik: bool = False, stream=None):
    """mlem_iterate without device allocation (static scratch, size-limited)."""
    import torch
    ll = np.zeros(max(n_iter, 1), np.float64) if loglik else None
    _check(load().mlem_iterate_noalloc(sys.handle, _dev_ptr(y, torch.float32), _dev_ptr(x, torch.float32),
                                       int(n_iter), ll.ctypes.data if loglik else None, _stream_ptr(stream)))
    return ll[:n_iter] if loglik else None


def mc_system_subset(parent: System, rows_per_view: int, n_subsets: int, subset: int, stream=None) -> System:
    h = ctypes.c_void_p()
    _check(load().mc_system_subset(parent.handle, int(rows_per_view), int(n_subsets), int(subset),
                                   _stream_ptr(stream), ctypes.byref(h)))
    return System(h)


def osem_iterate(fwd, back, y, x, n_iter: int, add=None, stream=None):
    """n_iter ordered-subset EM sweeps; fwd/back: lists of subset systems."""
    import torch
    if len(fwd) != len(back) or not fwd:
        raise ValueError("fwd and back need the same, non-zero number of subsets")
    arr = (ctypes.c_void_p * len(fwd))(*[f.handle for f in fwd])
    brr = (ctypes.c_void_p * len(back))(*[b.handle for b in back])
    _check(load().osem_iterate(arr, brr, len(fwd), _dev_ptr(y, torch.float32),
                               _dev_ptr(add, torch.float32) if add is not None else None,
                               _dev_ptr(x, torch.float32), int(n_iter), _stream_ptr(stream)))
    return x


def mc_project_ratio(sys: System, x, y, r, stream=None):
    import torch
    _check(load().mc_project_ratio(sys.handle, _dev_ptr(x, torch.float32), _dev_ptr(y, torch.float32),
                                   _dev_ptr(r, torch.float32), _stream_ptr(stream)))
    return r


def mc_loglik(sys: System, x, y, value, stream=None):
    import torch
    _check(load().mc_loglik(sys.handle, _dev_ptr(x, torch.float32), _dev_ptr(y, torch.float32),
                            _dev_ptr(value, torch.float64), _stream_ptr(stream)))
    return value


def mc_project_f64(sys: System, x, q, stream=None):
    import torch
    _check(load().mc_project_f64(sys.handle, _dev_ptr(x, torch.float64), _dev_ptr(q, torch.float64),
                                 _stream_ptr(stream)))
    return q


def mc_backproject_f64(sys: System, r, b, stream=None):
    import torch
    _check(load().mc_backproject_f64(sys.handle, _dev_ptr(r, torch.float64), _dev_ptr(b, torch.float64),
                                     _stream_ptr(stream)))
    return b


def mc_prior_quadratic(shape, beta: float, x, grad=None, value=None, stream=None):
    """Quadratic 6-neighbour prior of an image of shape (nz, ny, nx)."""
    import torch
    nz, ny, nx = shape
    f = load().mc_prior_quadratic if x.dtype == torch.float32 else load().mc_prior_quadratic_f64
    _check(f(int(nx), int(ny), int(nz), float(beta), _dev_ptr(x, x.dtype),
             _dev_ptr(grad, x.dtype) if grad is not None else None,
             _dev_ptr(value, torch.float64) if value is not None else None, _stream_ptr(stream)))
    return grad, value


def mc_pgd_step(alpha: float, sens, bp, x, gp=None, stream=None):
    import torch
    _check(load().mc_pgd_step(int(x.numel()), float(alpha), _dev_ptr(sens, torch.float64),
                              _dev_ptr(bp, torch.float32), _dev_ptr(gp, torch.float32) if gp is not None else None,
                              _dev_ptr(x, torch.float32), _stream_ptr(stream)))
    return x


def mc_system_set_spmv_layout(sys: System, fwd: int, bwd: int, stream=None):
    """Projector layouts: 0 streaming layout, 1..32 lanes per row (column)
    group, -1 keep; returns the layouts now in use."""
    _check(load().mc_system_set_spmv_layout(sys.handle, int(fwd), int(bwd), _stream_ptr(stream)))
    i = sys.info()
    return i["spmv_fwd"], i["spmv_bwd"]


def mc_system_autotune(sys: System, stream=None):
    _check(load().mc_system_autotune(sys.handle, _stream_ptr(stream)))
    i = sys.info()
    return i["spmv_fwd"], i["spmv_bwd"]


class Batch:
    """Batched ML-EM of many systems (mc_batch); keeps its tensors alive."""

    def __init__(self, systems, ys, xs):
        import torch
        if not (len(systems) == len(ys) == len(xs)) or not systems:
            raise ValueError("need the same, non-zero number of systems, projections and images")
        self._keep = (list(systems), list(ys), list(xs))
        n = len(systems)
        sarr = (ctypes.c_void_p * n)(*[s.handle for s in systems])
        yarr = (ctypes.c_void_p * n)(*[_dev_ptr(y, torch.float32).value for y in ys])
        xarr = (ctypes.c_void_p * n)(*[_dev_ptr(x, torch.float32).value for x in xs])
        h = ctypes.c_void_p()
        _check(load().mc_batch_create(sarr, n, yarr, xarr, ctypes.byref(h)))
        self._h = h

    def mlem(self, n_iter: int, stream=None):
        _check(load().mc_batch_mlem(self._h, int(n_iter), _stream_ptr(stream)))

    def mlem_persistent(self, n_iter: int, stream=None):
        _check(load().mc_batch_mlem_persistent(self._h, int(n_iter), _stream_ptr(stream)))

    def free(self):
        if self._h:
            _check(load().mc_batch_free(self._h))
            self._h = None

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.mc_batch_free(self._h)
                self._h = None
        except Exception:
            pass


def mc_batch_create(systems, ys, xs) -> Batch:
    return Batch(systems, ys, xs)


def mc_batch_mlem(batch: Batch, n_iter: int, stream=None):
    batch.mlem(n_iter, stream)


def mc_batch_mlem_persistent(batch: Batch, n_iter: int, stream=None):
    batch.mlem_persistent(n_iter, stream)


def mc_batch_free(batch: Batch):
    batch.free()


def mc_trace_histories(phantom, geometry, seed: int, first: int, count: int, precision="fp64",
                       primary_only=False, forced_direction=False) -> np.ndarray:
    inp = _Inputs(phantom, geometry, _precision(precision), primary_only, False, forced_direction)
    out = np.zeros(count, RECORD_DTYPE)
    _check(load().mc_trace_histories(ctypes.byref(inp.ph), ctypes.byref(inp.geo), int(seed), int(first),
                                     int(count), out.ctypes.data))
    return out


def mc_debug_kn(e_kev: float, seed: int, n: int, precision="fp64"):
    c = np.zeros(n, np.float64)
    e = np.zeros(n, np.float64)
    _check(load().mc_debug_kn(float(e_kev), _precision(precision), int(seed), int(n), c.ctypes.data, e.ctypes.data))
    return c, e


def mc_debug_distance_map(phantom) -> np.ndarray:
    """The float forced-detection traversal's distance map, shaped like the material grid."""
    mat = np.ascontiguousarray(phantom.material, dtype=np.uint8)
    rho = np.ascontiguousarray(phantom.rho, dtype=np.float64)
    zoa = np.ascontiguousarray(phantom.z_over_a, dtype=np.float64)
    zeff = np.ascontiguousarray(phantom.z_eff, dtype=np.float64)
    nz, ny, nx = mat.shape
    ph = MCPhantom(nx, ny, nz, float(phantom.voxel_mm), mat.ctypes.data, len(rho), rho.ctypes.data,
                   zoa.ctypes.data, zeff.ctypes.data)
    out = np.zeros(mat.shape, np.uint8)
    _check(load().mc_debug_distance_map(ctypes.byref(ph), out.ctypes.data))
    return out


def mc_debug_beam(phantom, geometry, seed: int, n: int, p0, d, e_kev: float, precision="fp64") -> int:
    inp = _Inputs(phantom, geometry, _precision(precision))
    p = np.ascontiguousarray(p0, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    out = ctypes.c_uint64(0)
    _check(load().mc_debug_beam(ctypes.byref(inp.ph), ctypes.byref(inp.geo), int(seed), int(n), p.ctypes.data,
                                dd.ctypes.data, float(e_kev), ctypes.byref(out)))
    return int(out.value)
