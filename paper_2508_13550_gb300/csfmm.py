"""Thin Python binding of the C ABI in include/csfmm.h.

Argument marshalling only: every step of the evaluation runs in the CUDA
library libcsfmm.so.  Tensors are torch CUDA tensors (float64, contiguous);
streams default to torch's current stream.  There is no CPU fallback: if the
library cannot be loaded, every call raises.

    plan = plan_create(points, kernel_id, degree, theta, max_leaf, precision=FP64,
                       shrink=False)
    plan = plan_create_targets(sources, targets, kernel_id, degree, theta, max_leaf)
    out  = evaluate(plan, weights)            # weights [nrhs, N] -> [nrhs, N, dim]
    out  = evaluate_host(plan, weights_np)    # host numpy in/out (copies inside)
    out  = evaluate_cstc(plan, weights)       # tree code on the same tree
    out  = direct(points, kernel_id, weights, precision=FP64)
    plan_stats(plan), plan_export_cells(plan), plan_export_list(plan, type), ...
    plan_destroy(plan)
    x, zeta = bve_step(x, zeta, area, dt, omega, degree)        # BVE vortex method, RK4
    grid = remesh_grid_create(grid_points, adj_offsets, adj)    # remeshing grid
    zeta, q = bve_step_remeshed(grid, zeta, area, dt, omega, degree, tracer=q)
    Server(...), autotune(...)                                   # serving, autotuner
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

KERNEL_LAPLACE = 0
KERNEL_BIOT_SAVART = 1
KERNEL_NEWTON = 2
KERNEL_BIHARMONIC = 3
KERNEL_SAL = 4  # bracket of Eq. G_SAL_approx (times 3 rho_w / (4 pi rho_e) for eta_SAL)
KERNEL_ONE = 100
FP64 = 0
FP32_BULK = 1
LIST_PP, LIST_PC, LIST_CP, LIST_CC = 0, 1, 2, 3

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NOT_ON_SPHERE", 3: "OUT_OF_MEMORY", 4: "CUDA",
          5: "TIMEOUT", 6: "UNSUPPORTED", 7: "BUSY", 8: "DEVICE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcsfmm.so")
_lock = threading.Lock()
_lib = None


class CsfmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"csfmm {STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_nrhs", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("rhs_chunk", ctypes.c_int),
                ("shrink", ctypes.c_int), ("no_persistent", ctypes.c_int),
                ("schedule", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


class TuneResult(ctypes.Structure):
    _fields_ = [("max_leaf", ctypes.c_int), ("rhs_chunk", ctypes.c_int),
                ("ms_per_eval", ctypes.c_double), ("rel_err", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("default_rel_err", ctypes.c_double),
                ("candidates", ctypes.c_int), ("from_cache", ctypes.c_int),
                ("no_persistent", ctypes.c_int), ("schedule", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("kernel_id", ctypes.c_int), ("degree", ctypes.c_int),
                ("max_leaf", ctypes.c_int), ("precision", ctypes.c_int),
                ("theta", ctypes.c_double), ("nlevels", ctypes.c_int32),
                ("ncells", ctypes.c_int32), ("nleaves", ctypes.c_int32),
                ("n_list", ctypes.c_int64 * 4), ("evals", ctypes.c_int64 * 4),
                ("pairs_covered", ctypes.c_int64), ("mac_margin", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("build_ms", ctypes.c_double),
                ("launches_per_evaluate", ctypes.c_int64), ("sym_pairs", ctypes.c_int64),
                ("sym_evals", ctypes.c_int64), ("cc_sym_pairs", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["n_list"] = list(self.n_list)
        d["evals"] = list(self.evals)
        return d


class Request(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("N", ctypes.c_int64), ("plan_key", ctypes.c_uint64),
                ("kernel_id", ctypes.c_int), ("degree", ctypes.c_int), ("max_leaf", ctypes.c_int),
                ("precision", ctypes.c_int), ("theta", ctypes.c_double),
                ("weights", ctypes.c_void_p), ("nrhs", ctypes.c_int), ("out", ctypes.c_void_p)]


class RequestTiming(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("submit_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("gpu_ms", ctypes.c_double), ("slot", ctypes.c_int), ("built_plan", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "plans_built",
                                              "plans_evicted", "bytes_held", "peak_bytes_held",
                                              "budget_bytes")] + \
               [("slots", ctypes.c_int), ("max_in_flight", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SERVER_MAX_NRHS = 8
SERVE_FIFO, SERVE_CHEAPEST_FIRST = 0, 1
SCHED_NEAR_64_THREADS, SCHED_ONE_TARGET, SCHED_CHUNK_16 = 1, 2, 4
SCHED_NO_SYMMETRIC, SCHED_NO_OVERLAP, SCHED_SIDE_FIRST, SCHED_TENSOR_NEAR = 8, 16, 32, 64

_VP, _I64, _I32, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_SIGS = {
    "csfmm_plan_create": [_VP, _I64, ctypes.c_int, ctypes.c_int, _D, ctypes.c_int,
                          ctypes.POINTER(Options), _VP, ctypes.POINTER(_VP)],
    "csfmm_plan_create_targets": [_VP, _I64, _VP, _I64, ctypes.c_int, ctypes.c_int, _D,
                                  ctypes.c_int, ctypes.POINTER(Options), _VP, ctypes.POINTER(_VP)],
    "csfmm_evaluate": [_VP, _VP, ctypes.c_int, _VP, _VP],
    "csfmm_evaluate_cstc": [_VP, _VP, ctypes.c_int, _VP, _VP],
    "csfmm_evaluate_host": [_VP, _VP, ctypes.c_int, _VP, _VP],
    "csfmm_evaluate_static": [_VP, _VP, ctypes.c_int, _VP, _VP],
    "csfmm_workspace_create": [_VP, ctypes.c_int, ctypes.POINTER(_VP)],
    "csfmm_workspace_destroy": [_VP],
    "csfmm_evaluate_ws": [_VP, _VP, _VP, ctypes.c_int, _VP, _VP],
    "csfmm_direct": [_VP, _I64, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP],
    "csfmm_direct_targets": [_VP, _I64, ctypes.c_int, _VP, ctypes.c_int, _VP, _I64, _VP,
                             ctypes.c_int, _VP],
    "csfmm_plan_stats": [_VP, ctypes.POINTER(Stats)],
    "csfmm_tune_cache_read": [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(TuneResult)],
    "csfmm_bve_step": [_VP, _VP, _VP, _I64, _D, _D, ctypes.c_int, _D, ctypes.c_int, ctypes.c_int,
                       _VP, _VP, _VP],
    "csfmm_bve_step_remeshed": [_VP, _VP, _VP, _VP, _VP, _D, _D, ctypes.c_int, _D, ctypes.c_int,
                                ctypes.c_int, _VP, _VP, _VP],
    "csfmm_remesh_grid_create": [_VP, _I64, _VP, _VP, _VP, ctypes.POINTER(_VP)],
    "csfmm_remesh": [_VP, _VP, _VP, ctypes.c_int, _VP, _VP],
    "csfmm_remesh_grid_destroy": [_VP],
    "csfmm_autotune": [_VP, _I64, ctypes.c_int, ctypes.c_int, _D, _VP, ctypes.c_int, ctypes.c_int,
                       ctypes.c_char_p, _D, ctypes.POINTER(TuneResult)],
    "csfmm_plan_export_cells": [_VP] + [_VP] * 10,
    "csfmm_plan_export_list": [_VP, ctypes.c_int, _VP, _VP],
    "csfmm_plan_export_order": [_VP, _VP],
    "csfmm_plan_export_proxies": [_VP, _VP],
    "csfmm_plan_export_proxy_weights": [_VP, ctypes.c_int, _VP],
    "csfmm_plan_enable_timing": [_VP, ctypes.c_int],
    "csfmm_plan_phase_times": [_VP, _VP, _VP],
    "csfmm_plan_sync": [_VP, _VP],
    "csfmm_plan_test_wait": [_VP, ctypes.c_int, ctypes.c_double],
    "csfmm_plan_destroy": [_VP],
    "csfmm_server_create": [_I64, ctypes.c_int, ctypes.POINTER(_VP)],
    "csfmm_server_set_policy": [_VP, ctypes.c_int, _D],
    "csfmm_server_submit": [_VP, ctypes.POINTER(Request), ctypes.POINTER(_I64)],
    "csfmm_server_poll": [_VP, _I64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(RequestTiming)],
    "csfmm_server_wait": [_VP, _I64, ctypes.POINTER(RequestTiming)],
    "csfmm_server_drain": [_VP],
    "csfmm_server_stats_get": [_VP, ctypes.POINTER(ServerStats)],
    "csfmm_server_destroy": [_VP],
    "csfmm_last_error": [],
    "csfmm_version": [],
}


def load(path: str | None = None):
    """Loads libcsfmm.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library {p} is missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(p)
        for name, args in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name in ("csfmm_last_error", "csfmm_version") else ctypes.c_int
        _lib = lib
        return lib


def exported_symbols():
    return list(_SIGS)


def _check(rc):
    if rc != 0:
        raise CsfmmError(rc, load().csfmm_last_error().decode())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def kernel_dim(kernel_id: int) -> int:
    return 3 if kernel_id == KERNEL_BIOT_SAVART else 1


class Plan:
    """Owns a csfmm_plan handle (destroyed with the object)."""

    def __init__(self, handle, N, kernel_id, points, nsrc=None, ntgt=None):
        self.handle = handle
        self.N = N  # points in the tree (sources and separate targets)
        self.nsrc = N if nsrc is None else nsrc
        self.ntgt = N if ntgt is None else ntgt
        self.kernel_id = kernel_id
        self.dim = kernel_dim(kernel_id)

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().csfmm_plan_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def plan_create(points, kernel_id: int, degree: int, theta: float, max_leaf: int,
                precision: int = FP64, max_nrhs: int = 16, use_graphs: int = 0, rhs_chunk: int = 0,
                shrink: bool = False, stream=None, no_persistent: bool = False,
                schedule: int = 0):
    import torch
    lib = load()
    opt = Options(precision, max_nrhs, use_graphs, rhs_chunk, int(bool(shrink)),
                  int(bool(no_persistent)), int(schedule))
    h = ctypes.c_void_p()
    N = points.shape[0]
    rc = lib.csfmm_plan_create(_dev(points, torch.float64), N, kernel_id, degree, theta,
                               max_leaf, ctypes.byref(opt), _stream(stream), ctypes.byref(h))
    _check(rc)
    return Plan(h, N, kernel_id, points)


def plan_create_targets(sources, targets, kernel_id: int, degree: int, theta: float,
                        max_leaf: int, precision: int = FP64, max_nrhs: int = 16,
                        use_graphs: int = 0, rhs_chunk: int = 0, shrink: bool = False,
                        stream=None, no_persistent: bool = False, schedule: int = 0):
    """csfmm_plan_create_targets: a plan whose evaluations take weights at the
    sources [nrhs, Ns] and return the sum at separate targets [nrhs, Nt, dim]."""
    import torch
    opt = Options(precision, max_nrhs, use_graphs, rhs_chunk, int(bool(shrink)),
                  int(bool(no_persistent)), int(schedule))
    h = ctypes.c_void_p()
    Ns, Nt = sources.shape[0], targets.shape[0]
    _check(load().csfmm_plan_create_targets(_dev(sources, torch.float64), Ns,
                                            _dev(targets, torch.float64), Nt, kernel_id, degree,
                                            theta, max_leaf, ctypes.byref(opt), _stream(stream),
                                            ctypes.byref(h)))
    return Plan(h, Ns + Nt, kernel_id, None, nsrc=Ns, ntgt=Nt)


def plan_destroy(plan: Plan):
    if plan.handle:
        _check(load().csfmm_plan_destroy(plan.handle))
        plan.handle = None


def evaluate(plan: Plan, weights, out=None, stream=None):
    import torch
    w = weights if weights.dim() == 2 else weights.unsqueeze(0)
    nrhs = w.shape[0]
    if out is None:
        out = torch.empty((nrhs, plan.ntgt, plan.dim), dtype=torch.float64, device=w.device)
    _check(load().csfmm_evaluate(plan.handle, _dev(w, torch.float64), nrhs,
                                 _dev(out, torch.float64), _stream(stream)))
    return out


def evaluate_cstc(plan: Plan, weights, out=None, stream=None):
    """csfmm_evaluate_cstc: the cubed sphere tree code (Algorithm "CSTC") on the
    plan's tree, degree, MAC and precision form; [nrhs, N] -> [nrhs, N, dim]."""
    import torch
    w = weights if weights.dim() == 2 else weights.unsqueeze(0)
    nrhs = w.shape[0]
    if out is None:
        out = torch.empty((nrhs, plan.ntgt, plan.dim), dtype=torch.float64, device=w.device)
    _check(load().csfmm_evaluate_cstc(plan.handle, _dev(w, torch.float64), nrhs,
                                      _dev(out, torch.float64), _stream(stream)))
    return out


STATIC_SCRATCH_BYTES = 64 << 20


def evaluate_static(plan: Plan, weights, out=None, stream=None):
    """csfmm_evaluate_static: same result as evaluate(), with the library's
    static device scratch instead of the plan's workspace (allocates no device
    memory inside the library; `out` may be passed preallocated)."""
    import torch
    w = weights if weights.dim() == 2 else weights.unsqueeze(0)
    nrhs = w.shape[0]
    if out is None:
        out = torch.empty((nrhs, plan.ntgt, plan.dim), dtype=torch.float64, device=w.device)
    _check(load().csfmm_evaluate_static(plan.handle, _dev(w, torch.float64), nrhs,
                                        _dev(out, torch.float64), _stream(stream)))
    return out


def evaluate_host(plan: Plan, weights, out=None, stream=None):
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if w.ndim == 1:
        w = w[None]
    nrhs = w.shape[0]
    if out is None:
        out = np.empty((nrhs, plan.ntgt, plan.dim))
    _check(load().csfmm_evaluate_host(plan.handle, ctypes.c_void_p(w.ctypes.data), nrhs,
                                      ctypes.c_void_p(out.ctypes.data), _stream(stream)))
    return out


def workspace_create(plan: Plan, max_nrhs: int):
    h = ctypes.c_void_p()
    _check(load().csfmm_workspace_create(plan.handle, max_nrhs, ctypes.byref(h)))
    return h


def workspace_destroy(ws):
    _check(load().csfmm_workspace_destroy(ws))


def evaluate_ws(plan: Plan, ws, weights, out=None, stream=None):
    import torch
    w = weights if weights.dim() == 2 else weights.unsqueeze(0)
    nrhs = w.shape[0]
    if out is None:
        out = torch.empty((nrhs, plan.ntgt, plan.dim), dtype=torch.float64, device=w.device)
    _check(load().csfmm_evaluate_ws(plan.handle, ws, _dev(w, torch.float64), nrhs,
                                    _dev(out, torch.float64), _stream(stream)))
    return out


def direct(points, kernel_id: int, weights, precision: int = FP64, targets=None, out=None,
           stream=None):
    import torch
    w = weights if weights.dim() == 2 else weights.unsqueeze(0)
    nrhs = w.shape[0]
    N = points.shape[0]
    dim = kernel_dim(kernel_id)
    lib = load()
    if targets is None:
        if out is None:
            out = torch.empty((nrhs, N, dim), dtype=torch.float64, device=w.device)
        _check(lib.csfmm_direct(_dev(points, torch.float64), N, kernel_id,
                                _dev(w, torch.float64), nrhs, _dev(out, torch.float64),
                                precision, _stream(stream)))
    else:
        nt = targets.shape[0]
        if out is None:
            out = torch.empty((nrhs, nt, dim), dtype=torch.float64, device=w.device)
        _check(lib.csfmm_direct_targets(_dev(points, torch.float64), N, kernel_id,
                                        _dev(w, torch.float64), nrhs,
                                        _dev(targets, torch.int64), nt,
                                        _dev(out, torch.float64), precision, _stream(stream)))
    return out


def bve_step(x, zeta, area, dt: float, omega: float, degree: int = 6, theta: float = 0.7,
             max_leaf: int = 0, precision: int = FP64, x_out=None, zeta_out=None, stream=None):
    """csfmm_bve_step: one RK4 step of the vortex method for the barotropic
    vorticity equation (Sec. 2.3, Eq. BVE_ODEs); degree 0 = direct sum.
    max_leaf 0 = 4 degree^2.  Returns (x_out, zeta_out) on the device."""
    import torch
    N = x.shape[0]
    if x_out is None:
        x_out = torch.empty((N, 3), dtype=torch.float64, device=x.device)
    if zeta_out is None:
        zeta_out = torch.empty((N,), dtype=torch.float64, device=x.device)
    leaf = max_leaf if max_leaf > 0 else max(1, 4 * degree * degree)
    _check(load().csfmm_bve_step(_dev(x, torch.float64), _dev(zeta, torch.float64),
                                 _dev(area, torch.float64), N, float(dt), float(omega),
                                 int(degree), float(theta), int(leaf), int(precision),
                                 _dev(x_out, torch.float64), _dev(zeta_out, torch.float64),
                                 _stream(stream)))
    return x_out, zeta_out


class RemeshGrid:
    """Owns a csfmm_remesh_grid handle (destroyed with the object)."""

    def __init__(self, handle, M, points):
        self.handle = handle
        self.M = M
        self.points = points

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().csfmm_remesh_grid_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def remesh_grid_create(grid, adj_offsets, adj, stream=None) -> RemeshGrid:
    """csfmm_remesh_grid_create: grid device [M,3] FP64, neighbour lists of
    its (Delaunay) triangulation as device int64 CSR (adj_offsets [M+1], adj)."""
    import torch
    h = ctypes.c_void_p()
    M = grid.shape[0]
    _check(load().csfmm_remesh_grid_create(_dev(grid, torch.float64), M,
                                           _dev(adj_offsets, torch.int64), _dev(adj, torch.int64),
                                           _stream(stream), ctypes.byref(h)))
    return RemeshGrid(h, M, grid)


def remesh_grid_destroy(g: RemeshGrid):
    if g.handle:
        _check(load().csfmm_remesh_grid_destroy(g.handle))
        g.handle = None


def remesh(g: RemeshGrid, x, f, out=None, stream=None):
    """csfmm_remesh: values at the grid points from moved particles x [M,3]
    (particle p started at grid point p) carrying f [M] or [nfield, M]."""
    import torch
    nf = 1 if f.dim() == 1 else f.shape[0]
    if out is None:
        out = torch.empty(f.shape, dtype=torch.float64, device=x.device)
    _check(load().csfmm_remesh(g.handle, _dev(x, torch.float64), _dev(f, torch.float64), nf,
                               _dev(out, torch.float64), _stream(stream)))
    return out


def bve_step_remeshed(g: RemeshGrid, zeta, area, dt: float, omega: float, degree: int = 6,
                      theta: float = 0.7, max_leaf: int = 0, precision: int = FP64,
                      grid_plan: Plan | None = None, tracer=None, zeta_out=None,
                      tracer_out=None, stream=None):
    """csfmm_bve_step_remeshed: one RK4 step from the grid points followed by
    remeshing; returns the vorticity at the grid points, or (vorticity,
    tracer) when a tracer is given."""
    import torch
    if zeta_out is None:
        zeta_out = torch.empty((g.M,), dtype=torch.float64, device=zeta.device)
    if tracer is not None and tracer_out is None:
        tracer_out = torch.empty((g.M,), dtype=torch.float64, device=zeta.device)
    leaf = max_leaf if max_leaf > 0 else max(1, 4 * degree * degree)
    _check(load().csfmm_bve_step_remeshed(
        g.handle, grid_plan.handle if grid_plan else None, _dev(zeta, torch.float64),
        _dev(tracer, torch.float64) if tracer is not None else None, _dev(area, torch.float64),
        float(dt), float(omega), int(degree), float(theta), int(leaf), int(precision),
        _dev(zeta_out, torch.float64),
        _dev(tracer_out, torch.float64) if tracer is not None else None, _stream(stream)))
    return zeta_out if tracer is None else (zeta_out, tracer_out)


def autotune(points, kernel_id: int, degree: int, theta: float, weights, precision: int = FP64,
             cache_path: str | None = None, err_factor: float = 2.0) -> dict:
    """csfmm_autotune: fastest leaf size, then launch schedule and tile
    shapes, within err_factor of the default's error (see include/csfmm.h)."""
    import torch
    w = weights if weights.dim() == 2 else weights.unsqueeze(0)
    res = TuneResult()
    _check(load().csfmm_autotune(_dev(points, torch.float64), points.shape[0], kernel_id, degree,
                                 theta, _dev(w, torch.float64), w.shape[0], precision,
                                 cache_path.encode() if cache_path else None, err_factor,
                                 ctypes.byref(res)))
    return res.as_dict()


def tune_cache_read(path: str, key: str) -> dict | None:
    """csfmm_tune_cache_read: the cached choice for key, or None."""
    res = TuneResult()
    rc = load().csfmm_tune_cache_read(path.encode(), key.encode(), ctypes.byref(res))
    if rc == 1 and "not found" in load().csfmm_last_error().decode():
        return None
    _check(rc)
    return res.as_dict()


def plan_stats(plan: Plan) -> dict:
    s = Stats()
    _check(load().csfmm_plan_stats(plan.handle, ctypes.byref(s)))
    return s.as_dict()


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def plan_export_cells(plan: Plan) -> dict:
    nc = plan_stats(plan)["ncells"]
    out = dict(face=np.zeros(nc, np.int32), level=np.zeros(nc, np.int32),
               ia=np.zeros(nc, np.int64), ib=np.zeros(nc, np.int64),
               begin=np.zeros(nc, np.int64), end=np.zeros(nc, np.int64),
               parent=np.zeros(nc, np.int32), child=np.zeros((nc, 4), np.int32),
               centre=np.zeros((nc, 3)), radius=np.zeros(nc))
    keys = ("face", "level", "ia", "ib", "begin", "end", "parent", "child", "centre", "radius")
    _check(load().csfmm_plan_export_cells(plan.handle, *[_np_ptr(out[k]) for k in keys]))
    return out


def plan_export_list(plan: Plan, list_type: int):
    n = plan_stats(plan)["n_list"][list_type]
    t = np.zeros(max(n, 1), np.int32)
    s = np.zeros(max(n, 1), np.int32)
    _check(load().csfmm_plan_export_list(plan.handle, list_type, _np_ptr(t), _np_ptr(s)))
    return t[:n], s[:n]


def plan_export_order(plan: Plan):
    o = np.zeros(plan.N, np.int64)
    _check(load().csfmm_plan_export_order(plan.handle, _np_ptr(o)))
    return o


def plan_export_proxies(plan: Plan):
    st = plan_stats(plan)
    P = (st["degree"] + 1) ** 2
    px = np.zeros((st["ncells"], P, 3))
    _check(load().csfmm_plan_export_proxies(plan.handle, _np_ptr(px)))
    return px


def plan_export_proxy_weights(plan: Plan, nrhs: int = 1):
    st = plan_stats(plan)
    P = (st["degree"] + 1) ** 2
    wb = np.zeros((st["ncells"], nrhs, P))
    _check(load().csfmm_plan_export_proxy_weights(plan.handle, nrhs, _np_ptr(wb)))
    return wb


PHASES = ("gather", "p2m", "m2m", "far", "ppsym", "near", "l2l", "l2p", "ccsym")


def plan_enable_timing(plan: Plan, on: bool = True):
    _check(load().csfmm_plan_enable_timing(plan.handle, 1 if on else 0))


def plan_phase_times(plan: Plan):
    """({phase: summed ms}, number of timed evaluations); clears the record."""
    ms = np.zeros(len(PHASES))
    calls = np.zeros(1, np.int64)
    _check(load().csfmm_plan_phase_times(plan.handle, _np_ptr(ms), _np_ptr(calls)))
    return dict(zip(PHASES, ms.tolist())), int(calls[0])


def plan_sync(plan: Plan, stream=None):
    _check(load().csfmm_plan_sync(plan.handle, _stream(stream)))


def plan_test_wait(plan: Plan, never_ready: bool, limit_ms: float = 2000.0):
    """csfmm_plan_test_wait: the bound of the persistent launch's dependency
    waits, and the test hook that makes every wait unsatisfiable."""
    _check(load().csfmm_plan_test_wait(plan.handle, int(bool(never_ready)), float(limit_ms)))


class Server:
    """csfmm_server: continuous batching over resident plans (one scheduler
    thread in the library; this class only marshals arguments)."""

    def __init__(self, budget_bytes: int, slots: int, policy: int | None = None,
                 age_ms: float = 250.0):
        self.handle = ctypes.c_void_p()
        _check(load().csfmm_server_create(int(budget_bytes), int(slots), ctypes.byref(self.handle)))
        if policy is not None:
            self.set_policy(policy, age_ms)

    def set_policy(self, policy: int, age_ms: float = 250.0):
        """csfmm_server_set_policy: SERVE_FIFO or SERVE_CHEAPEST_FIRST."""
        _check(load().csfmm_server_set_policy(self.handle, int(policy), float(age_ms)))

    def submit(self, points, plan_key, kernel_id, degree, theta, max_leaf, precision, weights,
               out):
        """Queues a request; points, weights and out are CUDA tensors that must
        stay alive until the request completes.  Returns the request id."""
        import torch
        req = Request(_dev(points, torch.float64).value, points.shape[0], int(plan_key),
                      int(kernel_id), int(degree), int(max_leaf), int(precision), float(theta),
                      _dev(weights, torch.float64).value, weights.shape[0],
                      _dev(out, torch.float64).value)
        rid = ctypes.c_int64()
        _check(load().csfmm_server_submit(self.handle, ctypes.byref(req), ctypes.byref(rid)))
        return rid.value

    def poll(self, rid):
        done = ctypes.c_int()
        t = RequestTiming()
        _check(load().csfmm_server_poll(self.handle, rid, ctypes.byref(done), ctypes.byref(t)))
        return bool(done.value), t.as_dict()

    def wait(self, rid):
        t = RequestTiming()
        rc = load().csfmm_server_wait(self.handle, rid, ctypes.byref(t))
        return rc, t.as_dict()

    def drain(self):
        _check(load().csfmm_server_drain(self.handle))

    def stats(self):
        s = ServerStats()
        _check(load().csfmm_server_stats_get(self.handle, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if self.handle:
            _check(load().csfmm_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def last_error() -> str:
    return load().csfmm_last_error().decode()


def version() -> str:
    return load().csfmm_version().decode()
