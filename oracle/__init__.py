"""CPU oracle for the cubed-sphere FMM (Chen & Krasny, arXiv 2508.13550).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it.

The arithmetic lives in ``csfmm_oracle.c`` (plain FP64 C, OpenMP over
independent targets), compiled on first use with the host C compiler and
``-ffp-contract=off`` so that geometric decisions are evaluated without fused
multiply-add.  This module only marshals numpy arrays through ctypes.

Functions
  direct(pts, kernel, w, targets=None)   Eq. (nbodysum), i = j omitted
  FMM(pts, n, theta, N0, shrink=False)    tree + lists (Sec. 3, Sec. 8); with shrink
                                          the cells' boxes bound their points (Sec. 3)
    .evaluate(kernel, w)                  Algorithm "CSFMM"
    .upward(w)                            proxy weights, Sec. 6
    .cells(), .lists(), .order(), .info() the plan's structures
  cheb_nodes(n), lagrange(n, u)           Sec. 4, Eq. (barycentric)
  direct_targets, fmm_targets             separate target and source sets (Sec. 1)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csfmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KERNEL_LAPLACE = 0
KERNEL_BIOT_SAVART = 1
KERNEL_NEWTON = 2
KERNEL_BIHARMONIC = 3
KERNEL_SAL = 4
KERNEL_ONE = 100

PP, PC, CP, CC = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler; returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i64, i32, vp = (ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                           ctypes.c_void_p)
        lib.oracle_direct.argtypes = [P(d), i64, ctypes.c_int, P(d), ctypes.c_int,
                                      P(i64), i64, P(d)]
        lib.oracle_direct.restype = ctypes.c_int
        lib.oracle_fmm_create.argtypes = [P(d), i64, ctypes.c_int, d, ctypes.c_int, ctypes.c_int]
        lib.oracle_fmm_create.restype = vp
        lib.oracle_fmm_destroy.argtypes = [vp]
        lib.oracle_fmm_info.argtypes = [vp, P(i64), P(d)]
        lib.oracle_fmm_cells.argtypes = [vp, P(i32), P(i32), P(i64), P(i64), P(i64),
                                         P(i64), P(i32), P(i32), P(d), P(d)]
        lib.oracle_fmm_list.argtypes = [vp, ctypes.c_int, P(i32), P(i32)]
        lib.oracle_fmm_order.argtypes = [vp, P(i64)]
        lib.oracle_fmm_proxies.argtypes = [vp, P(d)]
        lib.oracle_fmm_evaluate.argtypes = [vp, ctypes.c_int, P(d), ctypes.c_int, P(d)]
        lib.oracle_fmm_evaluate_targets.argtypes = [vp, ctypes.c_int, P(d), ctypes.c_int,
                                                    P(i64), i64, P(d)]
        lib.oracle_fmm_upward.argtypes = [vp, P(d), ctypes.c_int, P(d)]
        lib.oracle_cstc_evaluate.argtypes = [vp, ctypes.c_int, P(d), ctypes.c_int, P(i64), i64,
                                             P(d), P(i64), P(d)]
        lib.oracle_cstc_evaluate.restype = ctypes.c_int
        lib.oracle_fmm_local.argtypes = [vp, P(d), P(d), P(i32)]
        lib.oracle_cheb_nodes.argtypes = [ctypes.c_int, P(d)]
        lib.oracle_lagrange.argtypes = [ctypes.c_int, P(d), d, P(d)]
        lib.oracle_set_mutation.argtypes = [ctypes.c_int]
        lib.oracle_kernel_dim.argtypes = [ctypes.c_int]
        lib.oracle_dilog.argtypes = [d]
        lib.oracle_dilog.restype = d
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_num_threads.restype = None
        _lib = lib
        return lib


def _ptr(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def kernel_dim(kernel: int) -> int:
    return 3 if kernel == KERNEL_BIOT_SAVART else 1


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(n: int) -> None:
    """OpenMP threads of later oracle calls."""
    _load().oracle_set_num_threads(int(n))


def set_mutation(m: int) -> None:
    """Plant a numbered mistake in the oracle (0 restores it).  Used only by
    the tests that show each pin is sensitive to such mistakes."""
    _load().oracle_set_mutation(int(m))


def _weights(w, N):
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    if w.ndim == 1:
        w = w[None, :]
    if w.shape[1] != N:
        raise ValueError("weights must be [nrhs, N]")
    return w


def direct(pts, kernel: int, w, targets=None):
    """phi_i = sum_{j != i} K(x_i, x_j) w_j (Eq. nbodysum) for the given
    target indices (all if None).  Returns [nrhs, ntargets, dim]."""
    lib = _load()
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
    N = len(pts)
    w = _weights(w, N)
    nrhs = w.shape[0]
    dim = kernel_dim(kernel)
    if targets is None:
        tg = None
        nt = N
    else:
        tg = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
        nt = len(tg)
    out = np.zeros((nrhs, nt, dim))
    rc = lib.oracle_direct(_ptr(pts), N, kernel, _ptr(w), nrhs,
                           _ptr(tg, ctypes.c_int64) if tg is not None else None,
                           nt, _ptr(out))
    if rc != 0:
        raise ValueError("oracle_direct: invalid arguments")
    return out


def dilog(x: float) -> float:
    """dilog(x) = -int_0^x log(1 - t)/t dt for 0 <= x <= 1 (Eq. G_B)."""
    return float(_load().oracle_dilog(float(x)))


def cheb_nodes(n: int):
    s = np.zeros(n + 1)
    _load().oracle_cheb_nodes(n, _ptr(s))
    return s


def lagrange(n: int, u: float):
    """[L_0(u), ..., L_n(u)] at the Chebyshev points of degree n."""
    lib = _load()
    s = cheb_nodes(n)
    L = np.zeros(n + 1)
    lib.oracle_lagrange(n, _ptr(s), float(u), _ptr(L))
    return L


class FMM:
    """Tree and interaction lists of the oracle CSFMM for a point set."""

    def __init__(self, pts, n: int, theta: float, N0: int, shrink: bool = False):
        self._lib = _load()
        self.pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
        self.N = len(self.pts)
        self.n, self.theta, self.N0 = int(n), float(theta), int(N0)
        self.shrink = bool(shrink)
        self.P = (self.n + 1) ** 2
        self._h = self._lib.oracle_fmm_create(_ptr(self.pts), self.N, self.n,
                                              self.theta, self.N0, int(self.shrink))
        if not self._h:
            raise ValueError("oracle_fmm_create: invalid arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_fmm_destroy(h)
            self._h = None

    def info(self):
        a = np.zeros(10, dtype=np.int64)
        m = ctypes.c_double(0.0)
        self._lib.oracle_fmm_info(self._h, _ptr(a, ctypes.c_int64), ctypes.byref(m))
        keys = ("ncells", "nleaves", "nlevels", "nPP", "nPC", "nCP", "nCC",
                "n_mac_tests", "evals", "pairs_covered")
        d = {k: int(v) for k, v in zip(keys, a)}
        d["margin"] = m.value
        return d

    def cells(self):
        nc = self.info()["ncells"]
        out = dict(face=np.zeros(nc, np.int32), level=np.zeros(nc, np.int32),
                   ia=np.zeros(nc, np.int64), ib=np.zeros(nc, np.int64),
                   begin=np.zeros(nc, np.int64), end=np.zeros(nc, np.int64),
                   parent=np.zeros(nc, np.int32), child=np.zeros((nc, 4), np.int32),
                   centre=np.zeros((nc, 3)), radius=np.zeros(nc))
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        self._lib.oracle_fmm_cells(
            self._h, _ptr(out["face"], i32), _ptr(out["level"], i32),
            _ptr(out["ia"], i64), _ptr(out["ib"], i64), _ptr(out["begin"], i64),
            _ptr(out["end"], i64), _ptr(out["parent"], i32), _ptr(out["child"], i32),
            _ptr(out["centre"]), _ptr(out["radius"]))
        return out

    def lists(self):
        """{PP, PC, CP, CC: (targets int32[], sources int32[])} in cell indices."""
        inf = self.info()
        res = {}
        for ty, key in ((PP, "nPP"), (PC, "nPC"), (CP, "nCP"), (CC, "nCC")):
            t = np.zeros(inf[key], np.int32)
            s = np.zeros(inf[key], np.int32)
            self._lib.oracle_fmm_list(self._h, ty, _ptr(t, ctypes.c_int32),
                                      _ptr(s, ctypes.c_int32))
            res[ty] = (t, s)
        return res

    def order(self):
        o = np.zeros(self.N, np.int64)
        self._lib.oracle_fmm_order(self._h, _ptr(o, ctypes.c_int64))
        return o

    def proxies(self):
        nc = self.info()["ncells"]
        px = np.zeros((nc, self.P, 3))
        self._lib.oracle_fmm_proxies(self._h, _ptr(px))
        return px

    def local_coords(self):
        u = np.zeros(self.N)
        v = np.zeros(self.N)
        leaf = np.zeros(self.N, np.int32)
        self._lib.oracle_fmm_local(self._h, _ptr(u), _ptr(v), _ptr(leaf, ctypes.c_int32))
        return u, v, leaf

    def upward(self, w):
        """Proxy weights of every cell, [ncells, nrhs, P] (Sec. 6)."""
        w = _weights(w, self.N)
        nc = self.info()["ncells"]
        out = np.zeros((nc, w.shape[0], self.P))
        self._lib.oracle_fmm_upward(self._h, _ptr(w), w.shape[0], _ptr(out))
        return out

    def evaluate(self, kernel: int, w, targets=None):
        """CSFMM potentials [nrhs, N, dim] in input order, or
        [nrhs, len(targets), dim] at the given input indices (same
        arithmetic, restricted to the cells those targets need)."""
        w = _weights(w, self.N)
        nrhs = w.shape[0]
        if targets is not None:
            tg = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
            out = np.zeros((nrhs, len(tg), kernel_dim(kernel)))
            rc = self._lib.oracle_fmm_evaluate_targets(
                self._h, kernel, _ptr(w), nrhs, _ptr(tg, ctypes.c_int64), len(tg),
                _ptr(out))
            if rc != 0:
                raise ValueError("oracle_fmm_evaluate: invalid arguments")
            return out
        out = np.zeros((nrhs, self.N, kernel_dim(kernel)))
        rc = self._lib.oracle_fmm_evaluate(self._h, kernel, _ptr(w), nrhs, _ptr(out))
        if rc != 0:
            raise ValueError("oracle_fmm_evaluate: invalid arguments")
        return out

    def evaluate_cstc(self, kernel: int, w, targets=None, with_stats=False):
        """Cubed sphere tree code (Algorithm "CSTC") on the same tree, degree
        and MAC: potentials [nrhs, N or len(targets), dim] in input order.
        With with_stats, also {"pc", "pp", "evals", "margin"}: interaction
        counts and kernel evaluations over the targets, and the smallest
        relative distance of a separation test from its threshold."""
        w = _weights(w, self.N)
        nrhs = w.shape[0]
        tg = None if targets is None else np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
        nt = self.N if tg is None else len(tg)
        out = np.zeros((nrhs, nt, kernel_dim(kernel)))
        st = np.zeros(3, dtype=np.int64)
        m = ctypes.c_double(0.0)
        rc = self._lib.oracle_cstc_evaluate(
            self._h, kernel, _ptr(w), nrhs,
            None if tg is None else _ptr(tg, ctypes.c_int64), nt, _ptr(out),
            _ptr(st, ctypes.c_int64), ctypes.byref(m))
        if rc != 0:
            raise ValueError("oracle_cstc_evaluate: invalid arguments")
        if with_stats:
            return out, {"pc": int(st[0]), "pp": int(st[1]), "evals": int(st[2]),
                         "margin": m.value}
        return out


def _union(sources, targets, w):
    src = np.asarray(sources, dtype=np.float64)
    tgt = np.asarray(targets, dtype=np.float64)
    w = np.atleast_2d(np.asarray(w, dtype=np.float64))
    pts = np.ascontiguousarray(np.vstack([src, tgt]))
    wu = np.ascontiguousarray(np.hstack([w, np.zeros((w.shape[0], len(tgt)))]))
    return pts, wu, np.arange(len(src), len(src) + len(tgt))


def direct_targets(sources, kernel: int, w, targets):
    """phi(y_t) = sum_j K(y_t, x_j) w_j at target points that are not the
    sources (Sec. 1: separate target and source sets; the targets distinct
    from every source and from each other).  Computed as Eq. (nbodysum) over
    the union of both sets with weight zero at the targets, read at the
    targets: every added term is K(y_t, y_s) * 0.  Returns [nrhs, Nt, dim]."""
    pts, wu, tg = _union(sources, targets, w)
    return direct(pts, kernel, wu, tg)


def fmm_targets(sources, targets, n: int, theta: float, N0: int, kernel: int, w,
                cstc: bool = False, shrink: bool = False):
    """The CSFMM (or, with cstc, the CSTC) for separate targets on one tree
    built over the sources followed by the targets (a cell splits while it
    holds more than N0 points of both kinds together), the targets weighted
    zero, read at the targets.  Returns [nrhs, Nt, dim]."""
    pts, wu, tg = _union(sources, targets, w)
    f = FMM(pts, n, theta, N0, shrink)
    return f.evaluate_cstc(kernel, wu, tg) if cstc else f.evaluate(kernel, wu, tg)


def rel_l2(a, b, areas=None, ref=None):
    """Global relative error E of Sec. 10.2: sqrt(sum (a-b)^2 A / sum ref^2 A)
    (ref defaults to b; areas default to 1)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ref = b if ref is None else np.asarray(ref, dtype=np.float64)
    if areas is None:
        num = np.sum((a - b) ** 2)
        den = np.sum(ref ** 2)
    else:
        A = np.asarray(areas, dtype=np.float64)
        sh = [1] * a.ndim
        ax = next(i for i, s in enumerate(a.shape) if s == len(A))
        sh[ax] = len(A)
        A = A.reshape(sh)
        num = np.sum((a - b) ** 2 * A)
        den = np.sum(ref ** 2 * A)
    return float(np.sqrt(num / den))
