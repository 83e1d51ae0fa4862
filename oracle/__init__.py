"""Python handle on the serial CPU oracle (``oracle/ivs_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product path (``paper_1802_00330_gb300``) never imports it.

The shared library is compiled with gcc on first use (or by ``build()``) with
``-frounding-math -ffp-contract=off`` so that every directed operation is one IEEE
operation under ``fesetround`` and no multiply-add is fused.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ivs_oracle.c")
_HDR = os.path.join(_HERE, "ivs_oracle.h")
_LIB = os.path.join(_HERE, "libivs_oracle.so")
_lock = threading.Lock()
_lib = None

FLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-frounding-math", "-ffp-contract=off",
         "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU involved)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *FLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Sys(C.Structure):
    _fields_ = [("n_vars", C.c_int32), ("n_eqs", C.c_int32), ("n_terms", C.c_int32),
                ("eq_offsets", C.c_void_p), ("coef_lo", C.c_void_p), ("coef_hi", C.c_void_p),
                ("exps", C.c_void_p)]


class _Opt(C.Structure):
    _fields_ = [("tol", C.c_double), ("hs_enable", C.c_int32), ("hs_min_depth", C.c_int32),
                ("hs_iters", C.c_int32), ("root_depth", C.c_int32), ("max_depth", C.c_int32),
                ("order", C.c_int32), ("order_seed", C.c_uint64), ("max_boxes", C.c_int64),
                ("centred", C.c_int32), ("krawczyk", C.c_int32), ("split_mode", C.c_int32),
                ("gap_split", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("boxes", C.c_int64), ("excluded_eval", C.c_int64), ("hs_applied", C.c_int64),
                ("hs_empty", C.c_int64), ("hs_contracted", C.c_int64), ("hs_singular", C.c_int64),
                ("accepted", C.c_int64), ("unsplittable", C.c_int64), ("split", C.c_int64),
                ("max_depth_seen", C.c_int32), ("excluded_centred", C.c_int64), ("gap_splits", C.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            vp = C.c_void_p
            lib.orc_solve.argtypes = [C.POINTER(_Sys), vp, vp, C.POINTER(_Opt), C.POINTER(vp)]
            lib.orc_solve.restype = C.c_int
            lib.orc_result_count.argtypes = [vp]
            lib.orc_result_count.restype = C.c_int64
            lib.orc_result_status.argtypes = [vp]
            lib.orc_result_boxes.argtypes = [vp, vp, vp, vp, vp]
            lib.orc_result_stats.argtypes = [vp, C.POINTER(_Stats)]
            lib.orc_result_free.argtypes = [vp]
            lib.orc_result_depth_stats.argtypes = [vp, vp, vp]
            lib.orc_iv_op.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_int, vp]
            lib.orc_iv_extdiv.argtypes = [C.c_double] * 4 + [vp]
            lib.orc_eval.argtypes = [C.POINTER(_Sys), vp, vp, vp, vp]
            lib.orc_eval_f32.argtypes = [C.POINTER(_Sys), vp, vp, vp, vp]
            lib.orc_jacobian.argtypes = [C.POINTER(_Sys), vp, vp, vp, vp]
            lib.orc_gj_inverse.argtypes = [C.c_int, vp, vp]
            lib.orc_hs_step.argtypes = [C.POINTER(_Sys), vp, vp, vp, vp]
            lib.orc_kr_step.argtypes = [C.POINTER(_Sys), vp, vp, vp, vp, vp, vp]
            lib.orc_hs_gap_step.argtypes = [C.POINTER(_Sys), vp, vp, vp, vp, vp, vp, vp]
            lib.orc_centred.argtypes = [C.POINTER(_Sys), vp, vp, vp, vp]
            lib.orc_clusters.argtypes = [C.c_int, C.c_int64, vp, vp, vp]
            lib.orc_clusters.restype = C.c_int64
            lib.orc_backtrack.argtypes = [C.c_int, C.c_int64, vp, vp, vp, vp, C.c_int, C.c_int64, vp]
            lib.orc_backtrack.restype = C.c_int64
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class _SysHolder:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, s):
        self.off = np.ascontiguousarray(s.eq_offsets, dtype=np.int32)
        self.clo = np.ascontiguousarray(s.coef_lo, dtype=np.float64)
        self.chi = np.ascontiguousarray(s.coef_hi, dtype=np.float64)
        self.exps = np.ascontiguousarray(s.exps, dtype=np.uint8)
        self.c = _Sys(int(s.n_vars), int(s.n_eqs), int(self.off[-1]), _ptr(self.off),
                      _ptr(self.clo), _ptr(self.chi), _ptr(self.exps))


def solve(s, box_lo=None, box_hi=None, tol=None, hs_enable=True, hs_min_depth=0, hs_iters=1,
          root_depth=0, max_depth=200, order=0, order_seed=0, max_boxes=0, centred=False, krawczyk=False,
          split_mode=0, gap_split=False):
    """Run the serial solver.  Returns a dict with sorted boxes, flags, depths, stats, status."""
    lib = _load()
    h = _SysHolder(s)
    lo = np.ascontiguousarray(s.box_lo if box_lo is None else box_lo, dtype=np.float64)
    hi = np.ascontiguousarray(s.box_hi if box_hi is None else box_hi, dtype=np.float64)
    opt = _Opt(float(s.tol if tol is None else tol), int(hs_enable), int(hs_min_depth),
               int(hs_iters), int(root_depth), int(max_depth), int(order), int(order_seed),
               int(max_boxes), int(bool(centred)), int(bool(krawczyk)), int(split_mode), int(bool(gap_split)))
    res = C.c_void_p()
    lib.orc_solve(C.byref(h.c), _ptr(lo), _ptr(hi), C.byref(opt), C.byref(res))
    try:
        status = lib.orc_result_status(res)
        cnt = lib.orc_result_count(res)
        n = int(s.n_vars)
        out_lo = np.zeros((cnt, n))
        out_hi = np.zeros((cnt, n))
        flags = np.zeros(cnt, np.int32)
        depth = np.zeros(cnt, np.int32)
        if cnt:
            lib.orc_result_boxes(res, _ptr(out_lo), _ptr(out_hi), _ptr(flags), _ptr(depth))
        st = _Stats()
        lib.orc_result_stats(res, C.byref(st))
        stats = {k: getattr(st, k) for k, _ in _Stats._fields_}
        db = np.zeros(64, np.int64)
        dk = np.zeros(64, np.int64)
        lib.orc_result_depth_stats(res, _ptr(db), _ptr(dk))
        stats["depth_boxes"] = db
        stats["depth_kept"] = dk
    finally:
        lib.orc_result_free(res)
    return {"status": status, "lo": out_lo, "hi": out_hi, "flags": flags, "depth": depth,
            "stats": stats}


OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_POW, OP_NEG = range(6)


def iv_op(op, a, b=(0.0, 0.0), k=0):
    lib = _load()
    out = np.zeros(2)
    rc = lib.orc_iv_op(op, a[0], a[1], b[0], b[1], k, _ptr(out))
    if rc:
        raise ValueError("operation undefined for these operands")
    return float(out[0]), float(out[1])


def extdiv(x, y):
    lib = _load()
    out = np.zeros(4)
    np_ = lib.orc_iv_extdiv(x[0], x[1], y[0], y[1], _ptr(out))
    return [(float(out[2 * q]), float(out[2 * q + 1])) for q in range(np_)]


def eval_box(s, lo, hi):
    lib = _load()
    h = _SysHolder(s)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    ol = np.zeros(s.n_eqs)
    oh = np.zeros(s.n_eqs)
    lib.orc_eval(C.byref(h.c), _ptr(lo), _ptr(hi), _ptr(ol), _ptr(oh))
    return ol, oh


def eval_box_f32(s, lo, hi):
    lib = _load()
    h = _SysHolder(s)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    ol = np.zeros(s.n_eqs, np.float32)
    oh = np.zeros(s.n_eqs, np.float32)
    lib.orc_eval_f32(C.byref(h.c), _ptr(lo), _ptr(hi), _ptr(ol), _ptr(oh))
    return ol, oh


def jacobian(s, lo, hi):
    lib = _load()
    h = _SysHolder(s)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    jl = np.zeros((s.n_eqs, s.n_vars))
    jh = np.zeros((s.n_eqs, s.n_vars))
    lib.orc_jacobian(C.byref(h.c), _ptr(lo), _ptr(hi), _ptr(jl), _ptr(jh))
    return jl, jh


def gj_inverse(a):
    lib = _load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = a.shape[0]
    out = np.zeros((n, n))
    rc = lib.orc_gj_inverse(n, _ptr(a), _ptr(out))
    return rc, out


def hs_step(s, lo, hi):
    """One Hansen-Sengupta sweep.  Returns (status, lo', hi'); status 0 box, 1 empty,
    2 skipped (singular preconditioner)."""
    lib = _load()
    h = _SysHolder(s)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    ol = lo.copy()
    oh = hi.copy()
    rc = lib.orc_hs_step(C.byref(h.c), _ptr(lo), _ptr(hi), _ptr(ol), _ptr(oh))
    return rc, ol, oh


def kr_step(s, lo, hi):
    """One Krawczyk step (eq 15, 16).  Returns (status, lo', hi', k_lo, k_hi): K(X) in
    k_lo/k_hi (status 0 or 1), X intersected with K(X) in lo'/hi' (status 0)."""
    lib = _load()
    h = _SysHolder(s)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    ol, oh = lo.copy(), hi.copy()
    kl = np.full_like(lo, -np.inf)
    kh = np.full_like(hi, np.inf)
    rc = lib.orc_kr_step(C.byref(h.c), _ptr(lo), _ptr(hi), _ptr(ol), _ptr(oh), _ptr(kl), _ptr(kh))
    return rc, ol, oh, kl, kh


def hs_gap_step(s, lo, hi):
    """One Gauss-Seidel sweep with the two-box split of a gap.  Returns (status, boxes,
    gap_row): status 0 one box, 1 empty, 2 skipped (singular), 3 two boxes (the lower and
    the upper piece of coordinate gap_row); boxes = list of (lo, hi)."""
    lib = _load()
    h = _SysHolder(s)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    ol, oh, ol2, oh2 = lo.copy(), hi.copy(), lo.copy(), hi.copy()
    g = np.zeros(1, np.int32)
    rc = lib.orc_hs_gap_step(C.byref(h.c), _ptr(lo), _ptr(hi), _ptr(ol), _ptr(oh), _ptr(ol2), _ptr(oh2), _ptr(g))
    boxes = [] if rc in (1, 2) else [(ol, oh)] + ([(ol2, oh2)] if rc == 3 else [])
    return rc, boxes, int(g[0])


def centred(s, lo, hi):
    """Centred form F_c,i(X) = f_i(mid X) + sum_j J_ij(X) (X_j - mid X_j) of every
    equation (n_eqs == n_vars); returns (lo, hi) arrays."""
    lib = _load()
    h = _SysHolder(s)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    ol = np.zeros(s.n_eqs)
    oh = np.zeros(s.n_eqs)
    lib.orc_centred(C.byref(h.c), _ptr(lo), _ptr(hi), _ptr(ol), _ptr(oh))
    return ol, oh


def clusters(lo, hi):
    """Connected components of touching boxes (rows of lo/hi).  Returns (count, labels)."""
    lib = _load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    k, n = lo.shape if lo.ndim == 2 else (0, 1)
    labels = np.zeros(max(k, 1), np.int64)
    nc = lib.orc_clusters(int(n), int(k), _ptr(lo), _ptr(hi), _ptr(labels))
    return int(nc), labels[:k]


def backtrack(lo, hi, d_lo, d_hi, level, max_cells=1 << 26, groups=False):
    """Distinct cells of `level` of the initial box's dyadic grid met by the boxes
    (Algorithm 5 read on that grid); -1 if more than max_cells would be enumerated.
    With groups=True returns (cells, connected components of the cells)."""
    lib = _load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    d_lo = np.ascontiguousarray(d_lo, dtype=np.float64)
    d_hi = np.ascontiguousarray(d_hi, dtype=np.float64)
    k, n = lo.shape if lo.ndim == 2 else (0, len(d_lo))
    g = np.zeros(1, np.int64)
    c = int(lib.orc_backtrack(int(n), int(k), _ptr(lo), _ptr(hi), _ptr(d_lo), _ptr(d_hi), int(level),
                              int(max_cells), _ptr(g)))
    return (c, int(g[0])) if groups else c
