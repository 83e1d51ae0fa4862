"""ctypes binding of ``libivsolve.so`` (declared in ``include/ivsolve.h``).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.
There is no CPU fallback -- if the library is missing or no GPU is present the calls
raise.  Function names follow the C ABI; ``solve`` / ``solve_batch`` / ``Plan`` are thin
conveniences that return numpy arrays.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libivsolve.so")

IVS_OK, IVS_ERR_INVALID, IVS_ERR_NOMEM, IVS_ERR_BUDGET, IVS_ERR_TIMEOUT, IVS_ERR_CUDA = range(6)
IVS_BOX_WIDTH, IVS_BOX_UNSPLITTABLE, IVS_BOX_DEPTH_LIMIT = 1, 2, 4


class ivs_system(C.Structure):
    _fields_ = [("n_vars", C.c_int32), ("n_eqs", C.c_int32), ("n_terms", C.c_int32),
                ("eq_offsets", C.c_void_p), ("coef_lo", C.c_void_p), ("coef_hi", C.c_void_p),
                ("exps", C.c_void_p)]


class ivs_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("hs_enable", C.c_int32), ("hs_min_depth", C.c_int32),
                ("hs_iters", C.c_int32), ("prefilter_fp32", C.c_int32), ("root_depth", C.c_int32),
                ("max_depth", C.c_int32), ("max_boxes", C.c_int64), ("max_results", C.c_int64),
                ("time_budget_s", C.c_double), ("centred_form", C.c_int32), ("krawczyk", C.c_int32),
                ("split_mode", C.c_int32), ("gap_split", C.c_int32)]


class ivs_stats(C.Structure):
    _fields_ = [("boxes", C.c_int64), ("excluded_prefilter", C.c_int64), ("excluded_eval", C.c_int64),
                ("hs_applied", C.c_int64), ("hs_empty", C.c_int64), ("hs_contracted", C.c_int64),
                ("hs_singular", C.c_int64), ("accepted", C.c_int64), ("unsplittable", C.c_int64),
                ("split", C.c_int64), ("max_depth_seen", C.c_int32), ("waves", C.c_int32),
                ("device_ms", C.c_double), ("launches", C.c_int64), ("eval64_boxes", C.c_int64),
                ("kept_shadow", C.c_int64), ("queue_ms", C.c_double), ("solve_ms", C.c_double), ("excluded_centred", C.c_int64),
                ("gap_splits", C.c_int64)]


class ivs_plan_cfg(C.Structure):
    _fields_ = [("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t), ("stream", C.c_void_p),
                ("wave_children", C.c_int64), ("eval_blocks", C.c_int32), ("eval_threads", C.c_int32),
                ("device", C.c_int32), ("profile", C.c_int32)]


class ivs_server_cfg(C.Structure):
    _fields_ = [("workspace_bytes", C.c_size_t), ("wave_children", C.c_int64), ("results_per_slot", C.c_int64),
                ("max_slots", C.c_int32), ("max_vars", C.c_int32), ("sweeps_per_step", C.c_int32),
                ("device", C.c_int32), ("reserve_factor", C.c_double), ("min_region_entries", C.c_int64),
                ("schedule", C.c_int32)]


class ivs_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("in_flight", C.c_int64), ("waiting", C.c_int64), ("steps", C.c_int64), ("sweeps", C.c_int64),
                ("boxes", C.c_int64), ("busy_s", C.c_double), ("last_error", C.c_char * 160)]


class ivs_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("ms", C.c_double)]


# name -> (restype, argtypes); the full list of entry points of include/ivsolve.h
_VP = C.c_void_p
_PP = C.POINTER(C.c_void_p)
SIGNATURES = {
    "ivs_options_default": (None, [C.POINTER(ivs_options)]),
    "ivs_release_cached": (None, []),
    "ivs_clusters": (C.c_int, [C.c_int32, C.c_int64, _VP, _VP, C.POINTER(C.c_int64), _VP, _VP, _VP, C.c_int64]),
    "ivs_backtrack": (C.c_int, [C.c_int32, C.c_int64, _VP, _VP, _VP, _VP, C.c_int32, C.c_int64,
                                C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "ivs_clusters_gpu": (C.c_int, [C.c_int32, C.c_int64, _VP, _VP, C.POINTER(C.c_int64), _VP, _VP, _VP, C.c_int64,
                                   C.c_int32]),
    "ivs_backtrack_gpu": (C.c_int, [C.c_int32, C.c_int64, _VP, _VP, _VP, _VP, C.c_int32, C.c_int64,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int32]),
    "ivs_plan_backtrack": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int64, C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64)]),
    "ivs_plan_clusters": (C.c_int, [_VP, C.c_int32, C.POINTER(C.c_int64)]),
    "ivs_solve": (C.c_int, [C.POINTER(ivs_system), _VP, _VP, C.POINTER(ivs_options), _PP]),
    "ivs_solve_batch": (C.c_int, [C.c_int32, C.POINTER(ivs_system), _VP, _VP, C.POINTER(ivs_options),
                                  C.c_int32, _PP]),
    "ivs_result_count": (C.c_int64, [_VP]),
    "ivs_result_n_vars": (C.c_int32, [_VP]),
    "ivs_result_status": (C.c_int, [_VP]),
    "ivs_result_boxes": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "ivs_result_stats": (C.c_int, [_VP, C.POINTER(ivs_stats)]),
    "ivs_result_depth_stats": (C.c_int, [_VP, _VP, _VP, _VP]),
    "ivs_result_free": (None, [_VP]),
    "ivs_workspace_bytes": (C.c_size_t, [C.c_int32, C.POINTER(ivs_system), C.c_int64, C.c_int64, C.c_int64]),
    "ivs_plan_create": (C.c_int, [C.c_int32, C.POINTER(ivs_system), _VP, _VP, C.POINTER(ivs_options),
                                  C.c_int32, C.POINTER(ivs_plan_cfg), _PP]),
    "ivs_plan_run": (C.c_int, [_VP]),
    "ivs_plan_result": (C.c_int, [_VP, C.c_int32, _PP]),
    "ivs_plan_stats": (C.c_int, [_VP, C.POINTER(ivs_stats)]),
    "ivs_plan_depth_stats": (C.c_int, [_VP, C.c_int32, C.POINTER(ivs_stats), _VP, _VP, _VP]),
    "ivs_plan_destroy": (None, [_VP]),
    "ivs_plan_kernel_times": (C.c_int32, [_VP, _VP, C.c_int32]),
    "ivs_autotune": (C.c_int, [C.c_int32, C.POINTER(ivs_system), _VP, _VP, C.POINTER(ivs_options), C.c_int32,
                               C.c_int64, C.POINTER(ivs_plan_cfg), C.POINTER(C.c_double)]),
    "ivs_probe_rate": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ivs_solve_noalloc": (C.c_int, [C.POINTER(ivs_system), _VP, _VP, C.POINTER(ivs_options), _VP, _VP, _VP,
                                    _VP, C.c_int64, C.POINTER(C.c_int64), C.POINTER(ivs_stats), C.c_char_p,
                                    C.c_int32]),
    "ivs_server_cfg_default": (None, [C.POINTER(ivs_server_cfg)]),
    "ivs_server_create": (C.c_int, [C.POINTER(ivs_server_cfg), _PP]),
    "ivs_server_submit": (C.c_int, [_VP, C.POINTER(ivs_system), _VP, _VP, C.POINTER(ivs_options),
                                    C.POINTER(C.c_uint64)]),
    "ivs_server_poll": (C.c_int, [_VP, C.c_uint64, _PP]),
    "ivs_server_wait": (C.c_int, [_VP, C.c_uint64, C.c_double, _PP]),
    "ivs_server_get_stats": (C.c_int, [_VP, C.POINTER(ivs_server_stats)]),
    "ivs_server_destroy": (None, [_VP]),
    "ivs_status_str": (C.c_char_p, [C.c_int]),
    "ivs_last_error": (C.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def load():
    """Load the CUDA library; raises if it was not built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_1802_00330_gb300.build.build() (nvcc, sm_103a)")
            lib = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)


class IvsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(rc):
    if rc != IVS_OK:
        lib = load()
        raise IvsError(rc, f"{lib.ivs_status_str(rc).decode()}: {lib.ivs_last_error().decode()}")


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class _SysRef:
    """Owns contiguous copies of a system's arrays while a C struct points at them."""

    def __init__(self, s):
        self.off = np.ascontiguousarray(s.eq_offsets, dtype=np.int32)
        self.clo = np.ascontiguousarray(s.coef_lo, dtype=np.float64)
        self.chi = np.ascontiguousarray(s.coef_hi, dtype=np.float64)
        self.exps = np.ascontiguousarray(s.exps, dtype=np.uint8)
        self.lo = np.ascontiguousarray(s.box_lo, dtype=np.float64)
        self.hi = np.ascontiguousarray(s.box_hi, dtype=np.float64)
        self.c = ivs_system(int(s.n_vars), int(s.n_eqs), int(self.off[-1]), _ptr(self.off),
                            _ptr(self.clo), _ptr(self.chi), _ptr(self.exps))


def make_options(tol=1e-6, hs_enable=True, hs_min_depth=0, hs_iters=1, prefilter_fp32=True,
                 root_depth=0, max_depth=200, max_boxes=0, max_results=0, time_budget_s=0.0,
                 centred_form=False, krawczyk=False, split_mode=0, gap_split=False):
    o = ivs_options()
    load().ivs_options_default(C.byref(o))
    o.tol = float(tol)
    o.hs_enable = int(hs_enable)
    o.hs_min_depth = int(hs_min_depth)
    o.hs_iters = int(hs_iters)
    o.prefilter_fp32 = int(prefilter_fp32)
    o.root_depth = int(root_depth)
    o.max_depth = int(max_depth)
    o.max_boxes = int(max_boxes)
    o.max_results = int(max_results)
    o.time_budget_s = float(time_budget_s)
    o.centred_form = int(bool(centred_form))
    o.krawczyk = int(bool(krawczyk))
    o.split_mode = int(split_mode)
    o.gap_split = int(bool(gap_split))
    return o


def result_to_dict(r):
    lib = load()
    cnt = lib.ivs_result_count(r)
    n = lib.ivs_result_n_vars(r)
    lo = np.zeros((cnt, n))
    hi = np.zeros((cnt, n))
    flags = np.zeros(cnt, np.int32)
    depth = np.zeros(cnt, np.int32)
    _check(lib.ivs_result_boxes(r, _ptr(lo), _ptr(hi), _ptr(flags), _ptr(depth)))
    st = ivs_stats()
    _check(lib.ivs_result_stats(r, C.byref(st)))
    stats = {k: getattr(st, k) for k, _ in ivs_stats._fields_}
    db = np.zeros(64, np.int64)
    dk = np.zeros(64, np.int64)
    dh = np.zeros(64, np.int64)
    _check(lib.ivs_result_depth_stats(r, _ptr(db), _ptr(dk), _ptr(dh)))
    stats["depth_boxes"] = db
    stats["depth_kept"] = dk
    stats["depth_hs"] = dh
    return {"status": lib.ivs_result_status(r), "lo": lo, "hi": hi, "flags": flags, "depth": depth,
            "stats": stats}


def solve(s, box_lo=None, box_hi=None, **opts):
    """Solve one system (a ``synth.PolySystem``-like object) through ``ivs_solve``."""
    lib = load()
    ref = _SysRef(s)
    lo = ref.lo if box_lo is None else np.ascontiguousarray(box_lo, dtype=np.float64)
    hi = ref.hi if box_hi is None else np.ascontiguousarray(box_hi, dtype=np.float64)
    opts.setdefault("tol", s.tol)
    o = make_options(**opts)
    res = C.c_void_p()
    rc = lib.ivs_solve(C.byref(ref.c), _ptr(lo), _ptr(hi), C.byref(o), C.byref(res))
    if not res:
        _check(rc)
    try:
        return result_to_dict(res)
    finally:
        lib.ivs_result_free(res)


class Plan:
    """Device-resident plan over one or more systems (``ivs_plan_*``).  ``workspace`` may
    be a CUDA tensor (e.g. ``torch.empty(nbytes, dtype=torch.uint8, device='cuda')``) that
    the plan uses instead of allocating; ``stream`` a ``torch.cuda.Stream``."""

    def __init__(self, systems, opts=None, wave_children=0, workspace=None, workspace_bytes=0,
                 stream=None, eval_blocks=0, eval_threads=0, profile=False):
        lib = load()
        self._lib = lib
        self.refs = [_SysRef(s) for s in systems]
        self.n_sys = len(systems)
        arr = (ivs_system * self.n_sys)(*[r.c for r in self.refs])
        los = (C.c_void_p * self.n_sys)(*[_ptr(r.lo) for r in self.refs])
        his = (C.c_void_p * self.n_sys)(*[_ptr(r.hi) for r in self.refs])
        if opts is None:
            opts = [make_options(tol=s.tol) for s in systems]
        elif isinstance(opts, dict):
            opts = [make_options(**{"tol": s.tol, **opts}) for s in systems]
        oarr = (ivs_options * self.n_sys)(*opts)
        cfg = ivs_plan_cfg()
        self._workspace = workspace
        if workspace is not None:
            cfg.workspace = C.c_void_p(int(workspace.data_ptr()))
            cfg.workspace_bytes = int(workspace.numel() * workspace.element_size())
        else:
            cfg.workspace_bytes = int(workspace_bytes)
        if stream is not None:
            cfg.stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        cfg.wave_children = int(wave_children)
        cfg.eval_blocks = int(eval_blocks)
        cfg.eval_threads = int(eval_threads)
        cfg.profile = int(profile)
        self.p = C.c_void_p()
        _check(lib.ivs_plan_create(self.n_sys, arr, los, his, oarr, C.sizeof(ivs_options), C.byref(cfg),
                                   C.byref(self.p)))

    def run(self):
        rc = self._lib.ivs_plan_run(self.p)
        if rc not in (IVS_OK, IVS_ERR_TIMEOUT, IVS_ERR_NOMEM):
            _check(rc)
        return rc

    def stats(self):
        st = ivs_stats()
        _check(self._lib.ivs_plan_stats(self.p, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ivs_stats._fields_}

    def result(self, s=0):
        res = C.c_void_p()
        _check(self._lib.ivs_plan_result(self.p, int(s), C.byref(res)))
        try:
            return result_to_dict(res)
        finally:
            self._lib.ivs_result_free(res)

    def backtrack(self, s, level, max_cells=1 << 26):
        """Algorithm 5 on the GPU over system s's device-resident result: (distinct cells of
        the level, connected groups of them) -- ``ivs_plan_backtrack``."""
        cells, groups = C.c_int64(), C.c_int64()
        _check(self._lib.ivs_plan_backtrack(self.p, int(s), int(level), int(max_cells), C.byref(cells),
                                            C.byref(groups)))
        return cells.value, groups.value

    def clusters(self, s):
        """Connected components of touching boxes of system s's result, on the GPU."""
        nc = C.c_int64()
        _check(self._lib.ivs_plan_clusters(self.p, int(s), C.byref(nc)))
        return nc.value

    def result_stats(self, s=0):
        """Counters of system s's last run (with the per-depth counts) without copying its
        boxes to the host."""
        st = ivs_stats()
        db, dk, dh = (np.zeros(64, np.int64) for _ in range(3))
        _check(self._lib.ivs_plan_depth_stats(self.p, int(s), C.byref(st), _ptr(db), _ptr(dk), _ptr(dh)))
        out = {k: getattr(st, k) for k, _ in ivs_stats._fields_}
        out.update(depth_boxes=db, depth_kept=dk, depth_hs=dh)
        return out

    def kernel_times(self):
        arr = (ivs_kernel_time * 64)()
        k = self._lib.ivs_plan_kernel_times(self.p, arr, 64)
        return {arr[q].name.decode(): (arr[q].launches, arr[q].ms) for q in range(min(k, 64))}

    def close(self):
        if self.p:
            self._lib.ivs_plan_destroy(self.p)
            self.p = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_rate(kind=0, device=0):
    """Measured directed-rounding rate of the device in ops/s (kind 0 FP64, 1 FP32, 2 / 3
    FP64 with 8 / 1 active lanes, 4 / 5 FP64 division directed / to nearest)."""
    ops = C.c_double()
    ms = C.c_double()
    _check(load().ivs_probe_rate(int(kind), int(device), C.byref(ops), C.byref(ms)))
    return ops.value, ms.value


class Server:
    """Continuous-batching server (``ivs_server_*``): submit systems while others run;
    poll or wait for their results."""

    def __init__(self, workspace_bytes=0, wave_children=0, results_per_slot=0, max_slots=0, max_vars=0,
                 sweeps_per_step=0, device=0, reserve_factor=0.0, min_region_entries=0, schedule=0):
        lib = load()
        self._lib = lib
        cfg = ivs_server_cfg()
        lib.ivs_server_cfg_default(C.byref(cfg))
        for k, v in (("workspace_bytes", workspace_bytes), ("wave_children", wave_children),
                     ("results_per_slot", results_per_slot), ("max_slots", max_slots), ("max_vars", max_vars),
                     ("sweeps_per_step", sweeps_per_step), ("reserve_factor", reserve_factor),
                     ("min_region_entries", min_region_entries), ("schedule", schedule)):
            if v:
                setattr(cfg, k, v)
        cfg.device = int(device)
        self.p = C.c_void_p()
        self._refs = {}
        _check(lib.ivs_server_create(C.byref(cfg), C.byref(self.p)))

    def submit(self, s, **opts):
        ref = _SysRef(s)
        o = make_options(**{"tol": s.tol, **opts})
        t = C.c_uint64()
        _check(self._lib.ivs_server_submit(self.p, C.byref(ref.c), _ptr(ref.lo), _ptr(ref.hi), C.byref(o), C.byref(t)))
        return t.value

    def poll(self, ticket):
        r = C.c_void_p()
        _check(self._lib.ivs_server_poll(self.p, C.c_uint64(ticket), C.byref(r)))
        if not r:
            return None
        try:
            return result_to_dict(r)
        finally:
            self._lib.ivs_result_free(r)

    def wait(self, ticket, timeout_s=0.0):
        r = C.c_void_p()
        _check(self._lib.ivs_server_wait(self.p, C.c_uint64(ticket), float(timeout_s), C.byref(r)))
        if not r:
            return None
        try:
            return result_to_dict(r)
        finally:
            self._lib.ivs_result_free(r)

    def stats(self):
        st = ivs_server_stats()
        _check(self._lib.ivs_server_get_stats(self.p, C.byref(st)))
        d = {k: getattr(st, k) for k, _ in ivs_server_stats._fields_}
        d["last_error"] = st.last_error.decode(errors="replace")
        return d

    def close(self):
        if self.p:
            self._lib.ivs_server_destroy(self.p)
            self.p = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(systems, trial_boxes=200_000, **opts):
    """Best (wave_children, eval_blocks) for these systems by short trial solves."""
    lib = load()
    refs = [_SysRef(s) for s in systems]
    n = len(systems)
    arr = (ivs_system * n)(*[r.c for r in refs])
    los = (C.c_void_p * n)(*[_ptr(r.lo) for r in refs])
    his = (C.c_void_p * n)(*[_ptr(r.hi) for r in refs])
    oarr = (ivs_options * n)(*[make_options(**{"tol": s.tol, **opts}) for s in systems])
    cfg = ivs_plan_cfg()
    rate = C.c_double()
    _check(lib.ivs_autotune(n, arr, los, his, oarr, C.sizeof(ivs_options), int(trial_boxes), C.byref(cfg),
                            C.byref(rate)))
    return {"wave_children": cfg.wave_children, "eval_blocks": cfg.eval_blocks, "trial_boxes_per_s": rate.value}


def solve_batch(systems, **opts):
    """Solve many systems in one device run through ``ivs_solve_batch``."""
    lib = load()
    refs = [_SysRef(s) for s in systems]
    n = len(systems)
    arr = (ivs_system * n)(*[r.c for r in refs])
    los = (C.c_void_p * n)(*[_ptr(r.lo) for r in refs])
    his = (C.c_void_p * n)(*[_ptr(r.hi) for r in refs])
    oarr = (ivs_options * n)(*[make_options(**{"tol": s.tol, **opts}) for s in systems])
    outs = (C.c_void_p * n)()
    rc = lib.ivs_solve_batch(n, arr, los, his, oarr, C.sizeof(ivs_options), outs)
    try:
        if any(not o for o in outs):
            _check(rc)
        return [result_to_dict(o) for o in outs]
    finally:
        for o in outs:
            if o:
                lib.ivs_result_free(o)


def release_cached():
    """Frees the device memory, stream and graph that ivs_solve keeps from its last call."""
    load().ivs_release_cached()


def clusters(lo, hi, with_hulls=True):
    """Isolated roots of a box set (rows of lo/hi): connected components of touching boxes
    through ``ivs_clusters``.  Returns (count, labels, hull_lo, hull_hi)."""
    lib = load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    k = lo.shape[0]
    n = lo.shape[1] if lo.ndim == 2 and k else 1
    nc = C.c_int64()
    labels = np.zeros(max(k, 1), np.int64)
    hl = np.zeros((max(k, 1), n))
    hh = np.zeros((max(k, 1), n))
    _check(lib.ivs_clusters(n, k, _ptr(lo), _ptr(hi), C.byref(nc), _ptr(labels),
                            _ptr(hl) if with_hulls else None, _ptr(hh) if with_hulls else None, k))
    c = nc.value
    return c, labels[:k], hl[:c], hh[:c]


def clusters_gpu(lo, hi, device=0):
    """``ivs_clusters`` on the GPU (``ivs_clusters_gpu``): (count, labels, hull_lo, hull_hi)."""
    lib = load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    k = lo.shape[0]
    n = lo.shape[1] if lo.ndim == 2 and k else 1
    nc = C.c_int64()
    labels = np.zeros(max(k, 1), np.int64)
    hl = np.zeros((max(k, 1), n))
    hh = np.zeros((max(k, 1), n))
    _check(lib.ivs_clusters_gpu(n, k, _ptr(lo), _ptr(hi), C.byref(nc), _ptr(labels), _ptr(hl), _ptr(hh), k,
                                int(device)))
    c = nc.value
    return c, labels[:k], hl[:c], hh[:c]


def backtrack_gpu(lo, hi, box_lo, box_hi, level, max_cells=1 << 26, groups=False, device=0):
    """``ivs_backtrack`` on the GPU (``ivs_backtrack_gpu``)."""
    lib = load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    bl = np.ascontiguousarray(box_lo, dtype=np.float64)
    bh = np.ascontiguousarray(box_hi, dtype=np.float64)
    k = lo.shape[0]
    out = C.c_int64()
    grp = C.c_int64()
    _check(lib.ivs_backtrack_gpu(len(bl), k, _ptr(lo), _ptr(hi), _ptr(bl), _ptr(bh), int(level), int(max_cells),
                                 C.byref(out), C.byref(grp), int(device)))
    return (out.value, grp.value) if groups else out.value


def backtrack(lo, hi, box_lo, box_hi, level, max_cells=1 << 26, groups=False):
    """Distinct cells of `level` of the initial box's dyadic grid met by the boxes
    (Algorithm 5 read on that grid) through ``ivs_backtrack``; with groups=True also the
    connected components of those cells (the roots isolated at that width)."""
    lib = load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    bl = np.ascontiguousarray(box_lo, dtype=np.float64)
    bh = np.ascontiguousarray(box_hi, dtype=np.float64)
    k = lo.shape[0]
    out = C.c_int64()
    grp = C.c_int64()
    _check(lib.ivs_backtrack(len(bl), k, _ptr(lo), _ptr(hi), _ptr(bl), _ptr(bh), int(level), int(max_cells),
                             C.byref(out), C.byref(grp)))
    return (out.value, grp.value) if groups else out.value
