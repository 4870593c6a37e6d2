"""Python binding of libpd (include/pd.h): argument marshalling only.

Every step of the decimation runs in the library's CUDA kernels; this module
only converts torch tensors / numpy arrays to pointers, passes the current
CUDA stream, and routes the library's device allocations through PyTorch's
caching allocator.  The CUDA library must be built (``build.build()``);
importing this module on a machine without it raises immediately.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpd.so")

PD_OK, PD_EINVAL, PD_ERANGE, PD_ENOMEM, PD_ECUDA, PD_ETIMEOUT, PD_EINTERNAL = range(7)
PD_TERM_NONE, PD_TERM_COLOR, PD_TERM_ORIENT = 0, 1, 2
PD_BATCH_PACKED = -1      # pd_decimate_batch: every scan in one packed grid
PD_BATCH_MAX_SCANS = 4096
PD_KMAX = 16
PD_STATIC_MAX_POINTS = 65536

EXPORTED = ["pd_ctx_create", "pd_ctx_destroy", "pd_strerror", "pd_last_error", "pd_build_grid",
            "pd_grid_free", "pd_knn_cost", "pd_decimate_count", "pd_decimate_ratio",
            "pd_grid_stats", "pd_decimate_host", "pd_knn_cost_static", "pd_decimate_batch",
            "pd_autotune", "pd_decimate_wup", "pd_ctx_set_device_budget", "pd_ctx_memory",
            "pd_ctx_reset_peaks",
            # pd_normals.h
            "pd_normals_pca", "pd_mlp_init", "pd_mlp_forward", "pd_mlp_grad", "pd_mlp_train",
            "pd_normals_mlp",
            # pd_serve.h
            "pd_serve_open", "pd_serve_submit", "pd_serve_poll", "pd_serve_counts",
            "pd_serve_close",
            # pd_quality.h
            "pd_quality_report"]
PD_NORMAL_K, PD_MLP_IN, PD_MLP_HIDDEN = 16, 48, 64
PD_NORMAL_DEFINED, PD_NORMAL_PLANAR = 1, 2
PD_SERVE_BYTES_PER_POINT, PD_SERVE_BYTES_PER_POINT_NORMALS = 240, 400
PD_MLP_PARAMS = 64 * 48 + 64 + 64 * 64 + 64 + 3 * 64 + 3


class PdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_strerror(code), code, msg))
        self.code = code


class pd_allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p)),
                ("user", ctypes.c_void_p)]


class pd_grid_params(ctypes.Structure):
    _fields_ = [("leaf_max", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


class pd_cost_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("term", ctypes.c_int32), ("weight", ctypes.c_double),
                ("normals_dev", ctypes.c_void_p), ("band", ctypes.c_double),
                ("reserved", ctypes.c_int32 * 6)]


class pd_memory(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("device_peak", ctypes.c_uint64), ("host_bytes", ctypes.c_uint64),
                ("host_peak", ctypes.c_uint64), ("tracked", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class pd_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("rounds", ctypes.c_int32),
                ("grid_builds", ctypes.c_int32), ("dup_removed", ctypes.c_int64),
                ("requeries", ctypes.c_int64), ("filtered_queries", ctypes.c_int64),
                ("danger_queries", ctypes.c_int64), ("ms_total", ctypes.c_double),
                ("ms_knn", ctypes.c_double), ("ms_build", ctypes.c_double),
                ("ms_knn_first", ctypes.c_double), ("q_first", ctypes.c_int64),
                ("ms_knn_requery", ctypes.c_double), ("ms_rules", ctypes.c_double),
                ("launches", ctypes.c_int64), ("ms_select", ctypes.c_double),
                ("ms_danger", ctypes.c_double), ("pairs_first", ctypes.c_int64),
                ("leaf_max", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("ms_grid", ctypes.c_double), ("live_rounds", ctypes.c_int64),
                ("graph_rounds", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pd_scan_desc(ctypes.Structure):
    _fields_ = [("xyz_dev", ctypes.c_void_p), ("rgb_dev", ctypes.c_void_p),
                ("normals_dev", ctypes.c_void_p), ("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("ratio", ctypes.c_double), ("keep_dev", ctypes.c_void_p),
                ("status", ctypes.c_int32), ("stats", pd_stats)]


_lib = None


class pd_serve_params(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("mem_budget", ctypes.c_int64),
                ("cost", pd_cost_params), ("mlp_params_dev", ctypes.c_void_p),
                ("normals", ctypes.c_int)]


class pd_serve_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("gpu_ms", ctypes.c_double),
                ("stats", pd_stats)]


PD_QUALITY_MAX_RADII, PD_QUALITY_NFRAC, PD_QUALITY_HIST = 32, 7, 16384
QUALITY_FRACTILES = (1, 10, 25, 50, 75, 90, 99)  # percent


class pd_quality(ctypes.Structure):
    _fields_ = [("points", ctypes.c_int64), ("nr", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("radius_mm", ctypes.c_int32 * PD_QUALITY_MAX_RADII),
                ("mean", ctypes.c_double * PD_QUALITY_MAX_RADII),
                ("fractile", (ctypes.c_int32 * PD_QUALITY_NFRAC) * PD_QUALITY_MAX_RADII),
                ("slope_per_m2", ctypes.c_double), ("intercept", ctypes.c_double),
                ("r2", ctypes.c_double), ("rmse", ctypes.c_double),
                ("min_spacing2_mm2", ctypes.c_int64), ("mean_spacing_mm", ctypes.c_double),
                ("count_clipped", ctypes.c_int64), ("ms", ctypes.c_double),
                ("ms_counts", ctypes.c_double), ("reserved", ctypes.c_int64 * 6)]

    def as_dict(self):
        nr = self.nr
        return {"points": self.points, "radius_mm": list(self.radius_mm[:nr]),
                "mean": list(self.mean[:nr]),
                "fractile": [list(self.fractile[j]) for j in range(nr)],
                "slope_per_m2": self.slope_per_m2, "intercept": self.intercept, "r2": self.r2,
                "rmse": self.rmse, "min_spacing2_mm2": self.min_spacing2_mm2,
                "mean_spacing_mm": self.mean_spacing_mm, "count_clipped": self.count_clipped,
                "ms": self.ms, "ms_counts": self.ms_counts}


class pd_train_params(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


def lib():
    """The loaded libpd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libpd.so is not built: run paper_2311_17604_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I64 = ctypes.c_void_p, ctypes.c_int64
        L.pd_ctx_create.argtypes = [ctypes.POINTER(pd_allocator), ctypes.POINTER(P)]
        L.pd_ctx_destroy.argtypes = [P]
        L.pd_ctx_destroy.restype = None
        L.pd_strerror.argtypes = [ctypes.c_int]
        L.pd_strerror.restype = ctypes.c_char_p
        L.pd_last_error.argtypes = [P]
        L.pd_last_error.restype = ctypes.c_char_p
        L.pd_build_grid.argtypes = [P, P, P, I64, ctypes.POINTER(pd_grid_params), P,
                                    ctypes.POINTER(P)]
        L.pd_grid_free.argtypes = [P]
        L.pd_knn_cost.argtypes = [P, ctypes.POINTER(pd_cost_params), P, P, P]
        L.pd_decimate_count.argtypes = [P, ctypes.POINTER(pd_cost_params), I64, P, P]
        L.pd_decimate_ratio.argtypes = [P, ctypes.POINTER(pd_cost_params), ctypes.c_double, P, P]
        L.pd_decimate_wup.argtypes = [P, ctypes.POINTER(pd_cost_params), I64, P, P]
        L.pd_grid_stats.argtypes = [P, ctypes.POINTER(pd_stats)]
        L.pd_decimate_host.argtypes = [P, P, P, P, I64, ctypes.POINTER(pd_cost_params), I64, P,
                                       P, ctypes.POINTER(pd_stats)]
        L.pd_knn_cost_static.argtypes = [P, I64, ctypes.c_int, P, P, P]
        L.pd_decimate_batch.argtypes = [P, ctypes.POINTER(pd_scan_desc), ctypes.c_int,
                                        ctypes.POINTER(pd_cost_params), ctypes.c_int, P]
        L.pd_autotune.argtypes = [P, P, P, I64, ctypes.POINTER(pd_cost_params), ctypes.c_double,
                                  I64, P, ctypes.POINTER(ctypes.c_int32)]
        L.pd_normals_pca.argtypes = [P, P, P, P, P]
        L.pd_mlp_init.argtypes = [P, ctypes.c_uint64, P]
        L.pd_mlp_forward.argtypes = [P, P, I64, P, P, P]
        L.pd_mlp_grad.argtypes = [P, P, P, P, I64, P, P, P]
        L.pd_mlp_train.argtypes = [P, P, P, ctypes.c_int, P, P, P, I64,
                                   ctypes.POINTER(pd_train_params), P, P]
        L.pd_normals_mlp.argtypes = [P, P, P, P, I64, ctypes.c_float, P, P]
        L.pd_serve_open.argtypes = [P, ctypes.POINTER(pd_serve_params), ctypes.POINTER(P)]
        L.pd_serve_submit.argtypes = [P, P, P, I64, I64, ctypes.c_double, P]
        L.pd_serve_poll.argtypes = [P, I64, ctypes.c_int, ctypes.POINTER(pd_serve_result)]
        L.pd_serve_counts.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64),
                                      ctypes.POINTER(I64)]
        L.pd_serve_close.argtypes = [P]
        L.pd_quality_report.argtypes = [P, P, P, I64, P, ctypes.c_int,
                                        ctypes.POINTER(pd_quality), P]
        for f in EXPORTED:
            if f not in ("pd_ctx_destroy", "pd_strerror", "pd_last_error"):
                getattr(L, f).restype = ctypes.c_int
        L.pd_serve_submit.restype = I64
        _lib = L
    return _lib


def _strerror(code):
    try:
        return lib().pd_strerror(code).decode()
    except Exception:
        return "error"


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """pd_ctx with PyTorch's caching allocator as the device allocator."""

    def __init__(self, use_torch_allocator: bool = True):
        self._keep = []
        a = None
        if use_torch_allocator:
            torch = _torch()

            @ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
            def _alloc(user, nbytes, stream):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
                except Exception:
                    return None

            @ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
            def _free(user, ptr, stream):
                try:
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:
                    pass

            a = pd_allocator(_alloc, _free, None)
            self._keep += [_alloc, _free, a]
        h = ctypes.c_void_p()
        rc = lib().pd_ctx_create(ctypes.byref(a) if a is not None else None, ctypes.byref(h))
        if rc:
            raise PdError(rc, "pd_ctx_create")
        self.h = h

    def error(self) -> str:
        return lib().pd_last_error(self.h).decode()

    def set_device_budget(self, nbytes: int, spill_min: int = 0):
        """pd_ctx_set_device_budget: blocks beyond nbytes of device memory
        (and cold blocks) go to pinned host memory that the kernels address
        in place; 0 lifts the budget."""
        self.check(lib().pd_ctx_set_device_budget(self.h, ctypes.c_uint64(int(nbytes)),
                                                  ctypes.c_uint64(int(spill_min))),
                   "pd_ctx_set_device_budget")

    def memory(self) -> dict:
        m = pd_memory()
        self.check(lib().pd_ctx_memory(self.h, ctypes.byref(m)), "pd_ctx_memory")
        return {f: getattr(m, f) for f, _ in m._fields_ if f != "reserved"}

    def reset_peaks(self):
        self.check(lib().pd_ctx_reset_peaks(self.h), "pd_ctx_reset_peaks")

    def check(self, rc, what):
        if rc:
            raise PdError(rc, "%s: %s" % (what, self.error()))

    def close(self):
        if getattr(self, "h", None):
            lib().pd_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cost_params(k=1, term=PD_TERM_NONE, weight=0.0, normals=None, band=0.0):
    return pd_cost_params(int(k), int(term), float(weight), _ptr(normals), float(band))


class Grid:
    """A resident cloud (pd_grid) built from a device int32 [n,3] tensor."""

    def __init__(self, ctx: Context, xyz, rgb=None, leaf_max=0, stream=None):
        torch = _torch()
        assert xyz.is_cuda and xyz.dtype == torch.int32 and xyz.dim() == 2 and xyz.shape[1] == 3
        xyz = xyz.contiguous()
        if rgb is not None:
            assert rgb.is_cuda and rgb.dtype == torch.uint8
            rgb = rgb.contiguous()
        self.ctx = ctx
        self.n = int(xyz.shape[0])
        h = ctypes.c_void_p()
        p = pd_grid_params(int(leaf_max))
        rc = lib().pd_build_grid(ctx.h, _ptr(xyz), _ptr(rgb), self.n, ctypes.byref(p),
                                 _stream_ptr(stream), ctypes.byref(h))
        ctx.check(rc, "pd_build_grid")
        self.h = h

    def free(self):
        if getattr(self, "h", None):
            lib().pd_grid_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self) -> dict:
        s = pd_stats()
        self.ctx.check(lib().pd_grid_stats(self.h, ctypes.byref(s)), "pd_grid_stats")
        return s.as_dict()


def pd_build_grid(ctx, xyz, rgb=None, leaf_max=0, stream=None) -> Grid:
    return Grid(ctx, xyz, rgb, leaf_max, stream)


def pd_knn_cost(grid: Grid, k=1, term=PD_TERM_NONE, weight=0.0, normals=None, cost=None,
                knn=None, stream=None):
    """Cost (float64 [n]) and k nearest input indices (int32 [n,k]) of every point."""
    torch = _torch()
    dev = torch.device("cuda")
    if cost is None:
        cost = torch.empty(grid.n, dtype=torch.float64, device=dev)
    if knn is None:
        knn = torch.empty((grid.n, k), dtype=torch.int32, device=dev)
    cp = cost_params(k, term, weight, normals)
    rc = lib().pd_knn_cost(grid.h, ctypes.byref(cp), _ptr(cost), _ptr(knn), _stream_ptr(stream))
    grid.ctx.check(rc, "pd_knn_cost")
    return cost, knn


def pd_decimate_count(grid: Grid, m, k=1, term=PD_TERM_NONE, weight=0.0, normals=None,
                      keep=None, band=0.0, stream=None):
    """Greedy decimation to exactly m points; returns the uint8 keep mask [n]."""
    torch = _torch()
    if keep is None:
        keep = torch.empty(grid.n, dtype=torch.uint8, device="cuda")
    cp = cost_params(k, term, weight, normals, band)
    rc = lib().pd_decimate_count(grid.h, ctypes.byref(cp), int(m), _ptr(keep),
                                 _stream_ptr(stream))
    grid.ctx.check(rc, "pd_decimate_count")
    return keep


def pd_decimate_wup(grid: Grid, m, k=1, keep=None, stream=None):
    """The paper's iterative w_up scheme (parallel removal rounds); returns
    the uint8 keep mask [n] (exactly m ones)."""
    torch = _torch()
    if keep is None:
        keep = torch.empty(grid.n, dtype=torch.uint8, device="cuda")
    cp = cost_params(k)
    rc = lib().pd_decimate_wup(grid.h, ctypes.byref(cp), int(m), _ptr(keep), _stream_ptr(stream))
    grid.ctx.check(rc, "pd_decimate_wup")
    return keep


def pd_decimate_ratio(grid: Grid, ratio, k=1, term=PD_TERM_NONE, weight=0.0, normals=None,
                      keep=None, band=0.0, stream=None):
    torch = _torch()
    if keep is None:
        keep = torch.empty(grid.n, dtype=torch.uint8, device="cuda")
    cp = cost_params(k, term, weight, normals, band)
    rc = lib().pd_decimate_ratio(grid.h, ctypes.byref(cp), float(ratio), _ptr(keep),
                                 _stream_ptr(stream))
    grid.ctx.check(rc, "pd_decimate_ratio")
    return keep


def pd_decimate_host(ctx: Context, xyz: np.ndarray, m, k=1, term=PD_TERM_NONE, weight=0.0,
                     rgb=None, normals=None, keep=None, band=0.0, stream=None):
    """End to end on host arrays (numpy, ideally pinned): returns (keep, stats)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    n = xyz.shape[0]
    if keep is None:
        keep = np.empty(n, dtype=np.uint8)
    rgb = None if rgb is None else np.ascontiguousarray(rgb, dtype=np.uint8)
    normals = None if normals is None else np.ascontiguousarray(normals, dtype=np.float32)
    cp = cost_params(k, term, weight, None, band)
    st = pd_stats()
    rc = lib().pd_decimate_host(ctx.h, _ptr(xyz), _ptr(rgb), _ptr(normals), n, ctypes.byref(cp),
                                int(m), _ptr(keep), _stream_ptr(stream), ctypes.byref(st))
    ctx.check(rc, "pd_decimate_host")
    return keep, st.as_dict()


def pd_autotune(ctx: Context, xyz, ratio, k=1, term=PD_TERM_NONE, weight=0.0, normals=None,
                rgb=None, sample=0, stream=None):
    """Pick the octree leaf capacity for decimations like this one (timed on
    the first `sample` points); stored in the context for later grids.
    Returns the chosen capacity."""
    xyz = xyz.contiguous()
    out = ctypes.c_int32(0)
    cp = cost_params(k, term, weight, normals)
    rc = lib().pd_autotune(ctx.h, _ptr(xyz), _ptr(rgb), int(xyz.shape[0]), ctypes.byref(cp),
                           float(ratio), int(sample), _stream_ptr(stream), ctypes.byref(out))
    ctx.check(rc, "pd_autotune")
    return int(out.value)


def pd_quality_report(ctx: Context, xyz, keep, radii_mm, stream=None):
    """Quality report (neighbour count against area, fractile bands,
    regression slope / R^2 / RMSE, Eq. 2 spacing) of the retained points of a
    device int32 [n,3] cloud; keep: device uint8 [n] or None (all points)."""
    torch = _torch()
    assert xyz.is_cuda and xyz.dtype == torch.int32 and xyz.dim() == 2 and xyz.shape[1] == 3
    xyz = xyz.contiguous()
    if keep is not None:
        assert keep.is_cuda and keep.dtype == torch.uint8 and keep.numel() == xyz.shape[0]
        keep = keep.contiguous()
    r = np.ascontiguousarray(np.asarray(radii_mm, dtype=np.int32))
    out = pd_quality()
    rc = lib().pd_quality_report(ctx.h, _ptr(xyz), _ptr(keep), int(xyz.shape[0]), _ptr(r),
                                 len(r), ctypes.byref(out), _stream_ptr(stream))
    ctx.check(rc, "pd_quality_report")
    return out.as_dict()


def pd_knn_cost_static(xyz, k=1, cost=None, knn=None, stream=None):
    """Allocation-free neighbour/cost pass for clouds of at most
    PD_STATIC_MAX_POINTS points (device int32 [n,3]); same outputs as
    pd_knn_cost with the density cost.  Raises PdError on failure."""
    torch = _torch()
    assert xyz.is_cuda and xyz.dtype == torch.int32 and xyz.dim() == 2 and xyz.shape[1] == 3
    xyz = xyz.contiguous()
    n = int(xyz.shape[0])
    if cost is None:
        cost = torch.empty(n, dtype=torch.float64, device=xyz.device)
    if knn is None:
        knn = torch.empty((n, k), dtype=torch.int32, device=xyz.device)
    rc = lib().pd_knn_cost_static(_ptr(xyz), n, int(k), _ptr(cost), _ptr(knn),
                                  _stream_ptr(stream))
    if rc:
        raise PdError(rc, "pd_knn_cost_static")
    return cost, knn


def pd_decimate_batch(ctx: Context, clouds, k=1, term=PD_TERM_NONE, weight=0.0,
                      concurrency=PD_BATCH_PACKED, band=0.0, stream=None):
    """Decimate many independent scans; ``clouds`` is a list of dicts with
    ``xyz`` (device int32 [n,3]), ``m`` or ``ratio``, optional ``rgb`` (device
    uint8 [n,3]) and ``normals`` (device float32 [n,3]).  ``concurrency``:
    PD_BATCH_PACKED (all scans in one grid) or a number of concurrent slots
    (0 = 8).  Returns the keep masks (device uint8) and per-scan stats."""
    torch = _torch()
    descs = (pd_scan_desc * len(clouds))()
    keeps = []
    for i, c in enumerate(clouds):
        x = c["xyz"].contiguous()
        c["xyz"] = x
        n = int(x.shape[0])
        keep = torch.empty(n, dtype=torch.uint8, device=x.device)
        keeps.append(keep)
        descs[i].xyz_dev = x.data_ptr()
        descs[i].rgb_dev = c["rgb"].data_ptr() if c.get("rgb") is not None else None
        descs[i].normals_dev = c["normals"].data_ptr() if c.get("normals") is not None else None
        descs[i].n = n
        descs[i].m = int(c["m"]) if c.get("m") is not None else -1
        descs[i].ratio = float(c.get("ratio", 0.0))
        descs[i].keep_dev = keep.data_ptr()
    cp = cost_params(k, term, weight, None, band)
    rc = lib().pd_decimate_batch(ctx.h, descs, len(clouds), ctypes.byref(cp), int(concurrency),
                                 _stream_ptr(stream))
    ctx.check(rc, "pd_decimate_batch")
    return keeps, [descs[i].stats.as_dict() for i in range(len(clouds))]


# ---------------------------------------------------------------- normals (pd_normals.h)
def pd_normals_pca(grid: Grid, stream=None):
    """16-NN feature rows (bfloat16 bit patterns, int16 tensor [n, 48]), PCA
    normals (float32 [n, 3]) and validity (uint8 [n]) of every grid point."""
    torch = _torch()
    feat = torch.empty((grid.n, PD_MLP_IN), dtype=torch.int16, device="cuda")
    pca = torch.empty((grid.n, 3), dtype=torch.float32, device="cuda")
    valid = torch.empty(grid.n, dtype=torch.uint8, device="cuda")
    rc = lib().pd_normals_pca(grid.h, _ptr(feat), _ptr(pca), _ptr(valid), _stream_ptr(stream))
    grid.ctx.check(rc, "pd_normals_pca")
    return feat, pca, valid


def pd_mlp_init(seed=0, params=None, stream=None):
    torch = _torch()
    if params is None:
        params = torch.empty(PD_MLP_PARAMS, dtype=torch.float32, device="cuda")
    rc = lib().pd_mlp_init(_ptr(params), int(seed), _stream_ptr(stream))
    if rc:
        raise PdError(rc, "pd_mlp_init")
    return params


def pd_mlp_forward(params, feat, stream=None):
    """Network normals (float32 [n, 3]) and raw output norms (float32 [n])."""
    torch = _torch()
    n = int(feat.shape[0])
    normals = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    norm = torch.empty(n, dtype=torch.float32, device="cuda")
    rc = lib().pd_mlp_forward(_ptr(params), _ptr(feat), n, _ptr(normals), _ptr(norm),
                              _stream_ptr(stream))
    if rc:
        raise PdError(rc, "pd_mlp_forward")
    return normals, norm


def pd_mlp_grad(ctx: Context, params, feat, labels, stream=None):
    """(mean loss, gradient float32 [PD_MLP_PARAMS]) over all rows."""
    torch = _torch()
    grad = torch.empty(PD_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    rc = lib().pd_mlp_grad(ctx.h, _ptr(params), _ptr(feat), _ptr(labels.contiguous()),
                           int(feat.shape[0]), _ptr(grad), _ptr(loss), _stream_ptr(stream))
    ctx.check(rc, "pd_mlp_grad")
    return float(loss.item()), grad


class MlpTrainer:
    """Parameters plus Adam state, trained in place by pd_mlp_train."""

    def __init__(self, seed=0, params=None):
        torch = _torch()
        self.params = pd_mlp_init(seed) if params is None else params
        self.adam = torch.zeros(2 * PD_MLP_PARAMS, dtype=torch.float32, device="cuda")
        self.step = 0

    def train(self, ctx: Context, feat, labels, valid=None, steps=100, batch=4096, lr=1e-3,
              seed=0, stream=None):
        """Runs `steps` Adam steps; returns the per-step batch losses (float32)."""
        torch = _torch()
        loss = torch.empty(max(steps, 1), dtype=torch.float32, device="cuda")
        tp = pd_train_params(int(steps), int(batch), float(lr), int(seed))
        rc = lib().pd_mlp_train(ctx.h, _ptr(self.params), _ptr(self.adam), self.step, _ptr(feat),
                                _ptr(labels.contiguous()), _ptr(valid), int(feat.shape[0]),
                                ctypes.byref(tp), _ptr(loss), _stream_ptr(stream))
        ctx.check(rc, "pd_mlp_train")
        self.step += steps
        return loss[:steps]


def pd_normals_mlp(ctx: Context, params, feat, pca, min_norm=0.0, stream=None):
    """Normals for the orientation term: network where its output norm is at
    least min_norm (default 1e-3), PCA elsewhere; params=None gives PCA."""
    torch = _torch()
    n = int(pca.shape[0])
    out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    rc = lib().pd_normals_mlp(ctx.h, _ptr(params), _ptr(feat), _ptr(pca), n, float(min_norm),
                              _ptr(out), _stream_ptr(stream))
    ctx.check(rc, "pd_normals_mlp")
    return out


# ---------------------------------------------------------------- serving (pd_serve.h)
class Server:
    """pd_serve_* request loop.  ``submit`` takes host numpy arrays (kept
    alive here until the scan is polled done); page-locked arrays from
    ``pinned_like`` let the copies run asynchronously."""

    def __init__(self, ctx: Context, slots=4, mem_budget=0, k=1, term=PD_TERM_NONE, weight=0.0,
                 mlp_params=None, normals=False, band=0.0):
        self.ctx = ctx
        p = pd_serve_params()
        p.slots = int(slots)
        p.mem_budget = int(mem_budget)
        p.cost = cost_params(k, term, weight, None, band)
        p.mlp_params_dev = None if mlp_params is None else mlp_params.data_ptr()
        p.normals = 1 if normals else 0
        self._mlp = mlp_params
        h = ctypes.c_void_p()
        rc = lib().pd_serve_open(ctx.h, ctypes.byref(p), ctypes.byref(h))
        ctx.check(rc, "pd_serve_open")
        self.h = h
        self._live = {}

    def submit(self, xyz, m=-1, ratio=0.0, rgb=None, keep=None):
        """Queue one scan (host int32 [n,3]); returns its ticket."""
        xyz = np.ascontiguousarray(xyz, dtype=np.int32) if isinstance(xyz, np.ndarray) else xyz
        n = int(xyz.shape[0])
        if keep is None:
            keep = np.empty(n, dtype=np.uint8)
        t = lib().pd_serve_submit(self.h, _ptr(xyz), _ptr(rgb), n, int(m), float(ratio),
                                  _ptr(keep))
        if t < 0:
            raise PdError(int(-t), "pd_serve_submit")
        self._live[int(t)] = (xyz, rgb, keep)
        return int(t)

    def poll(self, ticket, wait_ms=-1):
        """(keep mask, result dict) when done, else None."""
        r = pd_serve_result()
        rc = lib().pd_serve_poll(self.h, int(ticket), int(wait_ms), ctypes.byref(r))
        if rc == PD_ETIMEOUT:
            return None
        if rc:
            raise PdError(rc, "pd_serve_poll")
        keep = self._live[int(ticket)][2]
        res = {f: getattr(r, f) for f, _ in pd_serve_result._fields_ if f != "stats"}
        res["stats"] = r.stats.as_dict()
        return keep, res

    def counts(self):
        q, r, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lib().pd_serve_counts(self.h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(d))
        return q.value, r.value, d.value

    def close(self):
        if self.h:
            lib().pd_serve_close(self.h)
            self.h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pinned_like(a):
    """A page-locked copy of a numpy array (a numpy view of a pinned torch tensor)."""
    torch = _torch()
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t.numpy()

