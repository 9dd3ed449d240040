"""Python binding of the C ABI in include/align.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but
check shapes, pick host/device flags and pass pointers: all of the method's work runs
in the library's CUDA kernels.  Host inputs are numpy arrays; device inputs and
outputs are torch CUDA tensors (torch supplies device memory and streams only).
If the shared library cannot be loaded the calls raise: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ALIGN_OK, ALIGN_NOT_READY = 0, 1
ALIGN_E_INVALID, ALIGN_E_OOM, ALIGN_E_CUDA, ALIGN_E_BUSY, ALIGN_E_TIMEOUT, ALIGN_E_NOREF, ALIGN_E_INTERNAL = (
    -1, -2, -3, -4, -5, -6, -7)
ALIGN_FEAT_COUNT, ALIGN_FEAT_ZVAR, ALIGN_FEAT_COUNT_ZVAR = 0, 1, 2
ALIGN_XYZ_DEVICE, ALIGN_POSES_DEVICE, ALIGN_OUT_DEVICE = 1, 2, 4
ALIGN_BATCH_GRAPH, ALIGN_BATCH_TUNE = 8, 16

_STATUS_NAMES = {0: "ALIGN_OK", 1: "ALIGN_NOT_READY", -1: "ALIGN_E_INVALID", -2: "ALIGN_E_OOM", -3: "ALIGN_E_CUDA",
                 -4: "ALIGN_E_BUSY", -5: "ALIGN_E_TIMEOUT", -6: "ALIGN_E_NOREF", -7: "ALIGN_E_INTERNAL"}

# Every entry point include/align.h declares (checked by the tests against the .so).
EXPORTS = ["align_create_grid", "align_destroy_grid", "align_grid_info", "align_set_reference",
           "align_get_reference", "align_round_poses", "align_eval_mi", "align_accumulate", "align_search",
           "align_search_ex", "align_eval_stats", "align_set_sweep", "align_set_spill", "align_eval_redo_poses", "align_profile", "align_microbench", "align_reference_noalloc", "align_batch_create",
           "align_batch_destroy", "align_eval_batch", "align_batch_set_shape", "align_batch_set_poses_per_cta",
           "align_batch_stats",
           "align_server_create", "align_server_add_reference", "align_submit", "align_poll", "align_wait",
           "align_server_now", "align_server_stats", "align_server_destroy", "align_refine_nm", "align_last_error"]


class AlignError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("res_m", C.c_float), ("dims", C.c_int32 * 3), ("feature", C.c_int32),
                ("count_levels", C.c_int32), ("var_levels", C.c_int32), ("count_thresh", C.c_void_p),
                ("var_thresh", C.c_void_p)]


class AlignPair(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("xyzB", C.c_void_p), ("nB", C.c_int64), ("poses12", C.c_void_p),
                ("eta6", C.c_void_p), ("P", C.c_int64), ("mi_out", C.c_void_p), ("argmax_out", C.c_void_p)]


class AlignRequest(C.Structure):
    _fields_ = [("ref_id", C.c_int32), ("xyzB", C.c_void_p), ("nB", C.c_int64), ("init", C.c_double * 6),
                ("range", C.c_double * 6), ("counts", C.c_int32 * 6), ("levels", C.c_int32)]


class AlignResult(C.Structure):
    _fields_ = [("T", C.c_double * 6), ("mi", C.c_float), ("status", C.c_int32), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the in-tree libmialign.so."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path}")
    lib = C.CDLL(path)
    P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "align_create_grid": [P, P, P],
        "align_destroy_grid": [P],
        "align_grid_info": [P, P, P],
        "align_set_reference": [P, P, i64, C.c_int],
        "align_get_reference": [P, P, P],
        "align_round_poses": [P, P, i64, P],
        "align_eval_mi": [P, P, i64, C.c_int, P, P, i64, P, P, P],
        "align_accumulate": [P, P, i64, C.c_int, P, P, P],
        "align_search": [P, P, i64, C.c_int, P, P, i32, P, P],
        "align_search_ex": [P, P, i64, C.c_int, P, P, P, i32, P, P, P],
        "align_eval_stats": [P, P],
        "align_set_sweep": [P, i32],
        "align_set_spill": [P, i32, i64],
        "align_eval_redo_poses": [P, P, i64, P],
        "align_profile": [P, i32, P],
        "align_reference_noalloc": [P, P, i64, P, P, P],
        "align_microbench": [i32, P, i64, i32, P, P],
        "align_batch_create": [P, P],
        "align_batch_destroy": [P],
        "align_eval_batch": [P, P, i32, C.c_int],
        "align_batch_set_shape": [P, i32],
        "align_batch_set_poses_per_cta": [P, i32],
        "align_batch_stats": [P, P],
        "align_server_create": [C.c_size_t, i32, P],
        "align_server_add_reference": [P, P, P, i64, P],
        "align_submit": [P, P, P],
        "align_poll": [P, C.c_uint64, P],
        "align_wait": [P, C.c_uint64, i64, P],
        "align_server_stats": [P, P],
        "align_server_destroy": [P],
        "align_refine_nm": [P, P, i64, C.c_int, P, i32, P, i32, C.c_double, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.align_server_now.argtypes = [P]
    lib.align_server_now.restype = C.c_double
    lib.align_last_error.argtypes = []
    lib.align_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def align_last_error() -> str:
    return load().align_last_error().decode()


def _check(status: int):
    if status != ALIGN_OK:
        raise AlignError(status, align_last_error())


# ---------------------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------------------
def _is_torch_cuda(x) -> bool:
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def _host(a, dtype, shape_tail=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape_tail is not None:
        a = a.reshape(-1, *shape_tail) if a.size else a.reshape(0, *shape_tail)
    return a


def _device_out(t, dtypes, numel, name):
    """Check a caller-owned CUDA output tensor: contiguous, of one of `dtypes`, with at least
    `numel` elements (the library writes that many)."""
    dtypes = dtypes if isinstance(dtypes, (tuple, list)) else (dtypes,)
    if not _is_torch_cuda(t):
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes or not t.is_contiguous() or t.numel() < numel:
        raise ValueError(f"{name} must be a contiguous {'/'.join(str(x) for x in dtypes)} CUDA tensor "
                         f"of at least {numel} elements")


def _points_arg(xyz):
    """(pointer, n, flags) for a points array (numpy host or torch CUDA)."""
    if _is_torch_cuda(xyz):
        import torch
        if xyz.dtype != torch.float32 or not xyz.is_contiguous() or xyz.dim() != 2 or xyz.shape[1] != 3:
            raise ValueError("device points must be a contiguous (n, 3) float32 CUDA tensor")
        return C.c_void_p(xyz.data_ptr()), int(xyz.shape[0]), ALIGN_XYZ_DEVICE, xyz
    a = _host(xyz, np.float32, (3,))
    return a.ctypes.data_as(C.c_void_p), int(a.shape[0]), 0, a


class Grid:
    """Owns an align_grid*.  `stream` is a torch.cuda.Stream, a raw cudaStream_t int, or None
    (torch's current stream at creation)."""

    def __init__(self, handle, desc_kw, stream_obj):
        self._h = handle
        self.desc = desc_kw
        self._stream_obj = stream_obj
        K = C.c_int32(0)
        V = C.c_int64(0)
        _check(load().align_grid_info(self._h, C.byref(K), C.byref(V)))
        self.K = int(K.value)
        self.V = int(V.value)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().align_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def align_create_grid(origin, res_m, dims, feature=ALIGN_FEAT_ZVAR, count_levels=7, var_levels=15,
                      count_thresh=None, var_thresh=None, stream=None) -> Grid:
    lib = load()
    d = GridDesc()
    d.origin = (C.c_float * 3)(*[float(v) for v in origin])
    d.res_m = float(res_m)
    d.dims = (C.c_int32 * 3)(*[int(v) for v in dims])
    d.feature = int(feature)
    d.count_levels = int(count_levels)
    d.var_levels = int(var_levels)
    ct = None if count_thresh is None else np.ascontiguousarray(count_thresh, dtype=np.uint32)
    vt = None if var_thresh is None else np.ascontiguousarray(var_thresh, dtype=np.int64)
    d.count_thresh = None if ct is None else ct.ctypes.data
    d.var_thresh = None if vt is None else vt.ctypes.data
    stream_obj = stream
    if stream is None:
        try:
            import torch
            stream_obj = torch.cuda.current_stream() if torch.cuda.is_available() else None
        except Exception:
            stream_obj = None
    raw = 0
    if stream_obj is not None:
        raw = stream_obj if isinstance(stream_obj, int) else int(stream_obj.cuda_stream)
    h = C.c_void_p()
    _check(lib.align_create_grid(C.byref(d), C.c_void_p(raw), C.byref(h)))
    return Grid(h, dict(origin=tuple(origin), res_m=res_m, dims=tuple(dims), feature=feature,
                        count_levels=count_levels, var_levels=var_levels), stream_obj)


def align_destroy_grid(grid: Grid):
    grid.close()


def align_set_reference(grid: Grid, xyzA):
    ptr, n, flags, keep = _points_arg(xyzA)
    _check(load().align_set_reference(grid.handle, ptr, n, flags))
    del keep


def align_get_reference(grid: Grid):
    sym = np.empty(grid.V, dtype=np.uint8)
    box = np.empty(6, dtype=np.int32)
    _check(load().align_get_reference(grid.handle, sym.ctypes.data_as(C.c_void_p), box.ctypes.data_as(C.c_void_p)))
    return sym, box


def align_round_poses(origin, eta6) -> np.ndarray:
    """FP64 eta rows -> FP32 pose12 rows for a grid with corner `origin` (host code, no GPU)."""
    o = np.ascontiguousarray(origin, dtype=np.float32).reshape(3)
    eta = _host(eta6, np.float64, (6,))
    out = np.empty((eta.shape[0], 12), dtype=np.float32)
    _check(load().align_round_poses(o.ctypes.data_as(C.c_void_p), eta.ctypes.data_as(C.c_void_p), eta.shape[0],
                                    out.ctypes.data_as(C.c_void_p)))
    return out


def align_eval_mi(grid: Grid, xyzB, poses12=None, eta6=None, with_hist=False, out=None):
    """MI for a batch of poses.  Host inputs -> (mi np.float32[P], argmax int, hist or None).
    With device tensors for `poses12` or `out=(mi, argmax, hist)`, outputs stay on the GPU
    (returned as the given tensors, not synchronised)."""
    lib = load()
    pptr, n, flags, keep_pts = _points_arg(xyzB)
    keep = [keep_pts]
    if (poses12 is None) == (eta6 is None):
        raise ValueError("give exactly one of poses12 and eta6")
    if poses12 is not None:
        if _is_torch_cuda(poses12):
            import torch
            if poses12.dtype != torch.float32 or not poses12.is_contiguous():
                raise ValueError("device poses must be contiguous float32")
            P = int(poses12.numel() // 12)
            poses_ptr = C.c_void_p(poses12.data_ptr())
            flags |= ALIGN_POSES_DEVICE
        else:
            ph = _host(poses12, np.float32, (12,))
            keep.append(ph)
            P = int(ph.shape[0])
            poses_ptr = ph.ctypes.data_as(C.c_void_p)
        eta_ptr = None
    else:
        eh = _host(eta6, np.float64, (6,))
        keep.append(eh)
        P = int(eh.shape[0])
        poses_ptr = None
        eta_ptr = eh.ctypes.data_as(C.c_void_p)
    if out is not None:
        import torch
        mi_t, am_t, hist_t = out
        _device_out(mi_t, torch.float32, P, "mi out")
        if am_t is not None:
            _device_out(am_t, torch.int64, 1, "argmax out")
        if hist_t is not None:
            _device_out(hist_t, (torch.int32, torch.uint32) if hasattr(torch, "uint32") else torch.int32,
                        P * grid.K * grid.K, "hist out")
        flags |= ALIGN_OUT_DEVICE
        _check(lib.align_eval_mi(grid.handle, pptr, n, flags, poses_ptr, eta_ptr, P, C.c_void_p(mi_t.data_ptr()),
                                 None if am_t is None else C.c_void_p(am_t.data_ptr()),
                                 None if hist_t is None else C.c_void_p(hist_t.data_ptr())))
        return out
    mi = np.empty(P, dtype=np.float32)
    am = C.c_int64(-1)
    hist = np.empty((P, grid.K, grid.K), dtype=np.uint32) if with_hist else None
    _check(lib.align_eval_mi(grid.handle, pptr, n, flags, poses_ptr, eta_ptr, P, mi.ctypes.data_as(C.c_void_p),
                             C.byref(am), None if hist is None else hist.ctypes.data_as(C.c_void_p)))
    del keep
    return mi, int(am.value), hist


def align_accumulate(grid: Grid, xyzB, pose12):
    """Per-voxel (n, S1, S2) int64 [V, 3] and B's occupied bbox under one pose."""
    pptr, n, flags, keep = _points_arg(xyzB)
    pose = _host(pose12, np.float32).reshape(12)
    acc = np.empty((grid.V, 3), dtype=np.int64)
    box = np.empty(6, dtype=np.int32)
    _check(load().align_accumulate(grid.handle, pptr, n, flags, pose.ctypes.data_as(C.c_void_p),
                                   acc.ctypes.data_as(C.c_void_p), box.ctypes.data_as(C.c_void_p)))
    del keep
    return acc, box


def align_search(grid: Grid, xyzB, init, rng, levels=6, counts=None):
    """Coarse-to-fine lattice search; returns (T eta[6], MI at T, per-level argmax)."""
    lib = load()
    pptr, n, flags, keep = _points_arg(xyzB)
    init = _host(init, np.float64).reshape(6)
    rng = _host(rng, np.float64).reshape(6)
    T = np.zeros(6, dtype=np.float64)
    mi = C.c_float(0.0)
    lb = np.zeros(max(levels, 1), dtype=np.int64)
    if counts is None:
        _check(lib.align_search(grid.handle, pptr, n, flags, init.ctypes.data_as(C.c_void_p),
                                rng.ctypes.data_as(C.c_void_p), int(levels), T.ctypes.data_as(C.c_void_p),
                                C.byref(mi)))
        del keep
        return T, float(mi.value), None
    cnt = np.ascontiguousarray(counts, dtype=np.int32)
    _check(lib.align_search_ex(grid.handle, pptr, n, flags, init.ctypes.data_as(C.c_void_p),
                               rng.ctypes.data_as(C.c_void_p), cnt.ctypes.data_as(C.c_void_p), int(levels),
                               T.ctypes.data_as(C.c_void_p), C.byref(mi), lb.ctypes.data_as(C.c_void_p)))
    del keep
    return T, float(mi.value), lb[:levels]


def align_refine_nm(grid: Grid, xyzB, starts, step=(8.0, 8.0, 1.0, 0.1, 0.1, 0.8), max_iter=100, ftol=0.0):
    """Nelder-Mead from every start (S x 6); returns (T [S, 6], MI [S], iterations [S])."""
    pptr, n, flags, keep = _points_arg(xyzB)
    st = _host(starts, np.float64, (6,))
    S = int(st.shape[0])
    stp = _host(step, np.float64).reshape(6)
    T = np.zeros((S, 6), dtype=np.float64)
    mi = np.zeros(S, dtype=np.float32)
    it = np.zeros(S, dtype=np.int32)
    _check(load().align_refine_nm(grid.handle, pptr, n, flags, st.ctypes.data_as(C.c_void_p), S,
                                  stp.ctypes.data_as(C.c_void_p), int(max_iter), float(ftol),
                                  T.ctypes.data_as(C.c_void_p), mi.ctypes.data_as(C.c_void_p),
                                  it.ctypes.data_as(C.c_void_p)))
    del keep
    return T, mi, it


SWEEP_KINDS = {0: "one pose per CTA", 1: "pose pairs", 2: "2-CTA cluster"}


def align_eval_stats(grid: Grid):
    out = np.zeros(6, dtype=np.int64)
    _check(load().align_eval_stats(grid.handle, out.ctypes.data_as(C.c_void_p)))
    return {"passes": int(out[0]), "wide_voxels": int(out[1]), "table_slots": int(out[2]), "ctas": int(out[3]),
            "kernel_launches": int(out[4]), "sweep": int(out[5])}


def align_set_sweep(grid: Grid, kind: int):
    """-1 automatic (default), or a kind of SWEEP_KINDS that every launch on the grid takes."""
    _check(load().align_set_sweep(grid.handle, int(kind)))


def align_set_spill(grid: Grid, on: bool, queue_runs: int = 0):
    """Sweep B once per pose (queueing the later key partitions' runs) or once per partition;
    queue_runs: runs per queue and CTA (0: half the points of B)."""
    _check(load().align_set_spill(grid.handle, 1 if on else 0, int(queue_runs)))


def align_eval_redo_poses(grid: Grid) -> np.ndarray:
    """Pose indices of the last evaluation that the exact path finished (ascending)."""
    lib = load()
    n = C.c_int64(0)
    _check(lib.align_eval_redo_poses(grid.handle, None, 0, C.byref(n)))
    out = np.zeros(max(int(n.value), 1), dtype=np.int64)
    _check(lib.align_eval_redo_poses(grid.handle, out.ctypes.data_as(C.c_void_p), int(n.value), C.byref(n)))
    return out[:int(n.value)]


def align_profile(grid: Grid, mode: int):
    """mode 1: enable + reset, 0: disable, 2: read.  Returns (eval ms total, compose ms total,
    eval launches timed)."""
    out = np.zeros(3, dtype=np.float64)
    _check(load().align_profile(grid.handle, int(mode), out.ctypes.data_as(C.c_void_p)))
    return float(out[0]), float(out[1]), int(out[2])


MICROBENCH_KINDS = {0: "fp32 ffma lane-ops", 1: "int32 add/xor lane-ops", 2: "voxel-map mix lane-ops",
                    3: "shared red.add (one bank per lane)", 4: "shared atom.add (one bank per lane)",
                    5: "shared red.add (random words)", 6: "shared atom.add (random words)",
                    7: "L2 atomic add (random words)"}


def align_microbench(kind: int, buf, reps: int = 5, stream=None):
    """(operations/s of the fastest run, its ms, operations per run) of micro-benchmark `kind`
    (MICROBENCH_KINDS) run on the caller's CUDA scratch tensor `buf` (>= 1 MiB)."""
    if not _is_torch_cuda(buf) or not buf.is_contiguous():
        raise ValueError("buf must be a contiguous CUDA tensor")
    raw, _ = _stream_raw(stream)
    out = np.zeros(3, dtype=np.float64)
    _check(load().align_microbench(int(kind), C.c_void_p(buf.data_ptr()), int(buf.numel() * buf.element_size()),
                                   int(reps), C.c_void_p(raw), out.ctypes.data_as(C.c_void_p)))
    return float(out[0]), float(out[1]), float(out[2])


def align_reference_noalloc(desc_kw: dict, xyzA, symA_out, boxA_out, stream=None):
    """A's symbols and bbox into caller-owned device tensors, without any device allocation
    by the library (for callers whose device memory is managed elsewhere or who may not
    allocate in their loop).  `xyzA` (n, 3) float32, `symA_out` (V,) uint8 and `boxA_out`
    (6,) int32 are CUDA tensors.  Asynchronous on `stream` (default: torch's current stream)."""
    lib = load()
    d = GridDesc()
    d.origin = (C.c_float * 3)(*[float(v) for v in desc_kw["origin"]])
    d.res_m = float(desc_kw["res_m"])
    d.dims = (C.c_int32 * 3)(*[int(v) for v in desc_kw["dims"]])
    d.feature = int(desc_kw.get("feature", ALIGN_FEAT_ZVAR))
    d.count_levels = int(desc_kw.get("count_levels", 7))
    d.var_levels = int(desc_kw.get("var_levels", 15))
    ct = desc_kw.get("count_thresh")
    vt = desc_kw.get("var_thresh")
    ct = None if ct is None else np.ascontiguousarray(ct, dtype=np.uint32)
    vt = None if vt is None else np.ascontiguousarray(vt, dtype=np.int64)
    d.count_thresh = None if ct is None else ct.ctypes.data
    d.var_thresh = None if vt is None else vt.ctypes.data
    if not (_is_torch_cuda(xyzA) and _is_torch_cuda(symA_out) and _is_torch_cuda(boxA_out)):
        raise ValueError("align_reference_noalloc takes CUDA tensors only")
    import torch
    xptr, nA, _, _ = _points_arg(xyzA)  # contiguous (n, 3) float32
    V = int(d.dims[0]) * int(d.dims[1]) * int(d.dims[2])
    _device_out(symA_out, torch.uint8, V, "symA_out")
    _device_out(boxA_out, torch.int32, 6, "boxA_out")
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in (xyzA, symA_out, boxA_out)):
        raise ValueError("align_reference_noalloc: tensors must be on the current device")
    if stream is None:
        stream = torch.cuda.current_stream()
    raw = stream if isinstance(stream, int) else int(stream.cuda_stream)
    _check(lib.align_reference_noalloc(C.byref(d), xptr, nA, C.c_void_p(symA_out.data_ptr()),
                                       C.c_void_p(boxA_out.data_ptr()), C.c_void_p(raw)))


# ---------------------------------------------------------------------------------------
# batching: many scan pairs in one launch sequence (one CUDA graph when captured)
# ---------------------------------------------------------------------------------------
def _stream_raw(stream):
    stream_obj = stream
    if stream is None:
        try:
            import torch
            stream_obj = torch.cuda.current_stream() if torch.cuda.is_available() else None
        except Exception:
            stream_obj = None
    raw = 0
    if stream_obj is not None:
        raw = stream_obj if isinstance(stream_obj, int) else int(stream_obj.cuda_stream)
    return raw, stream_obj


class Batch:
    """Owns an align_batch* (device workspace, captured graph)."""

    def __init__(self, handle, stream_obj):
        self._h = handle
        self._stream_obj = stream_obj

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().align_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def align_batch_create(stream=None) -> Batch:
    raw, obj = _stream_raw(stream)
    h = C.c_void_p()
    _check(load().align_batch_create(C.c_void_p(raw), C.byref(h)))
    return Batch(h, obj)


def align_batch_destroy(batch: Batch):
    batch.close()


def align_eval_batch(batch: Batch, pairs, graph=False, tune=False, out=None):
    """Evaluate many pairs in one launch.  `pairs`: sequence of (grid, xyzB, eta6) or
    (grid, xyzB, None, poses12).  Host inputs -> list of (mi np.float32[P], argmax int).
    With CUDA tensors for the points (all pairs), the poses (all pairs) or `out` (a list of
    (mi, argmax) CUDA tensors), those buffers are device memory."""
    lib = load()
    n = len(pairs)
    arr = (AlignPair * max(n, 1))()
    keep = []
    flags = (ALIGN_BATCH_GRAPH if graph else 0) | (ALIGN_BATCH_TUNE if tune else 0)
    results = []
    dev_pts = n > 0 and all(_is_torch_cuda(p[1]) for p in pairs)
    dev_poses = n > 0 and all(len(p) > 3 and p[3] is not None and _is_torch_cuda(p[3]) for p in pairs)
    if dev_pts:
        flags |= ALIGN_XYZ_DEVICE
    if dev_poses:
        flags |= ALIGN_POSES_DEVICE
    if out is not None:
        flags |= ALIGN_OUT_DEVICE
    for i, p in enumerate(pairs):
        grid, xyz = p[0], p[1]
        eta6 = p[2] if len(p) > 2 else None
        poses12 = p[3] if len(p) > 3 else None
        pptr, nB, fl, kp = _points_arg(xyz)
        if bool(fl & ALIGN_XYZ_DEVICE) != dev_pts:
            raise ValueError("points must be all host arrays or all CUDA tensors")
        keep.append(kp)
        arr[i].grid = grid.handle
        arr[i].xyzB = pptr
        arr[i].nB = nB
        if (eta6 is None) == (poses12 is None):
            raise ValueError("give exactly one of eta6 and poses12 per pair")
        if eta6 is not None:
            if dev_poses:
                raise ValueError("eta6 is host memory; give poses12 tensors for every pair")
            eh = _host(eta6, np.float64, (6,))
            keep.append(eh)
            arr[i].eta6 = eh.ctypes.data
            arr[i].P = int(eh.shape[0])
        elif dev_poses:
            arr[i].poses12 = poses12.data_ptr()
            arr[i].P = int(poses12.numel() // 12)
        else:
            ph = _host(poses12, np.float32, (12,))
            keep.append(ph)
            arr[i].poses12 = ph.ctypes.data
            arr[i].P = int(ph.shape[0])
        if out is not None:
            import torch
            mi_t, am_t = out[i]
            _device_out(mi_t, torch.float32, int(arr[i].P), "mi out")
            if am_t is not None:
                _device_out(am_t, torch.int64, 1, "argmax out")
            arr[i].mi_out = mi_t.data_ptr()
            arr[i].argmax_out = None if am_t is None else am_t.data_ptr()
            results.append((mi_t, am_t))
        else:
            mi = np.empty(int(arr[i].P), dtype=np.float32)
            am = np.full(1, -1, dtype=np.int64)
            arr[i].mi_out = mi.ctypes.data
            arr[i].argmax_out = am.ctypes.data
            results.append((mi, am))
    _check(lib.align_eval_batch(batch.handle, arr, n, flags))
    del keep
    if out is not None:
        return results
    return [(mi, int(am[0])) for mi, am in results]


def align_batch_set_shape(batch: Batch, shape: int):
    _check(load().align_batch_set_shape(batch.handle, int(shape)))


def align_batch_set_poses_per_cta(batch: Batch, poses_per_cta: int):
    _check(load().align_batch_set_poses_per_cta(batch.handle, int(poses_per_cta)))


def align_batch_stats(batch: Batch):
    out = np.zeros(9, dtype=np.int64)
    _check(load().align_batch_stats(batch.handle, out.ctypes.data_as(C.c_void_p)))
    keys = ["launches", "graph_captures", "graph_replays", "shape", "table_slots", "kernel_launches",
            "last_us", "tuner_trials", "poses_per_cta"]
    return {k: int(v) for k, v in zip(keys, out)}


# ---------------------------------------------------------------------------------------
# serving: continuous batching of alignment requests
# ---------------------------------------------------------------------------------------
class Server:
    """Owns an align_server* (worker thread, resident references, batch workspace)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().align_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def align_server_create(hbm_budget_bytes: int, max_slots: int) -> Server:
    h = C.c_void_p()
    _check(load().align_server_create(int(hbm_budget_bytes), int(max_slots), C.byref(h)))
    return Server(h)


def align_server_destroy(server: Server):
    server.close()


def align_server_add_reference(server: Server, xyzA, origin, res_m, dims, feature=ALIGN_FEAT_ZVAR, count_levels=7,
                               var_levels=15) -> int:
    d = GridDesc()
    d.origin = (C.c_float * 3)(*[float(v) for v in origin])
    d.res_m = float(res_m)
    d.dims = (C.c_int32 * 3)(*[int(v) for v in dims])
    d.feature = int(feature)
    d.count_levels = int(count_levels)
    d.var_levels = int(var_levels)
    a = _host(xyzA, np.float32, (3,))
    rid = C.c_int32(-1)
    _check(load().align_server_add_reference(server.handle, C.byref(d), a.ctypes.data_as(C.c_void_p),
                                             int(a.shape[0]), C.byref(rid)))
    return int(rid.value)


def align_submit(server: Server, ref_id: int, xyzB, init, rng, levels=6, counts=None) -> int:
    a = _host(xyzB, np.float32, (3,))
    r = AlignRequest()
    r.ref_id = int(ref_id)
    r.xyzB = a.ctypes.data
    r.nB = int(a.shape[0])
    r.init = (C.c_double * 6)(*[float(v) for v in init])
    r.range = (C.c_double * 6)(*[float(v) for v in rng])
    r.counts = (C.c_int32 * 6)(*([0] * 6 if counts is None else [int(v) for v in counts]))
    r.levels = int(levels)
    t = C.c_uint64(0)
    _check(load().align_submit(server.handle, C.byref(r), C.byref(t)))
    return int(t.value)


def _result_dict(res: AlignResult):
    return {"T": np.array(res.T[:], dtype=np.float64), "mi": float(res.mi), "status": int(res.status),
            "t_submit": float(res.t_submit), "t_start": float(res.t_start), "t_done": float(res.t_done)}


def align_poll(server: Server, ticket: int):
    """The result dict when done, else None."""
    res = AlignResult()
    st = load().align_poll(server.handle, C.c_uint64(ticket), C.byref(res))
    if st == ALIGN_NOT_READY:
        return None
    _check(st)
    return _result_dict(res)


def align_wait(server: Server, ticket: int, timeout_ms: int = -1):
    res = AlignResult()
    _check(load().align_wait(server.handle, C.c_uint64(ticket), int(timeout_ms), C.byref(res)))
    return _result_dict(res)


def align_server_now(server: Server) -> float:
    return float(load().align_server_now(server.handle))


def align_server_stats(server: Server):
    out = np.zeros(8, dtype=np.int64)
    _check(load().align_server_stats(server.handle, out.ctypes.data_as(C.c_void_p)))
    keys = ["steps", "admitted", "done", "max_active", "pose_evals", "bytes_held", "bytes_peak", "queued"]
    return {k: int(v) for k, v in zip(keys, out)}
