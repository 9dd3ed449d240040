"""CPU oracle for the voxelized-feature MI cost of arXiv 1709.06948 (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with the
CUDA library and never imports it.

The C source (``mi_oracle.c``) is the oracle proper: plain dense definitions of
Algorithm 1's steps, the overlap region, and Eqs. 1-5 in FP64.  This module only
marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FEAT_COUNT, FEAT_ZVAR, FEAT_COUNT_ZVAR = 0, 1, 2
_MAX_LEVELS = 63


class _Grid(C.Structure):
    _fields_ = [
        ("origin", C.c_float * 3),
        ("res_m", C.c_float),
        ("dims", C.c_int32 * 3),
        ("feature", C.c_int32),
        ("count_levels", C.c_int32),
        ("var_levels", C.c_int32),
        ("count_thresh", C.c_uint32 * _MAX_LEVELS),
        ("var_thresh", C.c_int64 * _MAX_LEVELS),
        ("inv_res", C.c_float),
        ("res_mm", C.c_int32),
        ("n_symbols", C.c_int32),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        P = C.c_void_p
        i64, i32, f64 = C.c_int64, C.c_int32, C.c_double
        sig = {
            "orc_grid_init": (C.c_int, [P, P, C.c_float, P, i32, i32, i32, P, P]),
            "orc_round_pose": (None, [P, P, P]),
            "orc_point_key": (i64, [P, P, P, P]),
            "orc_accumulate": (i64, [P, P, i64, P, P, P, P, P]),
            "orc_symbol": (i32, [P, i64, i64, i64]),
            "orc_reference": (None, [P, P, i64, P, P]),
            "orc_joint_hist": (i64, [P, P, P, P, i64, P, P, P]),
            "orc_mi_from_hist": (f64, [P, i32, i64]),
            "orc_entropy_rows": (f64, [P, i32, i64]),
            "orc_entropy_cols": (f64, [P, i32, i64]),
            "orc_entropy_joint": (f64, [P, i32, i64]),
            "orc_eval_mi": (None, [P, P, P, P, i64, P, i64, i64, P, P, P]),
            "orc_eval_mi_threads": (None, [P, P, P, P, i64, P, i64, P, P, P, i32]),
            "orc_argmax": (i64, [P, i64]),
            "orc_search": (None, [P, P, P, P, i64, P, P, P, i32, i32, P, P, P]),
            "orc_lattice": (None, [P, P, P, P]),
            "orc_nm_mi": (i32, [P, P, P, P, i64, P, P, i32, f64, P, P]),
            "orc_nm_quadratic": (i32, [P, P, P, P, i32, f64, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """A voxel grid with its feature definition (the oracle's own copy of the convention)."""

    def __init__(self, origin, res_m, dims, feature=FEAT_ZVAR, count_levels=7, var_levels=15,
                 count_thresh=None, var_thresh=None):
        lib = _load()
        self._g = _Grid()
        o = (C.c_float * 3)(*[float(x) for x in origin])
        d = (C.c_int32 * 3)(*[int(x) for x in dims])
        ct = None if count_thresh is None else np.ascontiguousarray(count_thresh, dtype=np.uint32)
        vt = None if var_thresh is None else np.ascontiguousarray(var_thresh, dtype=np.int64)
        rc = lib.orc_grid_init(C.byref(self._g), o, C.c_float(res_m), d, int(feature), int(count_levels),
                               int(var_levels), _ptr(ct), _ptr(vt))
        if rc != 0:
            raise ValueError("invalid grid description")

    @property
    def ref(self):
        return C.byref(self._g)

    @property
    def dims(self):
        return tuple(self._g.dims)

    @property
    def V(self) -> int:
        X, Y, Z = self.dims
        return X * Y * Z

    @property
    def K(self) -> int:
        return int(self._g.n_symbols)

    @property
    def res_mm(self) -> int:
        return int(self._g.res_mm)

    @property
    def inv_res(self) -> float:
        return float(self._g.inv_res)

    def thresholds(self):
        g = self._g
        return (np.array(g.count_thresh[: max(g.count_levels - 1, 0)], dtype=np.uint32),
                np.array(g.var_thresh[: max(g.var_levels - 1, 0)], dtype=np.int64))

    # --- single steps -------------------------------------------------------------
    def round_pose(self, eta) -> np.ndarray:
        eta = _f64(eta).reshape(-1, 6)
        out = np.empty((eta.shape[0], 12), dtype=np.float32)
        lib = _load()
        for i in range(eta.shape[0]):
            lib.orc_round_pose(self.ref, _ptr(eta[i]), _ptr(out[i]))
        return out

    def point_keys(self, pose12, xyz):
        """Per point: voxel key (-1 outside) and dz in mm under one pose."""
        lib = _load()
        pose12 = _f32(pose12).reshape(12)
        xyz = _f32(xyz).reshape(-1, 3)
        keys = np.empty(xyz.shape[0], dtype=np.int64)
        dzs = np.zeros(xyz.shape[0], dtype=np.int32)
        dz = C.c_int32(0)
        for i in range(xyz.shape[0]):
            keys[i] = lib.orc_point_key(self.ref, _ptr(pose12), _ptr(xyz[i]), C.byref(dz))
            dzs[i] = dz.value if keys[i] >= 0 else 0
        return keys, dzs

    def accumulate(self, xyz, pose12):
        """Dense (n, sum dz, sum dz^2) per voxel and the occupied bbox under one pose."""
        lib = _load()
        xyz = _f32(xyz).reshape(-1, 3)
        pose12 = _f32(pose12).reshape(12)
        cnt = np.empty(self.V, dtype=np.int64)
        s1 = np.empty(self.V, dtype=np.int64)
        s2 = np.empty(self.V, dtype=np.int64)
        box = np.empty(6, dtype=np.int32)
        inside = lib.orc_accumulate(self.ref, _ptr(xyz), xyz.shape[0], _ptr(pose12), _ptr(cnt), _ptr(s1),
                                    _ptr(s2), _ptr(box))
        return cnt, s1, s2, box, int(inside)

    def symbol(self, n, s1, s2) -> int:
        return int(_load().orc_symbol(self.ref, int(n), int(s1), int(s2)))

    def reference(self, xyzA):
        """Algorithm 1 initialisation: A's symbol per voxel and A's bbox."""
        xyzA = _f32(xyzA).reshape(-1, 3)
        sym = np.empty(self.V, dtype=np.uint8)
        box = np.empty(6, dtype=np.int32)
        _load().orc_reference(self.ref, _ptr(xyzA), xyzA.shape[0], _ptr(sym), _ptr(box))
        return sym, box

    def joint_hist(self, symA, boxA, xyzB, pose12):
        xyzB = _f32(xyzB).reshape(-1, 3)
        h = np.empty((self.K, self.K), dtype=np.uint64)
        box = np.empty(6, dtype=np.int32)
        N = _load().orc_joint_hist(self.ref, _ptr(np.ascontiguousarray(symA, dtype=np.uint8)),
                                   _ptr(np.ascontiguousarray(boxA, dtype=np.int32)), _ptr(xyzB),
                                   xyzB.shape[0], _ptr(_f32(pose12).reshape(12)), _ptr(h), _ptr(box))
        return h, int(N), box

    def eval_mi(self, symA, boxA, xyzB, poses12, nthreads=1, with_hist=False, p0=0, p1=None):
        lib = _load()
        xyzB = _f32(xyzB).reshape(-1, 3)
        poses12 = _f32(poses12).reshape(-1, 12)
        P = poses12.shape[0]
        mi = np.zeros(P, dtype=np.float64)
        nov = np.zeros(P, dtype=np.int64)
        hist = np.zeros((P, self.K, self.K), dtype=np.uint32) if with_hist else None
        symA = np.ascontiguousarray(symA, dtype=np.uint8)
        boxA = np.ascontiguousarray(boxA, dtype=np.int32)
        if p1 is None:
            p1 = P
        if nthreads > 1 and p0 == 0 and p1 == P:
            lib.orc_eval_mi_threads(self.ref, _ptr(symA), _ptr(boxA), _ptr(xyzB), xyzB.shape[0], _ptr(poses12), P,
                                    _ptr(mi), _ptr(hist), _ptr(nov), int(nthreads))
        else:
            lib.orc_eval_mi(self.ref, _ptr(symA), _ptr(boxA), _ptr(xyzB), xyzB.shape[0], _ptr(poses12), int(p0),
                            int(p1), _ptr(mi), _ptr(hist), _ptr(nov))
        return mi, hist, nov

    def search(self, symA, boxA, xyzB, init, rng, counts=(8, 8, 2, 2, 2, 8), levels=6, nthreads=1):
        lib = _load()
        xyzB = _f32(xyzB).reshape(-1, 3)
        T = np.zeros(6, dtype=np.float64)
        mi = C.c_double(0.0)
        lb = np.zeros(levels, dtype=np.int64)
        cnt = np.ascontiguousarray(counts, dtype=np.int32)
        lib.orc_search(self.ref, _ptr(np.ascontiguousarray(symA, dtype=np.uint8)),
                       _ptr(np.ascontiguousarray(boxA, dtype=np.int32)), _ptr(xyzB), xyzB.shape[0],
                       _ptr(_f64(init)), _ptr(_f64(rng)), _ptr(cnt), int(levels), int(nthreads), _ptr(T),
                       C.byref(mi), _ptr(lb))
        return T, float(mi.value), lb

    def nm(self, symA, boxA, xyzB, x0, step, max_iter, ftol=0.0):
        """Nelder-Mead on -MI (Algorithm 1's optimiser), FP64 MI of every vertex."""
        xyzB = _f32(xyzB).reshape(-1, 3)
        T = np.zeros(6, dtype=np.float64)
        mi = C.c_double(0.0)
        it = _load().orc_nm_mi(self.ref, _ptr(np.ascontiguousarray(symA, dtype=np.uint8)),
                               _ptr(np.ascontiguousarray(boxA, dtype=np.int32)), _ptr(xyzB), xyzB.shape[0],
                               _ptr(_f64(x0)), _ptr(_f64(step)), int(max_iter), float(ftol), _ptr(T), C.byref(mi))
        return T, float(mi.value), int(it)


def nm_quadratic(w, c, x0, step, max_iter, ftol=0.0):
    """Nelder-Mead (the oracle's implementation) on sum_i w_i (x_i - c_i)^2."""
    x = np.zeros(6, dtype=np.float64)
    f = C.c_double(0.0)
    it = _load().orc_nm_quadratic(_ptr(_f64(w)), _ptr(_f64(c)), _ptr(_f64(x0)), _ptr(_f64(step)), int(max_iter),
                                  float(ftol), _ptr(x), C.byref(f))
    return x, float(f.value), int(it)


def mi_from_hist(h, N=None) -> float:
    h = np.ascontiguousarray(h, dtype=np.uint64)
    K = h.shape[0]
    assert h.shape == (K, K)
    if N is None:
        N = int(h.sum())
    return float(_load().orc_mi_from_hist(_ptr(h), K, int(N)))


def entropies(h, N=None):
    """(H(X), H(Y), H(X,Y)) of a count table, rows = X."""
    h = np.ascontiguousarray(h, dtype=np.uint64)
    K = h.shape[0]
    if N is None:
        N = int(h.sum())
    lib = _load()
    return (float(lib.orc_entropy_rows(_ptr(h), K, int(N))), float(lib.orc_entropy_cols(_ptr(h), K, int(N))),
            float(lib.orc_entropy_joint(_ptr(h), K, int(N))))


def argmax(mi) -> int:
    mi = _f64(mi)
    return int(_load().orc_argmax(_ptr(mi), mi.shape[0]))


def lattice(center, rng, counts) -> np.ndarray:
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    P = int(np.prod(np.maximum(counts, 1)))
    out = np.empty((P, 6), dtype=np.float64)
    _load().orc_lattice(_ptr(_f64(center)), _ptr(_f64(rng)), _ptr(counts), _ptr(out))
    return out


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
