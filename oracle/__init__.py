"""CPU oracle for greedy kNN-cost decimation (arXiv 2311.17604).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this package; the library itself never does.

``pd_oracle.c`` is the plain C definition (brute-force or kd-tree kNN plus a
binary-heap sequential greedy); this module compiles it with gcc on first use
and wraps it with ctypes.  ``slow.py`` holds a second, independent pure-numpy
greedy that recomputes every cost from scratch at every step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BRUTE, KDTREE = 0, 1
TERM_NONE, TERM_COLOR, TERM_ORIENT = 0, 1, 2
D2_NONE = np.iinfo(np.int64).max


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP for the independent kNN queries).

    ``-ffp-contract=off`` keeps every floating-point operation separately
    rounded (no fused multiply-add), as the cost definition requires.
    """
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.orc_knn_cost.argtypes = [P, P, P, ctypes.c_int64, P, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, P, P, P]
            lib.orc_knn_cost.restype = ctypes.c_int
            lib.orc_decimate.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_int, P, P, P, P]
            lib.orc_decimate.restype = ctypes.c_int
            lib.orc_knn_query.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int, P,
                                          P, P]
            lib.orc_knn_query.restype = ctypes.c_int
            lib.orc_radius_counts.argtypes = [P, ctypes.c_int64, P, ctypes.c_int, P]
            lib.orc_radius_counts.restype = ctypes.c_int
            lib.orc_decimate_wup.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int64, ctypes.c_int, P, P, P, P,
                                             ctypes.c_int64]
            lib.orc_decimate_wup.restype = ctypes.c_int
            lib.orc_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(xyz, rgb, nrm, term):
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    assert xyz.ndim == 2 and xyz.shape[1] == 3
    rgb = None if rgb is None else np.ascontiguousarray(rgb, dtype=np.uint8)
    nrm = None if nrm is None else np.ascontiguousarray(nrm, dtype=np.float32)
    if term == TERM_COLOR and rgb is None:
        raise ValueError("colour term needs rgb")
    if term == TERM_ORIENT and nrm is None:
        raise ValueError("orientation term needs normals")
    return xyz, rgb, nrm


def threads() -> int:
    """OpenMP threads the oracle's parallel kNN loops use."""
    return int(_load().orc_threads())


def knn_cost(xyz, k, live=None, term=TERM_NONE, a=0.0, rgb=None, nrm=None, backend=KDTREE):
    """k nearest live neighbours of every point and its cost (Eq. 10/11).

    Returns (d2 [n,k] int64 ascending, idx [n,k] int32, cost [n] float64).
    Missing neighbours are D2_NONE / -1.  Removed points get cost 0.
    """
    xyz, rgb, nrm = _prep(xyz, rgb, nrm, term)
    n = xyz.shape[0]
    lv = None if live is None else np.ascontiguousarray(live, dtype=np.uint8)
    d2 = np.empty((n, k), dtype=np.int64)
    idx = np.empty((n, k), dtype=np.int32)
    cost = np.empty(n, dtype=np.float64)
    rc = _load().orc_knn_cost(_ptr(xyz), _ptr(rgb), _ptr(nrm), n, _ptr(lv), k, term, a, backend,
                              _ptr(d2), _ptr(idx), _ptr(cost))
    if rc != 0:
        raise ValueError("orc_knn_cost: invalid arguments")
    return d2, idx, cost


def knn_query(xyz, queries, k):
    """Brute-force k nearest neighbours and density cost (Eq. 10/11) of the
    given query points among all points (every point live).

    Returns (d2 [nq,k] int64 ascending, idx [nq,k] int32, cost [nq] float64).
    """
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    q = np.ascontiguousarray(queries, dtype=np.int64)
    nq = len(q)
    d2 = np.empty((nq, k), dtype=np.int64)
    idx = np.empty((nq, k), dtype=np.int32)
    cost = np.empty(nq, dtype=np.float64)
    rc = _load().orc_knn_query(_ptr(xyz), xyz.shape[0], _ptr(q), nq, k, _ptr(d2), _ptr(idx),
                               _ptr(cost))
    if rc != 0:
        raise ValueError("orc_knn_query: invalid arguments")
    return d2, idx, cost


def radius_counts(xyz, radii_mm):
    """counts[p, j] = #{q != p : d(p,q)^2 <= r_j^2} by brute force (int64)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    r2 = np.ascontiguousarray(np.asarray(radii_mm, dtype=np.int64) ** 2)
    n, nr = xyz.shape[0], len(r2)
    counts = np.empty((n, nr), dtype=np.int64)
    rc = _load().orc_radius_counts(_ptr(xyz), n, _ptr(r2), nr, _ptr(counts))
    if rc != 0:
        raise ValueError("orc_radius_counts: invalid arguments")
    return counts


def decimate(xyz, k, m, term=TERM_NONE, a=0.0, rgb=None, nrm=None, backend=KDTREE,
             want_order=False):
    """Sequential greedy decimation to exactly m points.

    Returns keep (uint8 [n]); with ``want_order`` also the removal order and
    the cost of each removed point at its removal (k = 1 density: d1^2).
    """
    xyz, rgb, nrm = _prep(xyz, rgb, nrm, term)
    n = xyz.shape[0]
    keep = np.empty(n, dtype=np.uint8)
    order = np.empty(max(n - m, 0), dtype=np.int32) if want_order else None
    pkey = np.empty(max(n - m, 0), dtype=np.float64) if want_order else None
    req = ctypes.c_int64(0)
    rc = _load().orc_decimate(_ptr(xyz), _ptr(rgb), _ptr(nrm), n, k, m, term, a, backend,
                              _ptr(keep), _ptr(order), _ptr(pkey), ctypes.byref(req))
    if rc != 0:
        raise ValueError("orc_decimate: invalid arguments")
    if want_order:
        return keep, order, pkey
    return keep


def wup_width(k: int) -> int:
    """Stored neighbours of the w_up mode for k (the k+b buffer): 8 for k <= 6."""
    if not 1 <= k <= 6:
        raise ValueError("the w_up mode supports k in [1, 6]")
    return 8


def decimate_wup(xyz, k, m, S=None, backend=KDTREE, want_log=False):
    """The paper's iterative w_up scheme (section "Sub-sampling algorithm")
    with each sweep restated as parallel rounds of non-interacting removals.

    Returns (keep uint8 [n], iterations, rounds); with ``want_log`` also the
    list of (iteration, points removed) of every round.
    """
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    n = xyz.shape[0]
    S = wup_width(k) if S is None else S
    keep = np.empty(n, dtype=np.uint8)
    it = ctypes.c_int32(0)
    rd = ctypes.c_int64(0)
    cap = 100000 if want_log else 0
    log = np.zeros(max(cap, 1), dtype=np.int64)
    rc = _load().orc_decimate_wup(_ptr(xyz), n, k, S, m, backend, _ptr(keep), ctypes.byref(it),
                                  ctypes.byref(rd), _ptr(log) if want_log else None, cap)
    if rc != 0:
        raise ValueError("orc_decimate_wup: invalid arguments")
    if want_log:
        nr = min(int(rd.value), cap)
        return keep, int(it.value), int(rd.value), [(int(v >> 40), int(v & ((1 << 40) - 1)))
                                                    for v in log[:nr]]
    return keep, int(it.value), int(rd.value)


def target_count(n: int, ratio: float) -> int:
    """m = floor(ratio * n), computed in double (Eq. 1: lambda = m / |C|)."""
    return int(np.floor(np.float64(ratio) * np.float64(n)))
