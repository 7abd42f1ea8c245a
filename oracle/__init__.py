"""Plain CPU oracle for exact Density Peaks Clustering (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The CUDA library never
does, and the two share no code, headers or helpers.

The arithmetic lives in ``dpc_oracle.c`` (plain C, built with
``-ffp-contract=off``); this module only compiles it and marshals numpy arrays.
Every routine evaluates the paper's definitions directly (Section 3,
Definitions 1-5): O(n^2) for full arrays, O(n) per selected point for the
sampled forms used on large point sets.

Points are ``(n, d)`` C-contiguous numpy arrays of ``int32`` or ``float32``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpc_oracle.c")
_SRC_TREE = os.path.join(_HERE, "dpc_oracle_tree.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

I32 = 0
F32 = 1

# planted deviations, used only by tests that show a pin catches a mistake
VAR_EXCLUSIVE = 1
VAR_NO_SELF = 2
VAR_TIE_LARGER_ID = 4
VAR_DIST_TIE_LARGER = 8
VAR_SQRT_COMPARE = 16
VAR_DROP_LAST_DIM = 32
VAR_CENTER_NO_RHO_MIN = 64  # labels only: a center need not reach rho_min


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_liboracle.so``."""
    srcs = (_SRC, _SRC_TREE)
    if not force and os.path.exists(_LIB_PATH) and \
            all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in srcs):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        lib.orc_density.argtypes = [vp, i32, i64, i32, dbl, vp, i64, i32, i32, vp]
        lib.orc_dependent.argtypes = [vp, i32, i64, i32, vp, ctypes.c_int32, i32, i32, vp, vp]
        lib.orc_dependent_at.argtypes = [vp, i32, i64, i32, dbl, vp, i64, i64, i32, i32, vp, vp, vp, vp]
        lib.orc_cluster.argtypes = [i64, vp, vp, vp, ctypes.c_int32, ctypes.c_int32, dbl, i32, vp]
        lib.orc_kth_sqdist.argtypes = [vp, i32, i64, i32, vp, i64, i32, i32, vp]
        lib.orc_threads.argtypes = [i32]
        lib.orc_tree_run.argtypes = [vp, i32, i64, i32, i32, vp, ctypes.c_int32, i32, vp, vp, vp]
        lib.orc_tree_batch.argtypes = [vp, i32, ctypes.c_int32, vp, vp, vp, i32, vp, ctypes.c_int32, i32,
                                       vp, vp, vp]
        lib.orc_tree_run.restype = ctypes.c_int
        lib.orc_tree_batch.restype = ctypes.c_int
        for f in (lib.orc_density, lib.orc_dependent, lib.orc_dependent_at, lib.orc_cluster,
                  lib.orc_kth_sqdist, lib.orc_threads):
            f.restype = ctypes.c_int
        _lib = lib
        return lib


def _points(pts):
    pts = np.asarray(pts)
    if pts.ndim == 1:
        pts = pts[:, None]
    if pts.dtype == np.int32:
        dtype = I32
    elif pts.dtype == np.float32:
        dtype = F32
    else:
        raise TypeError("points must be int32 or float32, got %s" % pts.dtype)
    pts = np.ascontiguousarray(pts)
    return pts, dtype, pts.shape[0], pts.shape[1]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def threads(requested: int = 0) -> int:
    """Number of worker threads the oracle uses for `requested` (0 = all cores)."""
    return _load().orc_threads(requested)


def density(pts, d_cut: float, idx=None, variant: int = 0, nthreads: int = 0) -> np.ndarray:
    """rho (Definition 1) of every point, or of the points ``idx`` only."""
    pts, dtype, n, d = _points(pts)
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        m = idx.shape[0]
    else:
        m = n
    out = np.zeros(m, dtype=np.int32)
    if n == 0 or m == 0:
        return out
    rc = _load().orc_density(_ptr(pts), dtype, n, d, float(d_cut), _ptr(idx), m, variant, nthreads, _ptr(out))
    if rc:
        raise RuntimeError("orc_density failed: %d" % rc)
    return out


def dependent(pts, rho, rho_skip: int = 0, variant: int = 0, nthreads: int = 0):
    """(lambda, delta) of every point from a full rho array (Definitions 2-3)."""
    pts, dtype, n, d = _points(pts)
    rho = np.ascontiguousarray(rho, dtype=np.int32)
    assert rho.shape == (n,)
    lam = np.zeros(n, dtype=np.int32)
    delta = np.zeros(n, dtype=np.float64)
    if n == 0:
        return lam, delta
    rc = _load().orc_dependent(_ptr(pts), dtype, n, d, _ptr(rho), int(rho_skip), variant, nthreads,
                               _ptr(lam), _ptr(delta))
    if rc:
        raise RuntimeError("orc_dependent failed: %d" % rc)
    return lam, delta


def dependent_at(pts, d_cut: float, idx, max_checks: int = 64, variant: int = 0, nthreads: int = 0):
    """(lambda, delta, rho, resolved) of the points ``idx``, with densities
    computed on demand; see ``orc_dependent_at``.  ``resolved[t]`` is False when
    more than ``max_checks`` nearer points had to be examined."""
    pts, dtype, n, d = _points(pts)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = idx.shape[0]
    lam = np.zeros(m, dtype=np.int32)
    delta = np.zeros(m, dtype=np.float64)
    rho = np.zeros(m, dtype=np.int32)
    status = np.zeros(m, dtype=np.int8)
    if m == 0:
        return lam, delta, rho, status.astype(bool)
    rc = _load().orc_dependent_at(_ptr(pts), dtype, n, d, float(d_cut), _ptr(idx), m, int(max_checks),
                                  variant, nthreads, _ptr(lam), _ptr(delta), _ptr(rho), _ptr(status))
    if rc:
        raise RuntimeError("orc_dependent_at failed: %d" % rc)
    return lam, delta, rho, status.astype(bool)


def cluster(rho, lam, delta, rho_noise: int, rho_min: int, delta_min: float, variant: int = 0) -> np.ndarray:
    """Labels (Definitions 4-5 and the assignment rule)."""
    rho = np.ascontiguousarray(rho, dtype=np.int32)
    lam = np.ascontiguousarray(lam, dtype=np.int32)
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    n = rho.shape[0]
    out = np.zeros(n, dtype=np.int32)
    if n == 0:
        return out
    rc = _load().orc_cluster(n, _ptr(rho), _ptr(lam), _ptr(delta), int(rho_noise), int(rho_min),
                             float(delta_min), int(variant), _ptr(out))
    if rc:
        raise RuntimeError("orc_cluster: dependent pointers do not form a valid forest (%d)" % rc)
    return out


# planted deviations of decision_graph, used only by the pin tests
DG_TIE_LARGER_ID = 1
DG_DROP_INF = 2
DG_DELTA_BIN_UP = 4
DG_SUM_NOT_PRODUCT = 8


def decision_graph(rho, delta, k: int, rho_bins: int = 0, delta_bins: int = 0, delta_lo: float = 1.0,
                   variant: int = 0):
    """Decision-graph summaries of one instance (Section 3: the hyper-parameters
    are read off the graph of delta against rho).

    top/gamma: the k points with the largest center score gamma = rho * delta
    (one binary64 product), descending, equal scores by the smaller id; a
    point whose score is NaN (delta NaN) or negative takes no part; the row is
    padded with (-1, NaN).  hist[a][b] counts the points with rho >= 1 and a
    non-NaN delta, a = floor(log2 rho), b = the binary exponent of the
    quotient delta / delta_lo (0 when delta <= delta_lo), both clipped to the
    last bin.  Plain numpy and Python loops; the rule is written out point by
    point.
    """
    rho = np.asarray(rho, dtype=np.int32)
    delta = np.asarray(delta, dtype=np.float64)
    n = rho.shape[0]
    score = []
    for i in range(n):
        r = float(rho[i])
        dl = float(delta[i])
        g = r + dl if variant & DG_SUM_NOT_PRODUCT else r * dl
        if math.isnan(g) or g < 0.0:
            continue
        if variant & DG_DROP_INF and math.isinf(g):
            continue
        score.append((g, i))
    if variant & DG_TIE_LARGER_ID:
        score.sort(key=lambda t: (-t[0], -t[1]))
    else:
        score.sort(key=lambda t: (-t[0], t[1]))
    top = np.full(k, -1, dtype=np.int32)
    gamma = np.full(k, np.nan, dtype=np.float64)
    for j, (g, i) in enumerate(score[:k]):
        top[j] = i
        gamma[j] = g
    out = {"top": top, "gamma": gamma}
    if rho_bins > 0 and delta_bins > 0:
        hist = np.zeros((rho_bins, delta_bins), dtype=np.int64)
        for i in range(n):
            r = int(rho[i])
            dl = float(delta[i])
            if r < 1 or math.isnan(dl):
                continue
            a = min(r.bit_length() - 1, rho_bins - 1)  # 2^a <= r < 2^(a+1)
            if not dl > delta_lo:
                b = 0
            else:
                q = dl / delta_lo
                if math.isinf(q):
                    b = delta_bins - 1
                else:
                    b = math.frexp(q)[1] - 1  # q = m * 2^(b+1), 0.5 <= m < 1
                    if variant & DG_DELTA_BIN_UP:
                        b += 1
                    b = min(max(b, 0), delta_bins - 1)
            hist[a, b] += 1
        out["hist"] = hist
    return out


# planted deviations of priority_range, used only by the pin tests
PR_GE = 1          # rho >= rho_q instead of rho > rho_q
PR_OPEN_BOX = 2    # lo < x < hi instead of lo <= x <= hi
PR_DROP_LAST = 4   # the last coordinate not tested


def priority_range(pts, rho, lo, hi, rho_q, variant: int = 0):
    """Priority range search (the appendix on range queries): the ids of the
    points x_i with x_i in the closed axis-parallel box [lo, hi] and priority
    rho_i > rho_q, in ascending order.  The priority is the density.  One query
    (lo, hi: length-d sequences); coordinates compared in binary64, where the
    int32 and float32 inputs are exact.  Written out point by point with numpy
    comparisons."""
    x = np.asarray(pts).astype(np.float64)
    if x.ndim == 1:
        x = x.reshape(-1, 1)
    n, d = x.shape
    rho = np.asarray(rho, dtype=np.int64)
    lo = np.asarray(lo, dtype=np.float64)[:d]
    hi = np.asarray(hi, dtype=np.float64)[:d]
    keep = rho >= rho_q if variant & PR_GE else rho > rho_q
    dims = d - 1 if variant & PR_DROP_LAST else d
    for a in range(dims):
        if variant & PR_OPEN_BOX:
            keep &= (x[:, a] > lo[a]) & (x[:, a] < hi[a])
        else:
            keep &= (x[:, a] >= lo[a]) & (x[:, a] <= hi[a])
    return np.flatnonzero(keep).astype(np.int32)


def kth_sqdist(pts, idx, k: int, nthreads: int = 0) -> np.ndarray:
    """k-th smallest squared distance from each point ``idx`` (self counted first)."""
    pts, dtype, n, d = _points(pts)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.shape[0], dtype=np.float64)
    if idx.shape[0] == 0:
        return out
    rc = _load().orc_kth_sqdist(_ptr(pts), dtype, n, d, _ptr(idx), idx.shape[0], int(k), nthreads, _ptr(out))
    if rc:
        raise RuntimeError("orc_kth_sqdist failed: %d" % rc)
    return out


def tree_run(pts, d_cuts, rho_skip: int = 0, dependent: bool = True, nthreads: int = 0):
    """rho, lambda, delta of every point of one set for every cutoff in
    ``d_cuts``, from the kd-tree oracle (``dpc_oracle_tree.c``: the same
    definitions as ``density``/``dependent``, searched on the paper's priority
    search kd-tree).  Returns arrays of shape (len(d_cuts), n); with
    ``dependent=False`` only rho."""
    pts, dtype, n, d = _points(pts)
    cuts = np.ascontiguousarray(np.atleast_1d(np.asarray(d_cuts, dtype=np.float64)))
    nc = cuts.shape[0]
    rho = np.zeros((nc, n), dtype=np.int32)
    lam = np.zeros((nc, n), dtype=np.int32) if dependent else None
    delta = np.zeros((nc, n), dtype=np.float64) if dependent else None
    if n:
        rc = _load().orc_tree_run(_ptr(pts), dtype, n, d, nc, _ptr(cuts), int(rho_skip), nthreads, _ptr(rho),
                                  _ptr(lam), _ptr(delta))
        if rc:
            raise RuntimeError("orc_tree_run failed: %d" % rc)
    return {"rho": rho, "lam": lam, "delta": delta}


def tree_batch(flat, pt_offset, coord_offset, dims, d_cuts, rho_skip: int = 0, nthreads: int = 0):
    """The kd-tree oracle over a batch of independent point sets packed back to
    back (``flat``: int32 or float32 coordinates; instance i has
    ``pt_offset[i+1] - pt_offset[i]`` points of ``dims[i]`` coordinates from
    element ``coord_offset[i]``), ``d_cuts[i]`` its cutoffs (the same number for
    every instance).  Returns rho, lam (instance-local ids), delta of shape
    (ncut, N), one thread per instance."""
    flat = np.ascontiguousarray(flat)
    if flat.dtype == np.int32:
        dtype = I32
    elif flat.dtype == np.float32:
        dtype = F32
    else:
        raise TypeError("points must be int32 or float32, got %s" % flat.dtype)
    po = np.ascontiguousarray(pt_offset, dtype=np.int64)
    co = np.ascontiguousarray(coord_offset, dtype=np.int64)
    dm = np.ascontiguousarray(dims, dtype=np.int32)
    cuts = np.ascontiguousarray(np.asarray(d_cuts, dtype=np.float64))
    ni = dm.shape[0]
    assert po.shape == (ni + 1,) and co.shape == (ni,) and cuts.ndim == 2 and cuts.shape[0] == ni
    nc = cuts.shape[1]
    N = int(po[-1])
    rho = np.zeros((nc, N), dtype=np.int32)
    lam = np.zeros((nc, N), dtype=np.int32)
    delta = np.zeros((nc, N), dtype=np.float64)
    rc = _load().orc_tree_batch(_ptr(flat), dtype, ni, _ptr(po), _ptr(co), _ptr(dm), nc, _ptr(cuts),
                                int(rho_skip), nthreads, _ptr(rho), _ptr(lam), _ptr(delta))
    if rc:
        raise RuntimeError("orc_tree_batch failed: %d" % rc)
    return {"rho": rho, "lam": lam, "delta": delta}


def run(pts, d_cut: float, rho_noise: int, rho_min: int, delta_min: float, rho_skip: int = 0,
        nthreads: int = 0):
    """Full DPC on a small point set: returns dict(rho, lam, delta, label)."""
    rho = density(pts, d_cut, nthreads=nthreads)
    lam, delta = dependent(pts, rho, rho_skip=rho_skip, nthreads=nthreads)
    label = cluster(rho, lam, delta, rho_noise, rho_min, delta_min)
    return {"rho": rho, "lam": lam, "delta": delta, "label": label}
