"""CPU oracle of exact K nearest neighbours (``knn.c``) and of the Chamfer loss
with its gradient (numpy, FP64) on packed heterogeneous batches of point
clouds (Sec. 3.1, "Chamfer loss" (Eq. 1) and "K Nearest Neighbors").

TEST INFRASTRUCTURE ONLY.  The tests and the benchmark's CPU-baseline leg are
the only callers; the product package never imports this module, and this
module never imports the product package.

Chamfer loss of cloud pair i (Eq. 1): the mean over p in P_i of the squared
distance to its nearest neighbour in Q_i, plus the mean over q in Q_i of the
squared distance to its nearest neighbour in P_i.  The neighbours are the
ones ``knn`` picks (K = 1, fp32 decision); the loss and its gradient are then
evaluated in FP64 from the coordinates.  An empty cloud contributes 0 to both
terms (its mean is over no points, and the other cloud's points have no
neighbour), and no gradient.  The batch loss is the mean of the N per-pair
losses.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn.c")
_LIB_PATH = os.path.join(_HERE, "libknn_oracle.so")
_lib = None

_f32p = ctypes.POINTER(ctypes.c_float)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile ``knn.c`` into ``libknn_oracle.so`` next to it (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(os.environ.get("ORACLE_KNN_LIB") or build())
        L.okn_knn.argtypes = [_f32p, _i64, _i64p, _i64p, _f32p, _i64p, _i64p, _i64, _int, _int, _i64p, _i64,
                              _i64p, _f32p]
        _lib = L
    return _lib


def _f(a, D=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a if D is None else a.reshape(-1, D)


def _i(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def knn(p1, first1, len1, p2, first2, len2, K, rows=None):
    """(idx (n, K) int64, dists (n, K) float32) for the query rows listed in
    ``rows`` (default: every row of p1).  idx is the global row in p2 of each
    neighbour (-1 past the end of a small cloud, with distance +inf)."""
    p1 = _f(p1)
    D = p1.shape[-1]
    p1 = p1.reshape(-1, D)
    p2 = _f(p2, D)
    first1, len1, first2, len2 = _i(first1), _i(len1), _i(first2), _i(len2)
    N = first1.shape[0]
    r = None if rows is None else _i(rows)
    n = p1.shape[0] if r is None else r.shape[0]
    idx = np.empty((n, K), np.int64)
    dists = np.empty((n, K), np.float32)
    L = _load()
    L.okn_knn(p1.ctypes.data_as(_f32p), p1.shape[0], first1.ctypes.data_as(_i64p), len1.ctypes.data_as(_i64p),
              p2.ctypes.data_as(_f32p), first2.ctypes.data_as(_i64p), len2.ctypes.data_as(_i64p), N, D, K,
              None if r is None else r.ctypes.data_as(_i64p), n, idx.ctypes.data_as(_i64p),
              dists.ctypes.data_as(_f32p))
    return idx, dists


def chamfer(p, first1, len1, q, first2, len2, idx_pq=None, idx_qp=None):
    """(loss, per_pair (N,), idx_pq (P1,), idx_qp (P2,)) in FP64 (Eq. 1).
    The nearest neighbours come from ``knn`` unless given."""
    p64 = np.asarray(p, np.float64)
    p64 = p64.reshape(-1, p64.shape[-1])
    q64 = np.asarray(q, np.float64).reshape(-1, p64.shape[1])
    first1, len1, first2, len2 = _i(first1), _i(len1), _i(first2), _i(len2)
    if idx_pq is None:
        idx_pq = knn(p, first1, len1, q, first2, len2, 1)[0][:, 0]
    if idx_qp is None:
        idx_qp = knn(q, first2, len2, p, first1, len1, 1)[0][:, 0]
    N = first1.shape[0]
    per = np.zeros(N)
    for i in range(N):
        for pts, other, first, n, nn in ((p64, q64, first1[i], len1[i], idx_pq), (q64, p64, first2[i], len2[i],
                                                                                   idx_qp)):
            rows = np.arange(first, first + n)
            rows = rows[nn[rows] >= 0]
            if n > 0 and rows.size:
                per[i] += np.sum((pts[rows] - other[nn[rows]]) ** 2) / n
    return per.mean() if N else 0.0, per, idx_pq, idx_qp


def chamfer_grad(p, first1, len1, q, first2, len2, idx_pq, idx_qp, grad_per_pair):
    """(grad_p, grad_q) in FP64 for an upstream gradient of the N per-pair
    losses (the batch mean's gradient is grad / N for each pair)."""
    p64 = np.asarray(p, np.float64)
    p64 = p64.reshape(-1, p64.shape[-1])
    q64 = np.asarray(q, np.float64).reshape(-1, p64.shape[1])
    gp, gq = np.zeros_like(p64), np.zeros_like(q64)
    first1, len1, first2, len2 = _i(first1), _i(len1), _i(first2), _i(len2)
    for i in range(first1.shape[0]):
        g = float(grad_per_pair[i])
        for pts, other, gs, go, first, n, nn in ((p64, q64, gp, gq, first1[i], len1[i], idx_pq),
                                                 (q64, p64, gq, gp, first2[i], len2[i], idx_qp)):
            rows = np.arange(first, first + n)
            rows = rows[nn[rows] >= 0]
            if n == 0 or rows.size == 0:
                continue
            # d/dx |x - y|^2 = 2 (x - y), d/dy = -2 (x - y), each term weighted by g / |cloud|
            t = 2.0 * g / n * (pts[rows] - other[nn[rows]])
            np.add.at(gs, rows, t)
            np.add.at(go, nn[rows], -t)
    return gp, gq


def knn_grad(p1, p2, idx, grad_dists):
    """(grad_p1, grad_p2) in FP64 of the squared distances of the listed
    neighbours (idx (P1, K), -1 slots ignored) for an upstream gradient (P1, K)."""
    p1 = np.asarray(p1, np.float64)
    D = p1.shape[-1]
    p1 = p1.reshape(-1, D)
    p2 = np.asarray(p2, np.float64).reshape(-1, D)
    g1, g2 = np.zeros_like(p1), np.zeros_like(p2)
    idx = np.asarray(idx)
    gd = np.asarray(grad_dists, np.float64)
    for k in range(idx.shape[1]):
        rows = np.nonzero(idx[:, k] >= 0)[0]
        t = 2.0 * gd[rows, k][:, None] * (p1[rows] - p2[idx[rows, k]])
        np.add.at(g1, rows, t)
        np.add.at(g2, idx[rows, k], -t)
    return g1, g2
