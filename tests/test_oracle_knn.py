"""Pins of the nearest-neighbour and Chamfer oracles (``oracle/knn.c``,
``oracle/knn.py``): scipy's k-d tree (an independent exact KNN) on random
heterogeneous batches, hand-placed ties and empty clouds, the naive
pairwise-distance Chamfer of Eq. 1 (the formulation the paper contrasts with),
closed forms of shifted clouds, and central differences of both gradients."""
import numpy as np
import pytest

from oracle import knn as ok


def _batch(rng, lens, D, scale=1.0):
    lens = np.asarray(lens, np.int64)
    first = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    pts = (rng.normal(size=(int(lens.sum()), D)) * scale).astype(np.float32)
    return pts, first, lens


@pytest.mark.parametrize("D", [1, 2, 3, 4])
@pytest.mark.parametrize("K", [1, 5, 32])
def test_knn_matches_kdtree(D, K):
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(10 * D + K)
    p1, f1, l1 = _batch(rng, [40, 0, 77, 3], D)
    p2, f2, l2 = _batch(rng, [60, 12, 0, 90], D)
    idx, dist = ok.knn(p1, f1, l1, p2, f2, l2, K)
    checked = 0
    for i in range(len(f1)):
        cand = p2[f2[i]:f2[i] + l2[i]].astype(np.float64)
        for r in range(f1[i], f1[i] + l1[i]):
            kk = min(K, int(l2[i]))
            assert (idx[r, kk:] == -1).all() and np.isinf(dist[r, kk:]).all()
            if kk == 0:
                continue
            tree = spatial.cKDTree(cand)
            dd, jj = tree.query(p1[r].astype(np.float64), k=min(kk + 1, int(l2[i])))
            dd, jj = np.atleast_1d(dd) ** 2, np.atleast_1d(jj)
            # the ranking is decided in fp32: compare where the FP64 gaps exceed its rounding
            for k in range(kk):
                lo = dd[k - 1] if k > 0 else -np.inf
                hi = dd[k + 1] if k + 1 < dd.size else np.inf
                if min(dd[k] - lo, hi - dd[k]) > 1e-5 * max(dd[k], 1e-30):
                    assert idx[r, k] == f2[i] + jj[k], (i, r, k)
                    checked += 1
                assert abs(float(dist[r, k]) - dd[k]) <= 1e-6 * dd[k] + 1e-30
    assert checked > 0.9 * sum(min(K, int(l2[i])) * int(l1[i]) for i in range(len(f1)))


def test_knn_ties_prefer_the_smaller_index_and_clouds_do_not_mix():
    # query at the origin; candidates at distance 1 in every axis direction,
    # one at 2, and (in cloud 1) one at distance 0.5 that cloud 0 must not see
    p1 = np.zeros((2, 3), np.float32)
    p2 = np.array([[0, 0, 2], [1, 0, 0], [0, -1, 0], [0, 0, 1], [-1, 0, 0], [0.5, 0, 0]], np.float32)
    f1, l1 = np.array([0, 1]), np.array([1, 1])
    f2, l2 = np.array([0, 5]), np.array([5, 1])
    idx, dist = ok.knn(p1, f1, l1, p2, f2, l2, 6)
    assert idx[0].tolist() == [1, 2, 3, 4, 0, -1]
    assert dist[0].tolist() == [1, 1, 1, 1, 4, np.inf]
    assert idx[1].tolist() == [5, -1, -1, -1, -1, -1] and dist[1, 0] == 0.25
    # a listed subset of rows gives the same rows
    i2, d2 = ok.knn(p1, f1, l1, p2, f2, l2, 6, rows=[1, 0])
    assert (i2 == idx[::-1]).all() and (d2 == dist[::-1]).all()


def test_knn_distance_is_the_stated_fp32_evaluation():
    # (1 + 2^-12)^2 = 1 + 2^-11 + 2^-24 is not a float: the single fp32 product
    # rounds it to 1 + 2^-11 (tie to even); the FP64 value sits between floats
    a = np.float32(1 + 2.0 ** -12)
    p1 = np.array([[a, 0]], np.float32)
    p2 = np.array([[0, 0]], np.float32)
    _, d = ok.knn(p1, [0], [1], p2, [0], [1], 1)
    assert d[0, 0] == np.float32(1 + 2.0 ** -11)
    # the second coordinate enters by one fma: 2^-24 + (1 + 2^-12)^2 = 1 + 2^-11 + 2^-23
    # exactly (a float); rounding the square first would give 1 + 2^-11 (tie to even)
    p1 = np.array([[2.0 ** -12, a]], np.float32)
    _, d = ok.knn(p1, [0], [1], p2, [0], [1], 1)
    assert d[0, 0] == np.float32(1 + 2.0 ** -11 + 2.0 ** -23)


def _naive_chamfer(p, f1, l1, q, f2, l2):
    # Eq. 1 via the full pairwise distance matrix of each pair of clouds
    per = []
    for i in range(len(f1)):
        P = p[f1[i]:f1[i] + l1[i]].astype(np.float64)
        Q = q[f2[i]:f2[i] + l2[i]].astype(np.float64)
        if len(P) == 0 or len(Q) == 0:
            per.append(0.0)
            continue
        M = ((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1)
        per.append(M.min(1).mean() + M.min(0).mean())
    return np.array(per)


def test_chamfer_matches_the_pairwise_matrix_form():
    rng = np.random.default_rng(3)
    p, f1, l1 = _batch(rng, [100, 7, 0, 64], 3)
    q, f2, l2 = _batch(rng, [33, 250, 5, 0], 3)
    loss, per, _, _ = ok.chamfer(p, f1, l1, q, f2, l2)
    ref = _naive_chamfer(p, f1, l1, q, f2, l2)
    np.testing.assert_allclose(per, ref, rtol=1e-6, atol=1e-12)
    assert loss == pytest.approx(ref.mean(), rel=1e-6)


def test_chamfer_closed_forms():
    # identical clouds: 0; a cloud on a coarse lattice shifted by t (|t| far below
    # the spacing): every nearest neighbour is the shifted partner, loss 2 |t|^2
    g = np.stack(np.meshgrid(np.arange(4.0), np.arange(3.0), np.arange(2.0)), -1).reshape(-1, 3).astype(np.float32)
    f, n = np.array([0]), np.array([len(g)])
    assert ok.chamfer(g, f, n, g, f, n)[0] == 0.0
    t = np.array([0.125, -0.0625, 0.25], np.float32)
    loss = ok.chamfer(g, f, n, g + t, f, n)[0]
    assert loss == pytest.approx(2 * float(np.dot(t, t)), rel=1e-12)


def test_chamfer_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    p, f1, l1 = _batch(rng, [12, 0, 9], 3)
    q, f2, l2 = _batch(rng, [7, 4, 15], 3)
    _, _, ipq, iqp = ok.chamfer(p, f1, l1, q, f2, l2)
    w = rng.normal(size=3)
    gp, gq = ok.chamfer_grad(p, f1, l1, q, f2, l2, ipq, iqp, w)
    p64, q64 = p.astype(np.float64), q.astype(np.float64)

    def L(pp, qq):
        return float(np.dot(w, ok.chamfer(pp, f1, l1, qq, f2, l2, ipq, iqp)[1]))

    h = 1e-6
    for arr, g, is_p in ((p64, gp, True), (q64, gq, False)):
        for ix in np.ndindex(arr.shape):
            a, b = arr.copy(), arr.copy()
            a[ix] += h
            b[ix] -= h
            fd = (L(a, q64) - L(b, q64)) / (2 * h) if is_p else (L(p64, a) - L(p64, b)) / (2 * h)
            assert g[ix] == pytest.approx(fd, rel=1e-6, abs=1e-8), ix


def test_knn_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    p1, f1, l1 = _batch(rng, [6, 5], 2)
    p2, f2, l2 = _batch(rng, [4, 8], 2)
    K = 5
    idx, _ = ok.knn(p1, f1, l1, p2, f2, l2, K)
    g = rng.normal(size=idx.shape)
    g1, g2 = ok.knn_grad(p1, p2, idx, g)

    def L(a1, a2):
        m = idx >= 0
        d = ((a1[:, None, :] - a2[np.where(m, idx, 0)]) ** 2).sum(-1)
        return float(np.sum(np.where(m, d, 0.0) * g))

    a1, a2 = p1.astype(np.float64), p2.astype(np.float64)
    h = 1e-6
    for arr, gr, first in ((a1, g1, True), (a2, g2, False)):
        for ix in np.ndindex(arr.shape):
            a, b = arr.copy(), arr.copy()
            a[ix] += h
            b[ix] -= h
            fd = (L(a, a2) - L(b, a2)) / (2 * h) if first else (L(a1, a) - L(a1, b)) / (2 * h)
            assert gr[ix] == pytest.approx(fd, rel=1e-6, abs=1e-8), ix
