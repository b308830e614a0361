"""Pins of the FP64 point-cloud oracle (``oracle/points.c``) against closed
forms, brute-force enumeration and central finite differences -- nothing here
re-types the oracle's own formulas.

Geometry: identity cameras (R = I, C = 0, f = 1) make the projection of a
point (a z, b z, z) exactly (a, b), so covered pixel sets are lattice points
inside a disc, computed independently here.
"""
import numpy as np
import pytest

from oracle import points as op

S = 32


def _cam(f=1.0, znear=0.1):
    row = np.zeros(16)
    row[0] = row[4] = row[8] = 1.0
    row[12] = f
    row[13] = znear
    return row


def _pix(i):
    return 1.0 - (2.0 * i + 1.0) / S


def _clouds(points, counts, cams=None):
    points = np.asarray(points, np.float64).reshape(-1, 3)
    counts = np.asarray(counts, np.int64)
    first = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    if cams is None:
        cams = np.stack([_cam()] * len(counts))
    return op.Clouds(points, first, counts, cams)


def _at(ndc_x, ndc_y, z):
    return [ndc_x * z, ndc_y * z, z]


def test_single_point_covers_the_lattice_points_of_its_disc():
    r = 0.2
    c = _clouds([_at(0.1, -0.23, 2.0)], [1])
    idx, zb, di = op.rasterize(c, S, 1, r)
    rows, cols = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
    d = (_pix(cols) - 0.1) ** 2 + (_pix(rows) + 0.23) ** 2
    expect = (d < r * r).reshape(-1)
    assert expect.sum() > 25
    np.testing.assert_array_equal(idx[:, 0] == 0, expect)
    np.testing.assert_allclose(di[expect, 0], d.reshape(-1)[expect], rtol=0, atol=1e-15)
    assert np.all(zb[expect, 0] == 2.0)
    assert np.all(idx[~expect] == -1) and np.all(zb[~expect] == -1) and np.all(di[~expect] == -1)


def test_points_along_one_ray_sort_by_depth_then_id():
    depths = [3.0, 1.5, 2.5, 1.5, 4.0]                      # ids 1 and 3 tie in depth
    c = _clouds([_at(0.0, 0.0, z) for z in depths], [5])
    K = 4
    idx, zb, _ = op.rasterize(c, S, K, 0.3)
    centre = (S // 2) * S + S // 2
    assert idx[centre].tolist() == [1, 3, 2, 0]             # z = 1.5 (id 1, 3), 2.5, 3.0; 4.0 dropped (K = 4)
    assert zb[centre].tolist() == [1.5, 1.5, 2.5, 3.0]


def test_clouds_see_only_their_own_points_and_znear_culls():
    pts = [_at(0.0, 0.0, 2.0), _at(0.0, 0.0, 0.05), _at(0.0, 0.0, 3.0)]   # second point nearer than znear
    c = _clouds(pts, [2, 1])
    idx, _, _ = op.rasterize(c, S, 3, 0.3)
    img0 = idx[: S * S]
    img1 = idx[S * S:]
    assert set(np.unique(img0)) == {-1, 0}
    assert set(np.unique(img1)) == {-1, 2}


def test_margins_flag_rims_and_depth_ties():
    r = 0.2
    # rim exactly through the centre of pixel (16, 16): distance r along x
    x0 = _pix(16) - r
    c = _clouds([_at(x0, _pix(16), 2.0), _at(_pix(5), _pix(5), 1.0), _at(_pix(5), _pix(5), 1.0 + 1e-9)], [3])
    fl = op.margins(c, S, 2, r)
    assert fl[16 * S + 16] & op.RIM
    assert fl[5 * S + 5] & op.DEPTH_TIE
    assert not fl[30 * S + 30]


def _alpha(d, r):
    return 1.0 - d / (r * r)


def test_alpha_and_norm_compositing_closed_forms():
    r = 0.5
    idx = np.array([[4, 1, 2, -1]])
    d = np.array([[0.05, 0.1, 0.2, -1.0]])
    feats = np.zeros((5, 2))
    feats[4], feats[1], feats[2] = [1.0, 2.0], [3.0, -1.0], [0.5, 0.25]
    a = _alpha(d[0, :3], r)
    w = [a[0], (1 - a[0]) * a[1], (1 - a[0]) * (1 - a[1]) * a[2]]
    expect = w[0] * feats[4] + w[1] * feats[1] + w[2] * feats[2]
    np.testing.assert_allclose(op.composite_fwd(idx, d, feats, r, op.ALPHA)[0], expect, rtol=1e-14)
    norm = (a[0] * feats[4] + a[1] * feats[1] + a[2] * feats[2]) / a.sum()
    np.testing.assert_allclose(op.composite_fwd(idx, d, feats, r, op.NORM)[0], norm, rtol=1e-14)


def test_alpha_silhouette_telescopes_and_a_centred_point_is_opaque():
    rng = np.random.default_rng(1)
    r = 0.3
    K = 7
    d = rng.uniform(0.0, r * r, size=(20, K))
    idx = np.tile(np.arange(K), (20, 1))
    ones = np.ones((K, 1))
    out = op.composite_fwd(idx, d, ones, r, op.ALPHA)[:, 0]
    np.testing.assert_allclose(out, 1.0 - np.prod(1.0 - _alpha(d, r), axis=1), rtol=1e-13)
    # a point exactly at the pixel centre (d = 0) hides everything behind it
    d[:, 0] = 0.0
    feats = rng.normal(size=(K, 3))
    np.testing.assert_allclose(op.composite_fwd(idx, d, feats, r, op.ALPHA), np.tile(feats[0], (20, 1)),
                               rtol=0, atol=1e-15)
    # empty pixel: 0 in both modes
    assert np.all(op.composite_fwd(np.full((1, K), -1), np.full((1, K), -1.0), feats, r, op.NORM) == 0)


@pytest.mark.parametrize("mode", [op.ALPHA, op.NORM])
def test_composite_adjoint_matches_central_differences(mode):
    rng = np.random.default_rng(2 + mode)
    r, K, D, npix = 0.4, 5, 3, 6
    idx = rng.integers(0, 9, size=(npix, K))
    idx[1, 3:] = -1
    d = rng.uniform(0.01, 0.15, size=(npix, K))
    feats = rng.normal(size=(9, D))
    g = rng.normal(size=(npix, D))
    gd, gf = op.composite_bwd(idx, d, feats, r, g, mode)
    h = 1e-6
    L = lambda dd, ff: float(np.sum(op.composite_fwd(idx, dd, ff, r, mode) * g))
    for p in range(npix):
        for k in range(K):
            if idx[p, k] < 0:
                assert gd[p, k] == 0
                continue
            dp, dm = d.copy(), d.copy()
            dp[p, k] += h
            dm[p, k] -= h
            assert gd[p, k] == pytest.approx((L(dp, feats) - L(dm, feats)) / (2 * h), rel=1e-6, abs=1e-8)
    for i in range(9):
        for c in range(D):
            fp, fm = feats.copy(), feats.copy()
            fp[i, c] += h
            fm[i, c] -= h
            assert gf[i, c] == pytest.approx((L(d, fp) - L(d, fm)) / (2 * h), rel=1e-6, abs=1e-8)


def test_rasterizer_adjoint_matches_central_differences():
    # a few points seen by a tilted camera; the loss composites the fragments,
    # differentiated with the selection held fixed (h far below every rim margin)
    rng = np.random.default_rng(5)
    cam = _cam(f=1.3)
    ang = 0.3
    Ry = np.array([[np.cos(ang), 0, np.sin(ang)], [0, 1, 0], [-np.sin(ang), 0, np.cos(ang)]])
    cam[0:9] = Ry.reshape(-1)
    cam[9:12] = [0.2, -0.1, -0.5]
    pts = np.array([_at(x, y, z) for x, y, z in rng.uniform([-0.4, -0.4, 1.5], [0.4, 0.4, 3.0], size=(6, 3))])
    c = op.Clouds(pts, np.array([0]), np.array([6]), cam[None])
    r, K = 0.35, 4
    feats = rng.normal(size=(6, 2))
    g = rng.normal(size=(S * S, 2))
    fl = op.margins(c, S, K, r, eps=1e-5)
    g[fl != 0] = 0
    idx, zb, di = op.rasterize(c, S, K, r)
    gdi, _ = op.composite_bwd(idx, di, feats, r, g, op.ALPHA)
    gz = rng.normal(size=idx.shape) * (idx >= 0)
    gz[fl != 0] = 0
    grad = op.rast_bwd(c, S, K, idx, gz, gdi)

    def loss(p):
        cc = op.Clouds(p, np.array([0]), np.array([6]), cam[None])
        i2, z2, d2 = op.rasterize(cc, S, K, r)
        assert np.array_equal(i2[fl == 0], idx[fl == 0])
        return float(np.sum(op.composite_fwd(i2, d2, feats, r, op.ALPHA) * g) + np.sum(z2 * gz * (i2 >= 0)))

    h = 1e-7
    for i in range(6):
        for j in range(3):
            pp, pm = pts.copy(), pts.copy()
            pp[i, j] += h
            pm[i, j] -= h
            fd = (loss(pp) - loss(pm)) / (2 * h)
            assert grad[i, j] == pytest.approx(fd, rel=1e-5, abs=1e-6 * (1 + abs(fd)))
