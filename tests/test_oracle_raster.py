"""Pins for the oracle's rasterizer (Section 3.2, "Rasterizer"; Fragment data).

Each check compares the oracle with something other than itself: integer
lattice counting, linear solves of the ray-triangle intersection, a
derivative-free 1D minimisation for the segment distances, exact stacked
geometry, and the binning completeness theorem.
"""
import numpy as np
import pytest

import oracle
from _scenes import identity_cam, ndc_triangle, pixel_centre, random_small_mesh, scene


def _mesh(sc):
    return oracle.Mesh(sc["verts"], sc["faces"], sc["first_face"], sc["num_faces"], sc["cams"])


# --------------------------------------------------------------------------
# coverage: lattice points of an axis-aligned right triangle
# --------------------------------------------------------------------------
@pytest.mark.parametrize("S", [8, 16, 32])
def test_right_triangle_coverage_is_lattice_set(S):
    # NDC corners (0.5, 0.5), (-0.5, 0.5), (0.5, -0.5) at constant depth 2.
    tri = ndc_triangle((0.5, 0.5), (-0.5, 0.5), (0.5, -0.5), 2.0)
    m = _mesh(scene([tri]))
    p2f, zb, ba, di = oracle.rasterize(m, S, 1, blur=0.0, persp=True, clip=False)
    got = (p2f[:, 0] == 0).reshape(S, S)
    # pixel centre x = (S-1-2c)/S, y = (S-1-2r)/S.  Inside the closed triangle iff
    # x <= 1/2, y <= 1/2 and x + y >= 0, i.e. in integers:
    #   2(S-1-2c) <= S,  2(S-1-2r) <= S,  (S-1-2c) + (S-1-2r) >= 0
    want = np.zeros((S, S), bool)
    for r in range(S):
        for c in range(S):
            X, Y = S - 1 - 2 * c, S - 1 - 2 * r
            want[r, c] = (2 * X <= S) and (2 * Y <= S) and (X + Y >= 0)
    np.testing.assert_array_equal(got, want)
    # constant-depth triangle: zbuf is exactly that depth wherever covered
    assert np.all(zb[p2f[:, 0] == 0, 0] == 2.0)
    assert np.all(zb[p2f[:, 0] < 0, 0] == -1.0)
    assert np.all(di[p2f[:, 0] < 0, 0] == -1.0)


def test_both_windings_rasterize_identically():
    a = ndc_triangle((0.5, 0.5), (-0.5, 0.5), (0.5, -0.5), 2.0)
    b = a[[0, 2, 1]]
    pa = oracle.rasterize(_mesh(scene([a])), 16, 1)[0]
    pb = oracle.rasterize(_mesh(scene([b])), 16, 1)[0]
    np.testing.assert_array_equal(pa, pb)


# --------------------------------------------------------------------------
# barycentrics
# --------------------------------------------------------------------------
def test_bary_at_vertices_and_centroid():
    S = 16
    # Pixel centres are (S-1-2c)/S; put v0 on the centre of (r=7,c=7) = (1/16, 1/16),
    # v1 on (r=7, c=1) = (13/16, 1/16), v2 on (r=1, c=7) = (1/16, 13/16).
    c = lambda i: pixel_centre(i, S)
    tri = ndc_triangle((c(7), c(7)), (c(1), c(7)), (c(7), c(1)), 3.0)
    m = _mesh(scene([tri]))
    p2f, zb, ba, di = oracle.rasterize(m, S, 1, persp=False, clip=False)
    ba = ba.reshape(S, S, 3)
    np.testing.assert_allclose(ba[7, 7], [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(ba[7, 1], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(ba[1, 7], [0, 0, 1], atol=1e-15)
    # centroid (5/16, 5/16)... is not a pixel centre; (r=5,c=5) is (5/16,5/16): check via solve
    p = np.array([c(5), c(5)])
    A = np.array([[c(1) - c(7), c(7) - c(7)], [c(7) - c(7), c(1) - c(7)]]).T
    lam = np.linalg.solve(A, p - np.array([c(7), c(7)]))
    np.testing.assert_allclose(ba[5, 5], [1 - lam.sum(), lam[0], lam[1]], atol=1e-15)
    # exact centroid: an equal-weights point; triangle chosen so that it is a pixel centre
    tri2 = ndc_triangle((c(4), c(4)), (c(10), c(4)), (c(4), c(10)), 1.0)
    # centroid x = (c4+c10+c4)/3 = c(6) because pixel centres are affine in the index
    _, _, b2, _ = oracle.rasterize(_mesh(scene([tri2])), S, 1, persp=False)
    np.testing.assert_allclose(b2.reshape(S, S, 3)[6, 6], [1 / 3, 1 / 3, 1 / 3], atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("persp,clip", [(False, False), (True, False), (True, True), (False, True)])
def test_bary_sums_to_one(seed, persp, clip):
    m = _mesh(random_small_mesh(seed, ntri=4))
    p2f, zb, ba, di = oracle.rasterize(m, 16, 4, blur=2e-3, persp=persp, clip=clip)
    v = p2f >= 0
    assert v.any()
    np.testing.assert_allclose(ba[v].sum(-1), 1.0, atol=1e-13)
    if clip:
        assert (ba[v] >= 0).all()


def _ray_hit(verts, cam, px, py):
    """World-space ray through NDC (px, py) intersected with the triangle's plane.
    Returns (3D barycentrics, view depth)."""
    R = cam[:9].reshape(3, 3)
    C = cam[9:12]
    f = cam[12]
    # R (fp32 rows upcast) is orthonormal only to ~1e-7: invert it exactly
    d_world = np.linalg.solve(R, np.array([px / f, py / f, 1.0]))
    a, b, c = verts
    M = np.stack([b - a, c - a, -d_world], 1)
    l1, l2, t = np.linalg.solve(M, C - a)
    return np.array([1 - l1 - l2, l1, l2]), t


@pytest.mark.parametrize("seed", range(6))
def test_perspective_bary_and_zbuf_equal_ray_plane_hit(seed):
    S = 48
    sc = random_small_mesh(seed, ntri=1)
    m = _mesh(sc)
    p2f, zb, ba, di = oracle.rasterize(m, S, 1, persp=True, clip=False)
    cam = sc["cams"][0]
    hits = 0
    for p in range(S * S):
        r, c = divmod(p, S)
        lam, t = _ray_hit(sc["verts"][sc["faces"][0]], cam, pixel_centre(c, S), pixel_centre(r, S))
        inside = (lam >= 0).all()
        assert (p2f[p, 0] == 0) == inside or np.min(np.abs(lam)) < 1e-12
        if p2f[p, 0] == 0:
            hits += 1
            np.testing.assert_allclose(ba[p, 0], lam, atol=1e-12)
            np.testing.assert_allclose(zb[p, 0], t, rtol=1e-12)
    assert hits > 0


def test_tilted_triangle_depth_is_plane_depth_not_affine():
    # a strongly tilted triangle: perspective-correct z differs from screen-affine z
    sc = scene([np.array([[-1.0, -1.0, 1.0], [1.0, -1.0, 5.0], [0.0, 1.5, 3.0]])])
    m = _mesh(sc)
    S = 16
    _, zp, bp, _ = oracle.rasterize(m, S, 1, persp=True)
    p2f, za, ba, _ = oracle.rasterize(m, S, 1, persp=False)
    v = p2f[:, 0] == 0
    cam = sc["cams"][0]
    for p in np.nonzero(v)[0]:
        r, c = divmod(p, S)
        lam, t = _ray_hit(sc["verts"], cam, pixel_centre(c, S), pixel_centre(r, S))
        assert abs(zp[p, 0] - t) < 1e-12 * t
    assert np.max(np.abs(za[v, 0] - zp[v, 0])) > 1e-3


# --------------------------------------------------------------------------
# dists: signed squared distance to the nearest edge segment
# --------------------------------------------------------------------------
def _seg_dist2_by_search(p, a, b):
    """min over t in [0,1] of |p - a - t(b-a)|^2 by ternary search (no closed form)."""
    lo, hi = 0.0, 1.0
    g = lambda t: float(np.sum((p - a - t * (b - a)) ** 2))
    for _ in range(200):
        m1 = lo + (hi - lo) / 3
        m2 = hi - (hi - lo) / 3
        if g(m1) <= g(m2):
            hi = m2
        else:
            lo = m1
    return min(g(0.0), g(1.0), g((lo + hi) / 2))


@pytest.mark.parametrize("seed", [10, 13, 15])
def test_dists_match_direct_minimisation(seed):
    S = 32
    blur = 0.05
    sc = random_small_mesh(seed, ntri=1)
    m = _mesh(sc)
    p2f, zb, ba, di = oracle.rasterize(m, S, 1, blur=blur, persp=True, clip=True)
    cam = sc["cams"][0]
    Pw = sc["verts"]
    R = cam[:9].reshape(3, 3)
    pv = (Pw - cam[9:12]) @ R.T
    ndc = np.stack([cam[12] * pv[:, 0] / pv[:, 2], cam[12] * pv[:, 1] / pv[:, 2]], 1)
    seen_in = seen_out = 0
    for p in range(S * S):
        r, c = divmod(p, S)
        q = np.array([pixel_centre(c, S), pixel_centre(r, S)])
        s = min(_seg_dist2_by_search(q, ndc[i], ndc[(i + 1) % 3]) for i in range(3))
        lam, _ = _ray_hit(Pw, cam, q[0], q[1])
        inside = (lam >= 0).all()
        want = -s if inside else s
        cand = inside or want < blur
        assert (p2f[p, 0] == 0) == cand
        if cand:
            assert abs(di[p, 0] - want) < 1e-12
            seen_in += inside
            seen_out += not inside
    assert seen_in > 0 and seen_out > 0


def test_dists_hand_cases():
    # triangle (0,0),(0.5,0),(0,0.5) at depth 1; 16x16 pixel centres are odd/16.
    tri = ndc_triangle((0.0, 0.0), (0.5, 0.0), (0.0, 0.5), 1.0)
    m = _mesh(scene([tri]))
    S = 16
    p2f, zb, ba, di = oracle.rasterize(m, S, 1, blur=1.0, persp=False)
    D = di[:, 0].reshape(S, S)
    # pixel (r=7, c=7) is at (1/16, 1/16): inside, nearest edges are the two legs
    assert abs(D[7, 7] - (-(1 / 16) ** 2)) < 1e-15
    # pixel (r=7, c=8) is at (-1/16, 1/16): outside, perpendicular foot on the leg x = 0
    assert abs(D[7, 8] - (1 / 16) ** 2) < 1e-15
    # pixel (r=8, c=8) is at (-1/16, -1/16): nearest point is the vertex (0,0)
    assert abs(D[8, 8] - 2 * (1 / 16) ** 2) < 1e-15
    # pixel (r=7, c=9) is at (-3/16, 1/16): foot (0, 1/16) on the leg x = 0
    assert abs(D[7, 9] - (3 / 16) ** 2) < 1e-15
    # pixel (r=1, c=1) is at (13/16, 13/16): nearest point on the hypotenuse x+y=1/2
    # is its midpoint (1/4,1/4): distance^2 = 2*(13/16-1/4)^2
    assert abs(D[1, 1] - 2 * (13 / 16 - 1 / 4) ** 2) < 1e-15
    # pixel (r=7, c=1) is at (13/16, 1/16): beyond vertex (1/2, 0) along the x axis side
    assert abs(D[7, 1] - ((13 / 16 - 1 / 2) ** 2 + (1 / 16) ** 2)) < 1e-15


# --------------------------------------------------------------------------
# z ordering / K nearest
# --------------------------------------------------------------------------
@pytest.mark.parametrize("K", [1, 3, 5, 8])
def test_stacked_parallel_triangles_sorted_by_depth(K):
    rng = np.random.default_rng(K)
    L = 6
    depths = np.arange(1, L + 1, dtype=float)
    order = rng.permutation(L)
    tris = [ndc_triangle((0.6, 0.6), (-0.6, 0.6), (0.6, -0.6), depths[i]) for i in order]
    m = _mesh(scene(tris))
    p2f, zb, ba, di = oracle.rasterize(m, 8, K)
    inv = np.argsort(order)                     # face id holding depth index j
    inside = p2f[:, 0] >= 0
    assert inside.sum() > 5
    for p in np.nonzero(inside)[0]:
        for k in range(K):
            if k < L:
                assert p2f[p, k] == inv[k]
                assert abs(zb[p, k] - depths[k]) <= 4e-16 * depths[k]
            else:
                assert p2f[p, k] == -1 and zb[p, k] == -1


def test_equal_depth_ties_break_by_face_id():
    tris = [ndc_triangle((0.6, 0.6), (-0.6, 0.6), (0.6, -0.6), 2.0)] * 3
    tris.insert(1, ndc_triangle((0.6, 0.6), (-0.6, 0.6), (0.6, -0.6), 1.5))
    m = _mesh(scene(tris))
    p2f, zb, _, _ = oracle.rasterize(m, 8, 4)
    p = np.nonzero(p2f[:, 0] >= 0)[0][0]
    assert list(p2f[p]) == [1, 0, 2, 3]


# --------------------------------------------------------------------------
# culling, batches
# --------------------------------------------------------------------------
def test_culled_faces_never_appear():
    good = ndc_triangle((0.6, 0.6), (-0.6, 0.6), (0.6, -0.6), 2.0)
    flat = ndc_triangle((0.6, 0.6), (0.0, 0.0), (-0.6, -0.6), 1.0)       # collinear in NDC
    near = good.copy()
    near[1, 2] = 0.05                                                      # corner before znear 0.1
    m = _mesh(scene([flat, near, good]))
    p2f, _, _, _ = oracle.rasterize(m, 16, 3, blur=0.01)
    assert set(np.unique(p2f)) <= {-1, 2}


def test_batch_isolation_and_per_mesh_equivalence():
    a = random_small_mesh(1, ntri=3)
    b = random_small_mesh(2, ntri=2)
    verts = np.concatenate([a["verts"], b["verts"]])
    faces = np.concatenate([a["faces"], b["faces"] + a["verts"].shape[0]])
    m = oracle.Mesh(verts, faces, [0, 3], [3, 2], np.concatenate([a["cams"], b["cams"]]))
    S, K = 16, 3
    p2f, zb, ba, di = oracle.rasterize(m, S, K, blur=1e-3, clip=True)
    p2f = p2f.reshape(2, S * S, K)
    assert set(np.unique(p2f[0])) <= {-1, 0, 1, 2}
    assert set(np.unique(p2f[1])) <= {-1, 3, 4}
    pb, zbb, _, _ = oracle.rasterize(_mesh(b), S, K, blur=1e-3, clip=True)
    np.testing.assert_array_equal(np.where(pb >= 0, pb + 3, -1), p2f[1])
    np.testing.assert_array_equal(zbb, zb.reshape(2, S * S, K)[1])


def test_empty_and_zero_face_meshes():
    a = random_small_mesh(3, level=1)
    F = a["faces"].shape[0]
    m = oracle.Mesh(a["verts"], a["faces"], [0, 0], [0, F],
                    np.concatenate([a["cams"], a["cams"]]))
    p2f, zb, _, _ = oracle.rasterize(m, 8, 2, blur=1e-3)
    assert (p2f.reshape(2, -1)[0] == -1).all()
    assert (p2f.reshape(2, -1)[1] >= 0).any()


def test_sampled_pixels_equal_full_image():
    m = _mesh(random_small_mesh(5, level=1))
    S, K = 16, 4
    full = oracle.rasterize(m, S, K, blur=1e-3, clip=True)
    px = np.array([[0, 3, 4], [0, 8, 8], [0, 15, 0], [0, 7, 9]])
    part = oracle.rasterize(m, S, K, blur=1e-3, clip=True, pixels=px)
    idx = px[:, 1] * S + px[:, 2]
    for a, b in zip(full, part):
        np.testing.assert_array_equal(a[idx], b)


# --------------------------------------------------------------------------
# binning
# --------------------------------------------------------------------------
@pytest.mark.parametrize("bin_size", [4, 8, 16, 5])
@pytest.mark.parametrize("blur", [0.0, 2e-3])
def test_bins_contain_every_candidate(bin_size, blur):
    m = _mesh(random_small_mesh(7, level=2))
    S = 32
    counts, offs, lists, amb = oracle.bins(m, S, bin_size, blur)
    nb = (S + bin_size - 1) // bin_size
    total = 0
    for r in range(S):
        for c in range(S):
            cf, _ = oracle.candidates(m, S, 0, r, c, blur=blur)
            b = (r // bin_size) * nb + c // bin_size
            members = set(lists[offs[b]:offs[b + 1]].tolist())
            assert set(cf.tolist()) <= members
            total += len(cf)
    assert total > 0
    # and binning restricted rasterization equals the unbinned one: every list is
    # ascending, and no list holds a face outside its image
    for b in range(counts.size):
        seg = lists[offs[b]:offs[b + 1]]
        assert np.all(np.diff(seg) > 0)


@pytest.mark.parametrize("seed", [10, 13, 15])
def test_clipped_bary_outside_face_is_clipped_ray_plane_bary(seed):
    """Outside the face (within blur) the perspective-correct barycentrics are the
    (partly negative) 3D barycentrics of the ray-plane hit; clipping comes after
    perspective correction, so b' = max(lambda, 0) / sum max(lambda, 0) and the
    depth is sum b'_i z_i."""
    S = 32
    sc = random_small_mesh(seed, ntri=1)
    m = _mesh(sc)
    p2f, zb, ba, di = oracle.rasterize(m, S, 1, blur=0.05, persp=True, clip=True)
    cam = sc["cams"][0]
    R = cam[:9].reshape(3, 3)
    zc = ((sc["verts"] - cam[9:12]) @ R.T)[:, 2]
    outside = 0
    for p in np.nonzero(p2f[:, 0] == 0)[0]:
        r, c = divmod(p, S)
        lam, _ = _ray_hit(sc["verts"], cam, pixel_centre(c, S), pixel_centre(r, S))
        cl = np.maximum(lam, 0)
        want = cl / cl.sum()
        np.testing.assert_allclose(ba[p, 0], want, atol=1e-12)
        np.testing.assert_allclose(zb[p, 0], want @ zc, rtol=1e-12)
        outside += (lam < 0).any()
    assert outside > 0
