"""Pins for the oracle's hand-written adjoints: central finite differences of
the oracle's own FP64 forward (Algorithms 1-2 and the rasterizer), on tiny
meshes, with the face selection held fixed and pixels near a kink masked.
"""
import numpy as np
import pytest

import oracle
from _scenes import random_small_mesh

SIG, ZN, ZF = 1e-4, 0.1, 100.0


def _rand_frags(rng, P, K, F):
    p2f = rng.integers(0, F, size=(P, K))
    p2f[rng.uniform(size=(P, K)) < 0.25] = -1
    zb = rng.uniform(1.8, 2.6, size=(P, K))
    ba = rng.dirichlet([1, 1, 1], size=(P, K))
    di = rng.uniform(-4e-4, 4e-4, size=(P, K))
    return p2f, zb, ba, di


@pytest.mark.parametrize("mode,sigma,gamma", [(0, 1e-4, 1e-4), (1, 1e-4, 1e-4), (1, 1e-2, 3e-2), (1, 2e-4, 1e-3)])
def test_blend_adjoint_matches_central_differences(mode, sigma, gamma):
    rng = np.random.default_rng(11)
    P, K, F, V = 6, 4, 5, 9
    faces = rng.integers(0, V, size=(F, 3))
    colors = rng.uniform(0, 1, size=(V, 3))
    p2f, zb, ba, di = _rand_frags(rng, P, K, F)
    g = rng.normal(size=(P, 4))
    bg = np.array([0.3, 0.5, 0.7])

    def L(zb_, ba_, di_, co_):
        return float(np.sum(g * oracle.blend_fwd(p2f, zb_, ba_, di_, faces, co_, sigma, gamma, ZN, ZF,
                                                 bg=bg, mode=mode)))

    gz, gb, gd, gc = oracle.blend_bwd(p2f, zb, ba, di, faces, colors, g, sigma, gamma, ZN, ZF, bg=bg,
                                      mode=mode)
    for arr, grad, h in ((di, gd, 1e-3 * sigma), (zb, gz, 1e-2 * gamma), (ba, gb, 1e-6),
                         (colors, gc, 1e-6)):
        num = np.zeros_like(arr)
        it = np.nditer(arr, flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            old = arr[i]
            arr[i] = old + h
            lp = L(zb, ba, di, colors)
            arr[i] = old - h
            lm = L(zb, ba, di, colors)
            arr[i] = old
            num[i] = (lp - lm) / (2 * h)
        scale = max(np.max(np.abs(num)), 1e-30)
        np.testing.assert_allclose(grad, num, atol=1e-6 * scale, rtol=1e-5)
    # invalid slots receive no gradient
    assert np.all(gd[p2f < 0] == 0) and np.all(gz[p2f < 0] == 0)


def _fd_rast(sc, S, K, blur, persp, clip, g_z, g_b, g_d, h=1e-7):
    m = oracle.Mesh(sc["verts"], sc["faces"], sc["first_face"], sc["num_faces"], sc["cams"])
    base = oracle.rasterize(m, S, K, blur, persp, clip)
    verts = sc["verts"].copy()
    num = np.zeros_like(verts)
    for v in range(verts.shape[0]):
        for j in range(3):
            vals = []
            for sgn in (1, -1):
                vv = verts.copy()
                vv[v, j] += sgn * h
                mm = oracle.Mesh(vv, sc["faces"], sc["first_face"], sc["num_faces"], sc["cams"])
                p2f, zb, ba, di = oracle.rasterize(mm, S, K, blur, persp, clip)
                keep = (base[0] >= 0)
                assert np.array_equal(p2f[keep.any(1)], base[0][keep.any(1)]), "selection changed"
                vals.append(np.sum(np.where(keep, g_z * zb, 0)) + np.sum(np.where(keep[..., None], g_b * ba, 0))
                            + np.sum(np.where(keep, g_d * di, 0)))
            num[v, j] = (vals[0] - vals[1]) / (2 * h)
    return base, num


@pytest.mark.parametrize("seed,ntri,blur,persp,clip", [
    (21, 1, 0.0, True, False),
    (22, 3, 0.0, False, False),
    (23, 2, 3e-3, True, True),
    (24, 4, 3e-3, True, False),
    (25, 3, 3e-3, False, True),
    (26, None, 1e-3, True, True),
])
def test_rast_adjoint_matches_central_differences(seed, ntri, blur, persp, clip):
    S, K = 16, 3
    sc = random_small_mesh(seed, ntri=ntri or 3, level=0 if ntri is None else None)
    m = oracle.Mesh(sc["verts"], sc["faces"], sc["first_face"], sc["num_faces"], sc["cams"])
    rng = np.random.default_rng(seed)
    P = S * S
    amb = oracle.margins(m, S, K, blur, persp, clip, eps=1e-4) & oracle.GRAD_AMBIGUOUS
    g_z = rng.normal(size=(P, K))
    g_b = rng.normal(size=(P, K, 3))
    g_d = rng.normal(size=(P, K)) * 300.0
    g_z[amb != 0] = 0
    g_b[amb != 0] = 0
    g_d[amb != 0] = 0
    base, num = _fd_rast(sc, S, K, blur, persp, clip, g_z, g_b, g_d)
    assert (base[0][amb == 0] >= 0).sum() > 5
    ana = oracle.rast_bwd(m, S, K, base[0], g_z, g_b, g_d, blur, persp, clip)
    scale = np.max(np.abs(num))
    assert scale > 0
    np.testing.assert_allclose(ana, num, atol=2e-6 * scale, rtol=2e-5)


def test_rast_then_blend_chain_matches_central_differences():
    """Whole differentiable path (rasterize -> softmax + silhouette blend) against
    finite differences of the composed FP64 forward."""
    S, K, blur = 16, 4, 3e-3
    sig, gam = 1e-3, 2e-3
    sc = random_small_mesh(31, level=0)
    faces = sc["faces"]
    rng = np.random.default_rng(31)
    colors = rng.uniform(0, 1, size=(sc["verts"].shape[0], 3))
    m = oracle.Mesh(sc["verts"], faces, sc["first_face"], sc["num_faces"], sc["cams"])
    amb = oracle.margins(m, S, K, blur, True, True, eps=1e-4) & oracle.GRAD_AMBIGUOUS
    g_img = rng.normal(size=(S * S, 4))
    g_img[amb != 0] = 0
    p2f, zb, ba, di = oracle.rasterize(m, S, K, blur, True, True)

    def loss(verts):
        mm = oracle.Mesh(verts, faces, sc["first_face"], sc["num_faces"], sc["cams"])
        q, z, b, d = oracle.rasterize(mm, S, K, blur, True, True)
        ok = amb == 0
        assert np.array_equal(q[ok], p2f[ok])
        img = oracle.blend_fwd(q, z, b, d, faces, colors, sig, gam, ZN, ZF)
        return float(np.sum(g_img * img))

    gz, gb, gd, gc = oracle.blend_bwd(p2f, zb, ba, di, faces, colors, g_img, sig, gam, ZN, ZF)
    ana = oracle.rast_bwd(m, S, K, p2f, gz, gb, gd, blur, True, True)
    h = 1e-7
    num = np.zeros_like(sc["verts"])
    for v in range(num.shape[0]):
        for j in range(3):
            vp = sc["verts"].copy(); vp[v, j] += h
            vm = sc["verts"].copy(); vm[v, j] -= h
            num[v, j] = (loss(vp) - loss(vm)) / (2 * h)
    scale = np.max(np.abs(num))
    assert scale > 0
    np.testing.assert_allclose(ana, num, atol=2e-6 * scale, rtol=2e-5)
