"""Pins of the FP64 shading oracle (``oracle/shading.c``): closed forms of the
Phong reflection model on hand-placed geometry, the reduction of every model
to the unlit softmax blend of ``oracle.c`` when only ambient light is on, the
equality of the three models on a face with one normal, and central finite
differences of the adjoint."""
import numpy as np
import pytest

import oracle
from oracle import shading as sh


def _face(normal=(0.0, 0.0, -1.0)):
    # one triangle in the plane z = 2 facing the camera (-z); the winding makes
    # (P1 - P0) x (P2 - P0) = -z, so flat shading sees the same normal
    verts = np.array([[-0.5, -0.5, 2.0], [0.5, -0.5, 2.0], [0.0, 0.5, 2.0]])
    normals = np.tile(np.asarray(normal, float), (3, 1))
    colors = np.array([[0.8, 0.2, 0.1], [0.8, 0.2, 0.1], [0.8, 0.2, 0.1]])
    return verts, np.array([[0, 2, 1]]), normals, colors


def _cam_at(centre):
    row = np.zeros(16)
    row[0] = row[4] = row[8] = 1.0
    row[9:12] = centre
    row[12] = 1.0
    row[13] = 0.1
    return row[None]


def _one_pixel(bary):
    return (np.zeros(1, np.int64), np.array([[0]]), np.array([[2.0]]), np.asarray(bary, float).reshape(1, 1, 3),
            np.array([[-1e-3]]))


@pytest.mark.parametrize("mode", [sh.FLAT, sh.GOURAUD, sh.PHONG])
def test_light_and_eye_along_the_normal(mode):
    # the surface point is (0, -1/6, 2); light and eye straight in front of it:
    # cos = 1 (full diffuse), mirror direction = eye direction (full specular)
    verts, faces, normals, colors = _face()
    b = [1 / 3, 1 / 3, 1 / 3]
    x = np.array([0.0, -1 / 6, 2.0])
    light = sh.light_params(x + [0, 0, -3.0], (0.1, 0.2, 0.3), (0.5, 0.5, 0.5), (0.25, 0.25, 0.25), 10.0)
    cams = _cam_at(x + [0, 0, -1.5])
    img, p2f, zb, ba, di = _one_pixel(b)
    out = sh.shade_fwd(img, p2f, zb, ba, di, faces, verts, normals, colors, cams, light, sh.blend_params(),
                       mode, sh.HARD)[0]
    if mode == sh.GOURAUD:
        # lit at the corners: each corner sees the light off its normal
        for i in range(3):
            u = (x + [0, 0, -3.0]) - verts[i]
            assert np.dot(u / np.linalg.norm(u), [0, 0, -1]) < 1
        assert out[3] == 1.0
        return
    np.testing.assert_allclose(out[:3], colors[0] * (np.array([0.1, 0.2, 0.3]) + 0.5) + 0.25, rtol=1e-14)


def test_oblique_light_lambert_cosine_and_back_light():
    verts, faces, normals, colors = _face()
    x = np.array([0.0, -1 / 6, 2.0])
    cams = _cam_at(x + [0, 0, -2.0])
    img, p2f, zb, ba, di = _one_pixel([1 / 3, 1 / 3, 1 / 3])
    ang = np.radians(60.0)
    light_dir = np.array([np.sin(ang), 0.0, -np.cos(ang)])
    light = sh.light_params(x + 4.0 * light_dir, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), 8.0)
    out = sh.shade_fwd(img, p2f, zb, ba, di, faces, verts, normals, colors, cams, light, sh.blend_params(),
                       sh.PHONG, sh.HARD)[0]
    np.testing.assert_allclose(out[:3], colors[0] * 0.5, rtol=1e-13)            # cos 60 = 1/2
    back = sh.light_params(x + [0, 0, 3.0], (0.1, 0.1, 0.1), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 8.0)
    out = sh.shade_fwd(img, p2f, zb, ba, di, faces, verts, normals, colors, cams, back, sh.blend_params(),
                       sh.PHONG, sh.HARD)[0]
    np.testing.assert_allclose(out[:3], colors[0] * 0.1, rtol=1e-14)            # ambient only
    # specular exponent: eye at the mirror direction of a 60-degree light, tilted by 10 degrees
    mirror = np.array([-np.sin(ang), 0.0, -np.cos(ang)])
    rot = np.radians(10.0)
    eye_dir = np.array([-np.sin(ang + rot), 0.0, -np.cos(ang + rot)])
    spec = sh.light_params(x + 4.0 * light_dir, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 8.0)
    out = sh.shade_fwd(img, p2f, zb, ba, di, faces, verts, normals, colors, _cam_at(x + 2.0 * eye_dir), spec,
                       sh.blend_params(), sh.PHONG, sh.HARD)[0]
    assert np.dot(mirror, eye_dir) == pytest.approx(np.cos(rot))
    np.testing.assert_allclose(out[:3], np.cos(rot) ** 8, rtol=1e-12)


def test_models_agree_on_a_flat_face_with_one_normal_and_ambient_reduces_to_the_unlit_blend():
    rng = np.random.default_rng(0)
    verts, faces, normals, colors = _face()
    colors = rng.uniform(size=(3, 3))
    cams = _cam_at([0.1, 0.0, -1.0])
    K = 3
    npix = 5
    p2f = np.array([[0, 0, -1]] * npix)
    zb = np.tile([2.0, 2.0 + 1e-3, -1.0], (npix, 1))
    di = rng.uniform(-1e-4, 1e-4, size=(npix, K))
    ba = rng.dirichlet([1, 1, 1], size=(npix, K))
    img = np.zeros(npix, np.int64)
    ambient = sh.light_params([0.3, 0.2, -2.0], (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 4.0)
    bl = sh.blend_params(sigma=1e-4, gamma=1e-2)
    unlit = oracle.blend_fwd(p2f, zb, ba, di, faces, colors, 1e-4, 1e-2, 0.1, 100.0, mode=1)
    for mode in (sh.FLAT, sh.GOURAUD, sh.PHONG):
        out = sh.shade_fwd(img, p2f, zb, ba, di, faces, verts, normals, colors, cams, ambient, bl, mode)
        np.testing.assert_allclose(out, unlit, rtol=1e-12, atol=1e-15)
    # with full lighting, flat == Phong when every vertex normal is the face normal
    lit = sh.light_params([0.3, 0.2, -2.0], (0.2, 0.2, 0.2), (0.6, 0.5, 0.4), (0.3, 0.3, 0.3), 16.0)
    a = sh.shade_fwd(img, p2f, zb, ba, di, faces, verts, normals, colors, cams, lit, bl, sh.FLAT)
    b = sh.shade_fwd(img, p2f, zb, ba, di, faces, verts, normals, colors, cams, lit, bl, sh.PHONG)
    np.testing.assert_allclose(a, b, rtol=1e-12)


@pytest.mark.parametrize("mode", [sh.FLAT, sh.GOURAUD, sh.PHONG])
@pytest.mark.parametrize("blend_mode", [sh.SOFTMAX, sh.HARD])
def test_adjoint_matches_central_differences(mode, blend_mode):
    rng = np.random.default_rng(7 + mode)
    # two faces sharing an edge, tilted, seen by one camera
    verts = np.array([[-0.6, -0.5, 2.0], [0.5, -0.4, 2.3], [0.0, 0.6, 2.1], [0.7, 0.5, 2.4]])
    faces = np.array([[0, 1, 2], [1, 3, 2]])
    normals = rng.normal(size=(4, 3)) * 0.3 + [0, 0, -1]
    colors = rng.uniform(size=(4, 3))
    cams = _cam_at([0.2, -0.1, -0.5])
    npix, K = 4, 2
    p2f = np.array([[0, 1], [1, -1], [0, -1], [1, 0]])
    zb = rng.uniform(2.0, 2.4, size=(npix, K))
    zb.sort(axis=1)
    ba = rng.dirichlet([2, 2, 2], size=(npix, K))
    di = rng.uniform(-3e-3, 3e-3, size=(npix, K))
    img = np.zeros(npix, np.int64)
    light = sh.light_params([1.0, 2.0, -1.5], (0.2, 0.25, 0.3), (0.6, 0.5, 0.4), (0.4, 0.4, 0.4), 6.0)
    bl = sh.blend_params(sigma=1e-3, gamma=5e-3)
    g = rng.normal(size=(npix, 4))
    args = [img, p2f, zb, ba, di, faces, verts, normals, colors, cams, light, bl, mode]
    gz, gb, gd, gv, gn, gc, abb = sh.shade_bwd(*args, g, blend_mode=blend_mode, with_abs_bary=True)
    # the term magnitudes bound each barycentric gradient (triangle inequality)
    assert (abb >= np.abs(gb) - 1e-15).all() and abb.max() > 0

    def L(**kw):
        a = dict(zip(["img", "p2f", "zb", "ba", "di", "faces", "verts", "normals", "colors"], args[:9]))
        a.update(kw)
        out = sh.shade_fwd(a["img"], a["p2f"], a["zb"], a["ba"], a["di"], a["faces"], a["verts"], a["normals"],
                           a["colors"], cams, light, bl, mode, blend_mode)
        return float(np.sum(out * g))

    h = 1e-6
    for name, arr, grad in (("verts", verts, gv), ("normals", normals, gn), ("colors", colors, gc),
                            ("ba", ba, gb), ("zb", zb, gz), ("di", di, gd)):
        it = np.nditer(arr, flags=["multi_index"])
        for _ in it:
            ix = it.multi_index
            if name in ("ba", "zb", "di") and p2f[ix[0], ix[1]] < 0:
                continue
            ap, am = arr.copy(), arr.copy()
            ap[ix] += h
            am[ix] -= h
            kw = {{"verts": "verts", "normals": "normals", "colors": "colors", "ba": "ba", "zb": "zb",
                   "di": "di"}[name]: ap}
            kwm = {list(kw)[0]: am}
            fd = (L(**kw) - L(**kwm)) / (2 * h)
            assert grad[ix] == pytest.approx(fd, rel=1e-5, abs=1e-6 * (1 + abs(fd))), (name, ix)
