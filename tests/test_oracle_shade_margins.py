"""Pins of the shading oracle's kink margin (``ors_shade_margins``): the
distance, in the reflection model's own terms, of a pixel's shading from the
places where a term switches on or off (the diffuse and specular terms at
c = m.l = 0, the specular term at s = r.v = 0 while c > 0).  The GPU shading
tests drop the upstream gradient where it is small.

Light and eye are placed by angle in the plane of incidence of a face that
faces the camera (normal (0, 0, -1)): a light at angle t_l from the normal
gives c = cos(t_l); its mirror direction lies at -t_l, so an eye at angle
t_e on the light's side gives s = cos(t_l + t_e).  The expected margins
follow from those angles, not from the model's formulas.
"""
import numpy as np
import pytest

from oracle import shading as sh

# one triangle in the plane z = 2, its winding giving the face normal (0, 0, -1)
VERTS = np.array([[-0.5, -0.5, 2.0], [0.5, -0.5, 2.0], [0.0, 0.5, 2.0]])
FACES = np.array([[0, 2, 1]])
NORMALS = np.tile([0.0, 0.0, -1.0], (3, 1))
CENTROID = VERTS.mean(0)
THIRD = [1 / 3, 1 / 3, 1 / 3]


def _dir(t):
    """Unit vector at angle t (radians) from the face normal (0, 0, -1), in the x-z plane."""
    return np.array([np.sin(t), 0.0, -np.cos(t)])


def _cam(centre):
    row = np.zeros(16)
    row[0] = row[4] = row[8] = 1.0
    row[9:12] = centre
    row[12] = 1.0
    row[13] = 0.1
    return row[None]


def _margin(t_l, t_e, shading, faces=FACES, verts=VERTS, normals=NORMALS, p2f=((0,),), bary=(THIRD,),
            blend=sh.SOFTMAX, at=CENTROID):
    light = sh.light_params(at + 3.0 * _dir(t_l))
    cams = _cam(at + 1.5 * _dir(t_e))
    p2f = np.asarray(p2f, np.int64)
    bary = np.asarray(bary, float).reshape(1, p2f.shape[1], 3)
    return float(sh.shade_margins(np.zeros(1, np.int64), p2f, bary, faces, verts, normals, cams, light, shading,
                                  blend)[0])


@pytest.mark.parametrize("shading", [sh.FLAT, sh.PHONG])
def test_specular_switch_within_1e_7(shading):
    # t_l = 40 deg, eye 90 deg - 1e-7 rad from the mirror direction: s = sin(1e-7)
    t_l = np.radians(40.0)
    m = _margin(t_l, np.pi / 2 - t_l - 1e-7, shading)
    assert m == pytest.approx(1e-7, rel=1e-6)


@pytest.mark.parametrize("shading", [sh.FLAT, sh.PHONG])
def test_away_from_both_switches(shading):
    # c = cos 40 deg = 0.766, s = cos 60 deg = 0.5
    m = _margin(np.radians(40.0), np.radians(20.0), shading)
    assert m == pytest.approx(0.5, rel=1e-12)


@pytest.mark.parametrize("shading", [sh.FLAT, sh.PHONG])
def test_grazing_light(shading):
    # c = cos(90 deg - 1e-7) = 1e-7; s = cos(120 deg) = -0.5
    m = _margin(np.pi / 2 - 1e-7, np.radians(30.0), shading)
    assert m == pytest.approx(1e-7, rel=1e-6)


def test_light_behind_ignores_the_specular_switch():
    # c = -0.3 (light behind the face): the specular term is off, so s = 0
    # (eye at 90 deg from the mirror direction) is no kink; the margin is |c|
    t_l = np.arccos(-0.3)
    m = _margin(t_l, np.pi / 2 - t_l, sh.PHONG)
    assert m == pytest.approx(0.3, rel=1e-12)


def test_hard_blend_reads_the_first_slot_only():
    # slot 1 holds a second face whose normals are perpendicular to the light
    # (c = 0: a kink); the hard blend shows slot 0 only
    light_at = CENTROID + 3.0 * _dir(np.radians(40.0))
    v2 = VERTS + np.array([0.0, 0.0, 1.0])
    n2 = np.cross(light_at - v2.mean(0), [0.0, 1.0, 0.0])
    n2 /= np.linalg.norm(n2)
    verts = np.concatenate([VERTS, v2])
    normals = np.concatenate([NORMALS, np.tile(n2, (3, 1))])
    faces = np.array([[0, 2, 1], [3, 5, 4]])
    kw = dict(faces=faces, verts=verts, normals=normals, p2f=((0, 1),), bary=(THIRD, THIRD))
    assert _margin(np.radians(40.0), np.radians(20.0), sh.PHONG, blend=sh.HARD, **kw) == pytest.approx(0.5)
    assert _margin(np.radians(40.0), np.radians(20.0), sh.PHONG, blend=sh.SOFTMAX, **kw) < 1e-12


def test_gouraud_takes_the_corners():
    # corner 0's normal is perpendicular to the light seen from corner 0
    # (c = 0 there); at the centroid the interpolated normal is far from that
    t_l = np.radians(40.0)
    light_at = CENTROID + 3.0 * _dir(t_l)
    n0 = np.cross(light_at - VERTS[0], [0.0, 1.0, 0.0])
    n0 /= np.linalg.norm(n0)
    normals = NORMALS.copy()
    normals[0] = n0 if np.dot(n0, [0, 0, -1]) > 0 else -n0
    assert _margin(t_l, np.radians(-20.0), sh.GOURAUD, normals=normals) < 1e-12
    assert _margin(t_l, np.radians(-20.0), sh.PHONG, normals=normals) > 0.5
