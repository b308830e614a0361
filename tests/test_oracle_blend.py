"""Pins for the oracle's blends (Algorithm 1, silhouette; Algorithm 2, softmax).

Closed-form special cases and limits: one face, no face, equal faces, far
separated depths, the logistic function at the blur radius, and slot
permutation invariance.
"""
import math

import numpy as np
import pytest
from scipy.special import expit

import oracle
from paper_2007_08501_gb300.workloads import BLUR_SIGMA_1E4

SIG, GAM, ZN, ZF = 1e-4, 1e-4, 0.1, 100.0


def _frag(K, slots):
    """slots: list of (face, z, bary(3), dist)"""
    p2f = -np.ones((1, K), np.int64)
    zb = -np.ones((1, K))
    ba = -np.ones((1, K, 3))
    di = -np.ones((1, K))
    for k, (f, z, b, d) in enumerate(slots):
        p2f[0, k] = f
        zb[0, k] = z
        ba[0, k] = b
        di[0, k] = d
    return p2f, zb, ba, di


FACES = np.array([[0, 1, 2], [3, 4, 5], [0, 3, 5]], np.int64)
COLORS = np.random.default_rng(0).uniform(0, 1, size=(6, 3))


def test_no_valid_face_gives_background_and_zero_alpha():
    p2f, zb, ba, di = _frag(4, [])
    out = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, GAM, ZN, ZF, bg=(0.2, 0.4, 0.6))
    np.testing.assert_array_equal(out[0], [0.2, 0.4, 0.6, 0.0])


@pytest.mark.parametrize("d", [-3e-4, -1e-5, 0.0, 2e-4, BLUR_SIGMA_1E4])
def test_single_face_alpha_is_logistic(d):
    p2f, zb, ba, di = _frag(1, [(1, 2.0, (0.2, 0.3, 0.5), d)])
    out = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, GAM, ZN, ZF, mode=0)
    assert abs(out[0, 3] - expit(-d / SIG)) < 1e-15
    assert out[0, 0] == out[0, 1] == out[0, 2] == 0.0


def test_alpha_at_blur_radius_is_1e4():
    # blur_radius = ln(1/1e-4 - 1) * 1e-4 is where sigmoid(-d / 1e-4) = 1e-4
    p2f, zb, ba, di = _frag(1, [(0, 2.0, (1, 0, 0), BLUR_SIGMA_1E4)])
    out = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, GAM, ZN, ZF, mode=0)
    assert abs(out[0, 3] - 1e-4) < 1e-15


def test_single_face_in_front_shows_interpolated_colour():
    # zinv = (100 - 2)/99.9 ~ 0.98, so the background weight exp((1e-10 - zinv)/1e-4) underflows
    b = np.array([0.2, 0.3, 0.5])
    p2f, zb, ba, di = _frag(3, [(1, 2.0, b, -1e-5)])
    out = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, GAM, ZN, ZF)
    np.testing.assert_allclose(out[0, :3], b @ COLORS[FACES[1]], rtol=1e-14)


def test_single_face_with_wide_gamma_blends_with_background():
    g = 1e3
    b = np.array([0.6, 0.3, 0.1])
    z, d = 5.0, 1e-5
    p2f, zb, ba, di = _frag(2, [(2, z, b, d)])
    bg = np.array([0.9, 0.1, 0.3])
    out = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, g, ZN, ZF, bg=bg)
    # one face: a two-way mix of the face colour (weight prob) and the background
    # (weight exp((eps - zinv)/gamma))
    prob = expit(-d / SIG)
    zinv = (ZF - z) / (ZF - ZN)
    wb = math.exp((1e-10 - zinv) / g)
    c = b @ COLORS[FACES[2]]
    np.testing.assert_allclose(out[0, :3], (prob * c + wb * bg) / (prob + wb), rtol=1e-13)


def test_equal_faces_average_and_alpha_power():
    K = 4
    d = -2e-5
    b1, b2 = np.array([1.0, 0, 0]), np.array([0, 0, 1.0])
    p2f, zb, ba, di = _frag(K, [(0, 2.0, b1, d), (1, 2.0, b2, d)])
    out = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, GAM, ZN, ZF)
    np.testing.assert_allclose(out[0, :3], 0.5 * (COLORS[0] + COLORS[5]), rtol=1e-14)
    p = expit(-d / SIG)
    assert abs(out[0, 3] - (1 - (1 - p) ** 2)) < 1e-15
    p2f, zb, ba, di = _frag(K, [(0, 2.0, b1, d)] * K)
    out = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, GAM, ZN, ZF, mode=0)
    assert abs(out[0, 3] - (1 - (1 - p) ** K)) < 1e-15


def test_depth_separated_faces_weight_ratio():
    # weights ratio between two faces = (p2/p1) exp(-(z2-z1)/((zfar-znear) gamma))
    g = 2e-3
    z1, z2 = 2.0, 2.1
    d1, d2 = -1e-4, 5e-5
    b1, b2 = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    p2f, zb, ba, di = _frag(2, [(0, z1, b1, d1), (1, z2, b2, d2)])
    out = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, g, ZN, ZF)
    r = expit(-d2 / SIG) / expit(-d1 / SIG) * math.exp(-(z2 - z1) / ((ZF - ZN) * g))
    want = (COLORS[0] + r * COLORS[4]) / (1 + r)
    np.testing.assert_allclose(out[0, :3], want, rtol=1e-12)
    # with gamma 1e-4 and a depth gap of 1 (exponent -100) the nearer face takes everything
    zb[0, 1] = z1 + 1.0
    out = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, GAM, ZN, ZF)
    np.testing.assert_allclose(out[0, :3], COLORS[0], rtol=1e-12)


def test_slot_permutation_and_invalid_slot_contents_do_not_matter():
    rng = np.random.default_rng(3)
    K = 5
    slots = [(int(rng.integers(0, 3)), float(rng.uniform(1.9, 2.1)), rng.dirichlet([1, 1, 1]),
              float(rng.uniform(-3e-4, 3e-4))) for _ in range(3)]
    p2f, zb, ba, di = _frag(K, slots)
    g = 5e-3
    a = oracle.blend_fwd(p2f, zb, ba, di, FACES, COLORS, SIG, g, ZN, ZF)
    perm = [2, 0, 4, 1, 3]
    zb2, ba2, di2 = zb.copy(), ba.copy(), di.copy()
    zb2[0, 3:] = 7.0
    di2[0, 3:] = -1.0
    b = oracle.blend_fwd(p2f[:, perm], zb2[:, perm], ba2[:, perm], di2[:, perm], FACES, COLORS, SIG, g,
                         ZN, ZF)
    np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-15)
