"""Pins of the oracle's margin flags (``orc_margins``): the mask that the GPU
parity tests use to exclude pixels whose face selection (or gradient) is
decided by rounding.

Each flag is checked on hand-placed geometry, seen through the identity
camera (NDC = (x/z, y/z), depth z), at one pixel centre: a case just inside
the flag's margin must raise exactly that flag, and a case just outside must
not.  The "outside" distances are chosen so that the plausible mistakes (a
squared distance compared with a Euclidean margin, an absolute instead of a
relative area margin, only the first depth pair compared, the inside of a
face counted as near its blur boundary, a shared corner counted as an edge
tie, the clip kink flagged without clipping, the extrapolated depth weighed
without its barycentrics) turn a "not flagged" case into a flagged one, or
the reverse.  Margins are the ones the parity tests use: eps = 1e-6.
"""
import numpy as np
import pytest

import oracle
from _scenes import ndc_triangle, pixel_centre, scene

S = 16
R0 = C0 = 7
PX = pixel_centre(C0, S)          # x of the test pixel centre (1/16)
PY = pixel_centre(R0, S)          # y of the test pixel centre (1/16)
EPS = 1e-6


def _flags(tris, K=1, blur=0.0, persp=True, clip=False, depths=None):
    """Margin flags at pixel (0, R0, C0) of a one-image scene.  ``tris`` holds
    NDC corner triples relative to the pixel centre; ``depths`` their depths."""
    world = []
    for i, t in enumerate(tris):
        z = 2.0 if depths is None else depths[i]
        world.append(ndc_triangle(*[(PX + p[0], PY + p[1]) for p in t], z))
    sc = scene(world)
    m = oracle.Mesh(sc["verts"], sc["faces"], sc["first_face"], sc["num_faces"], sc["cams"])
    px = np.array([[0, R0, C0]], np.int64)
    return int(oracle.margins(m, S, K, blur, persp, clip, pixels=px, eps=EPS)[0])


def _edge_at(dx):
    """A large triangle whose left edge is the vertical line x = dx (relative
    to the pixel), the triangle lying at x >= dx: the pixel is outside by dx
    for dx > 0, inside by |dx| for dx < 0."""
    return ((dx, -0.3), (dx, 0.3), (dx + 0.3, 0.0))


# --------------------------------------------------------------------------
# flag 1: blur == 0, a face boundary within eps of the pixel centre
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dx", [1e-7, -1e-7, 5e-7])
def test_flag1_edge_within_eps(dx):
    assert _flags([_edge_at(dx)]) == 1


def test_flag1_vertex_within_eps():
    # nearest point is a corner, 7e-7 away diagonally
    d = 5e-7
    assert _flags([((d, d), (d + 0.3, d), (d, d + 0.3))]) == 1


@pytest.mark.parametrize("dx", [5e-4, -5e-4])
def test_flag1_not_raised_at_5e_4(dx):
    # 5e-4 is far outside the margin; its square (2.5e-7) is inside it
    assert _flags([_edge_at(dx)]) == 0


def test_flag1_only_without_blur():
    assert _flags([_edge_at(1e-7)], blur=1e-4) == 0


# --------------------------------------------------------------------------
# flag 2: blur > 0, the pixel outside a face within eps of its blur boundary
# --------------------------------------------------------------------------
BLUR = 9.21e-4
RB = np.sqrt(BLUR)


@pytest.mark.parametrize("off", [5e-7, -5e-7])
def test_flag2_blur_boundary_within_eps(off):
    assert _flags([_edge_at(RB + off)], blur=BLUR) == 2


def test_flag2_not_raised_1e_5_from_the_boundary():
    # |dist - sqrt(blur)| = 1e-5 > eps, while |dist^2 - blur| = 6e-7 < eps
    assert _flags([_edge_at(RB + 1e-5)], blur=BLUR) == 0


def test_flag2_not_raised_inside_the_face():
    # inside, sqrt(blur) away from the nearest edge: the blur boundary is an
    # outside-only notion
    assert _flags([_edge_at(-RB)], blur=BLUR) == 0


# --------------------------------------------------------------------------
# flag 4: |A| within eps (relative) of the 1e-12 cull threshold
# --------------------------------------------------------------------------
def _small(area):
    a = np.sqrt(area)
    # far from the pixel; double area a*a
    return ((0.3, 0.3), (0.3 + a, 0.3), (0.3, 0.3 + a))


@pytest.mark.parametrize("rel", [5e-7, -5e-7])
def test_flag4_area_near_cull_threshold(rel):
    assert _flags([_small(1e-12 * (1 + rel))]) == 4


def test_flag4_relative_not_absolute():
    assert _flags([_small(5e-12)]) == 0
    assert _flags([_small(1e-12 * (1 + 5e-6))]) == 0


# --------------------------------------------------------------------------
# flag 8: two of the first K+1 candidates within eps in depth
# --------------------------------------------------------------------------
BIG = ((-0.3, -0.2), (0.35, -0.25), (0.05, 0.3))   # no edge tie at the pixel


def test_flag8_depth_tie_first_pair():
    assert _flags([BIG, BIG], K=1, depths=[2.0, 2.0 + 5e-7]) == 8
    assert _flags([BIG, BIG], K=1, depths=[2.0, 2.0 + 2e-6]) == 0


def test_flag8_depth_tie_within_the_first_k_plus_one():
    # tie between the 2nd and 3rd candidates: inside the first K+1 for K = 2
    # (the pair decides slot 2), beyond it for K = 1
    d = [1.0, 2.0, 2.0 + 5e-7]
    assert _flags([BIG] * 3, K=2, depths=d) == 8
    assert _flags([BIG] * 3, K=1, depths=d) == 0


# --------------------------------------------------------------------------
# flag 16: a corner (or a candidate's depth) within eps of znear (0.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dz", [5e-7, -5e-7])
def test_flag16_corner_near_znear(dz):
    far = ((0.3, 0.3), (0.4, 0.3), (0.3, 0.4))
    assert _flags([far], depths=[(0.1 + dz, 1.0, 1.0)]) == 16


def test_flag16_not_raised_1e_3_from_znear():
    far = ((0.3, 0.3), (0.4, 0.3), (0.3, 0.4))
    assert _flags([far], depths=[(0.1 + 1e-3, 1.0, 1.0)]) == 0


# --------------------------------------------------------------------------
# flag 32: two nearest edge segments tied in distance, reaching different points
# --------------------------------------------------------------------------
# isosceles triangle, apex above the pixel: on the symmetry axis the two
# slanted edges are equally near (0.134), the base is 0.7 away
ISO = ((-0.5, -0.7), (0.5, -0.7), (0.0, 0.3))


def test_flag32_symmetric_edge_tie():
    assert _flags([ISO]) == 32


def test_flag32_not_raised_off_the_axis():
    t = tuple((x + 1e-3, y) for x, y in ISO)
    assert _flags([t]) == 0


def test_flag32_shared_corner_is_not_a_tie():
    # the pixel 0.05 above the apex (a blur candidate): both slanted edges
    # reach the apex itself, so the tie does not change the gradient
    t = tuple((x, y - 0.35) for x, y in ISO)
    assert _flags([t], blur=0.01) == 0


# --------------------------------------------------------------------------
# flag 64: with clipping, a perspective-corrected barycentric within eps of 0
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dx", [1e-7, -1e-7])
def test_flag64_clip_kink(dx):
    # barycentric of the far corner = dx / 0.3
    assert _flags([_edge_at(dx)], blur=1e-4, clip=True) == 64


def test_flag64_not_raised_away_from_the_kink():
    assert _flags([_edge_at(1e-3)], blur=1e-4, clip=True) == 0


def test_flag64_only_with_clipping():
    assert _flags([_edge_at(1e-7)], blur=1e-4, clip=False) == 0


# --------------------------------------------------------------------------
# flag 128: unclipped extrapolation outside the face, ill-conditioned for fp32
# --------------------------------------------------------------------------
# The pixel lies 0.1 of the height beyond the apex v2 of a small triangle
# (screen barycentrics (-0.05, -0.05, 1.1)).
TIP = ((-0.01, -0.022), (0.01, -0.022), (0.0, -0.002))


def test_flag128_near_cancelling_perspective_extrapolation():
    # depths (1, 1, 10): sum b_i / z_i = -0.1 + 0.11 = 0.01 nearly cancels
    # (condition 21, extrapolated depth 100)
    assert _flags([TIP], blur=1e-5, depths=[(1.0, 1.0, 10.0)]) == 128


def test_flag128_not_raised_for_a_benign_extrapolation():
    # constant depth: condition 1.2, depth 1
    assert _flags([TIP], blur=1e-5, depths=[(1.0, 1.0, 1.0)]) == 0


def test_flag128_never_with_clipping():
    assert _flags([TIP], blur=1e-5, clip=True, depths=[(1.0, 1.0, 10.0)]) == 0


def test_flag128_weighs_the_extrapolated_barycentrics():
    # affine barycentrics (-10, 5.5, 5.5) at a constant depth of 0.2: the
    # depth is small (condition 21 x 0.2 = 4.2), the barycentrics are not
    # (21 x 10 = 210): an fp32 evaluation misses them by ~3e-5
    h = 1e-3
    tri = ((0.0, -10 * h - h), (-1e-3, -10 * h), (1e-3, -10 * h))
    assert _flags([tri], blur=2e-4, persp=False, depths=[0.2]) == 128


# --------------------------------------------------------------------------
# the flag groups the parity tests use
# --------------------------------------------------------------------------
def test_flag_groups():
    assert oracle.FWD_AMBIGUOUS == 1 | 2 | 4 | 8 | 16 | 128
    assert oracle.GRAD_COND_AMBIGUOUS & (2 | 8) == 0
    assert oracle.GRAD_COND_AMBIGUOUS & (32 | 64 | 1 | 16) == 32 | 64 | 1 | 16
