"""The synthetic input recipe (stand-ins for the paper's ShapeNet samples,
Appendix A): icosphere counts and geometry, displacement, cameras, the packed
layout, seeding, and the shapes of the benchmark batches."""
import math

import numpy as np
import pytest

from paper_2007_08501_gb300 import workloads as wl


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_icosphere_counts_closed_outward_surface(level):
    v, f = wl.icosphere(level)
    assert v.shape == (10 * 4 ** level + 2, 3) and f.shape == (20 * 4 ** level, 3)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-12)
    # closed 2-manifold: every undirected edge in exactly two faces, once each way
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], 0)
    directed = {tuple(x) for x in e.tolist()}
    assert len(directed) == e.shape[0]
    assert all((b, a) in directed for a, b in directed)
    # consistent outward winding: the face normal points away from the centre
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    assert (np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) > 0).all()
    # the previous level's vertices come first
    if level > 0:
        pv, _ = wl.icosphere(level - 1)
        np.testing.assert_array_equal(v[:pv.shape[0]], pv)


def test_displacement_is_radial():
    rng = np.random.default_rng(0)
    v, f = wl.displaced_sphere(3, 0.05, rng)
    u, _ = wl.icosphere(3)
    r = np.linalg.norm(v, axis=1)
    np.testing.assert_allclose(v / r[:, None], u, atol=1e-12)
    assert 0.02 < np.std(r) < 0.08


def test_look_at_camera_axes_and_centre():
    row = wl.look_at_camera(2.7, 20.0, 75.0, 60.0, 0.1).astype(np.float64)
    R, C = row[:9].reshape(3, 3), row[9:12]
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-6)
    assert np.linalg.norm(C) == pytest.approx(2.7, rel=1e-6)
    # the origin lies straight ahead at depth |C|; world up projects to view +y
    np.testing.assert_allclose(R @ (np.zeros(3) - C), [0, 0, 2.7], atol=1e-5)
    assert (R @ np.array([0.0, 1.0, 0.0]))[1] > 0
    assert row[12] == pytest.approx(1 / math.tan(math.radians(30.0)), rel=1e-6) and row[13] == pytest.approx(0.1)


def test_packed_layout_and_seeding():
    b = wl.sphere_batch([1, 0, 2], 0.05, seed_base=7)
    assert b.first_face.tolist() == [0, 80, 100] and b.num_faces.tolist() == [80, 20, 320]
    assert b.verts.shape == (42 + 12 + 162, 3) and b.cams.shape == (3, 16)
    # faces index their own mesh's vertices in the packed array
    assert b.faces[:80].max() < 42 and 42 <= b.faces[80:100].min() and b.faces[80:100].max() < 54
    assert (b.colors >= 0).all() and (b.colors <= 1).all()
    again = wl.sphere_batch([1, 0, 2], 0.05, seed_base=7)
    for x, y in ((b.verts, again.verts), (b.cams, again.cams), (b.colors, again.colors)):
        np.testing.assert_array_equal(x, y)


def test_benchmark_mesh_batch_shapes():
    w = wl.workload(1)
    b = w.batch
    assert (b.N, w.image_size, w.K) == (8, 256, 8)
    assert b.faces.shape[0] == 8 * 5120 and b.verts.shape[0] == 8 * 2562
    assert w.blur_radius == pytest.approx(math.log(1 / 1e-4 - 1) * 1e-4)
    assert wl.upstream_grad(b.N, 8, 3).shape == (8, 8, 8, 4)


def test_nearest_neighbour_batches():
    w = wl.knn_workload("knn_het")
    c = w.pairs
    assert c.N == 32 and w.K == 8
    assert (c.len1 >= 10_000).all() and (c.len1 <= 90_000).all() and (c.len2 >= 10_000).all()
    assert c.p.shape == (int(c.len1.sum()), 3) and c.q.shape == (int(c.len2.sum()), 3)
    np.testing.assert_array_equal(c.first1[1:], np.cumsum(c.len1)[:-1])
    # points lie on the displaced spheres' surfaces
    r = np.linalg.norm(c.q[:50_000], axis=1)
    assert 0.6 < r.min() and r.max() < 1.4
    ch = wl.knn_workload("chamfer")
    assert ch.chamfer and (ch.pairs.len1 == 1000).all() and (ch.pairs.len2 == 50_000).all()
    assert wl.pairs_per_batch(ch.pairs, both_ways=True) == 2 * 32 * 1000 * 50_000


def test_sampled_pixels_are_distinct_and_sorted():
    px = wl.sample_pixels(3, 16, 40, 5)
    assert px.shape == (120, 3)
    flat = (px[:, 0] * 16 + px[:, 1]) * 16 + px[:, 2]
    assert np.unique(flat).size == 120 and (np.diff(flat) > 0).all()
