"""Tiny hand-built scenes for the oracle pins and the GPU parity tests.

The "identity camera" (R = I, C = 0, f = 1) maps a world point (x, y, z) to
NDC (x/z, y/z) with depth z, so a triangle can be placed at exact NDC
positions by scaling its x, y by the wanted depth.
"""
import numpy as np

from paper_2007_08501_gb300 import workloads


def identity_cam(f=1.0, znear=0.1):
    c = np.zeros(16, np.float64)
    c[0] = c[4] = c[8] = 1.0
    c[12] = f
    c[13] = znear
    return c


def ndc_triangle(p0, p1, p2, z):
    """World vertices whose identity-camera NDC corners are p0, p1, p2 at depth z
    (z may be a scalar or a per-vertex triple)."""
    zs = np.broadcast_to(np.asarray(z, np.float64), (3,))
    return np.array([[p[0] * zz, p[1] * zz, zz] for p, zz in zip((p0, p1, p2), zs)], np.float64)


def scene(tris, cams=None, mesh_of=None):
    """Pack a list of (3,3) world triangles (unshared vertices) into one batch.
    ``mesh_of[i]`` gives the image of triangle i (default: all in image 0);
    triangles must be grouped by image."""
    tris = [np.asarray(t, np.float64) for t in tris]
    if mesh_of is None:
        mesh_of = [0] * len(tris)
    N = (max(mesh_of) + 1) if mesh_of else 1
    verts = np.concatenate(tris, 0) if tris else np.zeros((0, 3))
    faces = np.arange(3 * len(tris), dtype=np.int64).reshape(-1, 3)
    first = np.zeros(N, np.int64)
    num = np.zeros(N, np.int64)
    for n in range(N):
        idx = [i for i, m in enumerate(mesh_of) if m == n]
        first[n] = idx[0] if idx else (first[n - 1] + num[n - 1] if n else 0)
        num[n] = len(idx)
    if cams is None:
        cams = [identity_cam()] * N
    return dict(verts=verts, faces=faces, first_face=first, num_faces=num,
                cams=np.stack(cams, 0))


def random_small_mesh(seed, ntri=3, level=None):
    """A few random triangles (or a coarse displaced icosphere) seen by a
    look-at camera; vertices drawn in FP64."""
    rng = np.random.default_rng(seed)
    if level is not None:
        v, f = workloads.displaced_sphere(level, 0.05, rng)
    else:
        # well-shaped triangles: near-equilateral, random plane orientation
        tris = []
        for _ in range(ntri):
            c = rng.uniform(-0.3, 0.3, size=3)
            q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
            r = rng.uniform(0.3, 0.6)
            phi = rng.uniform(0, 2 * np.pi)
            th = phi + 2 * np.pi * np.arange(3) / 3 + rng.uniform(-0.4, 0.4, size=3)
            tris.append(c + r * (np.cos(th)[:, None] * q[0] + np.sin(th)[:, None] * q[1]))
        v = np.concatenate(tris, 0)
        f = np.arange(3 * ntri, dtype=np.int64).reshape(-1, 3)
    cam = workloads.look_at_camera(2.7, rng.uniform(-30, 30), rng.uniform(0, 360)).astype(np.float64)
    return dict(verts=v.astype(np.float64), faces=f.astype(np.int64),
                first_face=np.array([0], np.int64), num_faces=np.array([f.shape[0]], np.int64),
                cams=cam[None, :])


def pixel_centre(i, S):
    return 1.0 - (2.0 * i + 1.0) / S
