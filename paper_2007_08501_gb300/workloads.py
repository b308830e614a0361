"""Seeded synthetic inputs for the packed-mesh rasterizer.

This module generates DATA only: icosphere meshes, radial displacement, look-at
cameras, per-vertex colours and upstream gradients.  It holds none of the
rasterizer's or the blends' arithmetic, so both the CUDA path and the FP64 CPU
oracle can consume what it produces.

The paper benchmarks on ShapeNetCoreV1 meshes sampled as homogeneous
(one mesh repeated, sigma = 0) or heterogeneous (face counts drawn around a mean)
batches (Appendix A, "Sampling Batches for Benchmarks").  ShapeNet is not
available, so seeded icospheres stand in for it: repeated levels give the
homogeneous case, levels drawn from 3..7 give the heterogeneous one.

Packed layout (Section 3, "3D data structures": list / packed / padded):
  verts      (V, 3) float32   world-space positions of all meshes, concatenated
  faces      (F, 3) int64     global indices into ``verts``; mesh n owns the
                              contiguous face range [first_face[n], first_face[n] + num_faces[n])
  first_face (N,)   int64
  num_faces  (N,)   int64
  cams       (N, 16) float32  per image: R (3x3 row-major, world->view), C (camera
                              centre, 3), f = 1/tan(fov/2), znear, 0, 0
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CAM_STRIDE = 16


# --------------------------------------------------------------------------
# icosphere
# --------------------------------------------------------------------------
def _icosahedron():
    """The 12-vertex icosahedron on the unit sphere with 20 outward faces.

    Faces are found as the vertex triples that are pairwise at the minimum
    edge distance, sorted lexicographically, then oriented outward.
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    base = []
    for a in (-1.0, 1.0):
        for b in (-t, t):
            base.append((a, b, 0.0))
            base.append((0.0, a, b))
            base.append((b, 0.0, a))
    v = np.array(base, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    edge = np.min(d[d > 1e-9])
    adj = np.abs(d - edge) < 1e-9
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            if not adj[i, j]:
                continue
            for k in range(j + 1, 12):
                if adj[i, k] and adj[j, k]:
                    n = np.cross(v[j] - v[i], v[k] - v[i])
                    if np.dot(n, v[i] + v[j] + v[k]) < 0:
                        faces.append((i, k, j))
                    else:
                        faces.append((i, j, k))
    f = np.array(faces, dtype=np.int64)
    assert f.shape == (20, 3)
    return v, f


def icosphere(level: int):
    """Unit icosphere after ``level`` 4-way subdivisions.

    V = 10*4**level + 2, F = 20*4**level.  Level 3 gives 642 / 1,280,
    level 4 gives 2,562 / 5,120, level 8 gives 655,362 / 1,310,720.
    Vertex order: the previous level's vertices, then one new vertex per edge
    in order of the edge's first visit (faces in order, edges (a,b),(b,c),(c,a)).
    """
    v, f = _icosahedron()
    for _ in range(level):
        nv = v.shape[0]
        e = np.stack([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=1).reshape(-1, 2)
        key = np.sort(e, axis=1)
        key1 = key[:, 0] * (nv + 1) + key[:, 1]
        uniq, first, inv = np.unique(key1, return_index=True, return_inverse=True)
        # number unique edges by first visit
        order = np.argsort(first, kind="stable")
        rank = np.empty_like(order)
        rank[order] = np.arange(order.size)
        mid_id = nv + rank[inv].reshape(-1, 3)          # (F, 3): ids of mids of ab, bc, ca
        ue = key[first[order]]
        mids = v[ue[:, 0]] + v[ue[:, 1]]
        mids /= np.linalg.norm(mids, axis=1, keepdims=True)
        v = np.concatenate([v, mids], axis=0)
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        ab, bc, ca = mid_id[:, 0], mid_id[:, 1], mid_id[:, 2]
        f = np.stack(
            [np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
             np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)], axis=1
        ).reshape(-1, 3)
    return v, f


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------
def look_at_camera(dist: float, elev_deg: float, azim_deg: float, fov_deg: float = 60.0,
                   znear: float = 0.1):
    """One camera row (16 floats) looking at the origin from (dist, elev, azim).

    C = dist * (cos e sin a, sin e, cos e cos a); the rows of R are the view
    axes x = up x z, y = z x x, z = -C/|C| with up = +Y, so view +X points to
    the image's left, +Y up and +Z into the screen.
    """
    e = math.radians(elev_deg)
    a = math.radians(azim_deg)
    C = dist * np.array([math.cos(e) * math.sin(a), math.sin(e), math.cos(e) * math.cos(a)])
    z = -C / np.linalg.norm(C)
    x = np.cross(np.array([0.0, 1.0, 0.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], 0)
    row = np.zeros(CAM_STRIDE, dtype=np.float64)
    row[0:9] = R.reshape(-1)
    row[9:12] = C
    row[12] = 1.0 / math.tan(math.radians(fov_deg) / 2.0)
    row[13] = znear
    return row.astype(np.float32)


# --------------------------------------------------------------------------
# batches
# --------------------------------------------------------------------------
@dataclass
class MeshBatch:
    verts: np.ndarray        # (V,3) f32
    faces: np.ndarray        # (F,3) i64
    first_face: np.ndarray   # (N,) i64
    num_faces: np.ndarray    # (N,) i64
    cams: np.ndarray         # (N,16) f32
    colors: np.ndarray       # (V,3) f32
    levels: list = field(default_factory=list)

    @property
    def N(self):
        return int(self.first_face.shape[0])

    @property
    def V(self):
        return int(self.verts.shape[0])

    @property
    def F(self):
        return int(self.faces.shape[0])


_ICO_CACHE: dict = {}


def _ico(level):
    if level not in _ICO_CACHE:
        _ICO_CACHE[level] = icosphere(level)
    return _ICO_CACHE[level]


def displaced_sphere(level: int, sigma: float, rng: np.random.Generator):
    v, f = _ico(level)
    eps = rng.normal(0.0, sigma, size=(v.shape[0], 1)) if sigma > 0 else 0.0
    return (v * (1.0 + eps)), f


def random_camera(rng: np.random.Generator, dist=2.7, fov=60.0, znear=0.1,
                  elev_range=(-30.0, 30.0)):
    elev = rng.uniform(*elev_range)
    azim = rng.uniform(0.0, 360.0)
    return look_at_camera(dist, elev, azim, fov, znear)


def pack(meshes, cams, colors=None) -> MeshBatch:
    """Concatenate per-mesh (verts, faces) into the packed layout."""
    vs, fs, ff, nf = [], [], [], []
    voff = foff = 0
    for v, f in meshes:
        vs.append(v)
        fs.append(f + voff)
        ff.append(foff)
        nf.append(f.shape[0])
        voff += v.shape[0]
        foff += f.shape[0]
    verts = np.concatenate(vs, 0).astype(np.float32) if vs else np.zeros((0, 3), np.float32)
    faces = np.concatenate(fs, 0).astype(np.int64) if fs else np.zeros((0, 3), np.int64)
    if colors is None:
        colors = np.zeros_like(verts)
    return MeshBatch(verts, faces, np.array(ff, np.int64), np.array(nf, np.int64),
                     np.stack(cams, 0).astype(np.float32) if cams else np.zeros((0, 16), np.float32),
                     colors.astype(np.float32))


def first_images(b: MeshBatch, n: int) -> MeshBatch:
    """The first ``n`` images of a packed batch (all vertices kept)."""
    n = max(1, min(int(n), b.N))
    F = int(b.first_face[n - 1] + b.num_faces[n - 1])
    return MeshBatch(b.verts, b.faces[:F].copy(), b.first_face[:n].copy(), b.num_faces[:n].copy(),
                     b.cams[:n].copy(), b.colors, list(b.levels[:n]))


def sphere_batch(levels, sigma, seed_base, cam_seed=None, color_seed=None, cams=None):
    """One displaced icosphere per image; mesh i draws from seed ``seed_base + i``."""
    meshes, cam_rows = [], []
    for i, L in enumerate(levels):
        rng = np.random.default_rng(seed_base + i)
        meshes.append(displaced_sphere(L, sigma, rng))
        cam_rows.append(random_camera(rng) if cams is None else cams[i])
    b = pack(meshes, cam_rows)
    crng = np.random.default_rng(seed_base + 977 if color_seed is None else color_seed)
    b.colors = crng.uniform(0.0, 1.0, size=(b.V, 3)).astype(np.float32)
    b.levels = list(levels)
    return b


def upstream_grad(N, S, seed, channels=4):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0, size=(N, S, S, channels)).astype(np.float32)


# --------------------------------------------------------------------------
# the five benchmark workloads (restated as synthetic inputs)
# --------------------------------------------------------------------------
BLUR_SIGMA_1E4 = math.log(1.0 / 1e-4 - 1.0) * 1e-4   # sigma(-d/1e-4) = 1e-4 at d = blur


@dataclass
class Workload:
    name: str
    batch: MeshBatch
    image_size: int
    K: int
    blur_radius: float
    blend_mode: str          # "none" | "sil" | "rgb" (= silhouette alpha + softmax rgb)
    sigma: float = 1e-4
    gamma: float = 1e-4
    znear: float = 0.1
    zfar: float = 100.0
    perspective_correct: bool = True
    clip_barycentric_coords: bool = False
    bin_size: int = 16
    grad_seed: int = 0


def workload(index: int, variant: str = "") -> Workload:
    """Workload ``index`` (0..4) of the benchmark table; seeds are 1000*index + i."""
    seed = 1000 * index
    if index == 0:
        b = sphere_batch([3], 0.05, seed)
        return Workload("plain fwd: 1 icosphere (642 verts, 1280 faces), 64x64, K=1",
                        b, 64, 1, 0.0, "none", bin_size=0)
    if index == 1:
        b = sphere_batch([4] * 8, 0.05, seed)
        return Workload("8 icospheres level 4 (5120 faces), 256x256, K=8, soft sil + softmax rgb",
                        b, 256, 8, BLUR_SIGMA_1E4, "rgb", clip_barycentric_coords=True,
                        grad_seed=seed + 500)
    if index == 2:
        rng = np.random.default_rng(seed + 999)
        levels = [int(x) for x in rng.integers(3, 8, size=32)]
        b = sphere_batch(levels, 0.03, seed)
        return Workload("32 icospheres of level 3..7, 512x512, K=4, soft silhouette",
                        b, 512, 4, BLUR_SIGMA_1E4, "sil", clip_barycentric_coords=True,
                        grad_seed=seed + 500)
    if index == 3:
        b = sphere_batch([8], 0.02, seed)
        if variant == "hard":
            return Workload("1 icosphere level 8 (1.31M faces), 1024x1024, K=1 hard",
                            b, 1024, 1, 0.0, "sil", grad_seed=seed + 500)
        return Workload("1 icosphere level 8 (1.31M faces), 1024x1024, K=8 soft",
                        b, 1024, 8, BLUR_SIGMA_1E4, "sil", clip_barycentric_coords=True,
                        grad_seed=seed + 500)
    if index == 4:
        rng = np.random.default_rng(seed)
        v, f = displaced_sphere(6, 0.0, rng)
        cams = [look_at_camera(2.7, float(rng.uniform(-30, 30)), 360.0 * i / 20.0)
                for i in range(20)]
        b = pack([(v, f)], cams[:1])
        # 20 views of ONE mesh: faces of every image index the same packed verts
        F0 = f.shape[0]
        b.faces = np.tile(f.astype(np.int64), (20, 1))
        b.first_face = np.arange(20, dtype=np.int64) * F0
        b.num_faces = np.full(20, F0, np.int64)
        b.cams = np.stack(cams, 0).astype(np.float32)
        b.colors = np.zeros_like(b.verts)
        b.levels = [6] * 20
        return Workload("1 icosphere level 6 (81920 faces) x 20 views, 512x512, K=50, soft sil",
                        b, 512, 50, BLUR_SIGMA_1E4, "sil", clip_barycentric_coords=True,
                        grad_seed=seed + 500)
    raise ValueError(index)


def target_sphere(seed=4321, level=6, sigma=0.05):
    """The displaced sphere whose silhouettes are the analysis-by-synthesis target."""
    rng = np.random.default_rng(seed)
    return displaced_sphere(level, sigma, rng)


# --------------------------------------------------------------------------
# point clouds: points sampled uniformly from displaced sphere surfaces
# --------------------------------------------------------------------------
@dataclass
class PointBatch:
    points: np.ndarray       # (P,3) f32
    first_point: np.ndarray  # (N,) i64
    num_points: np.ndarray   # (N,) i64
    cams: np.ndarray         # (N,16) f32
    features: np.ndarray     # (P,D) f32

    @property
    def N(self):
        return int(self.first_point.shape[0])

    @property
    def P(self):
        return int(self.points.shape[0])


def sample_surface(verts, faces, n, rng):
    """``n`` points uniform over the surface: faces by area, then uniform barycentrics."""
    a, b, c = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    fi = rng.choice(faces.shape[0], size=n, p=area / area.sum())
    u, v = rng.random(n), rng.random(n)
    flip = u + v > 1.0
    u[flip], v[flip] = 1.0 - u[flip], 1.0 - v[flip]
    return a[fi] + u[:, None] * (b[fi] - a[fi]) + v[:, None] * (c[fi] - a[fi])


def point_batch(counts, seed_base, level=4, sigma=0.05, D=1, cams=None):
    """One cloud per image with ``counts[i]`` points; cloud i draws from seed ``seed_base + i``.
    Features are 1 (silhouette) for D == 1, else U[0,1]."""
    pts, cam_rows, feats = [], [], []
    for i, n in enumerate(counts):
        rng = np.random.default_rng(seed_base + i)
        v, f = displaced_sphere(level, sigma, rng)
        pts.append(sample_surface(v, f, int(n), rng))
        cam_rows.append(random_camera(rng) if cams is None else cams[i])
        feats.append(np.ones((int(n), 1)) if D == 1 else rng.uniform(0.0, 1.0, size=(int(n), D)))
    counts = np.asarray(counts, np.int64)
    first = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    return PointBatch(np.concatenate(pts, 0).astype(np.float32), first, counts,
                      np.stack(cam_rows, 0).astype(np.float32), np.concatenate(feats, 0).astype(np.float32))


POINT_RADIUS = 0.01   # NDC units: 1.28 pixels at 256 x 256


@dataclass
class PointWorkload:
    name: str
    batch: PointBatch
    image_size: int
    K: int
    radius: float
    mode: int                # 0: Alpha compositing, 1: Norm
    grad_seed: int = 0


def point_workload(mode: int = 0) -> PointWorkload:
    """The point renderer benchmark: 8 clouds x 200,000 points sampled from displaced
    level-4 spheres, 256 x 256, K = 50, silhouettes (D = 1)."""
    b = point_batch([200_000] * 8, 5000, level=4, sigma=0.05)
    return PointWorkload("8 clouds x 200,000 points, 256x256, K=50, silhouette, %s compositing"
                         % ("Alpha" if mode == 0 else "Norm"), b, 256, 50, POINT_RADIUS, mode, grad_seed=5500)


# --------------------------------------------------------------------------
# pixel sampling for oracle checks on large images
# --------------------------------------------------------------------------
def sample_pixels(N, S, per_image, seed):
    """Distinct (n, row, col) triples, ``per_image`` per image, sorted."""
    rng = np.random.default_rng(seed)
    out = []
    for n in range(N):
        m = min(per_image, S * S)
        idx = np.sort(rng.choice(S * S, size=m, replace=False))
        out.append(np.stack([np.full(m, n), idx // S, idx % S], 1))
    return np.concatenate(out, 0).astype(np.int64) if out else np.zeros((0, 3), np.int64)


# --------------------------------------------------------------------------
# nearest neighbours and Chamfer (Section 3.1; App. A: points sampled
# uniformly from a mesh surface, homogeneous or heterogeneous batch sizes)
# --------------------------------------------------------------------------
@dataclass
class CloudPairs:
    p: np.ndarray        # (P1, 3) f32 query clouds, packed
    first1: np.ndarray   # (N,) i64
    len1: np.ndarray     # (N,) i64
    q: np.ndarray        # (P2, 3) f32 candidate clouds, packed
    first2: np.ndarray
    len2: np.ndarray

    @property
    def N(self):
        return int(self.first1.shape[0])


def _packed_surface_samples(counts, seed_base, level, sigma):
    pts = []
    for i, n in enumerate(counts):
        rng = np.random.default_rng(seed_base + i)
        v, f = displaced_sphere(level, sigma, rng)
        pts.append(sample_surface(v, f, int(n), rng))
    counts = np.asarray(counts, np.int64)
    first = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64) if len(counts) else counts
    return (np.concatenate(pts, 0) if pts else np.zeros((0, 3))).astype(np.float32), first, counts


def cloud_pairs(len1, len2, seed_base, level=4, sigma=0.05):
    """Pair i: |P_i| = len1[i] and |Q_i| = len2[i] points sampled from two
    displaced spheres (seeds seed_base + i and seed_base + 50000 + i)."""
    p, f1, l1 = _packed_surface_samples(len1, seed_base, level, sigma)
    q, f2, l2 = _packed_surface_samples(len2, seed_base + 50000, level, sigma)
    return CloudPairs(p, f1, l1, q, f2, l2)


@dataclass
class KnnWorkload:
    name: str
    pairs: CloudPairs
    K: int
    chamfer: bool        # Chamfer loss forward + backward instead of KNN forward
    grad_seed: int = 0


def knn_workload(kind: str) -> KnnWorkload:
    """The operator benchmarks of Section 3.1 (batch size 32):
    'knn'      |P| = |Q| = 50,000 per cloud, K = 8, forward;
    'knn_het'  |P|, |Q| uniform in [10,000, 90,000] (mean 50,000), K = 8, forward;
    'chamfer'  |P| = 1,000, |Q| = 50,000, Chamfer loss forward + backward."""
    B = 32
    if kind == "knn":
        return KnnWorkload("32 pairs of clouds, |P| = |Q| = 50,000, K = 8", cloud_pairs([50_000] * B, [50_000] * B,
                                                                                        7000), 8, False)
    if kind == "knn_het":
        rng = np.random.default_rng(7100)
        l1 = rng.integers(10_000, 90_001, size=B)
        l2 = rng.integers(10_000, 90_001, size=B)
        return KnnWorkload("32 pairs of clouds, |P|, |Q| uniform in [10k, 90k], K = 8", cloud_pairs(l1, l2, 7200),
                           8, False)
    if kind == "chamfer":
        return KnnWorkload("32 pairs of clouds, |P| = 1,000, |Q| = 50,000, Chamfer fwd+bwd",
                           cloud_pairs([1_000] * B, [50_000] * B, 7400), 1, True, grad_seed=7500)
    raise ValueError(kind)


def pairs_per_batch(pairs: CloudPairs, both_ways=False):
    """Candidate distances one KNN pass evaluates: sum_i |P_i| |Q_i| (twice for Chamfer)."""
    n = int(np.sum(pairs.len1.astype(np.int64) * pairs.len2.astype(np.int64)))
    return 2 * n if both_ways else n
