"""``torch.autograd.Function`` wrappers over the C ABI.

``rasterize_meshes`` returns Fragment data (Section 3.2 "Rasterizer") and
differentiates to the packed vertices through ``rast_mesh_bwd``, which
recomputes barycentrics, depth and distance from ``pix_to_face`` instead of
keeping them for the backward pass.  ``blend`` applies Algorithm 1
(silhouette) or Algorithms 1 + 2 (softmax rgb + silhouette alpha) and
differentiates through ``blend_bwd``.  ``render_meshes`` does both in one
Function: its forward is ``rast_blend_fwd`` (the fine pass blends as it
writes the fragments) and its backward ``blend_rast_bwd`` (the blend adjoint
goes straight into the rasterizer adjoint without materialising fragment
gradients).  ``knn_points`` and ``chamfer_distance`` (Section 3.1, Eq. 1)
wrap the exact nearest-neighbour search on packed point-cloud batches.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import ops


@dataclass
class RasterSettings:
    image_size: int
    faces_per_pixel: int = 1
    blur_radius: float = 0.0
    bin_size: int = 16               # 0: plain per-image form
    max_faces_per_bin: int = 4096
    max_bin_entries: int = 0
    perspective_correct: bool = True
    clip_barycentric_coords: bool = False

    def params(self, N):
        return ops.make_rast_params(N, self.image_size, self.faces_per_pixel, self.blur_radius, self.bin_size,
                                    self.max_faces_per_bin, self.perspective_correct,
                                    self.clip_barycentric_coords, self.max_bin_entries)


@dataclass
class BlendSettings:
    sigma: float = 1e-4
    gamma: float = 1e-4
    znear: float = 0.1
    zfar: float = 100.0
    background: tuple = (1.0, 1.0, 1.0)
    eps: float = 1e-10
    rgb: bool = True

    def params(self):
        return ops.make_blend_params(self.sigma, self.gamma, self.znear, self.zfar, self.background, self.eps,
                                     ops.BLEND_RGB if self.rgb else ops.BLEND_SIL)


class Workspace:
    """Device workspace reused across calls; grows when a call needs more."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = None

    def get(self, p, V, F):
        n = ops.rast_workspace_bytes(p, V, F)
        if self.buf is None or self.buf.numel() < n:
            self.buf = torch.empty(n, dtype=torch.uint8, device=self.device)
        return self.buf

    def status(self):
        return 0 if self.buf is None else ops.rast_query_status(self.buf)


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, verts, faces, first_face, num_faces, cams, settings, ws):
        N = first_face.shape[0]
        S, K = settings.image_size, settings.faces_per_pixel
        p = settings.params(N)
        buf = ws.get(p, verts.shape[0], faces.shape[0])
        p2f, zbuf, bary, dists = ops.alloc_fragments(N, S, K, verts.device)
        ops.rast_mesh_fwd(p, verts, faces, first_face, num_faces, cams, p2f, zbuf, bary, dists, buf)
        ctx.save_for_backward(verts, faces, first_face, num_faces, cams, p2f)
        ctx.settings = settings
        ctx.ws = ws
        ctx.mark_non_differentiable(p2f)
        ctx.set_materialize_grads(False)
        return p2f, zbuf, bary, dists

    @staticmethod
    def backward(ctx, g_p2f, g_zbuf, g_bary, g_dists):
        verts, faces, first_face, num_faces, cams, p2f = ctx.saved_tensors
        p = ctx.settings.params(first_face.shape[0])
        buf = ctx.ws.get(p, verts.shape[0], faces.shape[0])
        gv = torch.empty_like(verts)
        c = lambda t: None if t is None else t.contiguous()
        ops.rast_mesh_bwd(p, verts, faces, first_face, num_faces, cams, p2f, c(g_zbuf), c(g_bary), c(g_dists), gv,
                          buf)
        return gv, None, None, None, None, None, None


def rasterize_meshes(verts, faces, first_face, num_faces, cams, settings: RasterSettings, ws: Workspace = None):
    """Fragments (pix_to_face, zbuf, bary, dists) of a packed mesh batch."""
    if ws is None:
        ws = Workspace(verts.device)
    return _Rasterize.apply(verts.contiguous(), faces.contiguous(), first_face.contiguous(),
                            num_faces.contiguous(), cams.contiguous(), settings, ws)


class _Blend(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pix_to_face, zbuf, bary, dists, faces, colors, settings):
        N, S, _, K = pix_to_face.shape
        bp = settings.params()
        img = torch.empty((N, S, S, 4), dtype=torch.float32, device=pix_to_face.device)
        rgb = settings.rgb
        ops.blend_fwd(bp, N, S, K, pix_to_face, zbuf if rgb else None, bary if rgb else None, dists,
                      faces if rgb else None, colors if rgb else None, img)
        ctx.save_for_backward(pix_to_face, zbuf, bary, dists, faces, colors)
        ctx.settings = settings
        return img

    @staticmethod
    def backward(ctx, g_img):
        pix_to_face, zbuf, bary, dists, faces, colors = ctx.saved_tensors
        s = ctx.settings
        N, S, _, K = pix_to_face.shape
        gd = torch.empty_like(dists)
        if s.rgb:
            gz = torch.empty_like(zbuf)
            gb = torch.empty_like(bary)
            gc = torch.empty_like(colors)
            ops.blend_bwd(s.params(), N, S, K, pix_to_face, zbuf, bary, dists, faces, colors, g_img.contiguous(),
                          gz, gb, gd, gc)
            return None, gz, gb, gd, None, gc, None
        ops.blend_bwd(s.params(), N, S, K, pix_to_face, None, None, dists, None, None, g_img.contiguous(), None,
                      None, gd, None)
        return None, None, None, gd, None, None, None


def blend(pix_to_face, zbuf, bary, dists, faces=None, colors=None, settings: BlendSettings = None):
    """RGBA image (N, S, S, 4): softmax rgb (if settings.rgb) and silhouette alpha."""
    settings = settings or BlendSettings()
    if settings.rgb:
        if faces is None or colors is None:
            raise ValueError("rgb blending needs faces and per-vertex colours")
        return _Blend.apply(pix_to_face, zbuf, bary, dists, faces, colors, settings)
    dummy = torch.zeros(0, device=pix_to_face.device)
    return _Blend.apply(pix_to_face, zbuf, bary, dists, dummy, dummy, settings)


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, verts, colors, faces, first_face, num_faces, cams, rs, bs, ws):
        N = first_face.shape[0]
        S, K = rs.image_size, rs.faces_per_pixel
        p = rs.params(N)
        buf = ws.get(p, verts.shape[0], faces.shape[0])
        p2f, zbuf, bary, dists = ops.alloc_fragments(N, S, K, verts.device)
        img = torch.empty((N, S, S, 4), dtype=torch.float32, device=verts.device)
        ops.rast_blend_fwd(p, bs.params(), verts, faces, first_face, num_faces, cams, colors if bs.rgb else None,
                           p2f, zbuf, bary, dists, img, buf)
        ctx.save_for_backward(verts, colors, faces, first_face, num_faces, cams, p2f, zbuf, bary, dists)
        ctx.rs, ctx.bs, ctx.ws = rs, bs, ws
        return img

    @staticmethod
    def backward(ctx, g_img):
        verts, colors, faces, first_face, num_faces, cams, p2f, zbuf, bary, dists = ctx.saved_tensors
        rs, bs = ctx.rs, ctx.bs
        p = rs.params(first_face.shape[0])
        buf = ctx.ws.get(p, verts.shape[0], faces.shape[0])
        gv = torch.empty_like(verts)
        rgb = bs.rgb
        gc = torch.empty_like(colors) if rgb else None
        ops.blend_rast_bwd(p, bs.params(), verts, faces, first_face, num_faces, cams, p2f, zbuf if rgb else None,
                           bary if rgb else None, dists, colors if rgb else None, g_img.contiguous(), gv, gc, buf)
        return gv, gc, None, None, None, None, None, None, None


def render_meshes(verts, faces, first_face, num_faces, cams, raster: RasterSettings, blend: BlendSettings,
                  colors=None, ws: Workspace = None):
    """RGBA image (N, S, S, 4) of a packed mesh batch: rasterize, then blend;
    differentiable in verts (and colors for the softmax blend) through the
    fused backward."""
    if ws is None:
        ws = Workspace(verts.device)
    if blend.rgb and colors is None:
        raise ValueError("rgb blending needs per-vertex colours")
    if colors is None:
        colors = torch.zeros(0, 3, device=verts.device)
    return _Render.apply(verts.contiguous(), colors.contiguous(), faces.contiguous(), first_face.contiguous(),
                         num_faces.contiguous(), cams.contiguous(), raster, blend, ws)


# ---------------------------------------------------------------------------
# point clouds (Section 3.2, differentiable point cloud renderer)
# ---------------------------------------------------------------------------
@dataclass
class PointSettings:
    image_size: int
    points_per_pixel: int = 8
    radius: float = 0.01             # NDC units
    bin_size: int = 16               # 0: plain per-image form
    max_points_per_bin: int = 8192
    max_bin_entries: int = 0
    mode: int = ops.PTS_ALPHA        # or ops.PTS_NORM

    def params(self, N):
        return ops.make_pts_params(N, self.image_size, self.points_per_pixel, self.radius, self.bin_size,
                                   self.max_points_per_bin, self.max_bin_entries)


class _RenderPoints(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, features, first_point, num_points, cams, settings, ws):
        N = first_point.shape[0]
        S, K = settings.image_size, settings.points_per_pixel
        p = settings.params(N)
        n = ops.pts_workspace_bytes(p, points.shape[0])
        if ws.buf is None or ws.buf.numel() < n:
            ws.buf = torch.empty(n, dtype=torch.uint8, device=points.device)
        idx, zbuf, dists = ops.alloc_pts_fragments(N, S, K, points.device)
        ops.pts_rasterize_fwd(p, points, first_point, num_points, cams, idx, zbuf, dists, ws.buf)
        img = torch.empty((N, S, S, features.shape[1]), dtype=torch.float32, device=points.device)
        ops.pts_composite_fwd(p, settings.mode, idx, dists, features, img)
        ctx.save_for_backward(points, features, first_point, num_points, cams, idx, dists)
        ctx.settings, ctx.ws = settings, ws
        return img

    @staticmethod
    def backward(ctx, g_img):
        points, features, first_point, num_points, cams, idx, dists = ctx.saved_tensors
        s = ctx.settings
        p = s.params(first_point.shape[0])
        gd = torch.empty_like(dists)
        gf = torch.empty_like(features)
        ops.pts_composite_bwd(p, s.mode, idx, dists, features, g_img.contiguous(), gd, gf)
        gp = torch.empty_like(points)
        ops.pts_rasterize_bwd(p, points, first_point, num_points, cams, idx, None, gd, gp, ctx.ws.buf)
        return gp, gf, None, None, None, None, None


def render_points(points, features, first_point, num_points, cams, settings: PointSettings, ws: Workspace = None):
    """(N, S, S, D) image of a packed batch of point clouds: K nearest splats per
    pixel, Alpha or Norm compositing; differentiable in points and features."""
    if ws is None:
        ws = Workspace(points.device)
    return _RenderPoints.apply(points.contiguous(), features.contiguous(), first_point.contiguous(),
                               num_points.contiguous(), cams.contiguous(), settings, ws)


# ---------------------------------------------------------------------------
# lit shading (flat / Gouraud / Phong with one point light; softmax or hard)
# ---------------------------------------------------------------------------
@dataclass
class ShadeSettings:
    light: tuple = (0.0, 0.0, -3.0)      # point light position (world)
    ambient: tuple = (0.5, 0.5, 0.5)
    diffuse: tuple = (0.3, 0.3, 0.3)
    specular: tuple = (0.2, 0.2, 0.2)
    shininess: float = 64.0
    shading: int = ops.SHADE_PHONG
    blend: int = ops.SHADE_SOFTMAX

    def params(self):
        return ops.make_shade_params(self.light, self.ambient, self.diffuse, self.specular, self.shininess,
                                     self.shading, self.blend)


class _Shade(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pix_to_face, zbuf, bary, dists, verts, normals, colors, faces, cams, bs, ss):
        N, S, _, K = pix_to_face.shape
        img = torch.empty((N, S, S, 4), dtype=torch.float32, device=pix_to_face.device)
        ops.shade_fwd(bs.params(), ss.params(), N, S, K, pix_to_face, zbuf, bary, dists, faces, verts, normals,
                      colors, cams, img)
        ctx.save_for_backward(pix_to_face, zbuf, bary, dists, verts, normals, colors, faces, cams)
        ctx.bs, ctx.ss = bs, ss
        return img

    @staticmethod
    def backward(ctx, g_img):
        pix_to_face, zbuf, bary, dists, verts, normals, colors, faces, cams = ctx.saved_tensors
        N, S, _, K = pix_to_face.shape
        gz, gb, gd = torch.empty_like(zbuf), torch.empty_like(bary), torch.empty_like(dists)
        gv, gn, gc = torch.empty_like(verts), torch.empty_like(normals), torch.empty_like(colors)
        ops.shade_bwd(ctx.bs.params(), ctx.ss.params(), N, S, K, pix_to_face, zbuf, bary, dists, faces, verts,
                      normals, colors, cams, g_img.contiguous(), gz, gb, gd, gv, gn, gc)
        return None, gz, gb, gd, gv, gn, gc, None, None, None, None


def shade(pix_to_face, zbuf, bary, dists, verts, normals, colors, faces, cams, blend: BlendSettings = None,
          shading: ShadeSettings = None):
    """RGBA (N, S, S, 4) of lit fragments: flat / Gouraud / Phong reflection of one point
    light, blended by softmax (Algorithm 2) or hard assignment.  Differentiable in the
    fragments (chain into rasterize_meshes), positions, normals and colours."""
    return _Shade.apply(pix_to_face, zbuf, bary, dists, verts.contiguous(), normals.contiguous(),
                        colors.contiguous(), faces.contiguous(), cams.contiguous(), blend or BlendSettings(),
                        shading or ShadeSettings())


# ---------------------------------------------------------------------------
# exact KNN and the Chamfer loss (Section 3.1, 3D operators; Eq. 1)
# ---------------------------------------------------------------------------
class _KnnPoints(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p1, p2, first1, len1, first2, len2, K):
        idx = torch.empty((p1.shape[0], K), dtype=torch.int64, device=p1.device)
        dists = torch.empty((p1.shape[0], K), dtype=torch.float32, device=p1.device)
        ws = ops.alloc_knn_workspace(first1.shape[0], p1.device)
        ops.knn_points(p1, first1, len1, p2, first2, len2, K, idx, dists, ws)
        ctx.save_for_backward(p1, p2, idx)
        ctx.mark_non_differentiable(idx)
        return dists, idx

    @staticmethod
    def backward(ctx, g_dists, g_idx):
        p1, p2, idx = ctx.saved_tensors
        g1, g2 = torch.empty_like(p1), torch.empty_like(p2)
        ops.knn_points_bwd(p1, p2, idx, g_dists.contiguous(), g1, g2)
        return g1, g2, None, None, None, None, None


def knn_points(p1, first1, len1, p2, first2, len2, K):
    """(dists (P1, K), idx (P1, K)): the K nearest rows of p2 (same cloud) to
    each row of p1, ascending squared distance; idx is -1 (dist +inf) past
    the end of a small cloud.  Differentiable in p1 and p2 through dists."""
    return _KnnPoints.apply(p1.contiguous(), p2.contiguous(), first1.contiguous(), len1.contiguous(),
                            first2.contiguous(), len2.contiguous(), int(K))


class _Chamfer(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, q, first1, len1, first2, len2):
        dev = p.device
        N = first1.shape[0]
        idx_pq = torch.empty(p.shape[0], dtype=torch.int64, device=dev)
        idx_qp = torch.empty(q.shape[0], dtype=torch.int64, device=dev)
        d_pq = torch.empty(p.shape[0], dtype=torch.float32, device=dev)
        d_qp = torch.empty(q.shape[0], dtype=torch.float32, device=dev)
        per = torch.empty(N, dtype=torch.float32, device=dev)
        loss = torch.empty((), dtype=torch.float32, device=dev)
        ws = ops.alloc_knn_workspace(N, dev)
        ops.chamfer_fwd(p, first1, len1, q, first2, len2, idx_pq, d_pq, idx_qp, d_qp, per, loss, ws)
        ctx.save_for_backward(p, q, first1, len1, first2, len2, idx_pq, idx_qp)
        return loss, per

    @staticmethod
    def backward(ctx, g_loss, g_per):
        p, q, first1, len1, first2, len2, idx_pq, idx_qp = ctx.saved_tensors
        gp, gq = torch.empty_like(p), torch.empty_like(q)
        gl = None if g_loss is None else g_loss.reshape(1).contiguous()
        gpp = None if g_per is None else g_per.contiguous()
        ops.chamfer_bwd(p, first1, len1, q, first2, len2, idx_pq, idx_qp, gl, gpp, gp, gq)
        return gp, gq, None, None, None, None


def chamfer_distance(p, first1, len1, q, first2, len2):
    """(loss, loss_per_pair): Eq. 1 for each pair of packed clouds (P_i, Q_i)
    and the batch mean; differentiable in p and q (neighbours held fixed)."""
    return _Chamfer.apply(p.contiguous(), q.contiguous(), first1.contiguous(), len1.contiguous(),
                          first2.contiguous(), len2.contiguous())
