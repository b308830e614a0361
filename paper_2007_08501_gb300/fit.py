"""Analysis by synthesis: fit a mesh to target silhouettes, one CUDA graph per step.

Each step renders soft silhouettes of one mesh from several cameras through the
differentiable rasterizer and the silhouette blend (Algorithm 1),
``autograd.render_meshes``, whose backward is the fused blend + rasterizer
adjoint, compares them with target silhouettes using the negative
IoU of Appendix B,

    L_s = 1 - sum(S_p * S_g) / sum(S_p + S_g - S_p * S_g),

averaged over the views, and takes an Adam step on per-vertex offsets.  All
views share the mesh's vertices, so the rasterizer's backward pass sums every
view's gradient into the same offsets.  The whole step (forward, loss,
backward, optimizer) is captured once in a CUDA graph and replayed; nothing
synchronises with the host inside the graph.
"""
from __future__ import annotations

import torch

from . import autograd as ag


def iou_loss(pred, target):
    """Negative silhouette IoU per view, averaged; inputs (V, S, S) in [0, 1]."""
    inter = (pred * target).flatten(1).sum(1)
    union = (pred + target - pred * target).flatten(1).sum(1)
    return (1.0 - inter / union.clamp_min(1e-12)).mean()


class SilhouetteFitter:
    """Optimises offsets of ``verts`` so that its silhouettes match ``target``.

    faces (F0, 3) index ``verts`` (V, 3); ``cams`` (N, 16) holds one camera per
    view; every view rasterizes the same F0 faces.
    """

    def __init__(self, verts, faces, cams, target, settings: ag.RasterSettings, blend: ag.BlendSettings,
                 lr=1e-3):
        dev = verts.device
        N = cams.shape[0]
        F0 = faces.shape[0]
        self.base = verts.detach().clone()
        self.offsets = torch.zeros_like(self.base, requires_grad=True)
        self.faces = faces.repeat(N, 1).contiguous()
        self.first_face = (torch.arange(N, device=dev, dtype=torch.int64) * F0).contiguous()
        self.num_faces = torch.full((N,), F0, device=dev, dtype=torch.int64)
        self.cams = cams.contiguous()
        self.target = target.contiguous()
        self.settings = settings
        self.blend = blend
        self.ws = ag.Workspace(dev)
        self.opt = torch.optim.Adam([self.offsets], lr=lr, capturable=True)
        self.loss = torch.zeros((), device=dev)
        self.graph = None

    def _step(self):
        self.opt.zero_grad(set_to_none=False)
        verts = self.base + self.offsets
        img = ag.render_meshes(verts, self.faces, self.first_face, self.num_faces, self.cams, self.settings,
                               self.blend, ws=self.ws)
        loss = iou_loss(img[..., 3], self.target)
        loss.backward()
        self.opt.step()
        self.loss.copy_(loss.detach())

    def eager_step(self):
        self._step()
        return self.loss

    def capture(self, warmup=3):
        """Warm up on a side stream (allocations, workspace, optimizer state), then
        capture one step."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self._step()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        self.opt.zero_grad(set_to_none=False)
        with torch.cuda.graph(self.graph):
            self._step()
        return self

    def replay(self, n):
        for _ in range(n):
            self.graph.replay()
        return self.loss
