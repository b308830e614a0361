"""Gradcheck-style finite differences of the GPU autograd path.

``render_meshes`` (rast_blend_fwd forward, blend_rast_bwd backward) on a few
triangles at 16x16: every vertex coordinate is moved by +-h, the loss
L = sum(G * image) is evaluated through the same forward on the GPU, and the
central difference (L(v + h) - L(v - h)) / 2h is compared with verts.grad.
Only pixels whose face selection (pix_to_face) is the same at every
perturbed position, and which the oracle finds at least 2e-3 (NDC) from every
kink of the loss (its margin flags at that width: edge-distance ties, clip
kinks, blur boundaries, depth ties; the perturbation moves corners by ~3e-4),
carry upstream gradient, so the loss is smooth in the perturbation.  The
comparison is loose (fp32 forward: its rounding divided by 2h), and stands
beside the strict comparison with the FP64 oracle adjoint in the other tests.
Both blends: silhouette (Algorithm 1) and softmax RGB (Algorithm 2); sigma
and gamma are widened so the loss is smooth at the scale of h.
"""
import numpy as np
import pytest
import torch

import oracle
from _scenes import random_small_mesh
from paper_2007_08501_gb300 import autograd as ag

pytestmark = pytest.mark.gpu

S, K = 16, 4
H = 5e-4            # world units; the triangles span ~0.5


def _scene(seed):
    sc = random_small_mesh(seed, ntri=3)
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    return (T(sc["verts"], torch.float32), T(sc["faces"], torch.int64), T(sc["first_face"], torch.int64),
            T(sc["num_faces"], torch.int64), T(sc["cams"], torch.float32))


def _away_from_kinks(verts, faces, ff, nf, cams, blur):
    """Pixels the oracle finds at least 2e-3 from every margin of the loss."""
    m = oracle.Mesh(verts.cpu().numpy(), faces.cpu().numpy(), ff.cpu().numpy(), nf.cpu().numpy(),
                    cams.cpu().numpy())
    flags = oracle.margins(m, S, K, blur, True, True, eps=2e-3)
    return torch.from_numpy(flags.reshape(S, S) == 0).cuda()


@pytest.mark.parametrize("rgb", [False, True])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_vertex_gradient_matches_central_differences(rgb, seed):
    verts, faces, ff, nf, cams = _scene(seed)
    rs = ag.RasterSettings(S, K, 2e-3, bin_size=16, max_faces_per_bin=64, clip_barycentric_coords=True)
    bs = ag.BlendSettings(sigma=1e-3, gamma=1e-2, rgb=rgb)
    colors = torch.rand(verts.shape[0], 3, device="cuda", generator=torch.Generator("cuda").manual_seed(seed))
    kw = dict(colors=colors if rgb else None)

    def frags(v):
        return ag.rasterize_meshes(v, faces, ff, nf, cams, rs)[0].clone()

    # pixels whose selection is the same at v and at every v +- h e_i
    base = frags(verts)
    stable = torch.ones(S, S, dtype=torch.bool, device="cuda")
    for i in range(verts.numel()):
        for sgn in (1.0, -1.0):
            v = verts.clone()
            v.view(-1)[i] += sgn * H
            stable &= (frags(v) == base).all(-1)[0]
    stable &= _away_from_kinks(verts, faces, ff, nf, cams, float(np.float32(rs.blur_radius)))
    assert stable.float().mean() > 0.5
    g = torch.randn(1, S, S, 4, device="cuda", generator=torch.Generator("cuda").manual_seed(100 + seed))
    if not rgb:
        g[..., :3] = 0.0
    g *= stable[None, :, :, None]

    def loss(v):
        img = ag.render_meshes(v, faces, ff, nf, cams, rs, ag.BlendSettings(sigma=1e-3, gamma=1e-2, rgb=rgb), **kw)
        return (img.double() * g.double()).sum()

    v = verts.clone().requires_grad_(True)
    loss(v).backward()
    grad = v.grad.double().view(-1)
    fd = torch.empty_like(grad)
    with torch.no_grad():
        for i in range(verts.numel()):
            vp, vm = verts.clone(), verts.clone()
            vp.view(-1)[i] += H
            vm.view(-1)[i] -= H
            fd[i] = (loss(vp) - loss(vm)) / (2 * H)
    scale = grad.abs().max().item()
    assert scale > 0
    err = (fd - grad).abs()
    tol = 2e-2 * torch.clamp(grad.abs(), min=0.05 * scale)
    worst = (err / tol).max().item()
    print("rgb=%s seed=%d: %d stable pixels, max |grad| %.3g, worst %.3f of the bound"
          % (rgb, seed, int(stable.sum()), scale, worst))
    assert worst <= 1.0, (fd.cpu().numpy(), grad.cpu().numpy())
