"""Lit shading (shade_fwd / shade_bwd) against the FP64 shading oracle on the
GPU's own fragments: images within 1e-5; fragment and vertex gradients within
1e-4 relative globally, every component within 1e-3 and 99% within 1e-4 of
max(|ref|, 1e-2 rms(ref)) -- for vertex sums, of the magnitudes of their
per-slot contributions -- (sums with cancellation, such as dL/dbary_i =
gx . P_i + ga . A_i, carry fp32 rounding of the size of their terms)."""
import numpy as np
import pytest
import torch

from _gpu import gpu_fwd, grad_close, to_dev
from oracle import shading as osh
from paper_2007_08501_gb300 import ops, workloads
from paper_2007_08501_gb300.workloads import BLUR_SIGMA_1E4

pytestmark = pytest.mark.gpu

BLUR = float(np.float32(BLUR_SIGMA_1E4))
LIGHT = dict(light=(1.5, 2.0, -2.5), ambient=(0.3, 0.25, 0.2), diffuse=(0.5, 0.5, 0.6),
             specular=(0.3, 0.3, 0.3), shininess=16.0)


def _f32(x):
    return float(np.float32(x))


@pytest.mark.parametrize("shading", [ops.SHADE_FLAT, ops.SHADE_GOURAUD, ops.SHADE_PHONG])
@pytest.mark.parametrize("blend", [ops.SHADE_SOFTMAX, ops.SHADE_HARD])
def test_shading_and_its_adjoint_match_oracle(shading, blend):
    b = workloads.sphere_batch([3, 2], 0.05, seed_base=300 + shading)
    d = to_dev(b)
    S, K = 40, 4
    fr, st, _, _ = gpu_fwd(d, S, K, BLUR, 16, True, True)
    assert st == 0
    p2f, zb, ba, di = fr
    N = b.N
    normals = (b.verts / np.linalg.norm(b.verts, axis=1, keepdims=True)).astype(np.float32)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    nrm, col = T(normals), T(b.colors)
    sigma, gamma = 1e-4, 1e-2
    bp = ops.make_blend_params(sigma, gamma, 1.0, 100.0, (1.0, 1.0, 1.0), 1e-10, ops.BLEND_RGB)
    sp = ops.make_shade_params(shading=shading, blend=blend, **LIGHT)
    img = torch.empty((N, S, S, 4), device="cuda")
    ops.shade_fwd(bp, sp, N, S, K, p2f, zb, ba, di, d["faces"], d["verts"], nrm, col, d["cams"], img)
    P = N * S * S
    fn = [x.cpu().numpy() for x in fr]
    image_of = np.repeat(np.arange(N), S * S)
    light = osh.light_params(*[np.float32(v) for v in (LIGHT["light"], LIGHT["ambient"], LIGHT["diffuse"],
                                                        LIGHT["specular"])], shininess=LIGHT["shininess"])
    bl = osh.blend_params(_f32(sigma), _f32(gamma), 1.0, 100.0, _f32(1e-10))
    args = [image_of, fn[0].reshape(P, K), fn[1].reshape(P, K), fn[2].reshape(P, K, 3), fn[3].reshape(P, K), b.faces,
            b.verts, normals, b.colors, b.cams, light, bl, shading]
    ref = osh.shade_fwd(*args, blend_mode=blend)
    got = img.cpu().numpy().reshape(P, 4)
    assert np.max(np.abs(got - ref)) <= 1e-5, np.max(np.abs(got - ref))
    assert (fn[0] >= 0).any()

    g = np.random.default_rng(5).normal(size=(P, 4)).astype(np.float32)
    # no upstream gradient where a reflection term switches on or off within 1e-4 (a kink:
    # fp32 and FP64 may fall on different sides)
    mg = osh.shade_margins(image_of, fn[0].reshape(P, K), fn[2].reshape(P, K, 3), b.faces, b.verts, normals,
                           b.cams, light, shading, blend)
    g[mg < 1e-4] = 0
    gz, gb, gd = torch.empty_like(zb), torch.empty_like(ba), torch.empty_like(di)
    gv, gn, gc = torch.empty_like(d["verts"]), torch.empty_like(nrm), torch.empty_like(col)
    ops.shade_bwd(bp, sp, N, S, K, p2f, zb, ba, di, d["faces"], d["verts"], nrm, col, d["cams"],
                  T(g.reshape(N, S, S, 4)), gz, gb, gd, gv, gn, gc)
    rz, rb, rd, rv, rn, rc, ab = osh.shade_bwd(*args, g, blend_mode=blend, with_abs=True)
    # vertex sums are judged against the magnitudes of their per-slot contributions
    for name, a, r, sc in (("grad_bary", gb, rb, None), ("grad_verts", gv, rv, ab[0]), ("grad_normals", gn, rn, ab[1]),
                           ("grad_colors", gc, rc, ab[2]), ("grad_zbuf", gz, rz, None), ("grad_dists", gd, rd, None)):
        an = a.cpu().numpy().reshape(r.shape)
        if not np.abs(r).max() > 0:
            assert np.abs(an).max() <= 1e-6, name
            continue
        worst, glob, n_over = grad_close(an, r, scale=sc, return_count=True)
        assert glob <= 1e-4 and worst <= 10 and n_over <= max(3, 0.01 * r.size), (name, worst, glob, n_over)


def test_shade_autograd_chains_into_the_rasterizer():
    from paper_2007_08501_gb300 import autograd as ag
    b = workloads.sphere_batch([3, 3], 0.05, seed_base=91)
    d = to_dev(b)
    normals = torch.nn.functional.normalize(d["verts"], dim=1)
    colors = torch.from_numpy(b.colors).cuda()
    rs = ag.RasterSettings(image_size=48, faces_per_pixel=4, blur_radius=BLUR, bin_size=16,
                           clip_barycentric_coords=True)
    bs = ag.BlendSettings(sigma=1e-4, gamma=1e-2, znear=1.0, zfar=100.0)
    ss = ag.ShadeSettings(shading=ops.SHADE_PHONG, **LIGHT)
    v = d["verts"].clone().requires_grad_(True)
    n = normals.clone().requires_grad_(True)
    c = colors.clone().requires_grad_(True)
    frags = ag.rasterize_meshes(v, d["faces"], d["first_face"], d["num_faces"], d["cams"], rs)
    img = ag.shade(*frags, v, n, c, d["faces"], d["cams"], bs, ss)
    g = torch.from_numpy(np.random.default_rng(2).normal(size=tuple(img.shape)).astype(np.float32)).cuda()
    (img * g).sum().backward()
    # by hand: shade_bwd, then rast_mesh_bwd on its fragment gradients, plus the direct term
    p2f, zb, ba, di = [x.detach() for x in frags]
    N, S, K = b.N, 48, 4
    gz, gb, gd = torch.empty_like(zb), torch.empty_like(ba), torch.empty_like(di)
    gv, gn, gc = torch.empty_like(v), torch.empty_like(n), torch.empty_like(c)
    ops.shade_bwd(bs.params(), ss.params(), N, S, K, p2f, zb, ba, di, d["faces"], d["verts"], normals, colors,
                  d["cams"], g, gz, gb, gd, gv, gn, gc)
    p = rs.params(N)
    ws = ops.alloc_workspace(p, b.V, b.F)
    gr = torch.empty_like(v)
    ops.rast_mesh_bwd(p, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], p2f, gz, gb, gd, gr, ws)
    tot = gv + gr
    # same kernels both ways; the float atomics may add in another order
    for got, want in ((v.grad, tot), (n.grad, gn), (c.grad, gc)):
        assert torch.linalg.norm(got - want) <= 1e-5 * torch.linalg.norm(want)


@pytest.mark.parametrize("shading", [ops.SHADE_GOURAUD, ops.SHADE_PHONG])
def test_benchmark_batch_sampled_pixels(shading):
    # the shaded benchmark step at full size (8 x 5,120 faces, 256x256, K = 8,
    # the bench's light), checked on 256 seeded pixels per image: image values
    # and the per-slot fragment gradients (which depend on the pixel alone)
    w = workloads.workload(1, "")
    b = w.batch
    d = to_dev(b)
    S, K = w.image_size, w.K
    fr, st, _, _ = gpu_fwd(d, S, K, float(np.float32(w.blur_radius)), 16, True, True)
    assert st == 0
    p2f, zb, ba, di = fr
    N = b.N
    nrm = torch.nn.functional.normalize(d["verts"], dim=1).contiguous()
    col = torch.from_numpy(b.colors).cuda()
    light = dict(light=(0.0, 3.0, -3.0), ambient=(0.3, 0.3, 0.3), diffuse=(0.6, 0.6, 0.6), specular=(0.3, 0.3, 0.3),
                 shininess=32.0)
    bp = ops.make_blend_params(w.sigma, w.gamma, w.znear, w.zfar, (1.0, 1.0, 1.0), 1e-10, ops.BLEND_RGB)
    sp = ops.make_shade_params(shading=shading, blend=ops.SHADE_SOFTMAX, **light)
    img = torch.empty((N, S, S, 4), device="cuda")
    ops.shade_fwd(bp, sp, N, S, K, p2f, zb, ba, di, d["faces"], d["verts"], nrm, col, d["cams"], img)
    g = torch.from_numpy(workloads.upstream_grad(N, S, w.grad_seed)).cuda()
    gz, gb, gd = torch.empty_like(zb), torch.empty_like(ba), torch.empty_like(di)
    gv, gn, gc = torch.empty_like(d["verts"]), torch.empty_like(nrm), torch.empty_like(col)
    ops.shade_bwd(bp, sp, N, S, K, p2f, zb, ba, di, d["faces"], d["verts"], nrm, col, d["cams"], g, gz, gb, gd, gv, gn,
                  gc)
    px = workloads.sample_pixels(N, S, 256, 77)
    flat = (px[:, 0] * S + px[:, 1]) * S + px[:, 2]
    P = N * S * S
    pick = lambda t, *tail: t.cpu().numpy().reshape(P, *tail)[flat]
    f_p2f, f_zb, f_ba, f_di = pick(p2f, K), pick(zb, K), pick(ba, K, 3), pick(di, K)
    normals = nrm.cpu().numpy()
    lt = osh.light_params(*[np.float32(v) for v in (light["light"], light["ambient"], light["diffuse"],
                                                    light["specular"])], shininess=light["shininess"])
    bl = osh.blend_params(_f32(w.sigma), _f32(w.gamma), _f32(w.znear), _f32(w.zfar), _f32(1e-10))
    args = [px[:, 0], f_p2f, f_zb, f_ba, f_di, b.faces, b.verts, normals, b.colors, b.cams, lt, bl, shading]
    ref = osh.shade_fwd(*args, blend_mode=osh.SOFTMAX)
    assert np.max(np.abs(pick(img, 4) - ref)) <= 1e-5
    # per-slot gradients, away from the reflection model's kinks
    gs = pick(g, 4)
    mg = osh.shade_margins(px[:, 0], f_p2f, f_ba, b.faces, b.verts, normals, b.cams, lt, shading, osh.SOFTMAX)
    keep = mg >= 1e-4
    rz, rb, rd, _, _, _, abb = osh.shade_bwd(*args, gs, blend_mode=osh.SOFTMAX, with_abs_bary=True)
    # barycentric gradients sum position, normal and colour terms: judged against their magnitudes
    for name, a, r, sc in (("grad_bary", pick(gb, K, 3), rb, abb), ("grad_zbuf", pick(gz, K), rz, None),
                           ("grad_dists", pick(gd, K), rd, None)):
        worst, glob, n_over = grad_close(a[keep], r[keep], scale=None if sc is None else sc[keep], return_count=True)
        assert glob <= 1e-4 and worst <= 10 and n_over <= max(3, 0.01 * r[keep].size), (name, worst, glob, n_over)
    assert keep.mean() > 0.9
