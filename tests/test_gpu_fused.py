"""The fused backward (blend adjoint pulled straight through the rasterizer
adjoint, one pass over the fragments) against

  * the FP64 oracle chain on the GPU's own fragments: oracle blend adjoint
    (Algorithms 1 and 2) -> oracle rasterizer adjoint, upstream gradient zeroed
    at gradient-ambiguous pixels, vertex and colour gradients compared with the
    same criterion as the separate adjoints;
  * the two separate C-ABI calls (blend_bwd then rast_mesh_bwd), which must
    agree up to the order of the float atomics.
"""
import numpy as np
import pytest
import torch

import oracle
from _gpu import assert_grad_close, gpu_fwd, grad_close, oracle_mesh, to_dev
from paper_2007_08501_gb300 import ops, workloads
from paper_2007_08501_gb300.workloads import BLUR_SIGMA_1E4

pytestmark = pytest.mark.gpu

BLUR = float(np.float32(BLUR_SIGMA_1E4))
SIGMA = GAMMA = 1e-4
ZNEAR, ZFAR = 1.0, 100.0


def _f32(x):
    return float(np.float32(x))


def _case(mode, K, persp, clip, blur, bin_size, S=48, levels=(3, 2), seed=0):
    b = workloads.sphere_batch(list(levels), 0.05, seed_base=500 + seed)
    d = to_dev(b)
    N = b.N
    fr, status, p, ws = gpu_fwd(d, S, K, blur, bin_size, persp, clip)
    assert status == 0
    p2f, zb, ba, di = fr
    colors = torch.from_numpy(b.colors).cuda()
    faces = d["faces"]
    bp = ops.make_blend_params(SIGMA, GAMMA, ZNEAR, ZFAR, (1.0, 1.0, 1.0), 1e-10, mode)
    m = oracle_mesh(b)
    amb = oracle.margins(m, S, K, blur, persp, clip) & oracle.GRAD_COND_AMBIGUOUS
    g = workloads.upstream_grad(N, S, 11 + seed).copy()
    if mode == ops.BLEND_SIL:
        g[..., :3] = 0
    g.reshape(N * S * S, 4)[amb != 0] = 0
    gimg = torch.from_numpy(g).cuda()

    # fused
    gv = torch.empty_like(d["verts"])
    gc = torch.empty_like(colors) if mode else None
    ops.blend_rast_bwd(p, bp, d["verts"], faces, d["first_face"], d["num_faces"], d["cams"], p2f,
                       zb if mode else None, ba if mode else None, di, colors if mode else None, gimg, gv, gc, ws)

    # two separate calls
    gd2 = torch.empty_like(di)
    gz2 = torch.empty_like(zb) if mode else None
    gb2 = torch.empty_like(ba) if mode else None
    gc2 = torch.empty_like(colors) if mode else None
    ops.blend_bwd(bp, N, S, K, p2f, zb, ba, di, faces, colors, gimg, gz2, gb2, gd2, gc2)
    gv2 = torch.empty_like(d["verts"])
    ops.rast_mesh_bwd(p, d["verts"], faces, d["first_face"], d["num_faces"], d["cams"], p2f, gz2, gb2, gd2, gv2, ws)
    assert ops.rast_query_status(ws) == 0

    # oracle chain on the GPU's fragments
    fn = [x.cpu().numpy() for x in (p2f, zb, ba, di)]
    P = N * S * S
    rz, rb, rd, rc, ra, _, _, _ = oracle.blend_bwd(
        fn[0].reshape(P, K), fn[1].reshape(P, K), fn[2].reshape(P, K, 3), fn[3].reshape(P, K), b.faces, b.colors,
        g.reshape(P, 4), _f32(SIGMA), _f32(GAMMA), _f32(ZNEAR), _f32(ZFAR), mode=mode, with_abs=True)
    ref, ref_abs = oracle.rast_bwd(m, S, K, fn[0].reshape(P, K), rz if mode else None, rb if mode else None, rd,
                                   blur, persp, clip, with_abs=True)
    assert np.abs(ref).max() > 0
    gvn = gv.cpu().numpy()
    assert_grad_close(gvn, ref, ref_abs, "fused grad_verts")
    # the separate calls: same sums in another atomic order
    worst, glob = grad_close(gvn, gv2.cpu().numpy(), rel=1e-5, scale=ref_abs)
    assert glob <= 1e-5 and worst <= 10, (worst, glob)
    if mode:
        worst, glob = grad_close(gc.cpu().numpy(), rc, scale=ra)
        assert worst <= 1 and glob <= 1e-4, ("grad_colors", worst, glob)
        worst, glob = grad_close(gc.cpu().numpy(), gc2.cpu().numpy(), rel=1e-5, scale=ra)
        assert glob <= 1e-5 and worst <= 1, ("grad_colors vs separate calls", worst, glob)


@pytest.mark.parametrize("mode,K,persp,clip,blur,bin_size", [
    (ops.BLEND_RGB, 8, True, True, BLUR, 16),
    (ops.BLEND_SIL, 8, True, True, BLUR, 16),
    (ops.BLEND_RGB, 4, True, False, BLUR, 0),
    (ops.BLEND_SIL, 1, False, False, 0.0, 8),
    (ops.BLEND_RGB, 2, False, True, BLUR, 8),
    (ops.BLEND_SIL, 16, True, True, BLUR, 16),
    (ops.BLEND_RGB, 16, True, True, BLUR, 16),
    (ops.BLEND_RGB, 5, True, True, BLUR, 16),   # generic K
    (ops.BLEND_SIL, 24, True, False, BLUR, 8),  # generic K
    (ops.BLEND_SIL, 13, True, True, BLUR, 16),  # generic K, odd: slots one at a time
    (ops.BLEND_SIL, 64, True, True, BLUR, 16),  # largest K: 64 KB of per-slot probabilities
])
def test_fused_backward_matches_oracle_chain(mode, K, persp, clip, blur, bin_size):
    _case(mode, K, persp, clip, blur, bin_size)


def test_fused_backward_ragged_image_and_shared_vertices():
    # S not a multiple of the 16 x 16 tile; two views of one mesh share its vertices
    v, f = workloads.displaced_sphere(2, 0.05, np.random.default_rng(8))
    cams = np.stack([workloads.look_at_camera(2.7, 10.0, 30.0), workloads.look_at_camera(2.7, -20.0, 200.0)])
    S, K = 37, 4
    verts = v.astype(np.float32)
    faces = np.concatenate([f, f]).astype(np.int64)
    batch = dict(verts=verts, faces=faces, first_face=np.array([0, f.shape[0]], np.int64),
                 num_faces=np.array([f.shape[0]] * 2, np.int64), cams=cams.astype(np.float32))
    d = to_dev(batch)
    fr, status, p, ws = gpu_fwd(d, S, K, BLUR, 16, True, True)
    assert status == 0
    p2f, zb, ba, di = fr
    colors = torch.from_numpy(np.random.default_rng(2).uniform(size=verts.shape).astype(np.float32)).cuda()
    bp = ops.make_blend_params(SIGMA, GAMMA, ZNEAR, ZFAR, (1.0, 1.0, 1.0), 1e-10, ops.BLEND_RGB)
    m = oracle_mesh(batch)
    amb = oracle.margins(m, S, K, BLUR, True, True) & oracle.GRAD_COND_AMBIGUOUS
    g = workloads.upstream_grad(2, S, 5).copy()
    g.reshape(2 * S * S, 4)[amb != 0] = 0
    gimg = torch.from_numpy(g).cuda()
    gv = torch.empty_like(d["verts"])
    gc = torch.empty_like(colors)
    ops.blend_rast_bwd(p, bp, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], p2f, zb, ba, di,
                       colors, gimg, gv, gc, ws)
    P = 2 * S * S
    fn = [x.cpu().numpy() for x in (p2f, zb, ba, di)]
    rz, rb, rd, rc, ra, _, _, _ = oracle.blend_bwd(
        fn[0].reshape(P, K), fn[1].reshape(P, K), fn[2].reshape(P, K, 3), fn[3].reshape(P, K), faces,
        colors.cpu().numpy(), g.reshape(P, 4), _f32(SIGMA), _f32(GAMMA), _f32(ZNEAR), _f32(ZFAR), mode=1,
        with_abs=True)
    ref, ref_abs = oracle.rast_bwd(m, S, K, fn[0].reshape(P, K), rz, rb, rd, BLUR, True, True, with_abs=True)
    assert_grad_close(gv.cpu().numpy(), ref, ref_abs, "fused shared verts")
    worst, glob = grad_close(gc.cpu().numpy(), rc, scale=ra)
    assert worst <= 1 and glob <= 1e-4


def test_fused_backward_empty_and_argument_errors():
    b = workloads.sphere_batch([2], 0.05, seed_base=4)
    d = to_dev(b)
    fr, _, p, ws = gpu_fwd(d, 16, 2, BLUR, 16)
    p2f, zb, ba, di = fr
    bp = ops.make_blend_params(SIGMA, GAMMA, ZNEAR, ZFAR, (1.0, 1.0, 1.0), 1e-10, ops.BLEND_SIL)
    # zero upstream gradient: zero vertex gradient (overwritten, not accumulated)
    gv = torch.full_like(d["verts"], 7.0)
    ops.blend_rast_bwd(p, bp, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], p2f, None, None,
                       di, None, torch.zeros((1, 16, 16, 4), device="cuda"), gv, None, ws)
    assert torch.count_nonzero(gv).item() == 0
    # rgb mode without colours is an argument error, nothing enqueued
    bp_rgb = ops.make_blend_params(SIGMA, GAMMA, ZNEAR, ZFAR, (1.0, 1.0, 1.0), 1e-10, ops.BLEND_RGB)
    with pytest.raises(ops.MeshRastError):
        ops.blend_rast_bwd(p, bp_rgb, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], p2f, zb, ba,
                           di, None, torch.zeros((1, 16, 16, 4), device="cuda"), gv, None, ws)


@pytest.mark.parametrize("rgb", [False, True])
def test_render_meshes_autograd_equals_separate_functions(rgb):
    from paper_2007_08501_gb300 import autograd as ag
    b = workloads.sphere_batch([3, 3], 0.05, seed_base=61)
    d = to_dev(b)
    rs = ag.RasterSettings(image_size=64, faces_per_pixel=4, blur_radius=BLUR, bin_size=16,
                           clip_barycentric_coords=True)
    bs = ag.BlendSettings(sigma=SIGMA, gamma=GAMMA, znear=ZNEAR, zfar=ZFAR, rgb=rgb)
    g = torch.from_numpy(workloads.upstream_grad(b.N, 64, 3)).cuda()
    out = []
    for fused in (True, False):
        v = d["verts"].clone().requires_grad_(True)
        c = torch.from_numpy(b.colors).cuda().requires_grad_(rgb)
        if fused:
            img = ag.render_meshes(v, d["faces"], d["first_face"], d["num_faces"], d["cams"], rs, bs,
                                   colors=c if rgb else None)
        else:
            p2f, zb, ba, di = ag.rasterize_meshes(v, d["faces"], d["first_face"], d["num_faces"], d["cams"], rs)
            img = ag.blend(p2f, zb, ba, di, d["faces"], c if rgb else None, settings=bs)
        (img * g).sum().backward()
        out.append((img.detach().cpu().numpy(), v.grad.cpu().numpy(), c.grad.cpu().numpy() if rgb else None))
    assert np.array_equal(out[0][0], out[1][0])
    ref = out[1][1]
    assert np.linalg.norm(out[0][1] - ref) <= 1e-5 * np.linalg.norm(ref)
    if rgb:
        assert np.linalg.norm(out[0][2] - out[1][2]) <= 1e-5 * np.linalg.norm(out[1][2])


@pytest.mark.parametrize("mode,K,bin_size,clip", [
    (ops.BLEND_RGB, 8, 16, True),     # fine pass blends (vector write path)
    (ops.BLEND_RGB, 8, 8, True),
    (ops.BLEND_SIL, 4, 16, True),
    (ops.BLEND_SIL, 1, 8, False),
    (ops.BLEND_RGB, 5, 16, True),     # fine pass blends (scalar write path, K < 8)
    (ops.BLEND_RGB, 16, 16, False),
    (ops.BLEND_RGB, 20, 8, True),     # K > 16: separate blend kernel inside the call
    (ops.BLEND_SIL, 20, 16, True),    # K > 16: the attribute pass blends the silhouette
    (ops.BLEND_SIL, 50, 8, True),
    (ops.BLEND_SIL, 4, 0, True),      # plain form: separate blend kernel
])
def test_fused_forward_equals_rasterize_then_blend(mode, K, bin_size, clip):
    b = workloads.sphere_batch([3, 2, 4], 0.05, seed_base=71)
    d = to_dev(b)
    N, S = b.N, 70                                   # ragged: 70 = 4 * 16 + 6
    blur = BLUR if clip or mode == ops.BLEND_RGB else 0.0
    p = ops.make_rast_params(N, S, K, np.float32(blur), bin_size, 4096, True, clip)
    ws = ops.alloc_workspace(p, b.V, b.F)
    colors = torch.from_numpy(b.colors).cuda()
    bp = ops.make_blend_params(SIGMA, GAMMA, ZNEAR, ZFAR, (1.0, 1.0, 1.0), 1e-10, mode)
    ref = ops.alloc_fragments(N, S, K)
    ops.rast_mesh_fwd(p, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], *ref, ws)
    ref_img = torch.empty((N, S, S, 4), device="cuda")
    ops.blend_fwd(bp, N, S, K, *ref[:4], d["faces"], colors, ref_img)
    got = ops.alloc_fragments(N, S, K)
    img = torch.full((N, S, S, 4), 7.0, device="cuda")
    ops.rast_blend_fwd(p, bp, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"],
                       colors if mode else None, *got, img, ws)
    assert ops.rast_query_status(ws) == 0
    for x, y in zip(ref, got):
        assert torch.equal(x, y)
    assert np.max(np.abs(img.cpu().numpy() - ref_img.cpu().numpy())) <= 1e-6
    # and the image matches the oracle blend of these fragments
    fn = [x.cpu().numpy() for x in got]
    P = N * S * S
    orc = oracle.blend_fwd(fn[0].reshape(P, K), fn[1].reshape(P, K), fn[2].reshape(P, K, 3), fn[3].reshape(P, K),
                           b.faces, b.colors, _f32(SIGMA), _f32(GAMMA), _f32(ZNEAR), _f32(ZFAR), mode=mode)
    assert np.max(np.abs(img.cpu().numpy().reshape(P, 4) - orc)) <= 1e-5


@pytest.mark.parametrize("K,bin_size", [(1, 8), (4, 16), (8, 16), (16, 8), (3, 16)])
def test_silhouette_without_fragments_equals_the_fragment_writing_forward(K, bin_size):
    # the fine pass blends and writes only the image: bit-identical to the call
    # that also writes the Fragment data (same arithmetic, stores skipped)
    b = workloads.sphere_batch([3, 2, 4], 0.05, seed_base=91)
    d = to_dev(b)
    N, S = b.N, 70
    p = ops.make_rast_params(N, S, K, np.float32(BLUR), bin_size, 4096, True, True)
    ws = ops.alloc_workspace(p, b.V, b.F)
    bp = ops.make_blend_params(SIGMA, GAMMA, ZNEAR, ZFAR, (1.0, 1.0, 1.0), 1e-10, ops.BLEND_SIL)
    frag = ops.alloc_fragments(N, S, K)
    ref = torch.empty((N, S, S, 4), device="cuda")
    args = (p, bp, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], None)
    ops.rast_blend_fwd(*args, *frag, ref, ws)
    img = torch.full((N, S, S, 4), 7.0, device="cuda")
    ops.rast_blend_fwd(*args, None, None, None, None, img, ws)
    assert ops.rast_query_status(ws) == 0
    assert torch.equal(img, ref)
    assert float(img[..., 3].max()) > 0.5


def test_fragment_free_forward_only_where_the_fine_pass_blends():
    b = workloads.sphere_batch([2], 0.05, seed_base=92)
    d = to_dev(b)
    colors = torch.from_numpy(b.colors).cuda()
    img = torch.empty((1, 32, 32, 4), device="cuda")
    for K, bin_size, mode in ((8, 16, ops.BLEND_RGB), (20, 16, ops.BLEND_SIL), (4, 0, ops.BLEND_SIL)):
        p = ops.make_rast_params(1, 32, K, np.float32(BLUR), bin_size, 4096, True, True)
        ws = ops.alloc_workspace(p, b.V, b.F)
        bp = ops.make_blend_params(SIGMA, GAMMA, ZNEAR, ZFAR, (1.0, 1.0, 1.0), 1e-10, mode)
        with pytest.raises(ops.MeshRastError):
            ops.rast_blend_fwd(p, bp, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], colors,
                               None, None, None, None, img, ws)
