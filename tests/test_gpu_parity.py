"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Fragments: pix_to_face bit-exact on every pixel whose depth / edge / blur /
cull margins exceed 1e-6 (the rest are counted); zbuf, bary and dists within
1e-5 absolute.  Blends within 1e-5.  Gradients within 1e-4 relative of the
oracle adjoint conditioned on the same face selection.
"""
import numpy as np
import pytest
import torch

import oracle
from _gpu import assert_grad_close, compare_frags, gpu_fwd, grad_close, np_frags, oracle_mesh, pick, to_dev
from _scenes import ndc_triangle, random_small_mesh, scene
from paper_2007_08501_gb300 import ops, workloads
from paper_2007_08501_gb300.workloads import BLUR_SIGMA_1E4

pytestmark = pytest.mark.gpu

BLUR = float(np.float32(BLUR_SIGMA_1E4))


def _full_check(batch, S, K, blur, bin_size, persp=True, clip=False, max_amb_frac=0.10, max_faces_per_bin=4096):
    d = to_dev(batch)
    fr, status, _, _ = gpu_fwd(d, S, K, blur, bin_size, persp, clip, max_faces_per_bin=max_faces_per_bin)
    assert status == 0
    m = oracle_mesh(batch)
    orc = oracle.rasterize(m, S, K, blur, persp, clip)
    amb = oracle.margins(m, S, K, blur, persp, clip) & oracle.FWD_AMBIGUOUS
    n_amb, n_bad = compare_frags(np_frags(fr), orc, amb)
    print("ambiguous pixels: %d of %d" % (n_amb, amb.size))
    assert n_bad == 0
    assert n_amb <= max_amb_frac * amb.size
    return fr


def test_config0_plain_form_full_image():
    w = workloads.workload(0)
    _full_check(w.batch, w.image_size, w.K, w.blur_radius, bin_size=0)


@pytest.mark.parametrize("bin_size", [8, 16])
def test_config0_binned_full_image(bin_size):
    w = workloads.workload(0)
    _full_check(w.batch, w.image_size, w.K, 0.0, bin_size)


@pytest.mark.parametrize("S,K,blur,bin_size,persp,clip", [
    (76, 4, BLUR, 16, True, True),     # ragged tail: 76 = 4*16 + 12
    (76, 3, BLUR, 8, True, False),     # K not a power of two, ragged 76 = 9*8 + 4
    (64, 1, 0.0, 16, False, False),    # hard, affine barycentrics
    (40, 8, BLUR, 8, False, True),
])
def test_small_multi_mesh_full_image(S, K, blur, bin_size, persp, clip):
    b = workloads.sphere_batch([3, 2, 3], 0.05, seed_base=77)
    _full_check(b, S, K, blur, bin_size, persp, clip)


def test_large_k_shared_memory_path():
    b = workloads.sphere_batch([3, 3], 0.05, seed_base=91)
    for bs in (0, 8):
        _full_check(b, 48, 50, BLUR, bs, True, True)


@pytest.mark.parametrize("S,K,bin_size", [(48, 50, 16), (70, 50, 16), (70, 20, 8), (40, 64, 16), (33, 17, 8)])
def test_large_k_streaming_path(S, K, bin_size):
    # clipped barycentrics, K > 16: the front-to-back streaming fine pass and
    # the attribute pass (ragged images, K up to the 64 maximum)
    b = workloads.sphere_batch([3, 3], 0.05, seed_base=91)
    _full_check(b, S, K, BLUR, bin_size, True, True)


def test_streaming_pass_equals_the_block_fine_pass_at_full_size():
    # The first 2 of the 20 views of the K = 50 benchmark batch (512 x 512),
    # rendered twice through rast_mesh_fwd: a bin capacity of 8192 takes the
    # streaming fine pass (bins sorted front to back, warps settling slots as
    # they go, the block-wide edge-line cull, the warp redo) and the attribute
    # pass; 8200 (above the streaming pass's limit) takes the block fine pass
    # with per-pixel lists in shared memory.  Both end in the same face tests,
    # depth keys and fragment arithmetic, so every output is identical.
    w = workloads.workload(4)
    b = workloads.first_images(w.batch, 2)
    d = to_dev(b)
    blur = float(np.float32(w.blur_radius))
    outs = []
    for cap in (8192, 8200):
        p = ops.make_rast_params(b.N, w.image_size, w.K, np.float32(blur), 16, cap, True, True)
        ws = ops.alloc_workspace(p, b.V, b.F)
        fr = ops.alloc_fragments(b.N, w.image_size, w.K)
        ops.rast_mesh_fwd(p, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], *fr, ws)
        assert ops.rast_query_status(ws) == 0
        outs.append(fr)
        del ws
    for x, y in zip(*outs):
        assert torch.equal(x, y)
    assert (outs[0][0][..., w.K - 1] >= 0).float().mean() > 0.3   # most pixels hold K faces


def test_large_k_ring_overflow_goes_to_the_second_pass():
    """30 faces tilted away from the camera: each has one corner at depth 1 (its
    sort key), while at the pixels near its far edge its depth is ~5.  No
    candidate settles before the bin's list ends, so more than the 16 a pixel
    keeps on chip in the first pass are unsettled at once: those pixels are
    queued and done by the second pass (a 64-entry ring)."""
    from _scenes import ndc_triangle, scene
    tris = [ndc_triangle((-0.6 + 0.002 * i, -0.6), (0.6, -0.6 + 0.001 * i), (0.0, 0.9), (5.0 + 0.01 * i, 5.0, 1.0))
            for i in range(30)]
    sc = scene(tris)
    S, K = 32, 40
    d = to_dev(sc)
    fr, status, p, ws = gpu_fwd(d, S, K, BLUR, 16, True, True)
    assert status == 0
    L = ops.rast_workspace_bin_layout(p, d["verts"].shape[0], d["faces"].shape[0])
    redo = int(ws[L["redo"]:L["redo"] + 4].cpu().numpy().view(np.uint32)[0])
    print("pixels handed to the second pass: %d" % redo)
    assert redo > 0
    m = oracle_mesh(sc)
    orc = oracle.rasterize(m, S, K, BLUR, True, True)
    amb = oracle.margins(m, S, K, BLUR, True, True) & oracle.FWD_AMBIGUOUS
    n_amb, n_bad = compare_frags(np_frags(fr), orc, amb)
    assert n_bad == 0 and n_amb < 0.5 * amb.size
    assert (orc[0][:, 20] >= 0).any()   # some pixels hold more than 20 faces


@pytest.mark.parametrize("level,S,K,bin_size,clip", [
    (6, 32, 4, 16, True),     # ~20k faces per bin: sorted in segments of 8192
    (6, 32, 4, 16, False),    # unclipped blur: no depth cull, every segment walked
    (5, 32, 50, 8, True),     # K > 16: segments of 2048 sorted before the walk
    (5, 32, 20, 16, False),
])
def test_bins_larger_than_the_sort_buffer(level, S, K, bin_size, clip):
    b = workloads.sphere_batch([level], 0.05, seed_base=17)
    # dense meshes at 32x32: many pixels sit within 1e-6 of some edge or depth tie
    _full_check(b, S, K, BLUR, bin_size, True, clip, max_amb_frac=0.6, max_faces_per_bin=65536)


@pytest.mark.parametrize("K", [2, 16, 20])
def test_binned_equals_plain(K):
    """The binned fine pass evaluates each face relative to its bin's first
    pixel, the plain form relative to the face's corner 0: face ids agree
    bitwise on every pixel outside the oracle's 1e-6 ambiguity band (the two
    roundings differ only within ~1e-8 of an edge), values to fp32 rounding."""
    b = workloads.sphere_batch([4, 3, 5], 0.05, seed_base=5)
    d = to_dev(b)
    S = 100
    m = oracle_mesh(b)
    amb = oracle.margins(m, S, K, BLUR, True, True) & oracle.FWD_AMBIGUOUS
    ok = (amb == 0).reshape(b.N, S, S)
    assert ok.mean() > 0.5
    ref = np_frags(gpu_fwd(d, S, K, BLUR, 0, True, True)[0])
    for bs in (8, 16):
        got = np_frags(gpu_fwd(d, S, K, BLUR, bs, True, True)[0])
        np.testing.assert_array_equal(ref[0][ok], got[0][ok])
        same = (ref[0] == got[0]) & (ref[0] >= 0)
        for x, y in zip(ref[1:], got[1:]):
            sel = same if x.ndim == 4 else same[..., None].repeat(3, -1)
            assert np.max(np.abs(x[sel] - y[sel])) <= 1e-5


def test_config1_sampled_pixels_at_full_size():
    w = workloads.workload(1)
    d = to_dev(w.batch)
    fr, status, p, ws = gpu_fwd(d, w.image_size, w.K, np.float32(w.blur_radius), 16, True, True)
    assert status == 0
    px = workloads.sample_pixels(w.batch.N, w.image_size, 256, seed=1)
    m = oracle_mesh(w.batch)
    orc = oracle.rasterize(m, w.image_size, w.K, np.float32(w.blur_radius), True, True, pixels=px)
    amb = oracle.margins(m, w.image_size, w.K, np.float32(w.blur_radius), True, True, pixels=px) \
        & oracle.FWD_AMBIGUOUS
    n_amb, n_bad = compare_frags(pick(np_frags(fr), px, w.image_size), orc, amb)
    assert n_bad == 0
    # invariants at every pixel: sorted depths, valid slots first, bary sums to 1
    p2f, zb, ba, di = np_frags(fr)
    valid = p2f >= 0
    assert np.all(valid[..., 1:] <= valid[..., :-1])
    z = np.where(valid, zb, np.inf)
    assert np.all(np.diff(z, axis=-1)[valid[..., 1:]] >= 0)
    assert np.allclose(ba[valid].sum(-1), 1.0, atol=1e-5)
    # inclusion is decided without divisions; the stored distance may sit ~1e-10 above blur
    assert np.all(di[valid] < np.float32(w.blur_radius) * (1 + 1e-5))


def test_blend_matches_oracle_on_same_fragments():
    w = workloads.workload(1)
    d = to_dev(w.batch)
    fr, _, _, _ = gpu_fwd(d, w.image_size, w.K, np.float32(w.blur_radius), 16, True, True)
    p2f, zb, ba, di = fr
    faces = d["faces"]
    colors = torch.from_numpy(w.batch.colors).cuda()
    N, S, K = w.batch.N, w.image_size, w.K
    for mode in (ops.BLEND_SIL, ops.BLEND_RGB):
        bp = ops.make_blend_params(w.sigma, w.gamma, w.znear, w.zfar, (1.0, 1.0, 1.0), 1e-10, mode)
        img = torch.empty((N, S, S, 4), device="cuda")
        ops.blend_fwd(bp, N, S, K, p2f, zb, ba, di, faces, colors, img)
        fn = [x.cpu().numpy() for x in (p2f, zb, ba, di)]
        ref = oracle.blend_fwd(*fn, w.batch.faces, w.batch.colors, float(np.float32(w.sigma)),
                               float(np.float32(w.gamma)), float(np.float32(w.znear)), float(np.float32(w.zfar)),
                               mode=mode)
        err = np.max(np.abs(img.cpu().numpy() - ref))
        assert err <= 1e-5, err
        # backward: same fragments, same upstream gradient
        g = torch.from_numpy(workloads.upstream_grad(N, S, 3)).cuda()
        gd = torch.empty_like(di)
        gz = torch.empty_like(zb) if mode else None
        gb = torch.empty_like(ba) if mode else None
        gc = torch.empty_like(colors) if mode else None
        ops.blend_bwd(bp, N, S, K, p2f, zb, ba, di, faces, colors, g, gz, gb, gd, gc)
        rz, rb, rd, rc, ra, az, ab, ad = oracle.blend_bwd(
            *fn, w.batch.faces, w.batch.colors, g.cpu().numpy(), float(np.float32(w.sigma)),
            float(np.float32(w.gamma)), float(np.float32(w.znear)), float(np.float32(w.zfar)), mode=mode,
            with_abs=True)
        checks = [("grad_dists", gd, rd, ad)]
        if mode:
            checks += [("grad_zbuf", gz, rz, az), ("grad_bary", gb, rb, ab), ("grad_colors", gc, rc, ra)]
        for name, a, r, sc in checks:
            worst, glob = grad_close(a.cpu().numpy(), r, scale=sc)
            assert worst <= 1 and glob <= 1e-4, (mode, name, worst, glob)


def _rast_bwd_check(batch, S, K, blur, bin_size, persp, clip, seed=0):
    """GPU rasterizer adjoint against the FP64 adjoint conditioned on the GPU's own
    face selection, upstream gradients zeroed at gradient-ambiguous pixels."""
    d = to_dev(batch)
    fr, _, p, ws = gpu_fwd(d, S, K, blur, bin_size, persp, clip)
    p2f = fr[0]
    N = batch["first_face"].shape[0] if isinstance(batch, dict) else batch.N
    m = oracle_mesh(batch)
    amb = oracle.margins(m, S, K, blur, persp, clip) & oracle.GRAD_COND_AMBIGUOUS
    rng = np.random.default_rng(seed)
    P = N * S * S
    gz = rng.normal(size=(P, K)).astype(np.float32)
    gb = rng.normal(size=(P, K, 3)).astype(np.float32)
    gd = (rng.normal(size=(P, K)) * 1e3).astype(np.float32)
    for g in (gz, gb, gd):
        g[amb != 0] = 0
    # the forward these gradients are conditioned on matches the oracle
    orc_p2f = oracle.rasterize(m, S, K, blur, persp, clip)[0]
    fwd_ok = (oracle.margins(m, S, K, blur, persp, clip) & oracle.FWD_AMBIGUOUS) == 0
    gp = p2f.cpu().numpy().reshape(P, K)
    assert np.array_equal(gp[fwd_ok], orc_p2f[fwd_ok])
    gv = torch.empty_like(d["verts"])
    T = lambda a: torch.from_numpy(a).cuda().reshape(*p2f.shape, *a.shape[2:])
    ops.rast_mesh_bwd(p, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], p2f, T(gz), T(gb),
                      T(gd), gv, ws)
    ref, ref_abs = oracle.rast_bwd(m, S, K, gp, gz, gb, gd, blur, persp, clip, with_abs=True)
    assert_grad_close(gv.cpu().numpy(), ref, ref_abs, "rast_bwd")


@pytest.mark.parametrize("persp,clip,blur", [(True, True, BLUR), (True, False, BLUR), (False, True, BLUR),
                                             (True, False, 0.0)])
@pytest.mark.parametrize("bin_size", [0, 16])
def test_rast_bwd_matches_oracle_adjoint(persp, clip, blur, bin_size):
    b = workloads.sphere_batch([3, 2], 0.05, seed_base=123)
    _rast_bwd_check(b, 48, 4, blur, bin_size, persp, clip)


def test_rast_bwd_at_clip_kinks_of_outside_pixels():
    # pixels outside a face near its corner, where the clipped barycentrics are
    # (0, 0, 1): the adjoint must see the forward's double-float barycentrics
    # (fp32 ones can put a clamped component on the wrong side of zero)
    b = workloads.sphere_batch([3, 3], 0.05, seed_base=2024)
    _rast_bwd_check(b, 64, 4, BLUR, 16, True, True)


def test_rast_bwd_shared_vertices_across_images():
    # two images of ONE mesh: both images' faces index the same vertices
    v, f = workloads.displaced_sphere(2, 0.05, np.random.default_rng(3))
    cams = [workloads.look_at_camera(2.7, 10.0, 30.0), workloads.look_at_camera(2.7, -20.0, 200.0)]
    b = dict(verts=v.astype(np.float32), faces=np.concatenate([f, f]).astype(np.int64),
             first_face=np.array([0, f.shape[0]], np.int64), num_faces=np.array([f.shape[0]] * 2, np.int64),
             cams=np.stack(cams))
    _rast_bwd_check(b, 40, 3, BLUR, 8, True, True)


def test_status_bits_and_degenerate_inputs():
    b = workloads.sphere_batch([2, 2], 0.05, seed_base=9)
    # bad vertex index
    bb = dict(verts=b.verts, faces=b.faces.copy(), first_face=b.first_face, num_faces=b.num_faces, cams=b.cams)
    bb["faces"][3, 1] = b.V + 5
    _, st, _, _ = gpu_fwd(to_dev(bb), 32, 2, BLUR, 16)
    assert st & ops.ST_BAD_INDEX
    # non-finite vertex
    bb = dict(verts=b.verts.copy(), faces=b.faces, first_face=b.first_face, num_faces=b.num_faces, cams=b.cams)
    bb["verts"][4, 0] = np.nan
    fr, st, _, _ = gpu_fwd(to_dev(bb), 32, 2, BLUR, 16)
    assert st & ops.ST_NONFINITE
    assert np.isfinite(np_frags(fr)[1]).all()
    # bin overflow with a tiny capacity: error bit, no fault
    _, st, _, _ = gpu_fwd(to_dev(b), 64, 2, BLUR, 16, max_faces_per_bin=2)
    assert st & ops.ST_BIN_OVERFLOW
    _, st, _, _ = gpu_fwd(to_dev(b), 64, 2, BLUR, 16, max_faces_per_bin=4096, max_bin_entries=10)
    assert st & ops.ST_BIN_OVERFLOW
    # bad packing
    bb = dict(verts=b.verts, faces=b.faces, first_face=np.array([0, 10], np.int64),
              num_faces=np.array([20, 20], np.int64), cams=b.cams)
    _, st, _, _ = gpu_fwd(to_dev(bb), 32, 2, BLUR, 16)
    assert st & ops.ST_BAD_MESH_RANGE


def test_empty_batches_and_zero_face_meshes():
    b = workloads.sphere_batch([2], 0.05, seed_base=4)
    two = dict(verts=b.verts, faces=b.faces, first_face=np.array([0, 0], np.int64),
               num_faces=np.array([0, b.F], np.int64), cams=np.concatenate([b.cams, b.cams]))
    fr, st, _, _ = gpu_fwd(to_dev(two), 32, 2, BLUR, 16)
    assert st == 0
    p2f = np_frags(fr)[0]
    assert (p2f[0] == -1).all() and (p2f[1] >= 0).any()
    none = dict(verts=b.verts, faces=np.zeros((0, 3), np.int64), first_face=np.array([0], np.int64),
                num_faces=np.array([0], np.int64), cams=b.cams)
    fr, st, _, _ = gpu_fwd(to_dev(none), 16, 1, 0.0, 8)
    assert (np_frags(fr)[0] == -1).all()
    # N = 0: nothing to do, still a valid call
    zero = dict(verts=b.verts, faces=b.faces, first_face=np.zeros(0, np.int64), num_faces=np.zeros(0, np.int64),
                cams=np.zeros((0, 16), np.float32))
    gpu_fwd(to_dev(zero), 16, 1, 0.0, 8)


def test_sub_pixel_faces_keep_bary_precision():
    # a face spanning ~2 pixels at 1024^2 placed away from the origin: fp32
    # projection alone would lose ~1e-4 in the barycentrics
    S = 1024
    c = lambda i: 1.0 - (2.0 * i + 1.0) / S
    tri = ndc_triangle((c(700.3), c(300.2)), (c(702.9), c(300.6)), (c(701.1), c(302.8)), 2.7)
    tri = tri.astype(np.float32)
    sc = scene([tri])
    sc["cams"] = sc["cams"].astype(np.float32)
    d = to_dev(sc)
    fr, st, _, _ = gpu_fwd(d, S, 1, 0.0, 16, True, False)
    px = np.array([[0, r, cc] for r in range(298, 306) for cc in range(698, 706)])
    m = oracle_mesh(sc)
    orc = oracle.rasterize(m, S, 1, 0.0, True, False, pixels=px)
    amb = oracle.margins(m, S, 1, 0.0, True, False, pixels=px) & oracle.FWD_AMBIGUOUS
    n_amb, n_bad = compare_frags(pick(np_frags(fr), px, S), orc, amb, atol=2e-6)
    assert n_bad == 0
    assert (orc[0] >= 0).sum() >= 2


def test_autotuner_picks_a_non_overflowing_configuration():
    from paper_2007_08501_gb300 import tune
    w = workloads.workload(1)
    d = to_dev(w.batch)
    best = tune.tune(d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], w.image_size, w.K,
                     BLUR, True, True, use_cache=False)
    assert best["bin_size"] in (8, 16)
    fr, st, _, _ = gpu_fwd(d, w.image_size, w.K, BLUR, best["bin_size"], True, True, best["max_faces_per_bin"],
                           best["max_bin_entries"])
    assert st == 0
