"""The benchmark's other workloads at full size, in the launch configuration the
autotuner picks, against the FP64 oracle on a seeded pixel sample:

  * 32 icospheres of levels 3..7 (heterogeneous packed batch), 512x512, K=4,
    soft silhouette;
  * 1 icosphere of 1.31M faces at 1024x1024, K=1 hard and K=8 soft;
  * 1 icosphere of 81,920 faces seen by 20 cameras (all images share the
    vertices), 512x512, K=50, soft silhouette.

Each runs forward, silhouette blend, blend adjoint and rasterizer adjoint over
the whole batch on the GPU; the upstream gradient is non-zero only at the
sampled, unambiguous pixels, so the vertex gradient can be checked against the
oracle adjoint evaluated at those pixels alone.  The sample is 256 pixels per
image (half of them in the central region the meshes cover); the oracle runs
over it in one spawned process per host core.
"""
import numpy as np
import pytest
import torch

import oracle
from _gpu import OraclePool, assert_grad_close, compare_frags, np_frags, oracle_mesh, pick, to_dev
from paper_2007_08501_gb300 import ops, tune, workloads

pytestmark = pytest.mark.gpu


def _sample(N, S, per_image, seed, centre=0.6):
    """Seeded pixels, per image: half anywhere, half in the central region."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi = int(S * (1 - centre) / 2), int(S * (1 + centre) / 2)
    for n in range(N):
        a = rng.integers(0, S, size=(per_image // 2, 2))
        b = rng.integers(lo, hi, size=(per_image - per_image // 2, 2))
        rc = np.unique(np.concatenate([a, b]), axis=0)
        out.append(np.concatenate([np.full((rc.shape[0], 1), n), rc], 1))
    return np.concatenate(out).astype(np.int64)


def _run(w, per_image, seed, check_grad=True):
    b = w.batch
    S, K = w.image_size, w.K
    blur = float(np.float32(w.blur_radius))
    persp, clip = w.perspective_correct, w.clip_barycentric_coords
    d = to_dev(b)
    best = tune.tune(d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], S, K, blur, persp, clip,
                     use_cache=False)
    p = ops.make_rast_params(b.N, S, K, blur, best["bin_size"], best["max_faces_per_bin"], persp, clip,
                             best["max_bin_entries"])
    ws = ops.alloc_workspace(p, b.V, b.F)
    frags = ops.alloc_fragments(b.N, S, K)
    ops.rast_mesh_fwd(p, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], *frags, ws)
    assert ops.rast_query_status(ws) == 0
    px = _sample(b.N, S, per_image, seed)
    m = oracle_mesh(b)
    pool = OraclePool(m)
    try:
        _check(w, b, d, p, ws, frags, px, pool, S, K, blur, persp, clip, seed, check_grad)
    finally:
        pool.close()


def _check(w, b, d, p, ws, frags, px, pool, S, K, blur, persp, clip, seed, check_grad):
    orc = pool.rasterize(S, K, blur, persp, clip, px)
    flags = pool.margins(S, K, blur, persp, clip, px)
    got = pick(np_frags(frags), px, S)
    n_amb, n_bad = compare_frags(got, orc, flags & oracle.FWD_AMBIGUOUS)
    assert n_bad == 0
    assert (orc[0] >= 0).any()
    # silhouette blend on the GPU's fragments
    bp = ops.make_blend_params(w.sigma, w.gamma, w.znear, w.zfar, (1.0, 1.0, 1.0), 1e-10, ops.BLEND_SIL)
    img = torch.empty((b.N, S, S, 4), device="cuda")
    p2f, zb, ba, di = frags
    ops.blend_fwd(bp, b.N, S, K, p2f, None, None, di, None, None, img)
    gfr = got
    ref_img = oracle.blend_fwd(gfr[0], gfr[1], gfr[2], gfr[3], None, None, float(np.float32(w.sigma)),
                               float(np.float32(w.gamma)), float(np.float32(w.znear)), float(np.float32(w.zfar)),
                               mode=0)
    assert np.max(np.abs(pick([img.cpu().numpy()], px, S)[0] - ref_img)) <= 1e-5
    if not check_grad:
        return
    # adjoints, with the upstream gradient restricted to sampled, unambiguous pixels
    keep = (flags & oracle.GRAD_COND_AMBIGUOUS) == 0
    assert keep.sum() >= 0.5 * keep.size
    rng = np.random.default_rng(seed + 1)
    gsel = np.zeros((px.shape[0], 4), np.float32)
    gsel[:, 3] = rng.normal(size=px.shape[0]).astype(np.float32) * keep
    gimg = torch.zeros((b.N, S, S, 4), device="cuda")
    gimg[px[:, 0], px[:, 1], px[:, 2]] = torch.from_numpy(gsel).cuda()
    gd = torch.empty_like(di)
    ops.blend_bwd(bp, b.N, S, K, p2f, None, None, di, None, None, gimg, None, None, gd, None)
    gv = torch.empty_like(d["verts"])
    ops.rast_mesh_bwd(p, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], p2f, None, None, gd,
                      gv, ws)
    _, _, rd, _ = oracle.blend_bwd(gfr[0], gfr[1], gfr[2], gfr[3], None, None, gsel, float(np.float32(w.sigma)),
                                   float(np.float32(w.gamma)), float(np.float32(w.znear)),
                                   float(np.float32(w.zfar)), mode=0, V=1)
    ref, ref_abs = pool.rast_bwd(S, K, gfr[0], None, None, rd, blur, persp, clip, px)
    assert np.abs(ref).max() > 0
    worst, glob, n_over = assert_grad_close(gv.cpu().numpy(), ref, ref_abs, w.name)
    print("%s: ambiguous %d / %d pixels, grad worst %.2f, global %.2e, over 1e-4: %d"
          % (w.name, n_amb, px.shape[0], worst, glob, n_over))
    # the fused backward the benchmark step runs (blend adjoint pulled straight
    # through the rasterizer adjoint), against the same oracle adjoint
    gv2 = torch.empty_like(d["verts"])
    ops.blend_rast_bwd(p, bp, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], p2f, None, None,
                       di, None, gimg, gv2, None, ws)
    assert_grad_close(gv2.cpu().numpy(), ref, ref_abs, w.name + " fused")


def test_heterogeneous_batch_of_32_meshes_512():
    _run(workloads.workload(2), per_image=256, seed=20)


@pytest.mark.parametrize("variant", ["hard", "soft"])
def test_large_mesh_1024(variant):
    _run(workloads.workload(3, variant), per_image=256, seed=30)


def test_twenty_views_shared_vertices_k50():
    _run(workloads.workload(4), per_image=256, seed=40)
