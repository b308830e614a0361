"""Point-cloud path (include/points.h) against the FP64 point oracle, element by
element: idx bit-exact on every pixel whose rim / depth-tie / znear margins
exceed 1e-6 (the rest are counted), zbuf and dists within 1e-5; compositing
within 1e-5; gradients within 1e-4 relative of the oracle adjoint conditioned
on the same selection."""
import numpy as np
import pytest
import torch

from _gpu import assert_grad_close, grad_close
from oracle import points as op
from paper_2007_08501_gb300 import ops, workloads

pytestmark = pytest.mark.gpu


def _dev(b):
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dict(points=T(b.points), first=T(b.first_point), num=T(b.num_points), cams=T(b.cams),
                feats=T(b.features))


def _fwd(d, N, S, K, r, bin_size, max_per_bin=8192, max_entries=0):
    p = ops.make_pts_params(N, S, K, r, bin_size, max_per_bin, max_entries)
    ws = ops.alloc_pts_workspace(p, d["points"].shape[0])
    fr = ops.alloc_pts_fragments(N, S, K)
    ops.pts_rasterize_fwd(p, d["points"], d["first"], d["num"], d["cams"], *fr, ws)
    return fr, ops.rast_query_status(ws), p, ws


def _compare(got, orc, flags):
    gi, gz, gd = [x.cpu().numpy().reshape(orc[0].shape) for x in got]
    oi, oz, od = orc
    ok = (flags & op.FWD_AMBIGUOUS) == 0
    assert np.array_equal(gi[ok], oi[ok]), np.argwhere(np.any(gi != oi, axis=1) & ok)[:5]
    same = (gi == oi) & (oi >= 0)
    assert np.all(gz[oi < 0] == -1) and np.all(gd[oi < 0] == -1)
    assert np.max(np.abs(gz[same] - oz[same]), initial=0) <= 1e-5
    assert np.max(np.abs(gd[same] - od[same]), initial=0) <= 1e-5
    return int((~ok).sum())


@pytest.mark.parametrize("S,K,r,bin_size", [
    (64, 4, 0.04, 16),
    (70, 8, 0.03, 8),      # ragged: 70 = 4 * 16 + 6
    (48, 1, 0.05, 0),      # plain form
    (64, 10, 0.04, 16),    # K > 8, shared-memory lists
    (40, 50, 0.06, 8),     # K = 50 as in the benchmark
])
def test_fragments_match_oracle(S, K, r, bin_size):
    b = workloads.point_batch([3000, 500, 8000], 31, level=3)
    d = _dev(b)
    fr, st, _, _ = _fwd(d, b.N, S, K, r, bin_size)
    assert st == 0
    c = op.Clouds.from_batch(b)
    orc = op.rasterize(c, S, K, float(np.float32(r)))
    fl = op.margins(c, S, K, float(np.float32(r)))
    n_amb = _compare(fr, orc, fl)
    assert n_amb <= 0.05 * fl.size
    assert (orc[0] >= 0).any()


@pytest.mark.parametrize("K", [2, 8, 24])
def test_binned_equals_plain(K):
    b = workloads.point_batch([4000, 9000], 7, level=4)
    d = _dev(b)
    ref = [x.cpu() for x in _fwd(d, b.N, 60, K, 0.035, 0)[0]]
    for bs in (8, 16):
        got = [x.cpu() for x in _fwd(d, b.N, 60, K, 0.035, bs)[0]]
        for x, y in zip(ref, got):
            assert torch.equal(x, y)


@pytest.mark.parametrize("mode", [ops.PTS_ALPHA, ops.PTS_NORM])
@pytest.mark.parametrize("D", [1, 3])
def test_compositing_and_its_adjoint_match_oracle(mode, D):
    b = workloads.point_batch([3000, 6000], 19, level=3, D=D)
    d = _dev(b)
    S, K, r = 56, 8, 0.04
    (idx, zb, di), st, p, _ = _fwd(d, b.N, S, K, r, 16)
    assert st == 0
    img = torch.empty((b.N, S, S, D), device="cuda")
    ops.pts_composite_fwd(p, mode, idx, di, d["feats"], img)
    fi, fd = idx.cpu().numpy(), di.cpu().numpy()
    ref = op.composite_fwd(fi.reshape(-1, K), fd.reshape(-1, K), b.features, np.float32(r), mode)
    assert np.max(np.abs(img.cpu().numpy().reshape(-1, D) - ref)) <= 1e-5
    g = torch.from_numpy(np.random.default_rng(3).normal(size=(b.N, S, S, D)).astype(np.float32)).cuda()
    gd = torch.empty_like(di)
    gf = torch.empty_like(d["feats"])
    ops.pts_composite_bwd(p, mode, idx, di, d["feats"], g, gd, gf)
    rd, rf, ra, rda = op.composite_bwd(fi.reshape(-1, K), fd.reshape(-1, K), b.features, np.float32(r),
                                       g.cpu().numpy().reshape(-1, D), mode, with_abs=True)
    w, glob = grad_close(gf.cpu().numpy(), rf, scale=ra)
    assert w <= 1 and glob <= 1e-4, (w, glob)
    # per slot, relative to the magnitudes of the terms (Norm of equal features has an
    # exactly zero gradient, which fp32 meets only to its rounding of those terms)
    w, _ = grad_close(gd.cpu().numpy().reshape(-1, K), rd, scale=rda)
    assert w <= 1, w
    if np.abs(rd).max() > 0:
        assert np.linalg.norm(gd.cpu().numpy().reshape(-1, K) - rd) <= 1e-4 * max(np.linalg.norm(rd), 1e-3 * np.linalg.norm(rda))


@pytest.mark.parametrize("bin_size", [0, 16])
def test_rasterizer_adjoint_matches_oracle(bin_size):
    b = workloads.point_batch([2500, 4000], 23, level=3)
    d = _dev(b)
    S, K, r = 48, 6, 0.05
    (idx, zb, di), st, p, ws = _fwd(d, b.N, S, K, r, bin_size)
    assert st == 0
    c = op.Clouds.from_batch(b)
    amb = op.margins(c, S, K, float(np.float32(r))) & op.GRAD_COND_AMBIGUOUS
    rng = np.random.default_rng(4)
    npix = b.N * S * S
    gz = rng.normal(size=(npix, K)).astype(np.float32)
    gdd = (rng.normal(size=(npix, K)) * 1e2).astype(np.float32)
    gz[amb != 0] = 0
    gdd[amb != 0] = 0
    gp = torch.empty_like(d["points"])
    T = lambda a: torch.from_numpy(a).cuda().reshape(idx.shape)
    ops.pts_rasterize_bwd(p, d["points"], d["first"], d["num"], d["cams"], idx, T(gz), T(gdd), gp, ws)
    ref, ref_abs = op.rast_bwd(c, S, K, idx.cpu().numpy().reshape(npix, K), gz, gdd, with_abs=True)
    assert np.abs(ref).max() > 0
    assert_grad_close(gp.cpu().numpy(), ref, ref_abs, "pts_rasterize_bwd")


def test_benchmark_clouds_sampled_pixels_at_full_size():
    w = workloads.point_workload()
    b = w.batch
    d = _dev(b)
    fr, st, p, ws = _fwd(d, b.N, w.image_size, w.K, w.radius, 16, max_per_bin=8192)
    assert st == 0
    px = workloads.sample_pixels(b.N, w.image_size, 24, 77)
    c = op.Clouds.from_batch(b)
    orc = op.rasterize(c, w.image_size, w.K, np.float32(w.radius), pixels=px)
    fl = op.margins(c, w.image_size, w.K, np.float32(w.radius), pixels=px)
    S = w.image_size
    sel = lambda t: t.cpu().numpy()[px[:, 0], px[:, 1], px[:, 2]]
    n_amb = _compare([torch.from_numpy(sel(x)) for x in fr], orc, fl)
    assert n_amb <= 0.2 * px.shape[0]
    assert (orc[0][:, -1] >= 0).any()    # some pixels hold the full K = 50


def test_status_bits_and_empty_inputs():
    b = workloads.point_batch([500, 500], 3, level=2)
    d = _dev(b)
    _, st, _, _ = _fwd(d, b.N, 32, 4, 0.05, 16, max_per_bin=2)
    assert st & ops.ST_BIN_OVERFLOW
    bad = dict(d)
    bad["points"] = d["points"].clone()
    bad["points"][7, 1] = float("nan")
    fr, st, _, _ = _fwd(bad, b.N, 32, 4, 0.05, 16)
    assert st & ops.ST_NONFINITE
    assert not (fr[0] == 7).any()
    bad = dict(d)
    bad["first"] = torch.tensor([0, 100], device="cuda")
    _, st, _, _ = _fwd(bad, b.N, 32, 4, 0.05, 16)
    assert st & ops.ST_BAD_MESH_RANGE
    empty = dict(d)
    empty["num"] = torch.zeros(2, dtype=torch.int64, device="cuda")
    empty["first"] = torch.zeros(2, dtype=torch.int64, device="cuda")
    fr, st, _, _ = _fwd(empty, b.N, 32, 4, 0.05, 8)
    assert st == 0 and bool((fr[0] == -1).all())


def test_render_points_autograd_equals_the_calls():
    from paper_2007_08501_gb300 import autograd as ag
    b = workloads.point_batch([3000, 5000], 41, level=3, D=3)
    d = _dev(b)
    st = ag.PointSettings(image_size=48, points_per_pixel=8, radius=0.05, bin_size=16, mode=ops.PTS_ALPHA)
    pts = d["points"].clone().requires_grad_(True)
    feats = d["feats"].clone().requires_grad_(True)
    img = ag.render_points(pts, feats, d["first"], d["num"], d["cams"], st)
    g = torch.from_numpy(np.random.default_rng(8).normal(size=tuple(img.shape)).astype(np.float32)).cuda()
    (img * g).sum().backward()
    (idx, zb, di), status, p, ws = _fwd(d, b.N, 48, 8, 0.05, 16)
    assert status == 0
    ref = torch.empty_like(img)
    ops.pts_composite_fwd(p, ops.PTS_ALPHA, idx, di, d["feats"], ref)
    assert torch.equal(ref, img.detach())
    gd, gf = torch.empty_like(di), torch.empty_like(d["feats"])
    ops.pts_composite_bwd(p, ops.PTS_ALPHA, idx, di, d["feats"], g, gd, gf)
    gp = torch.empty_like(d["points"])
    ops.pts_rasterize_bwd(p, d["points"], d["first"], d["num"], d["cams"], idx, None, gd, gp, ws)
    # the same kernels both ways; the float atomics may add in another order
    assert torch.linalg.norm(feats.grad - gf) <= 1e-5 * torch.linalg.norm(gf)
    assert torch.linalg.norm(pts.grad - gp) <= 1e-5 * torch.linalg.norm(gp)
