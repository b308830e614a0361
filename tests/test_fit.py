"""Analysis-by-synthesis loop: the silhouette IoU loss of Appendix B and the
graph-captured fitting step (20 views of one mesh, 512x512, K = 50)."""
import numpy as np
import pytest
import torch

from paper_2007_08501_gb300 import workloads


def test_iou_loss_limits():
    from paper_2007_08501_gb300.fit import iou_loss
    a = torch.rand(3, 8, 8)
    assert float(iou_loss(a, a > 2)) == pytest.approx(1.0)            # empty target: nothing overlaps
    m = (torch.rand(2, 8, 8) > 0.5).float()
    assert float(iou_loss(m, m)) == pytest.approx(0.0, abs=1e-7)      # identical binary masks
    assert float(iou_loss(m, 1 - m)) == pytest.approx(1.0)            # disjoint masks
    half = torch.zeros(1, 4, 4); half[0, :2] = 1
    full = torch.ones(1, 4, 4)
    assert float(iou_loss(half, full)) == pytest.approx(0.5)          # IoU = 8/16


def _fitter(views=20, S=512, K=50):
    from paper_2007_08501_gb300 import autograd as ag
    from paper_2007_08501_gb300.fit import SilhouetteFitter
    w = workloads.workload(4)
    dev = "cuda"
    F0 = int(w.batch.num_faces[0])
    verts = torch.from_numpy(w.batch.verts).to(dev)
    faces0 = torch.from_numpy(w.batch.faces[:F0]).to(dev)
    cams = torch.from_numpy(w.batch.cams[:views]).to(dev)
    rs = ag.RasterSettings(S, K, float(np.float32(w.blur_radius)), bin_size=8, max_faces_per_bin=4096,
                           clip_barycentric_coords=True)
    bs = ag.BlendSettings(sigma=w.sigma, gamma=w.gamma, rgb=False)
    tv, tf = workloads.target_sphere()
    tverts = torch.from_numpy(tv.astype(np.float32)).to(dev)
    tfaces = torch.from_numpy(tf.astype(np.int64)).to(dev).repeat(views, 1)
    ff = torch.arange(views, device=dev, dtype=torch.int64) * tf.shape[0]
    nf = torch.full((views,), tf.shape[0], device=dev, dtype=torch.int64)
    with torch.no_grad():
        target = ag.blend(*ag.rasterize_meshes(tverts, tfaces, ff, nf, cams, rs), settings=bs)[..., 3].clone()
    return SilhouetteFitter(verts, faces0, cams, target, rs, bs, lr=2e-3)


@pytest.mark.gpu
def test_graph_replay_equals_eager_step_and_loss_decreases():
    a = _fitter()
    for _ in range(4):
        la = float(a.eager_step())
    b = _fitter().capture(warmup=3)
    lb = float(b.replay(1))
    assert abs(la - lb) <= 1e-5 * max(1.0, abs(la)), (la, lb)
    l0 = lb
    l_end = float(b.replay(40))
    assert np.isfinite(l_end) and l_end < 0.99 * l0, (l0, l_end)
    assert b.ws.status() == 0
