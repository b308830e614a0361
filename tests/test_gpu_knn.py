"""Exact KNN and the Chamfer loss on the GPU against the CPU oracle
(``oracle/knn.c``, ``oracle/knn.py``).

Neighbour rows and their fp32 distances are bit-exact: both sides rank in
fp32 with the same evaluation order and the same tie-break.  Chamfer losses
agree within 1e-5 relative (the GPU sums fp32 distances in FP64; the oracle
evaluates Eq. 1 in FP64 from the same fp32 coordinates); gradients within
1e-4 relative (fp32 arithmetic and atomics), per component against 1e-2 of
their rms where they sum terms of both signs."""
import numpy as np
import pytest
import torch

from _gpu import grad_close
from oracle import knn as ok
from paper_2007_08501_gb300 import autograd as ag
from paper_2007_08501_gb300 import ops, workloads

pytestmark = pytest.mark.gpu


def _batch(rng, lens, D, scale=1.0):
    lens = np.asarray(lens, np.int64)
    first = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    return (rng.normal(size=(int(lens.sum()), D)) * scale).astype(np.float32), first, lens


def _T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_knn(p1, f1, l1, p2, f2, l2, K):
    P1 = p1.shape[0]
    idx = torch.full((P1, K), -7, dtype=torch.int64, device="cuda")
    dist = torch.full((P1, K), -7.0, dtype=torch.float32, device="cuda")
    ws = ops.alloc_knn_workspace(len(f1))
    ops.knn_points(_T(p1), _T(f1), _T(l1), _T(p2), _T(f2), _T(l2), K, idx, dist, ws)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


def _assert_same(gi, gd, ri, rd):
    np.testing.assert_array_equal(gi, ri)
    np.testing.assert_array_equal(gd.view(np.uint32), rd.view(np.uint32))


@pytest.mark.parametrize("D", [1, 2, 3, 4])
@pytest.mark.parametrize("K", [1, 2, 5, 8, 16, 32])
def test_knn_heterogeneous_batch_bit_exact(D, K):
    # empty clouds on either side, a candidate cloud smaller than K, ragged
    # query tiles, candidate clouds spanning several shared-memory chunks
    rng = np.random.default_rng(100 * D + K)
    p1, f1, l1 = _batch(rng, [300, 0, 1500, 7, 64], D)
    p2, f2, l2 = _batch(rng, [5000, 10, 0, 4100, 3], D)
    gi, gd = _gpu_knn(p1, f1, l1, p2, f2, l2, K)
    ri, rd = ok.knn(p1, f1, l1, p2, f2, l2, K)
    _assert_same(gi, gd, ri, rd)


@pytest.mark.parametrize("K", [1, 8, 32])
def test_knn_few_queries_many_candidates(K):
    # K = 1: 32 lanes share each query (wide groups) and merge their lists;
    # K >= 5: every lane on its own queries, lists inserted into by the warp
    rng = np.random.default_rng(K)
    p1, f1, l1 = _batch(rng, [40, 33], 3)
    p2, f2, l2 = _batch(rng, [40_000, 41_111], 3)
    _assert_same(*_gpu_knn(p1, f1, l1, p2, f2, l2, K), *ok.knn(p1, f1, l1, p2, f2, l2, K))


@pytest.mark.parametrize("K", [1, 4])
def test_knn_many_queries_few_candidates(K):
    # one lane per query group
    rng = np.random.default_rng(40 + K)
    p1, f1, l1 = _batch(rng, [3000, 2500, 1, 3100], 3)
    p2, f2, l2 = _batch(rng, [400, 300, 5, 333], 3)
    _assert_same(*_gpu_knn(p1, f1, l1, p2, f2, l2, K), *ok.knn(p1, f1, l1, p2, f2, l2, K))


def test_knn_ties_and_lattices():
    # integer lattices: many exactly equal distances; ranking by candidate row
    g = np.stack(np.meshgrid(np.arange(9.0), np.arange(7.0), np.arange(5.0)), -1).reshape(-1, 3).astype(np.float32)
    q = (g[::3] + np.float32(0.5)).astype(np.float32)
    f1, l1 = np.array([0]), np.array([len(q)])
    f2, l2 = np.array([0]), np.array([len(g)])
    for K in (1, 6, 27):
        _assert_same(*_gpu_knn(q, f1, l1, g, f2, l2, K), *ok.knn(q, f1, l1, g, f2, l2, K))


@pytest.mark.parametrize("kind", ["knn", "knn_het"])
def test_knn_benchmark_workloads_on_sampled_rows(kind):
    # the benchmark's batches and launch configuration, checked on 16 seeded query rows per cloud
    w = workloads.knn_workload(kind)
    c = w.pairs
    gi, gd = _gpu_knn(c.p, c.first1, c.len1, c.q, c.first2, c.len2, w.K)
    rng = np.random.default_rng(3)
    rows = np.concatenate([f + rng.choice(n, size=min(16, n), replace=False) for f, n in zip(c.first1, c.len1)])
    ri, rd = ok.knn(c.p, c.first1, c.len1, c.q, c.first2, c.len2, w.K, rows=rows)
    _assert_same(gi[rows], gd[rows], ri, rd)


def _gpu_chamfer(p, f1, l1, q, f2, l2, g_per=None, g_loss=None):
    N = len(f1)
    out = dict(idx_pq=torch.empty(p.shape[0], dtype=torch.int64, device="cuda"),
               d_pq=torch.empty(p.shape[0], device="cuda"),
               idx_qp=torch.empty(q.shape[0], dtype=torch.int64, device="cuda"),
               d_qp=torch.empty(q.shape[0], device="cuda"), per=torch.full((N,), -1.0, device="cuda"),
               loss=torch.full((1,), -1.0, device="cuda"))
    ws = ops.alloc_knn_workspace(N)
    P, Q = _T(p), _T(q)
    F1, L1, F2, L2 = _T(f1), _T(l1), _T(f2), _T(l2)
    ops.chamfer_fwd(P, F1, L1, Q, F2, L2, out["idx_pq"], out["d_pq"], out["idx_qp"], out["d_qp"], out["per"],
                    out["loss"], ws)
    gp, gq = torch.full_like(P, 5.0), torch.full_like(Q, 5.0)
    ops.chamfer_bwd(P, F1, L1, Q, F2, L2, out["idx_pq"], out["idx_qp"],
                    None if g_loss is None else _T(np.asarray([g_loss], np.float32)),
                    None if g_per is None else _T(np.asarray(g_per, np.float32)), gp, gq)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["gp"], res["gq"] = gp.cpu().numpy(), gq.cpu().numpy()
    return res


def test_chamfer_loss_and_gradients_match_oracle():
    rng = np.random.default_rng(9)
    p, f1, l1 = _batch(rng, [100, 0, 64, 900, 5, 3], 3)
    q, f2, l2 = _batch(rng, [3000, 7, 0, 2500, 1, 2600], 3)
    g_per = rng.normal(size=6)
    r = _gpu_chamfer(p, f1, l1, q, f2, l2, g_per=g_per, g_loss=0.75)
    loss, per, ipq, iqp = ok.chamfer(p, f1, l1, q, f2, l2)
    np.testing.assert_array_equal(r["idx_pq"], ipq)
    np.testing.assert_array_equal(r["idx_qp"], iqp)
    assert np.all(np.abs(r["per"] - per) <= 1e-5 * np.abs(per) + 1e-12), (r["per"], per)
    assert abs(r["loss"][0] - loss) <= 1e-5 * abs(loss)
    w = g_per + 0.75 / 6
    gp, gq = ok.chamfer_grad(p, f1, l1, q, f2, l2, ipq, iqp, w)
    for name, a, ref in (("grad_p", r["gp"], gp), ("grad_q", r["gq"], gq)):
        worst, glob = grad_close(a, ref)
        assert glob <= 1e-4 and worst <= 1, (name, worst, glob)


def test_chamfer_edge_cases():
    rng = np.random.default_rng(1)
    # every cloud empty on one side: no neighbours, zero loss, zero gradient
    p, f1, l1 = _batch(rng, [5, 0], 2)
    q, f2, l2 = _batch(rng, [0, 4], 2)
    r = _gpu_chamfer(p, f1, l1, q, f2, l2, g_per=[1.0, 1.0])
    assert (r["idx_pq"] == -1).all() and (r["idx_qp"] == -1).all() and np.isinf(r["d_pq"]).all()
    assert (r["per"] == 0).all() and r["loss"][0] == 0 and (r["gp"] == 0).all() and (r["gq"] == 0).all()
    # no clouds at all
    z = np.zeros((0, 3), np.float32)
    e = np.zeros(0, np.int64)
    r = _gpu_chamfer(z, e, e, z, e, e, g_loss=1.0)
    assert r["loss"][0] == 0


def test_knn_backward_and_autograd():
    rng = np.random.default_rng(12)
    p1, f1, l1 = _batch(rng, [50, 80], 3)
    p2, f2, l2 = _batch(rng, [30, 3], 3)
    K = 5
    P1 = _T(p1).requires_grad_(True)
    P2 = _T(p2).requires_grad_(True)
    dists, idx = ag.knn_points(P1, _T(f1), _T(l1), P2, _T(f2), _T(l2), K)
    g = rng.normal(size=(p1.shape[0], K)).astype(np.float32)
    valid = idx >= 0
    (torch.where(valid, dists, torch.zeros_like(dists)) * _T(g)).sum().backward()
    ri, _ = ok.knn(p1, f1, l1, p2, f2, l2, K)
    np.testing.assert_array_equal(idx.cpu().numpy(), ri)
    g1, g2 = ok.knn_grad(p1, p2, ri, np.where(ri >= 0, g, 0.0))
    for a, ref in ((P1.grad, g1), (P2.grad, g2)):
        worst, glob = grad_close(a.cpu().numpy(), ref)
        assert glob <= 1e-4 and worst <= 1


def test_chamfer_autograd_matches_the_direct_calls():
    rng = np.random.default_rng(13)
    p, f1, l1 = _batch(rng, [200, 150], 3)
    q, f2, l2 = _batch(rng, [300, 90], 3)
    P = _T(p).requires_grad_(True)
    Q = _T(q).requires_grad_(True)
    loss, per = ag.chamfer_distance(P, _T(f1), _T(l1), Q, _T(f2), _T(l2))
    (2.0 * loss + (per * _T(np.array([0.5, -1.0], np.float32))).sum()).backward()
    r = _gpu_chamfer(p, f1, l1, q, f2, l2, g_per=[0.5, -1.0], g_loss=2.0)
    # the same kernels both ways; the float atomics may add in another order
    for got, want in ((P.grad, _T(r["gp"])), (Q.grad, _T(r["gq"]))):
        assert torch.linalg.norm(got - want) <= 1e-6 * torch.linalg.norm(want)
    assert float(loss) == pytest.approx(float(r["loss"][0]), rel=1e-7)


def test_chamfer_benchmark_batch_in_full():
    # the benchmark's Chamfer batch (32 pairs of 1,000 and 50,000 points), every
    # neighbour both ways bit-exact, per-pair losses and both gradients
    w = workloads.knn_workload("chamfer")
    c = w.pairs
    N = c.N
    rng = np.random.default_rng(w.grad_seed)
    g_per = rng.normal(size=N)
    r = _gpu_chamfer(c.p, c.first1, c.len1, c.q, c.first2, c.len2, g_per=g_per, g_loss=1.0)
    loss, per, ipq, iqp = ok.chamfer(c.p, c.first1, c.len1, c.q, c.first2, c.len2)
    np.testing.assert_array_equal(r["idx_pq"], ipq)
    np.testing.assert_array_equal(r["idx_qp"], iqp)
    assert np.all(np.abs(r["per"] - per) <= 1e-5 * np.abs(per)), np.max(np.abs(r["per"] - per) / np.abs(per))
    assert abs(r["loss"][0] - loss) <= 1e-5 * abs(loss)
    gp, gq = ok.chamfer_grad(c.p, c.first1, c.len1, c.q, c.first2, c.len2, ipq, iqp, g_per + 1.0 / N)
    for name, a, ref in (("grad_p", r["gp"], gp), ("grad_q", r["gq"], gq)):
        worst, glob = grad_close(a, ref)
        assert glob <= 1e-4 and worst <= 1, (name, worst, glob)
