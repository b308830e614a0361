"""Helpers for the GPU parity tests: run the C-ABI path on a packed batch and
compare it with the FP64 oracle on the same inputs."""
import numpy as np
import torch

import oracle
from paper_2007_08501_gb300 import ops

DEV = "cuda"


def to_dev(b):
    """numpy batch (dict or MeshBatch) -> CUDA tensors"""
    g = (lambda k: b[k]) if isinstance(b, dict) else (lambda k: getattr(b, k))
    return dict(verts=torch.from_numpy(np.ascontiguousarray(g("verts"), np.float32)).to(DEV),
                faces=torch.from_numpy(np.ascontiguousarray(g("faces"), np.int64)).to(DEV),
                first_face=torch.from_numpy(np.ascontiguousarray(g("first_face"), np.int64)).to(DEV),
                num_faces=torch.from_numpy(np.ascontiguousarray(g("num_faces"), np.int64)).to(DEV),
                cams=torch.from_numpy(np.ascontiguousarray(g("cams"), np.float32)).to(DEV))


def oracle_mesh(b):
    """The oracle sees exactly the fp32 values the GPU sees, upcast."""
    g = (lambda k: b[k]) if isinstance(b, dict) else (lambda k: getattr(b, k))
    return oracle.Mesh(np.asarray(g("verts"), np.float32), g("faces"), g("first_face"), g("num_faces"),
                       np.asarray(g("cams"), np.float32))


def gpu_fwd(d, S, K, blur, bin_size=16, persp=True, clip=False, max_faces_per_bin=4096, max_bin_entries=0):
    N = d["first_face"].shape[0]
    p = ops.make_rast_params(N, S, K, np.float32(blur), bin_size, max_faces_per_bin, persp, clip, max_bin_entries)
    ws = ops.alloc_workspace(p, d["verts"].shape[0], d["faces"].shape[0])
    p2f, zb, ba, di = ops.alloc_fragments(N, S, K)
    ops.rast_mesh_fwd(p, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], p2f, zb, ba, di, ws)
    status = ops.rast_query_status(ws)
    return (p2f, zb, ba, di), status, p, ws


def np_frags(fr):
    return [t.detach().cpu().numpy() for t in fr]


def compare_frags(gpu, orc, amb, atol=1e-5):
    """pix_to_face bit-exact on unambiguous pixels; zbuf, bary, dists within atol
    wherever the face ids agree (except the flag-128 slots, which are counted
    and printed).  Returns (#ambiguous, #mismatched unambiguous)."""
    gp, gz, gb, gd = [np.asarray(x) for x in gpu]
    op, oz, ob, od = orc
    P, K = op.shape
    gp = gp.reshape(P, K)
    gz = gz.reshape(P, K)
    gb = gb.reshape(P, K, 3)
    gd = gd.reshape(P, K)
    ok = amb == 0
    bad = np.nonzero(np.any(gp[ok] != op[ok], axis=1))[0]
    # slots whose values are not compared: the unclipped extrapolations the
    # oracle marks as ill-conditioned for fp32 (flag 128), counted and shown
    n128 = int((((amb & 128) != 0)[:, None] & (gp == op) & (op >= 0)).sum())
    same = gp == op
    # empty slots carry exactly -1
    empty = op < 0
    assert np.all(gz[empty & same] == -1) and np.all(gd[empty & same] == -1)
    # values wherever the ids agree, except where the oracle marks the depth
    # extrapolation as ill-conditioned for fp32 (flag 128)
    v = same & ~empty & ((amb & 128) == 0)[:, None]
    if v.any():
        ez = np.max(np.abs(gz[v] - oz[v]))
        eb = np.max(np.abs(gb[v] - ob[v]))
        ed = np.max(np.abs(gd[v] - od[v]))

        def where(err):
            e = np.where(v, err, -1.0)
            i = np.unravel_index(np.argmax(e), e.shape)
            return dict(slot=tuple(int(x) for x in i), face=int(op[i]), gpu_z=float(gz[i]), orc_z=float(oz[i]),
                        gpu_b=gb[i].tolist(), orc_b=ob[i].tolist(), gpu_d=float(gd[i]), orc_d=float(od[i]),
                        flags=int(amb[i[0]]))
        assert ez <= atol, ("zbuf", ez, where(np.abs(gz - oz)))
        assert eb <= atol, ("bary", eb, where(np.max(np.abs(gb - ob), axis=-1)))
        assert ed <= atol, ("dists", ed, where(np.abs(gd - od)))
    print("compare_frags: %d of %d pixels ambiguous (ids not compared), %d slots' values not compared "
          "(ill-conditioned unclipped extrapolation), %d id mismatches" % (int((~ok).sum()), P, n128, int(bad.size)))
    return int((~ok).sum()), int(bad.size)


# ---------------------------------------------------------------------------
# the oracle over a pixel sample, split across spawned processes (one per host
# core; spawned, because this process holds a CUDA context)
# ---------------------------------------------------------------------------
_POOL_MESH = None


def _pool_init(arrs):
    global _POOL_MESH
    _POOL_MESH = oracle.Mesh(*arrs)


def _pool_job(job):
    kind, args, kw, px = job
    fn = {"rasterize": oracle.rasterize, "margins": oracle.margins, "rast_bwd": oracle.rast_bwd}[kind]
    return fn(_POOL_MESH, *args, pixels=px, **kw)


class OraclePool:
    """``rasterize`` / ``margins`` / ``rast_bwd`` of the oracle on a pixel sample,
    the sample cut into one slice per worker (results concatenated; vertex
    gradients summed)."""

    def __init__(self, m, workers=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        import os
        self.workers = workers or os.cpu_count() or 1
        arrs = (m.verts, m.faces, m.first_face, m.num_faces, m.cams)
        self.ex = cf.ProcessPoolExecutor(max_workers=self.workers, mp_context=mp.get_context("spawn"),
                                         initializer=_pool_init, initargs=(arrs,))

    def _map(self, kind, args, kw, px, extra=None):
        cuts = np.array_split(np.arange(px.shape[0]), self.workers)
        jobs = []
        for c in cuts:
            if c.size == 0:
                continue
            kwc = dict(kw)
            if extra is not None:
                kwc.update({k: (None if v is None else v[c]) for k, v in extra.items()})
            jobs.append((kind, args, kwc, px[c]))
        return list(self.ex.map(_pool_job, jobs))

    def rasterize(self, S, K, blur, persp, clip, px):
        parts = self._map("rasterize", (S, K, blur, persp, clip), {}, px)
        return tuple(np.concatenate([p[i] for p in parts]) for i in range(4))

    def margins(self, S, K, blur, persp, clip, px):
        return np.concatenate(self._map("margins", (S, K, blur, persp, clip), {}, px))

    def rast_bwd(self, S, K, p2f, grad_zbuf, grad_bary, grad_dists, blur, persp, clip, px):
        parts = self._map("rast_bwd", (S, K), dict(blur=blur, persp=persp, clip=clip, with_abs=True), px,
                          extra=dict(pix_to_face=p2f, grad_zbuf=grad_zbuf, grad_bary=grad_bary,
                                     grad_dists=grad_dists))
        return sum(p[0] for p in parts), sum(p[1] for p in parts)

    def close(self):
        self.ex.shutdown()


def pick(fr, pixels, S):
    """select (n, r, c) pixels out of full (N,S,S,K...) fragments"""
    n, r, c = pixels[:, 0], pixels[:, 1], pixels[:, 2]
    return [np.asarray(x)[n, r, c] for x in fr]


def grad_close(g, ref, rel=1e-4, scale=None, return_count=False):
    """Gradient check.  Per component |g - ref| <= rel * max(|ref|, floor), where
    floor is the component's scale when ``scale`` is given (the summed
    magnitudes of the terms that form it; an accumulated sum of signed terms is
    only defined relative to that; at least 1e-3 of the rms of those scales),
    else 1e-2 * rms(ref); and globally ||g - ref|| / ||ref|| <= rel.
    Returns (worst per-component ratio, global relative error[, number of
    components over the per-component bound])."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    if scale is None:
        rms = np.sqrt(np.mean(ref ** 2)) if ref.size else 0.0
        floor = 1e-2 * rms
    else:
        sc = np.asarray(scale, np.float64)
        floor = np.maximum(sc, 1e-3 * np.sqrt(np.mean(sc ** 2)))
    den = np.maximum(np.abs(ref), floor) + 1e-30
    ratio = np.abs(g - ref) / den / rel
    worst = float(np.max(ratio)) if ref.size else 0.0
    glob = float(np.linalg.norm(g - ref) / (np.linalg.norm(ref) + 1e-30))
    if return_count:
        return worst, glob, int((ratio > 1).sum())
    return worst, glob


def assert_grad_close(g, ref, scale, label=""):
    """Vertex-gradient criterion: global relative error <= 1e-4, and every
    component within 1e-4 of max(|ref|, its own term scale).  Prints the
    worst ratio and how many components were compared."""
    worst, glob, n_over = grad_close(g, ref, scale=scale, return_count=True)
    n_live = int((np.asarray(scale) > 0).sum())
    print("%s: %d live components, worst %.3f of the 1e-4 bound, global %.2e" % (label, n_live, worst, glob))
    assert glob <= 1e-4, (label, "global", glob)
    assert n_over == 0, (label, "over 1e-4", n_over, n_live, worst)
    return worst, glob, n_over
