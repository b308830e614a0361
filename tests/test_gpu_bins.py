"""GPU coarse binning (Section 3.2, "Rasterizer": faces are first assigned to
image tiles) against the oracle's bin assignment, bin by bin.

The GPU's counts and lists are read back from the workspace at the layout
``rast_workspace_bin_layout`` reports.  A face belongs to a bin when its bbox,
inflated by sqrt(blur), meets the rectangle spanned by the bin's pixel
centres.  Membership decided within eps = 1e-6 of a boundary is ambiguous:
  * every unambiguous member of the oracle's list must be in the GPU's list;
  * every GPU entry must be a member of the oracle's lists for the bbox grown
    by eps (a membership that rounding may decide either way);
  * the ambiguous entries are counted and printed;
  * the raw counts equal the list lengths (no overflow at these capacities).
"""
import numpy as np
import pytest
import torch

import oracle
from _gpu import oracle_mesh, to_dev
from paper_2007_08501_gb300 import ops, tune, workloads

pytestmark = pytest.mark.gpu

EPS = 1e-6


def _gpu_bins(d, N, S, K, blur, bin_size, max_per_bin, clip=True):
    p = ops.make_rast_params(N, S, K, np.float32(blur), bin_size, max_per_bin, True, clip)
    ws = ops.alloc_workspace(p, d["verts"].shape[0], d["faces"].shape[0])
    fr = ops.alloc_fragments(N, S, K)
    ops.rast_mesh_fwd(p, d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], *fr, ws)
    assert ops.rast_query_status(ws) == 0
    L = ops.rast_workspace_bin_layout(p, d["verts"].shape[0], d["faces"].shape[0])
    raw = ws.cpu().numpy().view(np.uint8)
    NB = L["NB"]
    counts = raw[L["counts"]:L["counts"] + 4 * NB].view(np.int32)
    eff = raw[L["eff"]:L["eff"] + 4 * NB].view(np.int32)
    offs = raw[L["offsets"]:L["offsets"] + 4 * (NB + 1)].view(np.int32)
    lists = raw[L["lists"]:L["lists"] + 8 * L["capacity"]].view(np.uint64)
    order = raw[L["order"]:L["order"] + 4 * NB].view(np.int32)
    # the fine pass's queue: every bin once, longest first by the bit length of its count
    np.testing.assert_array_equal(np.sort(order), np.arange(NB))
    bits = np.array([int(e).bit_length() for e in eff[order]])
    assert np.all(np.diff(bits) <= 0)
    return L, counts, eff, offs, lists


def _check(b, S, K, blur, bin_size, max_per_bin):
    blur = float(np.float32(blur))
    d = to_dev(b)
    L, counts, eff, offs, lists = _gpu_bins(d, b.N, S, K, blur, bin_size, max_per_bin)
    np.testing.assert_array_equal(counts, eff)
    m = oracle_mesh(b)
    oc, oo, ol, oa = oracle.bins(m, S, bin_size, blur, eps=EPS)
    grown = (np.sqrt(blur) + EPS) ** 2          # the bbox inflated by sqrt(blur) + eps
    gc, go, gl, _ = oracle.bins(m, S, bin_size, grown, eps=EPS)
    assert oc.size == L["NB"]
    n_amb = missing = extra = 0
    for bidx in range(L["NB"]):
        ids = (lists[offs[bidx]:offs[bidx] + eff[bidx]] & np.uint64(0xffffffff)).astype(np.int64)
        got = set(ids.tolist())
        assert len(got) == ids.size, "a face listed twice in bin %d" % bidx
        sl = slice(oo[bidx], oo[bidx + 1])
        sure = set(ol[sl][oa[sl] == 0].tolist())
        n_amb += int((oa[sl] != 0).sum())
        allowed = set(gl[go[bidx]:go[bidx + 1]].tolist())
        missing += len(sure - got)
        extra += len(got - allowed)
    print("bins %d x %d, bin %d, blur %.3g: %d entries, %d ambiguous, %d missing, %d extra"
          % (b.N, S, bin_size, blur, int(eff.sum()), n_amb, missing, extra))
    assert missing == 0 and extra == 0
    assert eff.sum() > 0


@pytest.mark.parametrize("bin_size", [8, 16])
@pytest.mark.parametrize("blur", [0.0, workloads.BLUR_SIGMA_1E4])
@pytest.mark.parametrize("S", [64, 70])
def test_bins_match_the_oracle(bin_size, blur, S):
    b = workloads.sphere_batch([3, 4, 2], 0.05, seed_base=801)
    _check(b, S, 4, blur, bin_size, 2048)


def test_bins_of_the_heterogeneous_512_batch():
    # the 32-mesh batch of levels 3..7 at its full size, bin size and
    # capacities from the autotuner
    w = workloads.workload(2)
    b = w.batch
    d = to_dev(b)
    blur = float(np.float32(w.blur_radius))
    best = tune.tune(d["verts"], d["faces"], d["first_face"], d["num_faces"], d["cams"], w.image_size, w.K, blur,
                     w.perspective_correct, w.clip_barycentric_coords, use_cache=False)
    del d
    torch.cuda.empty_cache()
    _check(b, w.image_size, w.K, blur, best["bin_size"], best["max_faces_per_bin"])
