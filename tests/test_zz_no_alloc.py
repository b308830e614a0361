"""rast_mesh_fwd_static: the forward for callers that cannot allocate device
memory (the library's built-in 16 MiB array stands in for the workspace).

Checked through the C ABI against rast_mesh_fwd on the same inputs, on two
calls in a row with different batches, so that contents left in the shared
array by the first call cannot leak into the second.  The same kernels run on
the same inputs, so the outputs must be identical bit for bit.  A warmed-up
call must not change the device's free memory, and its status word (read
with rast_query_static_status) must report a forced bin overflow.  This file
sorts last so that a run stopping at the first failure has already run every
other test.
"""
import numpy as np
import pytest
import torch

from paper_2007_08501_gb300 import ops, workloads

pytestmark = pytest.mark.gpu

BLUR = float(np.float32(workloads.BLUR_SIGMA_1E4))


def _dev(b):
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return T(b.verts), T(b.faces), T(b.first_face), T(b.num_faces), T(b.cams)


def _both(b, S, K, bin_size, max_per_bin, clip=True):
    v, f, ff, nf, cams = _dev(b)
    p = ops.make_rast_params(b.N, S, K, BLUR, bin_size, max_per_bin, True, clip)
    ref = ops.alloc_fragments(b.N, S, K)
    ws = ops.alloc_workspace(p, b.V, b.F)
    ops.rast_mesh_fwd(p, v, f, ff, nf, cams, *ref, ws)
    assert ops.rast_query_status(ws) == 0
    got = ops.alloc_fragments(b.N, S, K)
    for t in got:
        t.fill_(7)          # anything the call fails to write shows up
    ops.rast_mesh_fwd_static(p, v, f, ff, nf, cams, *got)
    torch.cuda.synchronize()
    assert ops.rast_query_static_status() == 0
    return ref, got


def _same(ref, got):
    # the same kernels run on the same inputs: every output identical
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


def test_static_workspace_forward_matches_rast_mesh_fwd_twice():
    w = workloads.workload(1)
    ref, got = _both(w.batch, w.image_size, w.K, 16, 256)
    _same(ref, got)
    # second call: a different batch, size and bin layout on the same shared array
    b2 = workloads.sphere_batch([3, 2, 4], 0.05, seed_base=31)
    ref2, got2 = _both(b2, 100, 3, 8, 512, clip=False)
    _same(ref2, got2)
    assert (ref2[0] >= 0).any()
    # third call: K > 16, the streaming fine pass and the attribute pass
    ref3, got3 = _both(b2, 64, 20, 16, 1024)
    _same(ref3, got3)
    assert (ref3[0] >= 0).any()


def test_static_call_allocates_nothing_and_reports_its_status():
    b = workloads.sphere_batch([2, 2], 0.05, seed_base=17)
    v, f, ff, nf, cams = _dev(b)
    fr = ops.alloc_fragments(b.N, 64, 4)
    p = ops.make_rast_params(b.N, 64, 4, BLUR, 16, 512, True, True)
    ops.rast_mesh_fwd_static(p, v, f, ff, nf, cams, *fr)      # warm-up: address lookup, lazy loading
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ops.rast_mesh_fwd_static(p, v, f, ff, nf, cams, *fr)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert ops.rast_query_static_status() == 0
    # a bin capacity of 1 face overflows: the status word says so
    tiny = ops.make_rast_params(b.N, 64, 4, BLUR, 16, 1, True, True)
    ops.rast_mesh_fwd_static(tiny, v, f, ff, nf, cams, *fr)
    assert ops.rast_query_static_status() & ops.ST_BIN_OVERFLOW
    # the next call starts from a clean status word
    ops.rast_mesh_fwd_static(p, v, f, ff, nf, cams, *fr)
    assert ops.rast_query_static_status() == 0


def test_static_workspace_rejects_requests_beyond_its_size():
    b = workloads.sphere_batch([2], 0.05, seed_base=5)
    v, f, ff, nf, cams = _dev(b)
    # 1 image at 1024^2 with bins of 8 and 4096 faces per bin needs > 16 MiB of bin lists
    p = ops.make_rast_params(1, 1024, 1, 0.0, 8, 4096, True, False)
    assert ops.rast_workspace_bytes(p, b.V, b.F) > ops.STATIC_WORKSPACE_BYTES
    fr = ops.alloc_fragments(1, 1024, 1)
    rc = ops.rast_mesh_fwd_static(p, v, f, ff, nf, cams, *fr, check=False)
    assert rc == ops.MESHRAST_ERR_STATIC_TOO_LARGE
    assert "16 MiB" in ops.rast_strerror(rc)
