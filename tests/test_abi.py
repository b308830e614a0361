"""The C ABI library builds for sm_103a, loads, and exports every symbol that
include/*.h declares; the binding's structs match the header's layout.
No GPU is needed (no compute calls)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"MESHRAST_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt))
    return names


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("rast_mesh_fwd", "rast_mesh_bwd", "blend_fwd", "blend_bwd", "rast_workspace_bytes",
              "rast_query_status", "rast_strerror"):
        assert n in names


@pytest.fixture(scope="module")
def lib():
    from paper_2007_08501_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_library_exports_every_declared_symbol(lib):
    from paper_2007_08501_gb300 import ops
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(ops.EXPORTED) == _declared()


def test_pure_host_entry_points(lib):
    from paper_2007_08501_gb300 import ops
    ops._lib = None
    L = ops.load()
    assert L.rast_strerror(-2).decode().startswith("workspace")
    p = ops.make_rast_params(2, 64, 4, 1e-3, 16, 128)
    n = L.rast_workspace_bytes(ctypes.byref(p), 100, 200)
    assert n > 0 and n % 256 == 0
    # a larger batch never needs less workspace
    assert L.rast_workspace_bytes(ctypes.byref(p), 100, 400) >= n
    bad = ops.make_rast_params(2, 64, 65, 1e-3, 16, 128)       # K > 64
    assert L.rast_workspace_bytes(ctypes.byref(bad), 100, 200) == 0
    bad = ops.make_rast_params(2, 64, 4, 1e-3, 12, 128)        # bin size 12
    assert L.rast_workspace_bytes(ctypes.byref(bad), 100, 200) == 0
    bad = ops.make_rast_params(2, 64, 4, -1.0, 16, 128)        # negative blur
    assert L.rast_workspace_bytes(ctypes.byref(bad), 100, 200) == 0
    # argument errors are reported before anything touches a device
    assert L.rast_mesh_fwd(ctypes.byref(bad), None, 0, None, 0, None, None, None, None, None, None, None,
                           None, 0, None) == ops.MESHRAST_ERR_INVALID_ARG
    bp = ops.make_blend_params(sigma=-1.0)
    assert L.blend_fwd(ctypes.byref(bp), 1, 4, 1, None, None, None, None, None, 0, None, 0, None,
                       None) == ops.MESHRAST_ERR_INVALID_ARG


def test_bin_layouts_past_32_bits_are_refused(lib):
    # bin keys, counts, offsets and list positions are 32-bit on the device: a
    # layout with 2^31 - 1 or more bins, or more bin-list entries, is refused
    # (workspace size 0, UNSUPPORTED from the calls) instead of being clamped
    from paper_2007_08501_gb300 import ops
    ops._lib = None
    L = ops.load()
    ok = ops.make_rast_params(16, 8192, 4, 1e-3, 16, 256)           # 2^22 bins x 256 entries
    assert L.rast_workspace_bytes(ctypes.byref(ok), 100, 200) > 0
    many_bins = ops.make_rast_params(65535, 8192, 4, 1e-3, 8, 1)    # 65535 x 1024^2 bins
    assert L.rast_workspace_bytes(ctypes.byref(many_bins), 100, 200) == 0
    big_cap = ops.make_rast_params(16, 8192, 4, 1e-3, 16, 1 << 20)  # 2^22 bins x 2^20 entries
    assert L.rast_workspace_bytes(ctypes.byref(big_cap), 100, 200) == 0
    big_entries = ops.make_rast_params(1, 64, 4, 1e-3, 16, 128, max_bin_entries=1 << 31)
    assert L.rast_workspace_bytes(ctypes.byref(big_entries), 100, 200) == 0
    for p in (many_bins, big_cap, big_entries):
        assert L.rast_mesh_fwd(ctypes.byref(p), None, 0, None, 0, None, None, None, None, None, None, None,
                               None, 0, None) == ops.MESHRAST_ERR_UNSUPPORTED
    pp = ops.make_pts_params(16, 8192, 4, 0.01, 16, 1 << 20)
    assert L.pts_workspace_bytes(ctypes.byref(pp), 100) == 0
    pp = ops.make_pts_params(16, 8192, 4, 0.01, 16, 256)
    assert L.pts_workspace_bytes(ctypes.byref(pp), 100) > 0


def test_fragment_free_forward_is_refused_outside_the_fine_pass_blend(lib):
    from paper_2007_08501_gb300 import ops
    ops._lib = None
    L = ops.load()
    img = ctypes.c_void_p(256)   # never dereferenced: the call returns before any device work
    for K, bin_size, mode in ((8, 16, ops.BLEND_RGB), (20, 16, ops.BLEND_SIL), (4, 0, ops.BLEND_SIL)):
        p = ops.make_rast_params(1, 32, K, 1e-3, bin_size, 128)
        bp = ops.make_blend_params(mode=mode)
        assert L.rast_blend_fwd(ctypes.byref(p), ctypes.byref(bp), None, 0, None, 0, None, None, None, None,
                                None, None, None, None, img, None, 0, None) == ops.MESHRAST_ERR_INVALID_ARG


def test_knn_host_checks(lib):
    from paper_2007_08501_gb300 import ops
    ops._lib = None
    L = ops.load()
    assert L.knn_workspace_bytes(0) == 256 and L.knn_workspace_bytes(-1) == 0
    assert L.knn_workspace_bytes(1000) % 256 == 0 and L.knn_workspace_bytes(1000) >= 2 * 1001 * 8
    # argument errors come back before anything touches a device
    for D, K in ((0, 1), (5, 1), (3, 0), (3, 33)):
        assert L.knn_points(None, 0, None, None, None, 0, None, None, 0, D, K, None, None, None, 0,
                            None) == ops.MESHRAST_ERR_INVALID_ARG
    assert L.knn_points(None, 0, None, None, None, 0, None, None, 0, 3, 4, None, None, None, 0,
                        None) == ops.MESHRAST_ERR_WORKSPACE
    assert L.chamfer_fwd(None, 0, None, None, None, 0, None, None, 1, 3, None, None, None, None, None, None, None,
                         0, None) == ops.MESHRAST_ERR_INVALID_ARG
    assert L.chamfer_bwd(None, 0, None, None, None, 0, None, None, -1, 3, None, None, None, None, None, None,
                         None) == ops.MESHRAST_ERR_INVALID_ARG


def test_struct_layouts_match_header():
    from paper_2007_08501_gb300 import ops
    assert ctypes.sizeof(ops.rast_params) == 48
    assert ops.rast_params.max_bin_entries.offset == 40
    assert ctypes.sizeof(ops.blend_params) == 40
    assert ctypes.sizeof(ops.pts_params) == 40
    assert ctypes.sizeof(ops.shade_params) == 64
    assert ops.pts_params.max_bin_entries.offset == 32


def test_autotune_capacities_have_headroom():
    from paper_2007_08501_gb300 import tune
    per_bin, entries = tune.capacities(218, 138191)
    assert per_bin % 64 == 0 and per_bin >= 218 * 1.25 and entries >= 138191 * 1.25
    assert tune.capacities(0, 0) == (64, 1024)


def test_binding_refuses_mismatched_knn_tensors():
    # the checks run before anything touches a device
    import torch
    from paper_2007_08501_gb300 import ops
    p = torch.zeros(10, 3)
    f, n = torch.zeros(2, dtype=torch.int64), torch.zeros(2, dtype=torch.int64)
    cases = [
        (lambda: ops.knn_points(p, f, n, p, f, n, 4, torch.zeros(10, 3, dtype=torch.int64), torch.zeros(10, 4), None),
         "idx"),
        (lambda: ops.knn_points(p, f, torch.zeros(3, dtype=torch.int64), p, f, n, 4, None, None, None), "lengths"),
        (lambda: ops.knn_points(p, f, n, torch.zeros(10, 2), f, n, 4, None, None, None), "dimension"),
        (lambda: ops.chamfer_fwd(p, f, n, p, f, n, None, None, None, None, torch.zeros(3), torch.zeros(1), None),
         "loss_per_pair"),
        (lambda: ops.chamfer_bwd(p, f, n, p, f, n, None, None, None, None, torch.zeros(9, 3), None), "grad_p"),
        (lambda: ops.knn_points_bwd(p, p, torch.zeros(10, 2, dtype=torch.int64), torch.zeros(10, 3), None, None),
         "grad_dists"),
    ]
    for call, what in cases:
        with pytest.raises(ops.MeshRastError, match=what):
            call()


def test_binding_sizes_accept_the_documented_shapes_and_refuse_short_tensors(lib):
    # correctly sized (CPU) tensors get past the size checks and stop at the
    # CUDA check; one short tensor is refused by name; no device is touched
    import torch
    from paper_2007_08501_gb300 import ops, workloads
    b = workloads.sphere_batch([1, 1], 0.05, seed_base=1)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    v, f, ff, nf, cams, col = T(b.verts), T(b.faces), T(b.first_face), T(b.num_faces), T(b.cams), T(b.colors)
    N, S, K = b.N, 8, 2
    p = ops.make_rast_params(N, S, K, 1e-3, 8, 64)
    bp = ops.make_blend_params()
    sp = ops.make_shade_params((0.0, 0.0, -3.0))
    fr = (torch.zeros(N, S, S, K, dtype=torch.int64), torch.zeros(N, S, S, K), torch.zeros(N, S, S, K, 3),
          torch.zeros(N, S, S, K))
    img = torch.zeros(N, S, S, 4)
    ws = torch.zeros(64, dtype=torch.uint8)
    pp = ops.make_pts_params(N, S, K, 0.05, 8, 64)
    pts = torch.zeros(20, 3)
    pf, pn = torch.tensor([0, 10]), torch.tensor([10, 10])
    pfr = (torch.zeros(N, S, S, K, dtype=torch.int64), torch.zeros(N, S, S, K), torch.zeros(N, S, S, K))
    feats = torch.zeros(20, 2)
    calls = {
        "rast_mesh_fwd": lambda fr=fr: ops.rast_mesh_fwd(p, v, f, ff, nf, cams, *fr, ws),
        "rast_mesh_bwd": lambda fr=fr: ops.rast_mesh_bwd(p, v, f, ff, nf, cams, fr[0], fr[1], fr[2], fr[3],
                                                         torch.zeros_like(v), ws),
        "blend_fwd": lambda fr=fr: ops.blend_fwd(bp, N, S, K, *fr, f, col, img),
        "blend_bwd": lambda fr=fr: ops.blend_bwd(bp, N, S, K, *fr, f, col, img, fr[1], fr[2], fr[3],
                                                 torch.zeros_like(col)),
        "rast_blend_fwd": lambda fr=fr: ops.rast_blend_fwd(p, bp, v, f, ff, nf, cams, col, *fr, img, ws),
        "blend_rast_bwd": lambda fr=fr: ops.blend_rast_bwd(p, bp, v, f, ff, nf, cams, *fr, col, img,
                                                           torch.zeros_like(v), torch.zeros_like(col), ws),
        "shade_fwd": lambda fr=fr: ops.shade_fwd(bp, sp, N, S, K, *fr, f, v, v, col, cams, img),
        "shade_bwd": lambda fr=fr: ops.shade_bwd(bp, sp, N, S, K, *fr, f, v, v, col, cams, img, fr[1], fr[2], fr[3],
                                                 torch.zeros_like(v), torch.zeros_like(v), torch.zeros_like(col)),
        "pts_rasterize_fwd": lambda fr=pfr: ops.pts_rasterize_fwd(pp, pts, pf, pn, cams, *fr, ws),
        "pts_rasterize_bwd": lambda fr=pfr: ops.pts_rasterize_bwd(pp, pts, pf, pn, cams, fr[0], fr[1], fr[2],
                                                                  torch.zeros_like(pts), ws),
        "pts_composite_fwd": lambda fr=pfr: ops.pts_composite_fwd(pp, 0, fr[0], fr[2], feats, torch.zeros(N, S, S, 2)),
        "pts_composite_bwd": lambda fr=pfr: ops.pts_composite_bwd(pp, 0, fr[0], fr[2], feats, torch.zeros(N, S, S, 2),
                                                                  fr[2], torch.zeros_like(feats)),
    }
    for name, call in calls.items():
        with pytest.raises(ops.MeshRastError, match="CUDA tensor"):
            call()
    short = (fr[0], fr[1], fr[2][..., :2].contiguous(), fr[3])      # barycentrics: 2 of 3 per slot
    with pytest.raises(ops.MeshRastError, match="bary holds"):
        calls["rast_mesh_fwd"](short)
    with pytest.raises(ops.MeshRastError, match="dists holds"):
        calls["pts_rasterize_fwd"]((pfr[0], pfr[1], pfr[2][:, :, :, :1].contiguous()))
