"""Autotuner for the binned rasterizer's launch parameters.

The two-pass rasterizer (Section 3.2, "Rasterizer": image tiles first, then
pixels) has three knobs whose best values depend on image size, K, blur and
face density: the bin size, the per-bin capacity ``max_faces_per_bin`` and
the capacity of all bin lists ``max_bin_entries``.  For each candidate bin
size the tuner runs one forward with generous capacities, reads the real
occupancy back (``rast_bin_occupancy``), sizes the capacities with headroom,
times a few forwards with CUDA events and keeps the fastest.  Results are
cached per (N, image size, K, blur > 0, clipping, perspective, log2 of the
face count, candidate bin sizes) in ``tuned.json`` next to this file.

Tuning synchronises and allocates; run it before capturing a CUDA graph.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

import torch

from . import ops

_CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")
_lock = threading.Lock()


def _key(N, S, K, blur, persp, clip, F, bin_sizes):
    return "N%d_S%d_K%d_b%d_c%d_p%d_F%d_bins%s" % (N, S, K, int(blur > 0), int(bool(clip)), int(bool(persp)),
                                                   int(math.log2(max(F, 1))), "-".join(str(b) for b in bin_sizes))


def _load_cache():
    try:
        with open(_CACHE_PATH) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(c):
    tmp = _CACHE_PATH + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE_PATH)


def capacities(max_count, total, headroom=1.25):
    """Per-bin capacity (a multiple of 64) and total list capacity with headroom."""
    per_bin = max(64, int(math.ceil(max_count * headroom / 64.0)) * 64)
    entries = max(1024, int(math.ceil(total * headroom)))
    return per_bin, entries


def tune(verts, faces, first_face, num_faces, cams, image_size, K, blur_radius=0.0, perspective_correct=True,
         clip_barycentric_coords=False, bin_sizes=(8, 16), reps=5, use_cache=True):
    """Returns dict(bin_size, max_faces_per_bin, max_bin_entries, ms, candidates)."""
    N, V, F = first_face.shape[0], verts.shape[0], faces.shape[0]
    key = _key(N, image_size, K, blur_radius, perspective_correct, clip_barycentric_coords, F, bin_sizes)
    with _lock:
        cache = _load_cache() if use_cache else {}
        if key in cache:
            return cache[key]
    frags = ops.alloc_fragments(N, image_size, K, verts.device)
    results = []
    for bs in bin_sizes:
        nb = (image_size + bs - 1) // bs
        # generous first pass: every bin may hold every face of the batch (capped)
        probe_cap = max(256, min(F, 1 << 20))
        probe_entries = min(N * nb * nb * probe_cap, (1 << 31) - 1)
        probe_entries = min(probe_entries, max(1 << 20, 64 * max(F, 1)))
        p = ops.make_rast_params(N, image_size, K, blur_radius, bs, probe_cap, perspective_correct,
                                 clip_barycentric_coords, probe_entries)
        ws = ops.alloc_workspace(p, V, F, verts.device)
        ops.rast_mesh_fwd(p, verts, faces, first_face, num_faces, cams, *frags, ws)
        mc, tot = ops.rast_bin_occupancy(p, V, F, ws)
        per_bin, entries = capacities(mc, tot)
        p = ops.make_rast_params(N, image_size, K, blur_radius, bs, per_bin, perspective_correct,
                                 clip_barycentric_coords, entries)
        del ws
        ws = ops.alloc_workspace(p, V, F, verts.device)
        ts = []
        for i in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ops.rast_mesh_fwd(p, verts, faces, first_face, num_faces, cams, *frags, ws)
            e1.record()
            e1.synchronize()
            if i >= 2:
                ts.append(e0.elapsed_time(e1))
        status = ops.rast_query_status(ws)
        if status & ops.ST_BIN_OVERFLOW:
            continue
        results.append(dict(bin_size=bs, max_faces_per_bin=per_bin, max_bin_entries=entries,
                            ms=statistics.median(ts), max_count=mc, total_entries=tot))
        del ws
    if not results:
        raise ops.MeshRastError("autotune: every candidate bin size overflowed")
    best = dict(min(results, key=lambda r: r["ms"]))
    best["candidates"] = results
    if use_cache:
        with _lock:
            cache = _load_cache()
            cache[key] = best
            _save_cache(cache)
    return best
