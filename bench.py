#!/usr/bin/env python
"""Throughput of the differentiable packed-mesh rasterizer + soft blends on GB300.

One step = the whole differentiable path over one batch, through the C ABI:
  rast_blend_fwd (stage, bin count/scan/fill, fine top-K, blend) ->
  blend_rast_bwd (blend adjoint pulled through the rasterizer adjoint, upstream
  grad N(0,1), grad to the packed vertices).
Default workload (the largest configuration): 1 displaced icosphere of 81,920
faces (level 6) seen by 20 cameras, 512x512, K = 50, blur_radius =
ln(1/1e-4 - 1) 1e-4, soft silhouette (sigma = 1e-4); the same step as four
separate calls and the plain per-mesh form (one unbinned launch per image) are
timed beside it.  --workload 1 is the 8 x 5,120-face batch at 256x256, K = 8,
softmax RGB + silhouette.

Each C-ABI call is captured in its own CUDA graph; a step replays the
graphs with CUDA events between them, so every stage's device time is
measured live on the launching stream inside the timed region.  L2 is
flushed (256 MiB write) between steps, outside the events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank renders its own
copy of the batch (independent replicas, no collective on the data path);
value = all ranks' slots / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd raster+blend ms/batch & Mpix·K/s, % HBM roofline, vs per-mesh plain form"
UNIT = "Mpix*K/s"
WORKLOADS = {
    "1": (1, "", "8 icospheres level 4 (5,120 faces each, radial N(0,0.05)), random cameras, 256x256, K=8, "
                 "blur=ln(1/1e-4-1)*1e-4, softmax rgb + silhouette (sigma=gamma=1e-4), fwd+bwd to verts"),
    "2": (2, "", "32 icospheres of levels 3..7 (heterogeneous packed batch, radial N(0,0.03)), random cameras, "
                 "512x512, K=4, blur=ln(1/1e-4-1)*1e-4, soft silhouette, fwd+bwd to verts"),
    "3hard": (3, "hard", "1 icosphere level 8 (1,310,720 faces, radial N(0,0.02)), 1024x1024, K=1, blur 0, "
                         "silhouette, fwd+bwd to verts"),
    "3soft": (3, "soft", "1 icosphere level 8 (1,310,720 faces, radial N(0,0.02)), 1024x1024, K=8, "
                         "blur=ln(1/1e-4-1)*1e-4, soft silhouette, fwd+bwd to verts"),
    "4": (4, "", "1 icosphere level 6 (81,920 faces) seen by 20 cameras (shared vertices), 512x512, K=50, "
                 "blur=ln(1/1e-4-1)*1e-4, soft silhouette, fwd+bwd to verts"),
    "1gouraud": (1, "", "8 icospheres level 4 (5,120 faces each), random cameras, 256x256, K=8, "
                        "blur=ln(1/1e-4-1)*1e-4, Gouraud-shaded per-vertex colours (one point light) + softmax blend, "
                        "fwd+bwd to verts, normals and colours"),
    "1phong": (1, "", "8 icospheres level 4 (5,120 faces each), random cameras, 256x256, K=8, "
                      "blur=ln(1/1e-4-1)*1e-4, Phong-shaded per-vertex colours (one point light) + softmax blend, "
                      "fwd+bwd to verts, normals and colours"),
    "points": (None, "alpha", "point clouds: 8 x 200,000 points sampled from displaced level-4 spheres, 256x256, "
                              "K=50, splat radius 0.01 NDC, Alpha-composited silhouettes, fwd+bwd to points"),
    "knn": (None, "knn", "exact KNN, 32 pairs of point clouds sampled from displaced level-4 spheres, |P| = |Q| = "
                         "50,000, D = 3, K = 8, forward"),
    "knn_het": (None, "knn_het", "exact KNN, 32 pairs of point clouds sampled from displaced level-4 spheres, |P|, |Q| "
                                 "uniform in [10,000, 90,000], D = 3, K = 8, forward"),
    "chamfer": (None, "chamfer", "Chamfer loss, 32 pairs of point clouds sampled from displaced level-4 spheres, "
                                 "|P| = 1,000, |Q| = 50,000, D = 3, forward + backward"),
    "points_norm": (None, "norm", "point clouds: 8 x 200,000 points sampled from displaced level-4 spheres, "
                                  "256x256, K=50, splat radius 0.01 NDC, Norm-composited silhouettes, fwd+bwd to "
                                  "points"),
}
# kernels one step launches: rast_blend_fwd = k_stage, k_scan, k_fill, then
#   K <= 16: k_fine (+ k_blend_fwd for the softmax blend);
#   K > 16 with clipped barycentrics (or no blur): k_sort_bins, k_fine_stream,
#   k_frag_attr (which blends the silhouette; + k_blend_fwd for softmax);
# blend_rast_bwd = k_stage, k_blend_rast_bwd


def mesh_kernels_per_step(w):
    rgb = w.blend_mode == "rgb"
    if w.K <= 16:
        fwd = 4 + (1 if rgb else 0)
    elif w.clip_barycentric_coords or not w.blur_radius > 0:
        fwd = 6 + (1 if rgb else 0)
    else:
        fwd = 5          # k_fine with shared-memory lists, then k_blend_fwd
    return fwd + 2
# DRAM bytes (read + write) per C-ABI call of a stage -- every kernel of the
# call, from one ncu capture (gpu__time_duration, dram__bytes_read/write,
# --clock-control none) of the current kernel source -- keyed by (workload,
# stage, bin size); a combination without an entry reports null.  Workload 4
# is captured on its first 2 of 20 views (--max-images 2) and scaled by 10:
# every view carries the same mesh, so each kernel's traffic grows with the
# views.
TRAFFIC_BYTES = {
    ("1", "fwd", 16): {"kernel": "rast_blend_fwd call: k_stage + k_scan + k_fill + k_fine<8,16,0> + k_blend_fwd<8>",
                       "bytes": 141800000, "profile": "profiles/launch_list_8x5120faces_256px_K8.md"},
    ("1", "bwd", 16): {"kernel": "blend_rast_bwd call: k_stage + k_blend_rast_bwd<8,1>", "bytes": 106100000,
                       "profile": "profiles/launch_list_8x5120faces_256px_K8.md"},
    ("4", "fwd", 16): {"kernel": "rast_blend_fwd call: k_stage + k_scan + k_fill + k_sort_bins + "
                                 "k_fine_stream<16,16,8,0> + k_fine_stream<16,64,4,1> + k_frag_attr<1>", "bytes": 11634000000,
                       "profile": "profiles/launch_list_20x81920faces_512px_K50.md (2 views x 10)"},
    ("4", "bwd", 16): {"kernel": "blend_rast_bwd call: k_stage + k_blend_rast_bwd_any<0>", "bytes": 4209000000,
                       "profile": "profiles/launch_list_20x81920faces_512px_K50.md (2 views x 10)"},
    ("points", "rast_fwd", 8): {"kernel": "pts_rasterize_fwd call: k_pstage + k_scan + k_pfill + k_pfine<0,8>",
                                "bytes": 552453578, "profile": "profiles/points_8x200000pts_256px_K50.md"},
    # the same rasterizer call (compositing mode does not enter it)
    ("points_norm", "rast_fwd", 8): {"kernel": "pts_rasterize_fwd call: k_pstage + k_scan + k_pfill + "
                                               "k_pfine<0,8>", "bytes": 552453578,
                                     "profile": "profiles/points_8x200000pts_256px_K50.md"},
}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="4", choices=sorted(WORKLOADS),
                    help="4 (default: the largest configuration, 20 views x 81,920 faces, 512^2, K = 50) or "
                         "another workload")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain per-mesh form")
    ap.add_argument("--plain", action="store_true",
                    help="also time the plain per-mesh form on workloads other than 1 and 4 (slow)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fit", action="store_true", help="workload 4: skip timing the fitting loop")
    ap.add_argument("--bin-size", type=int, default=0, choices=[0, 8, 16],
                    help="fix the bin size (0: the autotuner picks 8 or 16)")
    ap.add_argument("--max-images", type=int, default=0,
                    help="keep only the first N images of the workload (small cases for profiling)")
    ap.add_argument("--no-separate", action="store_true",
                    help="skip timing the step as four separate calls (no fused forward or backward)")
    return ap.parse_args()


def max_over_ranks(x, dist, device):
    """The slowest rank's value: every replica renders its own batch, and the
    job ends when the last one finishes (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms, scale=1e6):
    """Units all ranks processed per second (/ scale), timed by the slowest rank."""
    return world * units_per_rank / (ms / 1e3) / scale


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measure_fp32_peak(device, target_ms=40.0, reps=5):
    """FP32 FMA throughput of this GPU (``meshrast_fma_probe``: 8 blocks of 256
    threads per SM, 8 independent FMA chains per thread), CUDA events on the
    launching stream, best of ``reps`` after a warm-up.  Returns FMA lane
    operations per second (one FMA per lane per clock at peak; 2 FLOPs each)."""
    import torch
    from paper_2007_08501_gb300 import ops
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float32, device=device)
    iters = 64
    ops.fma_probe(out, blocks, iters)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ops.fma_probe(out, blocks, iters)
    e1.record()
    e1.synchronize()
    iters = max(64, int(iters * target_ms / max(e0.elapsed_time(e1), 1e-3)))
    best = None
    for _ in range(reps):
        e0.record()
        flops = ops.fma_probe(out, blocks, iters)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return flops / 2 / (best / 1e3)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


# ---------------------------------------------------------------------------
# our path
# ---------------------------------------------------------------------------
class Pipeline:
    """Static device buffers + one CUDA graph per C-ABI call."""

    def __init__(self, w, bin_size, max_faces_per_bin, device, max_bin_entries=0, fused=True, shading=None):
        import torch
        from paper_2007_08501_gb300 import ops
        self.torch, self.ops = torch, ops
        b = w.batch
        self.N, self.S, self.K = b.N, w.image_size, w.K
        self.dev = device
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.verts, self.faces = T(b.verts), T(b.faces)
        self.ff, self.nf, self.cams = T(b.first_face), T(b.num_faces), T(b.cams)
        self.colors = T(b.colors)
        self.gimg = T(workloads_upstream(w))
        self.p = ops.make_rast_params(b.N, w.image_size, w.K, np.float32(w.blur_radius), bin_size,
                                      max_faces_per_bin, w.perspective_correct, w.clip_barycentric_coords,
                                      max_bin_entries)
        self.bp = ops.make_blend_params(w.sigma, w.gamma, w.znear, w.zfar, (1.0, 1.0, 1.0), 1e-10,
                                        ops.BLEND_RGB if w.blend_mode == "rgb" else ops.BLEND_SIL)
        self.rgb = w.blend_mode == "rgb"
        self.ws = ops.alloc_workspace(self.p, b.V, b.F, device)
        self.frag = ops.alloc_fragments(b.N, w.image_size, w.K, device)
        self.img = torch.empty((b.N, w.image_size, w.image_size, 4), device=device)
        p2f, zb, ba, di = self.frag
        self.gz, self.gb, self.gd = torch.empty_like(zb), torch.empty_like(ba), torch.empty_like(di)
        self.gc = torch.empty_like(self.colors)
        self.gv = torch.empty_like(self.verts)
        self.fused = fused
        self.shading = shading
        if shading is not None:
            self.normals = torch.nn.functional.normalize(self.verts, dim=1).contiguous()
            self.sp = ops.make_shade_params((0.0, 3.0, -3.0), (0.3, 0.3, 0.3), (0.6, 0.6, 0.6), (0.3, 0.3, 0.3), 32.0,
                                            shading, ops.SHADE_SOFTMAX)
            self.gn = torch.empty_like(self.verts)
            self.gvd = torch.empty_like(self.verts)
        self.graphs = None

    def stages(self):
        ops, p2f, zb, ba, di = (self.ops, *self.frag)
        N, S, K = self.N, self.S, self.K
        rgb = self.rgb
        if self.shading is not None:
            return [
                ("rast_fwd", lambda: ops.rast_mesh_fwd(self.p, self.verts, self.faces, self.ff, self.nf, self.cams,
                                                       p2f, zb, ba, di, self.ws)),
                ("shade_fwd", lambda: ops.shade_fwd(self.bp, self.sp, N, S, K, p2f, zb, ba, di, self.faces,
                                                    self.verts, self.normals, self.colors, self.cams, self.img)),
                ("shade_bwd", lambda: ops.shade_bwd(self.bp, self.sp, N, S, K, p2f, zb, ba, di, self.faces,
                                                    self.verts, self.normals, self.colors, self.cams, self.gimg,
                                                    self.gz, self.gb, self.gd, self.gvd, self.gn, self.gc)),
                ("rast_bwd", lambda: ops.rast_mesh_bwd(self.p, self.verts, self.faces, self.ff, self.nf, self.cams,
                                                       p2f, self.gz, self.gb, self.gd, self.gv, self.ws)),
            ]
        if self.fused:
            return [
                ("fwd", lambda: ops.rast_blend_fwd(self.p, self.bp, self.verts, self.faces, self.ff, self.nf,
                                                   self.cams, self.colors if rgb else None, p2f, zb, ba, di,
                                                   self.img, self.ws)),
                ("bwd", lambda: ops.blend_rast_bwd(self.p, self.bp, self.verts, self.faces, self.ff, self.nf,
                                                   self.cams, p2f, zb if rgb else None, ba if rgb else None, di,
                                                   self.colors if rgb else None, self.gimg, self.gv,
                                                   self.gc if rgb else None, self.ws)),
            ]
        return [
            ("rast_fwd", lambda: ops.rast_mesh_fwd(self.p, self.verts, self.faces, self.ff, self.nf, self.cams,
                                                   p2f, zb, ba, di, self.ws)),
            ("blend_fwd", lambda: ops.blend_fwd(self.bp, N, S, K, p2f, zb, ba, di, self.faces, self.colors,
                                                self.img)),
            ("blend_bwd", lambda: ops.blend_bwd(self.bp, N, S, K, p2f, zb, ba, di, self.faces, self.colors,
                                                self.gimg, self.gz if rgb else None, self.gb if rgb else None,
                                                self.gd, self.gc if rgb else None)),
            ("rast_bwd", lambda: ops.rast_mesh_bwd(self.p, self.verts, self.faces, self.ff, self.nf, self.cams,
                                                   p2f, self.gz if rgb else None, self.gb if rgb else None,
                                                   self.gd, self.gv, self.ws)),
        ]

    def run_eager(self):
        for _, fn in self.stages():
            fn()

    def capture(self):
        torch = self.torch
        s = torch.cuda.Stream(self.dev)
        s.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(s):
            for _ in range(2):
                self.run_eager()
        torch.cuda.current_stream(self.dev).wait_stream(s)
        torch.cuda.synchronize(self.dev)
        self.graphs = []
        for name, fn in self.stages():
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn()
            self.graphs.append((name, g))
        torch.cuda.synchronize(self.dev)

    def status(self):
        return self.ops.rast_query_status(self.ws)


def workloads_upstream(w):
    from paper_2007_08501_gb300 import workloads
    return workloads.upstream_grad(w.batch.N, w.image_size, w.grad_seed)


def timed_steps(pipe, steps, warmup, flush, use_graph=True):
    """Returns per-step dict of stage -> ms, measured with CUDA events."""
    torch = pipe.torch
    names = [n for n, _ in pipe.stages()]
    fns = [g.replay for _, g in pipe.graphs] if use_graph else [fn for _, fn in pipe.stages()]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)] for _ in range(steps)]
    for i in range(warmup):
        flush.zero_()
        for fn in fns:
            fn()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        e = evs[i]
        e[0].record()
        for j, fn in enumerate(fns):
            fn()
            e[j + 1].record()
    torch.cuda.synchronize()
    out = []
    for e in evs:
        out.append({names[j]: e[j].elapsed_time(e[j + 1]) for j in range(len(fns))})
    return out


def algorithmic_bytes(w):
    """Bytes each stage must move per launch (fragments materialised as the C ABI requires)."""
    b = w.batch
    N, S, K = b.N, w.image_size, w.K
    slots, pix, V, F = N * S * S * K, N * S * S, b.V, b.F
    cams = 64 * N
    mesh_in = 12 * V + 24 * F + cams + 16 * N
    rgb_extra = 24 * F + 12 * V if w.blend_mode == "rgb" else 0   # faces + colours gathered by the rgb blend
    # fragment bytes a blend reads per slot: the silhouette (Algorithm 1) needs
    # only the face id and the distance (8 + 4), the softmax blend all 28
    frag_in = 12 if w.blend_mode == "sil" else 28
    return {
        "rast_fwd": mesh_in + 28 * slots,                                  # write fragments
        "fwd": mesh_in + 28 * slots + 16 * pix + rgb_extra,                # fused: fragments + rgba out
        "shade_fwd": 28 * slots + 16 * pix + 24 * F + 36 * V,              # fragments + faces, verts, normals, colours
        "shade_bwd": 28 * slots + 16 * pix + 20 * slots + 24 * F + 72 * V,
        "blend_fwd": frag_in * slots + 16 * pix + rgb_extra,               # read fragments, write rgba
        "blend_bwd": frag_in * slots + 16 * pix + 20 * slots + rgb_extra + 12 * V,
        "rast_bwd": mesh_in + 28 * slots + 12 * V,                         # ids + grad fragments
        "bwd": mesh_in + frag_in * slots + 16 * pix + rgb_extra + 24 * V,  # fused: fragments + grad image in,
    }                                                                      # vertex + colour grads out


def cpu_baseline(w, target_s=15.0):
    """The FP64 oracle, as it stands, on a bounded pixel sample of the same workload
    (single-threaded: rasterize + blend fwd/bwd + rasterizer adjoint)."""
    import oracle
    from paper_2007_08501_gb300 import workloads
    m = oracle.Mesh.from_batch(w.batch)
    blur = float(np.float32(w.blur_radius))
    S, K = w.image_size, w.K
    g_full = workloads.upstream_grad(w.batch.N, S, w.grad_seed)

    def run(per_image, seed):
        px = workloads.sample_pixels(w.batch.N, S, per_image, seed)
        t0 = time.perf_counter()
        fr = oracle.rasterize(m, S, K, blur, True, w.clip_barycentric_coords, pixels=px)
        g = g_full[px[:, 0], px[:, 1], px[:, 2]]
        mode = 1 if w.blend_mode == "rgb" else 0
        oracle.blend_fwd(*fr, w.batch.faces, w.batch.colors, w.sigma, w.gamma, w.znear, w.zfar, mode=mode)
        gz, gb, gd, _ = oracle.blend_bwd(*fr, w.batch.faces, w.batch.colors, g, w.sigma, w.gamma, w.znear,
                                         w.zfar, mode=mode)
        oracle.rast_bwd(m, S, K, fr[0], gz, gb, gd, blur, True, w.clip_barycentric_coords, pixels=px)
        return px.shape[0], time.perf_counter() - t0

    n0, t0 = run(32, 11)
    per_image = int(max(32, min(S * S, 32 * target_s / max(t0, 1e-3))))
    n, t = run(per_image, 12)
    return {"value": n * K / t / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d pixels (%d per image, seeded) of the same batch through the FP64 oracle "
                      "(rasterize all faces per pixel + blend fwd/bwd + adjoint), %.1f s" % (n, per_image, t),
            "per_image": per_image}


def _oracle_pixels(job):
    """One worker's share of the parallel CPU baseline: the oracle calls of
    ``cpu_baseline`` on a slice of the pixel sample (runs in a spawned process)."""
    import oracle
    (verts, faces, ff, nf, cams, colors, S, K, blur, clip, sigma, gamma, znear, zfar, mode, px, g) = job
    m = oracle.Mesh(verts, faces, ff, nf, cams)
    fr = oracle.rasterize(m, S, K, blur, True, clip, pixels=px)
    oracle.blend_fwd(*fr, faces, colors, sigma, gamma, znear, zfar, mode=mode)
    gz, gb, gd, _ = oracle.blend_bwd(*fr, faces, colors, g, sigma, gamma, znear, zfar, mode=mode)
    oracle.rast_bwd(m, S, K, fr[0], gz, gb, gd, blur, True, clip, pixels=px)
    return int(px.shape[0])


def cpu_baseline_parallel(w, per_image, workers=None):
    """The same oracle calls as ``cpu_baseline`` spread over a pool of
    processes, one per host core (spawned: this process already holds a CUDA
    context), the pixel sample split evenly."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from paper_2007_08501_gb300 import workloads
    workers = workers or os.cpu_count() or 1
    b = w.batch
    S, K = w.image_size, w.K
    blur = float(np.float32(w.blur_radius))
    mode = 1 if w.blend_mode == "rgb" else 0
    g_full = workloads.upstream_grad(b.N, S, w.grad_seed)
    head = (b.verts, b.faces, b.first_face, b.num_faces, b.cams, b.colors, S, K, blur, w.clip_barycentric_coords,
            w.sigma, w.gamma, w.znear, w.zfar, mode)

    def jobs(per, seed):
        px = workloads.sample_pixels(b.N, S, per, seed)
        g = g_full[px[:, 0], px[:, 1], px[:, 2]]
        order = np.random.default_rng(seed).permutation(px.shape[0])   # every share mixes the images
        return [head + (px[np.sort(sl)], g[np.sort(sl)]) for sl in np.array_split(order, workers) if sl.size]

    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_pixels, jobs(max(1, workers // b.N + 1), 21)))   # start the workers, load the oracle
        todo = jobs(per_image, 22)
        t0 = time.perf_counter()
        n = sum(ex.map(_oracle_pixels, todo))
        t = time.perf_counter() - t0
    return {"value": n * K / t / 1e6, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": "%d pixels (%d per image, seeded) through the same FP64 oracle calls, split over %d "
                      "spawned processes, %.1f s" % (n, per_image, workers, t)}


def time_fit_loop(w, tuned, dev, flush, iters=100):
    """Workload 4's analysis-by-synthesis loop: ``iters`` graph replays of one
    fitting step (render 20 soft silhouettes, negative IoU, fused backward,
    Adam) against the silhouettes of a differently seeded sphere."""
    import torch
    from paper_2007_08501_gb300 import autograd as ag
    from paper_2007_08501_gb300 import workloads
    from paper_2007_08501_gb300.fit import SilhouetteFitter
    b = w.batch
    views = b.N
    F0 = int(b.num_faces[0])
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    verts, faces0, cams = T(b.verts), T(b.faces[:F0]), T(b.cams)
    # the mesh moves while it is fitted: four times the capacities tuned on the start mesh
    rs = ag.RasterSettings(w.image_size, w.K, float(np.float32(w.blur_radius)), bin_size=tuned["bin_size"],
                           max_faces_per_bin=4 * tuned["max_faces_per_bin"],
                           max_bin_entries=4 * tuned["max_bin_entries"],
                           clip_barycentric_coords=w.clip_barycentric_coords)
    bs = ag.BlendSettings(sigma=w.sigma, gamma=w.gamma, znear=w.znear, zfar=w.zfar, rgb=False)
    tv, tf = workloads.target_sphere()
    tverts = T(tv.astype(np.float32))
    tfaces = T(tf.astype(np.int64)).repeat(views, 1)
    ff = torch.arange(views, device=dev, dtype=torch.int64) * tf.shape[0]
    nf = torch.full((views,), tf.shape[0], device=dev, dtype=torch.int64)
    trs = ag.RasterSettings(w.image_size, w.K, float(np.float32(w.blur_radius)), bin_size=tuned["bin_size"],
                            max_faces_per_bin=4096, clip_barycentric_coords=w.clip_barycentric_coords)
    with torch.no_grad():
        target = ag.blend(*ag.rasterize_meshes(tverts, tfaces, ff, nf, cams, trs), settings=bs)[..., 3].clone()
    fitter = SilhouetteFitter(verts, faces0, cams, target, rs, bs, lr=2e-3).capture(warmup=3)
    l0 = float(fitter.replay(1))
    flush.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fitter.replay(iters)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    return {"iterations": iters, "ms_per_iteration": round(ms / iters, 4), "loss_first": round(l0, 6),
            "loss_last": round(float(fitter.loss), 6), "status": fitter.ws.status(),
            "step": "render 20 soft silhouettes + negative IoU + fused backward + Adam, one CUDA graph"}


def run_ours(args):
    import torch
    from paper_2007_08501_gb300 import ops, workloads

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ops.load()
    widx, wvar, wdesc = WORKLOADS[args.workload]
    w = workloads.workload(widx, wvar)
    if args.max_images:
        w.batch = workloads.first_images(w.batch, args.max_images)
        wdesc += " (first %d images)" % w.batch.N
    b = w.batch
    slots = b.N * w.image_size * w.image_size * w.K

    # launch parameters from the autotuner (outside the timed region)
    from paper_2007_08501_gb300 import tune
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    tuned = tune.tune(T(b.verts), T(b.faces), T(b.first_face), T(b.num_faces), T(b.cams), w.image_size, w.K,
                      float(np.float32(w.blur_radius)), w.perspective_correct, w.clip_barycentric_coords,
                      bin_sizes=(args.bin_size,) if args.bin_size else (8, 16))
    shading = {"1gouraud": ops.SHADE_GOURAUD, "1phong": ops.SHADE_PHONG}.get(args.workload)
    pipe = Pipeline(w, bin_size=tuned["bin_size"], max_faces_per_bin=tuned["max_faces_per_bin"], device=dev,
                    max_bin_entries=tuned["max_bin_entries"], shading=shading)
    pipe.run_eager()
    torch.cuda.synchronize()
    st = pipe.status()
    if st != 0:
        raise RuntimeError("device status %d after the first step" % st)
    mc, tot = ops.rast_bin_occupancy(pipe.p, b.V, b.F, pipe.ws)
    fine_tests = int(tot) * tuned["bin_size"] ** 2
    # pixels the large-K streaming fine pass handed to its second pass (ring overflow)
    lay = ops.rast_workspace_bin_layout(pipe.p, b.V, b.F)
    redo_pixels = int(pipe.ws[lay["redo"]:lay["redo"] + 4].cpu().numpy().view(np.uint32)[0])
    pipe.capture()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    gpu_index = None
    try:
        gpu_index = torch.cuda.get_device_properties(dev).uuid
        gpu_index = "GPU-" + str(gpu_index) if not str(gpu_index).startswith("GPU-") else str(gpu_index)
    except Exception:
        gpu_index = None
    clocks = ClockSampler(gpu_index)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    per_step = timed_steps(pipe, args.steps, args.warmup, flush, use_graph=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [sum(s.values()) for s in per_step]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms = total_ms / args.steps
    value = whole_job_rate(slots, world, ms)
    st = pipe.status()

    stages = {k: statistics.mean(s[k] for s in per_step) for k in per_step[0]}
    dom = max(stages, key=stages.get)
    alg = algorithmic_bytes(w)
    peak, peak_kind = _peaks()
    achieved = alg[dom] / (stages[dom] / 1e3) / 1e9
    tr = TRAFFIC_BYTES.get((args.workload, dom, tuned["bin_size"]))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": tr["bytes"] if tr else None,
                "traffic_kernel": tr["kernel"] if tr else None,
                "traffic_source": ("ncu capture, " + tr["profile"]) if tr else None,
                "algorithmic_bytes": alg[dom], "kernel": dom,
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
                else "fallback 6.8 TB/s"}
    stage_frac = {k: round(alg[k] / (stages[k] / 1e3) / 1e9 / peak, 4) for k in stages}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    pin = lambda t: t.cpu().pin_memory()
    h_in = [(pipe.verts, pin(pipe.verts)), (pipe.faces, pin(pipe.faces)), (pipe.ff, pin(pipe.ff)),
            (pipe.nf, pin(pipe.nf)), (pipe.cams, pin(pipe.cams)), (pipe.colors, pin(pipe.colors)),
            (pipe.gimg, pin(pipe.gimg))]
    h_out = [(pipe.img, torch.empty_like(pipe.img, device="cpu").pin_memory()),
             (pipe.gv, torch.empty_like(pipe.gv, device="cpu").pin_memory())]
    h2d = sum(h.numel() * h.element_size() for _, h in h_in)
    d2h = sum(h.numel() * h.element_size() for _, h in h_out)
    # (a) serial: every copy and every call on one stream
    e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for d, h in h_in:
            d.copy_(h, non_blocking=True)
        for _, g in pipe.graphs:
            g.replay()
        for d, h in h_out:
            h.copy_(d, non_blocking=True)
        e1.record()
        e1.synchronize()
        if i >= args.warmup:
            e_ms.append(e0.elapsed_time(e1))
    # (b) overlapped, as a serving loop would run it: the upstream gradient
    # goes up on a second stream while the forward runs, and the image comes
    # down on it while the backward runs (the calls take the stream to use)
    main = torch.cuda.current_stream(dev)
    cs = torch.cuda.Stream(dev)
    h_gimg = dict((id(d), h) for d, h in h_in)[id(pipe.gimg)]
    fwd_in = [(d, h) for d, h in h_in if d is not pipe.gimg]
    fwd_graphs = [g for name, g in pipe.graphs if "fwd" in name]
    bwd_graphs = [g for name, g in pipe.graphs if "fwd" not in name]
    h_img = h_out[0][1]
    o_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev_g, ev_f, ev_i = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
        e0.record(main)
        cs.wait_event(e0)
        with torch.cuda.stream(cs):
            pipe.gimg.copy_(h_gimg, non_blocking=True)
            ev_g.record(cs)
        for d, h in fwd_in:
            d.copy_(h, non_blocking=True)
        for g in fwd_graphs:
            g.replay()
        ev_f.record(main)
        cs.wait_event(ev_f)
        with torch.cuda.stream(cs):
            h_img.copy_(pipe.img, non_blocking=True)
            ev_i.record(cs)
        main.wait_event(ev_g)
        for g in bwd_graphs:
            g.replay()
        for d, h in h_out[1:]:
            h.copy_(d, non_blocking=True)
        main.wait_event(ev_i)
        e1.record(main)
        e1.synchronize()
        if i >= args.warmup:
            o_ms.append(e0.elapsed_time(e1))
    e2e_serial_ms = max_over_ranks(statistics.mean(e_ms), dist, dev)
    e2e_ms = max_over_ranks(statistics.mean(o_ms), dist, dev)
    e2e = {"value": round(whole_job_rate(slots, world, e2e_ms), 1), "unit": UNIT,
           "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "copies": "upstream gradient uploaded on a second stream during the forward, image downloaded on it "
                     "during the backward; other inputs before the forward, vertex gradients after the backward",
           "serial_ms_per_step": round(e2e_serial_ms, 4),
           "serial_value": round(whole_job_rate(slots, world, e2e_serial_ms), 1)}

    separate = None
    if not args.no_separate and shading is None:
        # the same step as four C-ABI calls (rast_mesh_fwd, blend_fwd, blend_bwd, rast_mesh_bwd)
        sp = Pipeline(w, bin_size=tuned["bin_size"], max_faces_per_bin=tuned["max_faces_per_bin"], device=dev,
                      max_bin_entries=tuned["max_bin_entries"], fused=False)
        sp.capture()
        ss = timed_steps(sp, args.steps, 3, flush, use_graph=True)
        sstages = {k: round(statistics.mean(s[k] for s in ss), 4) for k in ss[0]}
        separate = {"ms_per_step": round(statistics.mean(sum(s.values()) for s in ss), 4),
                    **{k + "_ms": v for k, v in sstages.items()}}
        del sp

    # silhouette forward without Fragment data (the fine pass blends and writes
    # only the image; nothing is left for a backward pass): forward-only use
    sil_only = None
    if shading is None and w.blend_mode != "rgb" and w.K <= 16 and tuned["bin_size"] > 0:
        import torch as _t
        img2 = _t.empty_like(pipe.img)
        fn = lambda: ops.rast_blend_fwd(pipe.p, pipe.bp, pipe.verts, pipe.faces, pipe.ff, pipe.nf, pipe.cams, None,
                                        None, None, None, None, img2, pipe.ws)
        fn()
        _t.cuda.synchronize()
        g = _t.cuda.CUDAGraph()
        with _t.cuda.graph(g):
            fn()
        ts = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = _t.cuda.Event(enable_timing=True), _t.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            e1.synchronize()
            if i >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        same = bool(_t.equal(img2, pipe.img))
        sil_only = {"fwd_ms": round(statistics.mean(ts), 4), "fwd_with_fragments_ms": round(stages["fwd"], 4),
                    "fragment_bytes_not_written": slots * 28, "image_identical": same}
        del g, img2

    plain = None
    if not args.no_plain and (args.workload in ("1", "4") or args.plain):
        # the plain per-mesh form: one unbinned launch per image (no graph);
        # a few steps, each of them seconds long at the larger workloads
        pp = Pipeline(w, bin_size=0, max_faces_per_bin=1, device=dev)
        pp.run_eager()
        small = args.workload == "1"
        ps = timed_steps(pp, max(3, args.steps // 2) if small else 2, 2 if small else 1, flush, use_graph=False)
        pms = statistics.mean(sum(s.values()) for s in ps)
        pstages = {k: round(statistics.mean(s[k] for s in ps), 4) for k in ps[0]}
        plain = {"ms_per_step": round(pms, 4), "value": round(slots / (pms / 1e3) / 1e6, 1),
                 "fwd_ms": pstages["fwd"], "launches_per_step": b.N + 1 + 1 + 2,
                 "speedup_of_binned": round(pms / ms, 3)}

    # the FP32 FMA peak of this GPU (the ALU ceiling of the fine pass's face tests)
    fp32_fma = measure_fp32_peak(dev)
    fp32 = {"fma_lane_ops_per_s": round(fp32_fma, 1), "tflops": round(2 * fp32_fma / 1e12, 2),
            "probe": "meshrast_fma_probe: 8 blocks x 256 threads per SM, 8 FMA chains per thread, best of 5",
            "derived_at_max_clock_tflops": round(2 * FP32_LANE_OPS_PEAK / 1e12, 2)}

    fit_loop = None
    if args.workload == "4" and not args.no_fit:
        fit_loop = time_fit_loop(w, tuned, dev, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w)
    cpu_par = None
    if cpu is not None and (os.cpu_count() or 1) > 1:
        ncores = os.cpu_count()
        per = min(w.image_size * w.image_size, cpu.pop("per_image") * ncores)
        cpu_par = cpu_baseline_parallel(w, per, ncores)
    elif cpu is not None:
        cpu.pop("per_image")

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wdesc, "N": b.N, "image_size": w.image_size, "K": w.K, "faces": b.F,
                       "verts": b.V, "slots": slots, "blur_radius": float(np.float32(w.blur_radius)),
                       "bin_size": tuned["bin_size"], "max_faces_per_bin": tuned["max_faces_per_bin"],
                       "max_bin_entries": tuned["max_bin_entries"], "autotuned": True,
                       "graph": "one CUDA graph per C-ABI call",
                       "calls": "rast_blend_fwd (%s) + blend_rast_bwd (blend adjoint fused with the rasterizer "
                                "adjoint)" % ("the silhouette blend applied as the Fragment data is written: by the "
                                              "fine pass for K <= 16, by the attribute pass for K > 16"
                                              if w.blend_mode == "sil" else
                                              "softmax blend kernel inside the call, after the fine pass"),
                       "l2": "flushed between steps (256 MiB write), outside the timed events",
                       "bin_occupancy": {"max_faces_in_a_bin": mc, "total_entries": tot},
                       "redo_pixels": redo_pixels,
                       "parallelism": "replicas x%d" % world},
            "roofline": roofline,
            "stages_ms": {k: round(v, 4) for k, v in stages.items()},
            "stages_hbm_frac": stage_frac,
            "cpu_baseline": cpu, "cpu_baseline_parallel": cpu_par, "e2e": e2e,
            "gpu_launches": (8 if shading is not None else mesh_kernels_per_step(w)) * args.steps,
            "ms_per_step_median": round(statistics.median(step_ms), 4),
            "fine_pass": {"face_pixel_tests": fine_tests,
                          "tests_per_s": round(fine_tests / (stages.get("fwd", stages.get("rast_fwd")) / 1e3), 1),
                          "note": "sum over bins of (pixels in bin x faces in bin)"},
            "clocks": clk, "fp32_peak": fp32, "unfused": separate, "silhouette_without_fragments": sil_only,
            "plain_form": plain,
            "fit_loop": fit_loop,
            "status": st,
            "wall_s_timed_region": round(wall, 3),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


class PointPipeline:
    """Static buffers + one CUDA graph per C-ABI call of the point renderer step:
    rasterize, composite, composite adjoint, rasterizer adjoint."""

    def __init__(self, w, bin_size, max_per_bin, max_entries, device):
        import torch
        from paper_2007_08501_gb300 import ops
        self.torch, self.ops = torch, ops
        b = w.batch
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.points, self.first, self.num, self.cams = T(b.points), T(b.first_point), T(b.num_points), T(b.cams)
        self.feats = T(b.features)
        self.mode = w.mode
        self.dev = device
        N, S, K = b.N, w.image_size, w.K
        self.p = ops.make_pts_params(N, S, K, w.radius, bin_size, max_per_bin, max_entries)
        self.ws = ops.alloc_pts_workspace(self.p, b.P, device)
        self.frag = ops.alloc_pts_fragments(N, S, K, device)
        self.img = torch.empty((N, S, S, b.features.shape[1]), device=device)
        rng = np.random.default_rng(w.grad_seed)
        self.gimg = T(rng.normal(size=(N, S, S, b.features.shape[1])).astype(np.float32))
        self.gd = torch.empty_like(self.frag[2])
        self.gf = torch.empty_like(self.feats)
        self.gp = torch.empty_like(self.points)
        self.graphs = None

    def stages(self):
        ops = self.ops
        idx, zb, di = self.frag
        return [
            ("rast_fwd", lambda: ops.pts_rasterize_fwd(self.p, self.points, self.first, self.num, self.cams, idx, zb,
                                                       di, self.ws)),
            ("composite_fwd", lambda: ops.pts_composite_fwd(self.p, self.mode, idx, di, self.feats, self.img)),
            ("composite_bwd", lambda: ops.pts_composite_bwd(self.p, self.mode, idx, di, self.feats, self.gimg,
                                                            self.gd, self.gf)),
            ("rast_bwd", lambda: ops.pts_rasterize_bwd(self.p, self.points, self.first, self.num, self.cams, idx,
                                                       None, self.gd, self.gp, self.ws)),
        ]

    run_eager = Pipeline.run_eager
    capture = Pipeline.capture

    def status(self):
        return self.ops.rast_query_status(self.ws)


def point_bytes(w):
    b = w.batch
    N, S, K, D = b.N, w.image_size, w.K, b.features.shape[1]
    slots, pix, P = N * S * S * K, N * S * S, b.P
    return {"rast_fwd": 12 * P + 16 * slots,                       # points in, idx + zbuf + dists out
            "composite_fwd": 12 * slots + 4 * D * pix,             # idx + dists in, image out
            "composite_bwd": 12 * slots + 4 * D * pix + 4 * slots + 4 * D * P,
            "rast_bwd": 12 * P + 12 * slots + 12 * P}              # idx + grad dists in, grad points out


def point_cpu_baseline(w, target_s=15.0):
    from oracle import points as op
    from paper_2007_08501_gb300 import workloads
    c = op.Clouds.from_batch(w.batch)
    r = float(np.float32(w.radius))
    S, K = w.image_size, w.K
    rng = np.random.default_rng(w.grad_seed)

    def run(per_image, seed):
        px = workloads.sample_pixels(w.batch.N, S, per_image, seed)
        t0 = time.perf_counter()
        idx, zb, di = op.rasterize(c, S, K, r, pixels=px)
        g = rng.normal(size=(px.shape[0], w.batch.features.shape[1]))
        op.composite_fwd(idx, di, w.batch.features, r, w.mode)
        gd, _ = op.composite_bwd(idx, di, w.batch.features, r, g, w.mode)
        op.rast_bwd(c, S, K, idx, None, gd, pixels=px)
        return px.shape[0], time.perf_counter() - t0

    n0, t0 = run(4, 11)
    per_image = int(max(4, min(S * S, 4 * target_s / max(t0, 1e-3))))
    n, t = run(per_image, 12)
    return {"value": n * K / t / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d pixels (%d per image, seeded) through the FP64 point oracle (every point of the cloud "
                      "per pixel + compositing fwd/bwd + adjoint), %.1f s" % (n, per_image, t)}


def run_points(args):
    import torch
    from paper_2007_08501_gb300 import ops, workloads
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ops.load()
    _, variant, wdesc = WORKLOADS[args.workload]
    w = workloads.point_workload(ops.PTS_ALPHA if variant == "alpha" else ops.PTS_NORM)
    b = w.batch
    slots = b.N * w.image_size * w.image_size * w.K
    # bin size and capacities: one generous probe run per candidate bin size, then
    # a few timed forwards with the sized capacities (outside the timed region)
    best = None
    for bs in ((args.bin_size,) if args.bin_size else (8, 16)):
        probe = PointPipeline(w, bs, 1 << 16, 0, dev)
        probe.stages()[0][1]()
        mc_, tot_ = ops.pts_bin_occupancy(probe.p, b.P, probe.ws)
        del probe
        per_bin_ = max(64, int(np.ceil(mc_ * 1.25 / 64.0)) * 64)
        entries_ = max(1024, int(np.ceil(tot_ * 1.25)))
        trial = PointPipeline(w, bs, per_bin_, entries_, dev)
        fwd = trial.stages()[0][1]
        ts = []
        for i in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fwd()
            e1.record()
            e1.synchronize()
            if i >= 2:
                ts.append(e0.elapsed_time(e1))
        del trial
        if best is None or statistics.median(ts) < best[0]:
            best = (statistics.median(ts), bs, per_bin_, entries_, mc_, tot_)
    _, bin_size, per_bin, entries, mc, tot = best
    pipe = PointPipeline(w, bin_size, per_bin, entries, dev)
    pipe.run_eager()
    torch.cuda.synchronize()
    st = pipe.status()
    if st != 0:
        raise RuntimeError("device status %d after the first step" % st)
    pipe.capture()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    per_step = timed_steps(pipe, args.steps, args.warmup, flush, use_graph=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(sum(s.values()) for s in per_step), dist, dev)
    ms = total_ms / args.steps
    value = whole_job_rate(slots, world, ms)
    stages = {k: statistics.mean(s[k] for s in per_step) for k in per_step[0]}
    dom = max(stages, key=stages.get)
    alg = point_bytes(w)
    peak, peak_kind = _peaks()
    achieved = alg[dom] / (stages[dom] / 1e3) / 1e9
    tr = TRAFFIC_BYTES.get((args.workload, dom, bin_size))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": tr["bytes"] if tr else None,
                "traffic_kernel": tr["kernel"] if tr else None,
                "traffic_source": ("ncu capture, " + tr["profile"]) if tr else None,
                "algorithmic_bytes": alg[dom], "kernel": dom,
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
                else "fallback 6.8 TB/s"}
    # end to end with host buffers
    pin = lambda t: t.cpu().pin_memory()
    h_in = [(pipe.points, pin(pipe.points)), (pipe.first, pin(pipe.first)), (pipe.num, pin(pipe.num)),
            (pipe.cams, pin(pipe.cams)), (pipe.feats, pin(pipe.feats)), (pipe.gimg, pin(pipe.gimg))]
    h_out = [(pipe.img, torch.empty_like(pipe.img, device="cpu").pin_memory()),
             (pipe.gp, torch.empty_like(pipe.gp, device="cpu").pin_memory())]
    e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for d_, h in h_in:
            d_.copy_(h, non_blocking=True)
        for _, g in pipe.graphs:
            g.replay()
        for d_, h in h_out:
            h.copy_(d_, non_blocking=True)
        e1.record()
        e1.synchronize()
        if i >= args.warmup:
            e_ms.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(statistics.mean(e_ms), dist, dev)
    e2e = {"value": round(whole_job_rate(slots, world, e2e_ms), 1), "unit": UNIT, "ms_per_step": round(e2e_ms, 4),
           "h2d_bytes_per_step": sum(h.numel() * h.element_size() for _, h in h_in),
           "d2h_bytes_per_step": sum(h.numel() * h.element_size() for _, h in h_out)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = point_cpu_baseline(w)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wdesc, "N": b.N, "image_size": w.image_size, "K": w.K, "points": b.P,
                       "slots": slots, "radius": w.radius, "bin_size": bin_size, "max_points_per_bin": per_bin,
                       "max_bin_entries": entries, "graph": "one CUDA graph per C-ABI call",
                       "l2": "flushed between steps (256 MiB write), outside the timed events",
                       "bin_occupancy": {"max_points_in_a_bin": mc, "total_entries": tot},
                       "parallelism": "replicas x%d" % world},
            "roofline": roofline, "stages_ms": {k: round(v, 4) for k, v in stages.items()},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 7 * args.steps, "clocks": clk, "status": st,
            "paper_context": {"ms_per_step": 75.0, "hardware": "V100", "what": "8 clouds x 200k points, 256x256, "
                              "K=50, fwd+bwd, ShapeNet samples (radius not stated)"}}), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_reference_points(args, variant, wdesc):
    """The FP64 point oracle on host cores, a bounded pixel sample per step."""
    from oracle import points as op
    from paper_2007_08501_gb300 import workloads
    w = workloads.point_workload(0 if variant == "alpha" else 1)
    c = op.Clouds.from_batch(w.batch)
    r = float(np.float32(w.radius))
    S, K = w.image_size, w.K
    per_image = 4
    rng = np.random.default_rng(w.grad_seed)

    def step(seed):
        px = workloads.sample_pixels(w.batch.N, S, per_image, seed)
        idx, zb, di = op.rasterize(c, S, K, r, pixels=px)
        op.composite_fwd(idx, di, w.batch.features, r, w.mode)
        gd, _ = op.composite_bwd(idx, di, w.batch.features, r, rng.normal(size=(px.shape[0], 1)), w.mode)
        op.rast_bwd(c, S, K, idx, None, gd, pixels=px)
        return px.shape[0]

    for i in range(args.warmup):
        step(100 + i)
    t0 = time.perf_counter()
    n = sum(step(1000 + i) for i in range(args.steps))
    t = time.perf_counter() - t0
    value = n * K / t / 1e6
    sample = "%d pixels per step (%d per image, seeded), FP64 point oracle: rasterize + composite fwd/bwd + " \
             "adjoint" % (per_image * w.batch.N, per_image)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get(
            "WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": {"workload": wdesc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def run_reference(args):
    """The FP64 CPU oracle, timed on host cores on a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2007_08501_gb300 import workloads
    oracle.build()
    widx, wvar, wdesc = WORKLOADS[args.workload]
    if args.workload in KNN_WORKLOADS:
        return run_reference_knn(args, wdesc)
    if widx is None:
        return run_reference_points(args, wvar, wdesc)
    w = workloads.workload(widx, wvar)
    m = oracle.Mesh.from_batch(w.batch)
    blur = float(np.float32(w.blur_radius))
    S, K = w.image_size, w.K
    g_full = workloads.upstream_grad(w.batch.N, S, w.grad_seed)
    per_image = max(8, 2048 // w.batch.N) if args.workload == "1" else max(4, 256 // w.batch.N)

    def step(seed):
        px = workloads.sample_pixels(w.batch.N, S, per_image, seed)
        fr = oracle.rasterize(m, S, K, blur, True, w.clip_barycentric_coords, pixels=px)
        g = g_full[px[:, 0], px[:, 1], px[:, 2]]
        mode = 1 if w.blend_mode == "rgb" else 0
        oracle.blend_fwd(*fr, w.batch.faces, w.batch.colors, w.sigma, w.gamma, w.znear, w.zfar, mode=mode)
        gz, gb, gd, _ = oracle.blend_bwd(*fr, w.batch.faces, w.batch.colors, g, w.sigma, w.gamma, w.znear, w.zfar,
                                         mode=mode)
        oracle.rast_bwd(m, S, K, fr[0], gz, gb, gd, blur, True, w.clip_barycentric_coords, pixels=px)
        return px.shape[0]

    for i in range(args.warmup):
        step(100 + i)
    t0 = time.perf_counter()
    n = 0
    for i in range(args.steps):
        n += step(1000 + i)
    t = time.perf_counter() - t0
    value = n * K / t / 1e6
    sample = "%d pixels per step (%d per image, seeded), FP64 oracle: rasterize + blend fwd/bwd + adjoint" % (
        per_image * w.batch.N, per_image)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get(
            "WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": {"workload": wdesc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


# ---------------------------------------------------------------------------
# exact KNN and the Chamfer loss (Section 3.1 operators)
# ---------------------------------------------------------------------------
KNN_WORKLOADS = ("knn", "knn_het", "chamfer")
KNN_METRIC = "exact KNN / Chamfer ms per batch & candidate distances per second (Gpair/s), % FP32 ALU roofline"
KNN_UNIT = "Gpair/s"
# FP32 lane operations one candidate distance needs at least: D subtractions,
# one multiply and D - 1 fused multiply-adds (D = 3)
KNN_OPS_PER_PAIR = 6
FP32_LANE_OPS_PEAK = 152 * 128 * 2.07e9   # SMs x FP32 lanes x max SM clock (derived, not measured)


class KnnPipeline:
    """Static buffers + one CUDA graph per C-ABI call: knn_points, or
    chamfer_fwd then chamfer_bwd."""

    def __init__(self, w, device):
        import torch
        from paper_2007_08501_gb300 import ops
        self.torch, self.ops = torch, ops
        c = w.pairs
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.p, self.q = T(c.p), T(c.q)
        self.f1, self.l1, self.f2, self.l2 = T(c.first1), T(c.len1), T(c.first2), T(c.len2)
        self.K, self.chamfer = w.K, w.chamfer
        self.dev = device
        self.ws = ops.alloc_knn_workspace(c.N, device)
        P1, P2 = c.p.shape[0], c.q.shape[0]
        if self.chamfer:
            self.idx_pq = torch.empty(P1, dtype=torch.int64, device=device)
            self.d_pq = torch.empty(P1, device=device)
            self.idx_qp = torch.empty(P2, dtype=torch.int64, device=device)
            self.d_qp = torch.empty(P2, device=device)
            self.per = torch.empty(c.N, device=device)
            self.loss = torch.empty(1, device=device)
            self.gl = torch.ones(1, device=device)
            self.gp, self.gq = torch.empty_like(self.p), torch.empty_like(self.q)
        else:
            self.idx = torch.empty((P1, w.K), dtype=torch.int64, device=device)
            self.dists = torch.empty((P1, w.K), device=device)
        self.graphs = None

    def stages(self):
        ops = self.ops
        if not self.chamfer:
            return [("knn", lambda: ops.knn_points(self.p, self.f1, self.l1, self.q, self.f2, self.l2, self.K,
                                                   self.idx, self.dists, self.ws))]
        return [
            ("chamfer_fwd", lambda: ops.chamfer_fwd(self.p, self.f1, self.l1, self.q, self.f2, self.l2, self.idx_pq,
                                                    self.d_pq, self.idx_qp, self.d_qp, self.per, self.loss, self.ws)),
            ("chamfer_bwd", lambda: ops.chamfer_bwd(self.p, self.f1, self.l1, self.q, self.f2, self.l2, self.idx_pq,
                                                    self.idx_qp, self.gl, None, self.gp, self.gq)),
        ]

    run_eager = Pipeline.run_eager
    capture = Pipeline.capture

    def inputs(self):
        return [self.p, self.f1, self.l1, self.q, self.f2, self.l2]

    def outputs(self):
        return [self.loss, self.gp, self.gq] if self.chamfer else [self.idx, self.dists]


def knn_cpu_baseline(w, target_s=10.0, seed=17):
    """The oracle on host cores (one core): (candidate distances per second, seconds, sample text).
    KNN: a seeded sample of query rows per cloud, sized to take about target_s.
    Chamfer: the whole Eq. 1 loss and gradient (KNN both ways + FP64 sums) on
    the first cloud pairs of the batch, as many as fit in about target_s."""
    from oracle import knn as ok
    from paper_2007_08501_gb300 import workloads
    c = w.pairs
    if w.chamfer:
        def run(npair):
            sub = workloads.CloudPairs(c.p[:int(c.first1[npair - 1] + c.len1[npair - 1])], c.first1[:npair],
                                       c.len1[:npair], c.q[:int(c.first2[npair - 1] + c.len2[npair - 1])],
                                       c.first2[:npair], c.len2[:npair])
            t0 = time.perf_counter()
            _, _, ipq, iqp = ok.chamfer(sub.p, sub.first1, sub.len1, sub.q, sub.first2, sub.len2)
            ok.chamfer_grad(sub.p, sub.first1, sub.len1, sub.q, sub.first2, sub.len2, ipq, iqp, np.ones(npair))
            return workloads.pairs_per_batch(sub, both_ways=True), time.perf_counter() - t0
        n, t = run(1)
        k = int(max(1, min(c.N, target_s / max(t, 1e-3))))
        n, t = run(k)
        return n / t, t, "the first %d of %d cloud pairs through the oracle's Chamfer loss and gradient (KNN " \
                         "both ways in C, sums in FP64), %.1f s" % (k, c.N, t)
    rng = np.random.default_rng(seed)

    def run(per_cloud):
        rows = np.concatenate([f + rng.choice(n, size=min(per_cloud, n), replace=False)
                               for f, n in zip(c.first1, c.len1) if n > 0])
        npairs = int(np.sum(c.len2 * np.minimum(per_cloud, c.len1)))
        t0 = time.perf_counter()
        ok.knn(c.p, c.first1, c.len1, c.q, c.first2, c.len2, w.K, rows=rows)
        return npairs, time.perf_counter() - t0, rows.size

    n, t, _ = run(2)
    per_cloud = int(max(2, 2 * target_s / max(t, 1e-3)))
    n, t, nrows = run(per_cloud)
    return n / t, t, "%d seeded query rows (%d per cloud) against every candidate of their cloud through the " \
                     "oracle's KNN (K = %d), %.1f s" % (nrows, per_cloud, w.K, t)


def run_knn(args):
    import torch
    from paper_2007_08501_gb300 import ops, workloads
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ops.load()
    wdesc = WORKLOADS[args.workload][2]
    w = workloads.knn_workload(args.workload)
    c = w.pairs
    pairs = workloads.pairs_per_batch(c, both_ways=w.chamfer)
    pipe = KnnPipeline(w, dev)
    pipe.run_eager()
    torch.cuda.synchronize()
    pipe.capture()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    per_step = timed_steps(pipe, args.steps, args.warmup, flush, use_graph=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(sum(s.values()) for s in per_step), dist, dev)
    ms = total_ms / args.steps
    value = whole_job_rate(pairs, world, ms, 1e9)
    stages = {k: statistics.mean(s[k] for s in per_step) for k in per_step[0]}
    dom = "chamfer_fwd" if w.chamfer else "knn"
    achieved = pairs * KNN_OPS_PER_PAIR / (stages[dom] / 1e3)
    peak_ops = measure_fp32_peak(dev)
    roofline = {"bound": "alu", "achieved": round(achieved / 1e12, 3), "peak": round(peak_ops / 1e12, 2),
                "unit": "T FP32 lane-op/s", "frac": round(achieved / peak_ops, 4), "traffic": None,
                "kernel": "k_knn (%s call)" % dom,
                "ops_per_pair": KNN_OPS_PER_PAIR, "pairs_per_launch": pairs,
                "peak_source": "measured in this run: meshrast_fma_probe (FMA lane operations per second)",
                "derived_peak": round(FP32_LANE_OPS_PEAK / 1e12, 2)}
    # end to end with host buffers: inputs in, results out, every step
    pin = lambda t: t.cpu().pin_memory()
    h_in = [(d_, pin(d_)) for d_ in pipe.inputs()]
    h_out = [(d_, torch.empty_like(d_, device="cpu").pin_memory()) for d_ in pipe.outputs()]
    e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for d_, h in h_in:
            d_.copy_(h, non_blocking=True)
        for _, g in pipe.graphs:
            g.replay()
        for d_, h in h_out:
            h.copy_(d_, non_blocking=True)
        e1.record()
        e1.synchronize()
        if i >= args.warmup:
            e_ms.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(statistics.mean(e_ms), dist, dev)
    e2e = {"value": round(whole_job_rate(pairs, world, e2e_ms, 1e9), 2), "unit": KNN_UNIT, "ms_per_step": round(e2e_ms, 4),
           "h2d_bytes_per_step": sum(h.numel() * h.element_size() for _, h in h_in),
           "d2h_bytes_per_step": sum(h.numel() * h.element_size() for _, h in h_out)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, t, sample = knn_cpu_baseline(w)
        cpu = {"value": round(v / 1e9, 5), "unit": KNN_UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps({
            "metric": KNN_METRIC, "value": round(value, 2), "unit": KNN_UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wdesc, "N": c.N, "P1": int(c.p.shape[0]), "P2": int(c.q.shape[0]), "D": 3,
                       "K": w.K, "candidate_distances_per_step": pairs, "graph": "one CUDA graph per C-ABI call",
                       "l2": "flushed between steps (256 MiB write), outside the timed events",
                       "parallelism": "replicas x%d" % world},
            "roofline": roofline, "stages_ms": {k: round(v, 4) for k, v in stages.items()},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": (5 if w.chamfer else 2) * args.steps, "clocks": clk,
            "ms_per_step_median": round(statistics.median(sum(s.values()) for s in per_step), 4)}), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_reference_knn(args, wdesc):
    """The oracle's KNN on host cores, a bounded sample of query rows per step."""
    from paper_2007_08501_gb300 import workloads
    w = workloads.knn_workload(args.workload)
    for i in range(args.warmup):
        knn_cpu_baseline(w, 0.5, seed=100 + i)
    n = t = 0.0
    sample = ""
    for i in range(args.steps):
        v, ti, sample = knn_cpu_baseline(w, 5.0, seed=1000 + i)
        n += v * ti
        t += ti
    value = n / t / 1e9
    print(json.dumps({
        "impl": "reference", "metric": KNN_METRIC, "value": value, "unit": KNN_UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": {"workload": wdesc},
        "cpu_baseline": {"value": value, "unit": KNN_UNIT, "cores": 1, "kind": "oracle",
                         "sample": "per step: " + sample},
        "e2e": {"value": value, "unit": KNN_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


if __name__ == "__main__":
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload in KNN_WORKLOADS:
        run_knn(a)
    elif a.workload.startswith("points"):
        run_points(a)
    else:
        run_ours(a)
