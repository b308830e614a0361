// Point-cloud rasterizer and compositing for sm_103a (Section 3.2 of the
// paper, "Differentiable point cloud renderer"), with the C ABI of
// include/points.h.
//
//   k_pstage   one thread per point: double-float projection, 32-byte record
//              (NDC position hi/lo, depth), warp-aggregated bin counts
//   k_scan     (shared with the mesh rasterizer) clamp counts, prefix scan
//   k_pfill    one thread per point: append depth-keyed entries to its bins
//   k_pfine    persistent blocks over (image, bin) items: the bin's entries
//              sorted front to back, staged in shared memory, 32 points per
//              warp ballot; per-pixel top-K by (depth, id); stops a bin once
//              every lane's K-th depth lies in front of the next point
//   k_pnaive   the plain form: one launch per image, every pixel against
//              every point of its cloud
//   k_pcomp_fwd / k_pcomp_bwd   Alpha / Norm compositing and its adjoint
//   k_prast_bwd  dL/d(zbuf, dists) -> dL/dpoints through the projection
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "bin_common.cuh"
#include "meshrast.h"
#include "points.h"
#include "rast_common.cuh"
#include "rast_internal.h"

namespace mr {

// Point record (32 bytes): a = (x_hi, y_hi, x_lo, y_lo) in NDC, b = (depth,
// 0, 0, 0); culled points have depth +inf and are never binned.
struct __align__(16) PtRec {
    float4 a, b;
};
static_assert(sizeof(PtRec) == 32, "point record is 32 bytes");

constexpr float kPtSlack = 1e-5f;  // relative widening of a splat's box for binning

struct PtArgs {
    const float *points;
    int64_t P;
    const int64_t *first, *num;
    int N;
    const float *cams;
    float radius, r2;
    int S, K, bin, nb;
    int64_t items;
    PtRec *rec;
    int *cloud;
    int *counts, *cursor;
    const int *eff, *offsets;
    unsigned long long *lists;
    unsigned *queue, *status;
    int sort_cap;
    int64_t *idx;
    float *zbuf, *dists;
};

// box of a splat, widened so that every pixel passing d < r^2 in fp32 lies in it
__device__ __forceinline__ float4 splat_box(const PtRec &R, float radius) {
    const float w = radius * (1.f + kPtSlack);
    return make_float4(__fsub_rd(R.a.x, w), __fadd_ru(R.a.x, w), __fsub_rd(R.a.y, w), __fadd_ru(R.a.y, w));
}

// squared NDC distance from the pixel centre to the point (corner-relative
// double-float difference, then fp32 squares)
__device__ __forceinline__ float splat_d(const float4 &a, const PixC &p) {
    const float qx = __fadd_rn(__fsub_rn(p.xh, a.x), __fsub_rn(p.xl, a.z));
    const float qy = __fadd_rn(__fsub_rn(p.yh, a.y), __fsub_rn(p.yl, a.w));
    return __fmaf_rn(qx, qx, __fmul_rn(qy, qy));
}

// ---------------------------------------------------------------------------
// staging and binning
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_pstage(PtArgs a, int do_count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    PtRec R;
    R.a = make_float4(0.f, 0.f, 0.f, 0.f);
    R.b = make_float4(__int_as_float(0x7f800000), 0.f, 0.f, 0.f);
    int n = block_find_mesh(a.first, a.num, a.N, a.P, i);
    if (i < a.P) {
        if (n >= 0) {
            const float *cam = a.cams + 16 * n;
            const float px = a.points[3 * i], py = a.points[3 * i + 1], pz = a.points[3 * i + 2];
            if (!(isfinite(px) && isfinite(py) && isfinite(pz))) {
                set_status(a.status, MESHRAST_ST_NONFINITE);
                n = -1;
            } else {
                df X, Y, Z;
                project_corner(cam, px, py, pz, X, Y, Z);
                const float z = __fadd_rn(Z.hi, Z.lo);
                if (!(z >= cam[13]) || !isfinite(z) || !isfinite(X.hi) || !isfinite(Y.hi)) {
                    n = -1;
                } else {
                    R.a = make_float4(X.hi, Y.hi, X.lo, Y.lo);
                    R.b.x = z;
                }
            }
        }
        reinterpret_cast<float4 *>(a.rec + i)[0] = R.a;
        reinterpret_cast<float4 *>(a.rec + i)[1] = R.b;
        a.cloud[i] = n;
    }
    if (!do_count) return;
    int bx0 = 1, bx1 = 0, by0 = 1, by1 = 0;
    if (n >= 0) bin_rect_box(splat_box(R, a.radius), a.S, a.bin, bx0, bx1, by0, by1);
    const int nbx = max(0, bx1 - bx0 + 1), nby = max(0, by1 - by0 + 1);
    const int cnt = nbx * nby;
    const int wmax = __reduce_max_sync(0xffffffffu, cnt);
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < wmax; ++j) {
        int key = -1;
        if (j < cnt) key = (n * a.nb + by0 + j / nbx) * a.nb + bx0 + j % nbx;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && lane == __ffs(grp) - 1) atomicAdd(a.counts + key, __popc(grp));
    }
}

__global__ void __launch_bounds__(256) k_pfill(PtArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int n = -1;
    PtRec R;
    if (i < a.P) {
        n = a.cloud[i];
        if (n >= 0) {
            R.a = reinterpret_cast<const float4 *>(a.rec + i)[0];
            R.b = reinterpret_cast<const float4 *>(a.rec + i)[1];
        }
    }
    int bx0 = 1, bx1 = 0, by0 = 1, by1 = 0;
    if (n >= 0) bin_rect_box(splat_box(R, a.radius), a.S, a.bin, bx0, bx1, by0, by1);
    const int nbx = max(0, bx1 - bx0 + 1), nby = max(0, by1 - by0 + 1);
    const int cnt = nbx * nby;
    // depth bits (positive float) in the high word: integer order = front to back, ties by id
    const unsigned long long entry =
        n >= 0 ? (((unsigned long long)__float_as_uint(R.b.x) << 32) | (unsigned)i) : 0ull;
    const int wmax = __reduce_max_sync(0xffffffffu, cnt);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int j = 0; j < wmax; ++j) {
        int key = -1;
        if (j < cnt) key = (n * a.nb + by0 + j / nbx) * a.nb + bx0 + j % nbx;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(grp) - 1;
        int base = 0;
        if (key >= 0 && lane == leader) base = atomicAdd(a.cursor + key, __popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (key >= 0) {
            const int slot = base + __popc(grp & lt);
            if (slot < a.eff[key]) a.lists[a.offsets[key] + slot] = entry;
        }
    }
}

// ---------------------------------------------------------------------------
// writing one pixel's K fragments
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pt_slot(const PtArgs &a, int64_t s, int id, float z, const PixC &p) {
    if (id == 0x7fffffff) {
        a.idx[s] = -1;
        a.zbuf[s] = -1.f;
        a.dists[s] = -1.f;
    } else {
        a.idx[s] = id;
        a.zbuf[s] = z;
        a.dists[s] = splat_d(__ldg(reinterpret_cast<const float4 *>(a.rec + id)), p);
    }
}

template <int KM>
__device__ __forceinline__ void pt_write(const PtArgs &a, int64_t pix, const TopK<KM> &tk, const PixC &p) {
    const int64_t s0 = pix * (int64_t)a.K;
    if (a.K == KM && (KM % 4) == 0) {
        longlong2 *ip = reinterpret_cast<longlong2 *>(a.idx + s0);
        float4 *zp = reinterpret_cast<float4 *>(a.zbuf + s0);
        float4 *dp = reinterpret_cast<float4 *>(a.dists + s0);
#pragma unroll
        for (int j = 0; j < KM / 2; ++j) {
            longlong2 v;
            v.x = tk.f[2 * j] == 0x7fffffff ? -1ll : (long long)tk.f[2 * j];
            v.y = tk.f[2 * j + 1] == 0x7fffffff ? -1ll : (long long)tk.f[2 * j + 1];
            ip[j] = v;
        }
#pragma unroll
        for (int j = 0; j < KM / 4; ++j) {
            float zz[4], dd[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * j + i;
                const bool e = tk.f[k] == 0x7fffffff;
                zz[i] = e ? -1.f : tk.z[k];
                dd[i] = e ? -1.f : splat_d(__ldg(reinterpret_cast<const float4 *>(a.rec + tk.f[k])), p);
            }
            zp[j] = make_float4(zz[0], zz[1], zz[2], zz[3]);
            dp[j] = make_float4(dd[0], dd[1], dd[2], dd[3]);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (k >= a.K) break;
        pt_slot(a, s0 + k, tk.f[k], tk.z[k], p);
    }
}

// ---------------------------------------------------------------------------
// fine pass
// ---------------------------------------------------------------------------
template <int KM, int BS>
__global__ void __launch_bounds__(BS *BS) k_pfine(PtArgs a) {
    constexpr int BD = BS * BS;
    __shared__ float4 s_pt[BD];
    __shared__ int s_id[BD];
    __shared__ float s_key[BD];
    __shared__ int s_item;
    // dynamic: sort_cap bin entries; K > 16: afterwards the per-thread lists
    extern __shared__ unsigned long long s_sort[];
    const int tid = threadIdx.x, lane = tid & 31;
    const int ty = tid / BS, tx = tid % BS;
    const int nb2 = a.nb * a.nb;
    const float w = a.radius * (1.f + kPtSlack);
    while (true) {
        if (tid == 0) s_item = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if ((int64_t)item >= a.items) break;
        const int n = item / nb2, rem = item - n * nb2;
        const int by = rem / a.nb, bx = rem - by * a.nb;
        const int r = by * BS + ty, c = bx * BS + tx;
        const bool valid = (r < a.S) && (c < a.S);
        const PixC p = pixel_centre(r, c, a.S);
        float wx0 = 1.f, wx1 = -1.f, wy0 = 1.f, wy1 = -1.f;
        {
            const unsigned cmin = __reduce_min_sync(0xffffffffu, valid ? (unsigned)c : 0xffffffffu);
            const unsigned cmax = __reduce_max_sync(0xffffffffu, valid ? (unsigned)c : 0u);
            const unsigned rmin = __reduce_min_sync(0xffffffffu, valid ? (unsigned)r : 0xffffffffu);
            const unsigned rmax = __reduce_max_sync(0xffffffffu, valid ? (unsigned)r : 0u);
            if (cmin <= cmax) {
                wx1 = pc_hi((int)cmin, a.S);
                wx0 = pc_hi((int)cmax, a.S);
                wy1 = pc_hi((int)rmin, a.S);
                wy0 = pc_hi((int)rmax, a.S);
            }
        }
        const int cnt = a.eff[item];
        const int off = a.offsets[item];
        TopK<(KM > 0 ? KM : 1)> tk;
        SmemTopK stk;
        if constexpr (KM > 0) {
            tk.init();
        } else {
            // every segment sorted first and written back, then the same shared
            // memory holds the per-pixel lists (rows of K per thread)
            for (int seg = 0; seg < cnt; seg += a.sort_cap) {
                const int m = min(a.sort_cap, cnt - seg);
                sort_entries<BD>(s_sort, a.lists + off + seg, m);
                for (int i = tid; i < m; i += BD) a.lists[off + seg + i] = s_sort[i];
                __syncthreads();
            }
            stk.z = reinterpret_cast<float *>(s_sort) + tid * a.K;
            stk.f = reinterpret_cast<int *>(s_sort) + BD * a.K + tid * a.K;
            stk.stride = 1;
            stk.K = a.K;
            stk.init();
        }
        for (int seg = 0; seg < cnt; seg += a.sort_cap) {
            const int m = min(a.sort_cap, cnt - seg);
            if constexpr (KM > 0) sort_entries<BD>(s_sort, a.lists + off + seg, m);
            const unsigned long long *ent = (KM > 0) ? s_sort : a.lists + off + seg;
            for (int base = 0; base < m; base += BD) {
                const int mc = min(BD, m - base);
                if (tid < mc) {
                    const unsigned long long v = ent[base + tid];
                    const int id = (int)(unsigned)(v & 0xffffffffull);
                    s_id[tid] = id;
                    s_key[tid] = __uint_as_float((unsigned)(v >> 32));
                    s_pt[tid] = __ldg(reinterpret_cast<const float4 *>(a.rec + id));
                }
                __syncthreads();
                bool warp_done = false;
                for (int jb = 0; jb < mc; jb += 32) {
                    float thr;
                    if constexpr (KM > 0) thr = tk.z[KM - 1];
                    else thr = stk.thr();
                    const float wthr =
                        __int_as_float(__reduce_max_sync(0xffffffffu, valid ? __float_as_int(thr) : 0));
                    if (s_key[jb] > wthr) {  // depths are exact keys: the rest lies behind every lane
                        warp_done = true;
                        break;
                    }
                    const int jl = jb + lane;
                    bool hit = false;
                    if (jl < mc) {
                        const float4 q = s_pt[jl];
                        hit = q.x - w <= wx1 && q.x + w >= wx0 && q.y - w <= wy1 && q.y + w >= wy0 &&
                              !(s_key[jl] > wthr);
                    }
                    unsigned mask = __ballot_sync(0xffffffffu, hit);
                    while (mask) {
                        const int jj = jb + __ffs(mask) - 1;
                        mask &= mask - 1;
                        if (!valid) continue;
                        const float z = s_key[jj];
                        if constexpr (KM > 0) thr = tk.z[KM - 1];
                        else thr = stk.thr();
                        if (z > thr) continue;
                        if (!(splat_d(s_pt[jj], p) < a.r2)) continue;
                        const int id = s_id[jj];
                        if constexpr (KM > 0) {
                            if (tk.admits(z, id)) tk.insert(z, id);
                        } else {
                            if (stk.admits(z, id)) stk.insert(z, id);
                        }
                    }
                }
                if (!warp_done && base + BD < m) {
                    float thr;
                    if constexpr (KM > 0) thr = tk.z[KM - 1];
                    else thr = stk.thr();
                    const float wthr =
                        __int_as_float(__reduce_max_sync(0xffffffffu, valid ? __float_as_int(thr) : 0));
                    warp_done = __uint_as_float((unsigned)(ent[base + BD] >> 32)) > wthr;
                }
                if (__syncthreads_and(warp_done)) break;
            }
            __syncthreads();
        }
        if constexpr (KM > 0) {
            if (valid) pt_write<KM>(a, ((int64_t)n * a.S + r) * a.S + c, tk, p);
        } else {
            // the block writes its tile slot by slot (coalesced along a tile row)
            s_id[tid] = valid ? stk.n : 0;
            __syncthreads();
            const int K = a.K;
            const int rows = min(BS, a.S - by * BS), cols = min(BS, a.S - bx * BS);
            const int per_row = cols * K;
            const float *lz = reinterpret_cast<const float *>(s_sort);
            const int *lf = reinterpret_cast<const int *>(s_sort) + BD * K;
            for (int i = tid; i < rows * per_row; i += BD) {
                const int ry = i / per_row, rr = i - ry * per_row;
                const int cx = rr / K, k = rr - cx * K;
                const int t = ry * BS + cx;
                const int64_t sl = (((int64_t)n * a.S + by * BS + ry) * a.S + bx * BS + cx) * K + k;
                if (k < s_id[t]) pt_slot(a, sl, lf[t * K + k], lz[t * K + k], pixel_centre(by * BS + ry, bx * BS + cx, a.S));
                else pt_slot(a, sl, 0x7fffffff, 0.f, p);
            }
            __syncthreads();
        }
    }
}

// plain form: one launch per image, every pixel against every point of the cloud
template <int KM>
__global__ void __launch_bounds__(256) k_pnaive(PtArgs a, int n) {
    extern __shared__ unsigned long long s_dyn[];
    const int64_t pidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = pidx < (int64_t)a.S * a.S;
    const int r = (int)(pidx / a.S), c = (int)(pidx % a.S);
    const PixC p = pixel_centre(r, c, a.S);
    int64_t lo = a.first[n], hi = lo + a.num[n];
    lo = max(lo, (int64_t)0);
    hi = min(hi, a.P);
    TopK<(KM > 0 ? KM : 1)> tk;
    SmemTopK stk;
    if constexpr (KM > 0) {
        tk.init();
    } else {
        stk.z = reinterpret_cast<float *>(s_dyn) + threadIdx.x;
        stk.f = reinterpret_cast<int *>(s_dyn) + blockDim.x * a.K + threadIdx.x;
        stk.stride = blockDim.x;
        stk.K = a.K;
        stk.init();
    }
    if (!valid) return;
    for (int64_t i = lo; i < hi; ++i) {
        if (a.cloud[i] != n) continue;
        const float4 q = __ldg(reinterpret_cast<const float4 *>(a.rec + i));
        if (!(splat_d(q, p) < a.r2)) continue;
        const float z = __ldg(reinterpret_cast<const float *>(a.rec + i) + 4);
        if constexpr (KM > 0) {
            if (tk.admits(z, (int)i)) tk.insert(z, (int)i);
        } else {
            if (stk.admits(z, (int)i)) stk.insert(z, (int)i);
        }
    }
    const int64_t pix = (int64_t)n * a.S * a.S + pidx;
    if constexpr (KM > 0) {
        pt_write<KM>(a, pix, tk, p);
    } else {
        for (int k = 0; k < a.K; ++k)
            pt_slot(a, pix * a.K + k, k < stk.n ? stk.f[k * stk.stride] : 0x7fffffff,
                    k < stk.n ? stk.z[k * stk.stride] : 0.f, p);
    }
}

// ---------------------------------------------------------------------------
// compositing
// ---------------------------------------------------------------------------
struct CompArgs {
    int64_t npix;
    int N, S, K, D, mode;
    float inv_r2;
    int64_t P;
    const int64_t *idx;
    const float *dists, *features;
    float *image;
    const float *grad_image;
    float *grad_dists, *grad_features;
};

__device__ __forceinline__ int pt_id(const CompArgs &a, int64_t s) {
    const long long v = __ldg(a.idx + s);
    return (v >= 0 && v < a.P) ? (int)v : -1;
}

__global__ void __launch_bounds__(256) k_pcomp_fwd(CompArgs a) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= a.npix) return;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float T = 1.f, asum = 0.f;
    for (int k = 0; k < a.K; ++k) {
        const int64_t s = pix * a.K + k;
        const int i = pt_id(a, s);
        if (i < 0) continue;
        const float q = __ldg(a.dists + s) * a.inv_r2;  // 1 - alpha, without the cancellation
        const float al = 1.f - q;
        const float wgt = a.mode == PTS_COMPOSITE_ALPHA ? al * T : al;
        for (int ch = 0; ch < a.D; ++ch) acc[ch] += wgt * __ldg(a.features + (int64_t)i * a.D + ch);
        T *= q;
        asum += al;
    }
    const float sc = (a.mode == PTS_COMPOSITE_NORM) ? (asum > 0.f ? 1.f / asum : 0.f) : 1.f;
    for (int ch = 0; ch < a.D; ++ch) a.image[pix * a.D + ch] = acc[ch] * sc;
}

// One thread per pixel of a 16 x 16 tile; feature gradients are summed over
// the warp's lanes holding the same point before the atomics.  The forward
// recompute keeps only the transmittance at the start of every chunk of 8
// slots (in shared memory); the reverse pass recomputes each chunk's
// opacities and transmittances into registers.
constexpr int kCompChunk = 8;
constexpr int kCompChunks = (kMaxK + kCompChunk - 1) / kCompChunk;

template <int DM>
__global__ void __launch_bounds__(256) k_pcomp_bwd(CompArgs a) {
    __shared__ float s_T[kCompChunks][256];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    const bool valid = row < a.S && col < a.S;
    const int64_t pix = ((int64_t)blockIdx.z * a.S + row) * a.S + col;
    float g[DM];
#pragma unroll
    for (int ch = 0; ch < DM; ++ch) g[ch] = (valid && ch < a.D) ? a.grad_image[pix * a.D + ch] : 0.f;
    // forward recompute; 1 - alpha = d / r^2 is taken directly (no cancellation)
    float T = 1.f, asum = 0.f, out[DM];
#pragma unroll
    for (int ch = 0; ch < DM; ++ch) out[ch] = 0.f;
    for (int k = 0; valid && k < a.K; ++k) {
        if (k % kCompChunk == 0) s_T[k / kCompChunk][tid] = T;
        const int64_t s = pix * a.K + k;
        const int i = pt_id(a, s);
        if (i < 0) continue;
        const float q = __ldg(a.dists + s) * a.inv_r2;
#pragma unroll
        for (int ch = 0; ch < DM; ++ch)
            if (ch < a.D) out[ch] += (1.f - q) * __ldg(a.features + (int64_t)i * a.D + ch);
        T *= q;
        asum += 1.f - q;
    }
    const bool norm = a.mode == PTS_COMPOSITE_NORM;
    const float inv_a = asum > 0.f ? 1.f / asum : 0.f;
    // Alpha: df/dalpha_k = T_k (f_k - S_k), S_k the composite of the later
    // slots alone.  E_k = f_k - S_k follows the recursion
    //   E_last = f_last,  E_k = (f_k - f_next) + (1 - alpha_next) E_next,
    // exact when neighbouring features are equal (a silhouette: E_k is the
    // transmittance of the later slots), where f_k - S_k would cancel.
    // Norm: df/dalpha_k = (f_k - f) / sum alpha.
    float E[DM], f_next[DM];
    float q_next = 0.f;
    bool has_next = false;
#pragma unroll
    for (int ch = 0; ch < DM; ++ch) {
        E[ch] = 0.f;
        f_next[ch] = 0.f;
        if (norm) out[ch] *= inv_a;
    }
    const int nch = (a.K + kCompChunk - 1) / kCompChunk;
    for (int c = nch - 1; c >= 0; --c) {  // uniform trip counts: every lane reaches the warp grouping
        // this chunk's ids, 1 - alpha and transmittances, in registers
        int ids[kCompChunk];
        float qv[kCompChunk], Tv[kCompChunk];
        float Tc = valid ? s_T[c][tid] : 1.f;
#pragma unroll
        for (int j = 0; j < kCompChunk; ++j) {
            const int k = c * kCompChunk + j;
            const int64_t s = pix * a.K + k;
            ids[j] = (valid && k < a.K) ? pt_id(a, s) : -1;
            qv[j] = ids[j] >= 0 ? __ldg(a.dists + s) * a.inv_r2 : 1.f;
            Tv[j] = Tc;
            Tc *= qv[j];
        }
#pragma unroll
        for (int j = kCompChunk - 1; j >= 0; --j) {
            const int k = c * kCompChunk + j;
            if (k >= a.K) continue;  // uniform: K is the same for every lane
            const int64_t s = pix * a.K + k;
            const int i = ids[j];
            const float al = 1.f - qv[j];
            float gf[DM];
            float ga = 0.f;
#pragma unroll
            for (int ch = 0; ch < DM; ++ch) {
                gf[ch] = 0.f;
                if (i < 0 || ch >= a.D) continue;
                const float fc = __ldg(a.features + (int64_t)i * a.D + ch);
                if (norm) {
                    gf[ch] = al * inv_a * g[ch];
                    ga += g[ch] * (fc - out[ch]) * inv_a;
                } else {
                    E[ch] = has_next ? (fc - f_next[ch]) + q_next * E[ch] : fc;
                    f_next[ch] = fc;
                    gf[ch] = al * Tv[j] * g[ch];
                    ga += g[ch] * Tv[j] * E[ch];
                }
            }
            if (i >= 0) {
                q_next = qv[j];
                has_next = true;
            }
            if (valid) a.grad_dists[s] = (i < 0) ? 0.f : -ga * a.inv_r2;
            const unsigned peers = __match_any_sync(0xffffffffu, i);
            group_sum<DM>(peers, gf);
            if (i >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
#pragma unroll
                for (int ch = 0; ch < DM; ++ch)
                    if (ch < a.D) atomicAdd(a.grad_features + (int64_t)i * a.D + ch, gf[ch]);
            }
        }
    }
}

// dL/d(zbuf, dists) -> dL/dpoints: d = |p - x|^2, x = f x_v / z_v, then R^T.
// The point is projected here in fp32 (its selection is fixed by idx; the
// gradient needs no double-float positions), so no staging pass is needed.
__global__ void __launch_bounds__(256) k_prast_bwd(PtArgs a, const float *grad_zbuf, const float *grad_dists,
                                                 float *grad_points) {
    // each warp covers an 8 x 4 block of the 16 x 16 tile: neighbouring pixels
    // share points, so the warp's grouping by point finds more peers
    const int tx = ((threadIdx.x >> 5) & 1) * 8 + (threadIdx.x & 7), ty = (threadIdx.x >> 6) * 4 + ((threadIdx.x >> 3) & 3);
    const int n = blockIdx.z;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    const bool valid = row < a.S && col < a.S;
    const PixC p = pixel_centre(row, col, a.S);
    const int64_t pix = ((int64_t)n * a.S + row) * a.S + col;
    const float *cam = a.cams + 16 * n;
    const int64_t lo = a.first[n], hi = lo + a.num[n];
    for (int k = 0; k < a.K; ++k) {
        const int64_t s = pix * a.K + k;
        int i = -1;
        if (valid) {
            const long long v = a.idx[s];
            // an id outside this image's range contributes nothing
            i = (v >= 0 && v < a.P && v >= lo && v < hi) ? (int)v : -1;
        }
        float g3[3] = {0.f, 0.f, 0.f};
        float x = 0.f, y = 0.f, iz = 0.f;
        if (i >= 0) {
            const float d0 = __ldg(a.points + 3 * (int64_t)i) - cam[9];
            const float d1 = __ldg(a.points + 3 * (int64_t)i + 1) - cam[10];
            const float d2 = __ldg(a.points + 3 * (int64_t)i + 2) - cam[11];
            const float xv = cam[0] * d0 + cam[1] * d1 + cam[2] * d2;
            const float yv = cam[3] * d0 + cam[4] * d1 + cam[5] * d2;
            const float zv = cam[6] * d0 + cam[7] * d1 + cam[8] * d2;
            if (zv >= cam[13] && isfinite(zv)) {
                iz = 1.f / zv;
                x = cam[12] * xv * iz;
                y = cam[12] * yv * iz;
                const float gd = grad_dists ? grad_dists[s] : 0.f;
                const float gz = grad_zbuf ? grad_zbuf[s] : 0.f;
                const float qx = __fadd_rn(__fsub_rn(p.xh, x), p.xl);
                const float qy = __fadd_rn(__fsub_rn(p.yh, y), p.yl);
                g3[0] = -2.f * gd * qx;  // dL/dx_ndc
                g3[1] = -2.f * gd * qy;  // dL/dy_ndc
                g3[2] = gz;              // dL/dz_view (direct)
            } else {
                i = -1;                  // culled: never selected by the forward
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, i);
        group_sum<3>(peers, g3);
        if (i >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
            const float fo = cam[12];
            const float gxv = g3[0] * fo * iz, gyv = g3[1] * fo * iz;
            const float gzv = g3[2] - (g3[0] * x + g3[1] * y) * iz;
            float *gp = grad_points + 3 * (int64_t)i;
            atomicAdd(gp + 0, cam[0] * gxv + cam[3] * gyv + cam[6] * gzv);
            atomicAdd(gp + 1, cam[1] * gxv + cam[4] * gyv + cam[7] * gzv);
            atomicAdd(gp + 2, cam[2] * gxv + cam[5] * gyv + cam[8] * gzv);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int km_for_points(int K) {
    if (K <= 1) return 1;
    if (K <= 2) return 2;
    if (K <= 4) return 4;
    if (K <= 8) return 8;
    if (K <= 16) return 16;
    return 0;
}

struct PtLayout {
    size_t records, cloud, counts, eff, offsets, cursor, lists, bytes;
    int64_t nb, NB, capacity;
};

static bool pt_params_ok(const pts_params *p, int64_t P) {
    if (!p) return false;
    if (p->N < 0 || p->N > 65535 || p->image_size < 1 || p->image_size > 8192) return false;
    if (p->points_per_pixel < 1) return false;
    if (!(p->radius > 0.f) || !(p->radius < 4.f)) return false;
    if (p->reserved != 0 || p->reserved_f != 0.f) return false;
    if (P < 0 || P >= 0x7fffffffLL) return false;
    if (p->bin_size > 0 && p->max_points_per_bin <= 0) return false;
    if (p->max_bin_entries < 0) return false;
    return true;
}

static bool pt_unsupported(const pts_params *p) {
    if (p->points_per_pixel > kMaxK || (p->bin_size != 0 && p->bin_size != 8 && p->bin_size != 16)) return true;
    if (p->bin_size > 0) {
        // bin keys, counts, offsets and list positions are 32-bit on the device
        const int64_t nb = (p->image_size + p->bin_size - 1) / p->bin_size;
        const int64_t NB = (int64_t)p->N * nb * nb;
        if (NB >= 0x7fffffffLL) return true;
        const int64_t cap = p->max_bin_entries > 0 ? p->max_bin_entries : NB * (int64_t)p->max_points_per_bin;
        if (cap > 0x7fffffffLL) return true;
    }
    return false;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static void pt_layout(const pts_params *p, int64_t P, PtLayout *L) {
    std::memset(L, 0, sizeof(*L));
    size_t off = 256;  // header: status @0, queue @4, total @8, max count @16 (as the mesh workspace)
    L->records = off;
    off = al256(off + (size_t)P * sizeof(PtRec));
    L->cloud = off;
    off = al256(off + (size_t)P * 4);
    if (p->bin_size > 0) {
        const int64_t nb = (p->image_size + p->bin_size - 1) / p->bin_size;
        const int64_t NB = (int64_t)p->N * nb * nb;
        const int64_t cap = p->max_bin_entries > 0 ? p->max_bin_entries : NB * (int64_t)p->max_points_per_bin;
        L->nb = nb;
        L->NB = NB;
        L->capacity = cap;
        L->counts = off;
        off = al256(off + (size_t)NB * 4);
        L->eff = off;
        off = al256(off + (size_t)NB * 4);
        L->offsets = off;
        off = al256(off + (size_t)(NB + 1) * 4);
        L->cursor = off;
        off = al256(off + (size_t)NB * 4);
        L->lists = off;
        off = al256(off + (size_t)cap * 8);
    }
    L->bytes = off;
}

static void pt_fill_args(PtArgs &a, const pts_params *p, const float *points, int64_t P, const int64_t *first,
                         const int64_t *num, const float *cams, char *ws, const PtLayout &L) {
    std::memset(&a, 0, sizeof(a));
    a.points = points;
    a.P = P;
    a.first = first;
    a.num = num;
    a.N = p->N;
    a.cams = cams;
    a.radius = p->radius;
    a.r2 = p->radius * p->radius;
    a.S = p->image_size;
    a.K = p->points_per_pixel;
    a.bin = p->bin_size > 0 ? p->bin_size : 1;
    a.nb = (int)L.nb;
    a.items = L.NB;
    a.rec = reinterpret_cast<PtRec *>(ws + L.records);
    a.cloud = reinterpret_cast<int *>(ws + L.cloud);
    if (p->bin_size > 0) {
        a.counts = reinterpret_cast<int *>(ws + L.counts);
        a.cursor = reinterpret_cast<int *>(ws + L.cursor);
        a.eff = reinterpret_cast<const int *>(ws + L.eff);
        a.offsets = reinterpret_cast<const int *>(ws + L.offsets);
        a.lists = reinterpret_cast<unsigned long long *>(ws + L.lists);
    }
    a.queue = reinterpret_cast<unsigned *>(ws + 4);
    a.status = reinterpret_cast<unsigned *>(ws);
    a.sort_cap = fine_sort_cap(p->max_points_per_bin, p->points_per_pixel,
                               p->bin_size > 0 ? p->bin_size * p->bin_size : 256);
}

template <int KM, int BS>
static cudaError_t launch_pfine_t(const PtArgs &a, cudaStream_t st) {
    constexpr int BD = BS * BS;
    const size_t dyn = std::max((size_t)a.sort_cap * 8, (KM > 0) ? (size_t)0 : (size_t)BD * a.K * 8);
    auto kern = k_pfine<KM, BS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, BD, dyn);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.items, (int64_t)mr_host::num_sms() * std::max(1, bps)));
    kern<<<grid, BD, dyn, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_pfine(const PtArgs &a, int bin, cudaStream_t st) {
    const int km = km_for_points(a.K);
#define MR_PFINE(KM_)                                              \
    if (km == KM_) {                                               \
        if (bin == 8) return launch_pfine_t<KM_, 8>(a, st);        \
        if (bin == 16) return launch_pfine_t<KM_, 16>(a, st);      \
    }
    MR_PFINE(1) MR_PFINE(2) MR_PFINE(4) MR_PFINE(8) MR_PFINE(16) MR_PFINE(0)
#undef MR_PFINE
    return cudaErrorInvalidValue;
}

template <int KM>
static cudaError_t launch_pnaive_t(const PtArgs &a, cudaStream_t st) {
    const int BD = 256;
    const size_t dyn = (KM > 0) ? 0 : (size_t)BD * a.K * 8;
    if (KM == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_pnaive<KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    const int64_t npx = (int64_t)a.S * a.S;
    const int grid = (int)((npx + BD - 1) / BD);
    for (int n = 0; n < a.N; ++n) {
        k_pnaive<KM><<<grid, BD, dyn, st>>>(a, n);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t launch_pnaive(const PtArgs &a, cudaStream_t st) {
    switch (km_for_points(a.K)) {
        case 1: return launch_pnaive_t<1>(a, st);
        case 2: return launch_pnaive_t<2>(a, st);
        case 4: return launch_pnaive_t<4>(a, st);
        case 8: return launch_pnaive_t<8>(a, st);
        case 16: return launch_pnaive_t<16>(a, st);
        default: return launch_pnaive_t<0>(a, st);
    }
}

static bool al16(const void *q) { return ((uintptr_t)q & 15u) == 0; }

static int check_pws(const pts_params *p, int64_t P, void *ws, size_t ws_bytes, PtLayout *L) {
    pt_layout(p, P, L);
    if (!ws || ((uintptr_t)ws & 255u) != 0 || ws_bytes < L->bytes) return MESHRAST_ERR_WORKSPACE;
    return MESHRAST_OK;
}

}  // namespace mr

using mr::PtLayout;

extern "C" {

size_t pts_workspace_bytes(const pts_params *p, int64_t P) {
    if (!mr::pt_params_ok(p, P) || mr::pt_unsupported(p)) return 0;
    PtLayout L;
    mr::pt_layout(p, P, &L);
    return L.bytes;
}

int pts_rasterize_fwd(const pts_params *p, const float *points, int64_t P, const int64_t *first_point,
                      const int64_t *num_points, const float *cams, int64_t *idx, float *zbuf, float *dists,
                      void *workspace, size_t workspace_bytes, void *stream) {
    if (!mr::pt_params_ok(p, P)) return MESHRAST_ERR_INVALID_ARG;
    if (mr::pt_unsupported(p)) return MESHRAST_ERR_UNSUPPORTED;
    if (p->N > 0 && (!first_point || !num_points || !cams)) return MESHRAST_ERR_INVALID_ARG;
    if (P > 0 && !points) return MESHRAST_ERR_INVALID_ARG;
    const int64_t slots = (int64_t)p->N * p->image_size * p->image_size * p->points_per_pixel;
    if (slots > 0 && (!idx || !zbuf || !dists || !mr::al16(idx) || !mr::al16(zbuf) || !mr::al16(dists)))
        return MESHRAST_ERR_INVALID_ARG;
    PtLayout L;
    int rc = mr::check_pws(p, P, workspace, workspace_bytes, &L);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    if (cudaMemsetAsync(ws, 0, 256, st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    if (p->N == 0) return MESHRAST_OK;
    const bool binned = p->bin_size > 0;
    if (binned && L.NB > 0 && cudaMemsetAsync(ws + L.counts, 0, (size_t)L.NB * 4, st) != cudaSuccess)
        return MESHRAST_ERR_CUDA;
    mr::PtArgs a;
    mr::pt_fill_args(a, p, points, P, first_point, num_points, cams, ws, L);
    a.idx = idx;
    a.zbuf = zbuf;
    a.dists = dists;
    if (P > 0) {
        mr::k_pstage<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(a, binned ? 1 : 0);
        if (cudaGetLastError() != cudaSuccess) return MESHRAST_ERR_CUDA;
    }
    if (!binned) return mr::launch_pnaive(a, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
    mr::ScanArgs sa;
    sa.counts = a.counts;
    sa.eff = reinterpret_cast<int *>(ws + L.eff);
    sa.offsets = reinterpret_cast<int *>(ws + L.offsets);
    sa.cursor = a.cursor;
    sa.order = nullptr;
    sa.NB = L.NB;
    sa.capacity = L.capacity;
    sa.max_per_bin = p->max_points_per_bin;
    sa.queue = a.queue;
    sa.status = a.status;
    sa.total = reinterpret_cast<long long *>(ws + 8);
    sa.maxcount = reinterpret_cast<int *>(ws + 16);
    sa.first_face = first_point;
    sa.num_faces = num_points;
    sa.N = p->N;
    sa.F = P;
    if (mr::launch_scan(sa, st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    if (P > 0) {
        mr::k_pfill<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(a);
        if (cudaGetLastError() != cudaSuccess) return MESHRAST_ERR_CUDA;
    }
    return mr::launch_pfine(a, p->bin_size, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

int pts_rasterize_bwd(const pts_params *p, const float *points, int64_t P, const int64_t *first_point,
                      const int64_t *num_points, const float *cams, const int64_t *idx, const float *grad_zbuf,
                      const float *grad_dists, float *grad_points, void *workspace, size_t workspace_bytes,
                      void *stream) {
    if (!mr::pt_params_ok(p, P)) return MESHRAST_ERR_INVALID_ARG;
    if (mr::pt_unsupported(p)) return MESHRAST_ERR_UNSUPPORTED;
    if (p->N > 0 && (!first_point || !num_points || !cams)) return MESHRAST_ERR_INVALID_ARG;
    if (P > 0 && (!points || !grad_points)) return MESHRAST_ERR_INVALID_ARG;
    const int64_t slots = (int64_t)p->N * p->image_size * p->image_size * p->points_per_pixel;
    if (slots > 0 && !idx) return MESHRAST_ERR_INVALID_ARG;
    PtLayout L;
    int rc = mr::check_pws(p, P, workspace, workspace_bytes, &L);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    if (P > 0 && cudaMemsetAsync(grad_points, 0, (size_t)P * 3 * sizeof(float), st) != cudaSuccess)
        return MESHRAST_ERR_CUDA;
    if (slots == 0 || (!grad_zbuf && !grad_dists)) return MESHRAST_OK;
    mr::PtArgs a;
    mr::pt_fill_args(a, p, points, P, first_point, num_points, cams, ws, L);
    a.idx = const_cast<int64_t *>(idx);
    const unsigned tiles = (unsigned)((p->image_size + 15) / 16);
    mr::k_prast_bwd<<<dim3(tiles, tiles, (unsigned)p->N), 256, 0, st>>>(a, grad_zbuf, grad_dists, grad_points);
    return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

static int check_comp(const pts_params *p, int32_t mode, int64_t P, int32_t D) {
    if (!p || p->N < 0 || p->N > 65535 || p->image_size < 0 || p->image_size > 8192) return MESHRAST_ERR_INVALID_ARG;
    if (p->points_per_pixel < 1) return MESHRAST_ERR_INVALID_ARG;
    if (p->points_per_pixel > mr::kMaxK) return MESHRAST_ERR_UNSUPPORTED;
    if (!(p->radius > 0.f)) return MESHRAST_ERR_INVALID_ARG;
    if (mode != PTS_COMPOSITE_ALPHA && mode != PTS_COMPOSITE_NORM) return MESHRAST_ERR_INVALID_ARG;
    if (D < 1 || D > 8 || P < 0) return MESHRAST_ERR_INVALID_ARG;
    return MESHRAST_OK;
}

static void fill_comp(mr::CompArgs &c, const pts_params *p, int32_t mode, const int64_t *idx, const float *dists,
                      const float *features, int64_t P, int32_t D) {
    std::memset(&c, 0, sizeof(c));
    c.N = p->N;
    c.S = p->image_size;
    c.K = p->points_per_pixel;
    c.npix = (int64_t)p->N * p->image_size * p->image_size;
    c.D = D;
    c.mode = mode;
    c.inv_r2 = 1.f / (p->radius * p->radius);
    c.P = P;
    c.idx = idx;
    c.dists = dists;
    c.features = features;
}

int pts_composite_fwd(const pts_params *p, int32_t mode, const int64_t *idx, const float *dists,
                      const float *features, int64_t P, int32_t D, float *image, void *stream) {
    int rc = check_comp(p, mode, P, D);
    if (rc) return rc;
    mr::CompArgs c;
    fill_comp(c, p, mode, idx, dists, features, P, D);
    if (c.npix == 0) return MESHRAST_OK;
    if (!idx || !dists || !image || (P > 0 && !features)) return MESHRAST_ERR_INVALID_ARG;
    c.image = image;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    mr::k_pcomp_fwd<<<(unsigned)((c.npix + 255) / 256), 256, 0, st>>>(c);
    return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

int pts_composite_bwd(const pts_params *p, int32_t mode, const int64_t *idx, const float *dists,
                      const float *features, int64_t P, int32_t D, const float *grad_image, float *grad_dists,
                      float *grad_features, void *stream) {
    int rc = check_comp(p, mode, P, D);
    if (rc) return rc;
    mr::CompArgs c;
    fill_comp(c, p, mode, idx, dists, features, P, D);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (P > 0) {
        if (!grad_features) return MESHRAST_ERR_INVALID_ARG;
        if (cudaMemsetAsync(grad_features, 0, (size_t)P * D * sizeof(float), st) != cudaSuccess)
            return MESHRAST_ERR_CUDA;
    }
    if (c.npix == 0) return MESHRAST_OK;
    if (!idx || !dists || !grad_image || !grad_dists || (P > 0 && !features)) return MESHRAST_ERR_INVALID_ARG;
    c.grad_image = grad_image;
    c.grad_dists = grad_dists;
    c.grad_features = grad_features;
    const unsigned tiles = (unsigned)((p->image_size + 15) / 16);
    const dim3 grid(tiles, tiles, (unsigned)p->N);
    if (D == 1) mr::k_pcomp_bwd<1><<<grid, 256, 0, st>>>(c);
    else if (D <= 4) mr::k_pcomp_bwd<4><<<grid, 256, 0, st>>>(c);
    else mr::k_pcomp_bwd<8><<<grid, 256, 0, st>>>(c);
    return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

int pts_bin_occupancy(const pts_params *p, int64_t P, const void *workspace, int32_t *max_count,
                      int64_t *total_entries, void *stream) {
    if (!mr::pt_params_ok(p, P) || !workspace || !max_count || !total_entries || p->bin_size <= 0)
        return MESHRAST_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    const char *ws = reinterpret_cast<const char *>(workspace);
    int32_t mc = 0;
    long long tot = 0;
    if (cudaMemcpy(&mc, ws + 16, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return MESHRAST_ERR_CUDA;
    if (cudaMemcpy(&tot, ws + 8, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return MESHRAST_ERR_CUDA;
    *max_count = mc;
    *total_entries = tot;
    return MESHRAST_OK;
}

}  // extern "C"
