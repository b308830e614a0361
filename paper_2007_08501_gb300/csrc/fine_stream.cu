// Fine pass for large K (K > 16) with front-to-back finalisation, and the
// Fragment attribute pass that follows it (sm_103a).
//
// Section 3.2 of the paper ("Rasterizer"): per pixel, the K nearest faces
// along z among the faces binned to the pixel's image tile.  Keeping all K
// (depth, face) pairs of every pixel on chip (K x 8 bytes per pixel: 400 bytes
// at K = 50) limits a block of 256 pixels to one per SM.  This pass keeps far
// less: each bin's face list is sorted front to back by the nearest-corner
// depth of the face (a lower bound on its depth at any pixel where it is a
// candidate, when the depth is a convex combination of the corner depths:
// with clipped barycentrics, or without blur).  When a pixel meets a face
// whose bound is b, every candidate it holds with depth < b keeps its rank
// for good: no later face can come before it.  Such entries leave the pixel's
// list at once, written to their final slot, and only the still-unsettled
// candidates stay on chip, in a ring of kRing entries per pixel in shared
// memory (the settled prefix is a counter).
//
// A pixel whose unsettled candidates outgrow the ring (rare: dense, steeply
// tilted depth overlap) is redone at the end of the bin by a whole warp: the
// warp walks the bin's sorted list 32 faces at a time and keeps the pixel's K
// nearest in registers spread over its lanes (two list rows of 32), inserting
// each admitted face with a ballot (its rank) and lane shuffles (the shift).
//
// The fine pass writes each slot as one 64-bit key: (depth bits << 32) | face
// id, or -1 for an empty slot, into pix_to_face.  k_frag_attr, one warp per
// pixel and one lane per slot (coalesced, full occupancy), expands it into
// pix_to_face, zbuf, barycentrics and distance, and applies the silhouette
// blend (Algorithm 1) when asked.
#include <cuda_runtime.h>

#include <algorithm>

#include "bin_common.cuh"
#include "blend_common.cuh"
#include "rast_common.cuh"
#include "rast_internal.h"

namespace mr {

constexpr int kRing = 16;  // unsettled candidates a pixel keeps on chip

__device__ __forceinline__ long long pack_key(float z, int f) {
    return (long long)(((unsigned long long)__float_as_uint(z) << 32) | (unsigned)f);
}

// ---------------------------------------------------------------------------
// redo of one pixel by a warp: warp-distributed sorted K-list (K <= 64),
// entry i in row i / 32 of lane i % 32
// ---------------------------------------------------------------------------
struct WarpList {
    float z0, z1;
    int f0, f1;
    int m;  // entries held (<= K)
};

__device__ __forceinline__ void warp_list_insert(WarpList &L, float z, int f, int K) {
    const int lane = (int)(threadIdx.x & 31u);
    const unsigned b0 = __ballot_sync(0xffffffffu, key_less(L.z0, L.f0, z, f));
    const unsigned b1 = __ballot_sync(0xffffffffu, key_less(L.z1, L.f1, z, f));
    const int rank = __popc(b0) + __popc(b1);   // empty entries (+inf, INT_MAX) never count
    // entry i of the new list: i < rank the old i, i == rank the new one, i > rank the old i - 1
    const float pz0 = __shfl_up_sync(0xffffffffu, L.z0, 1), pz1 = __shfl_up_sync(0xffffffffu, L.z1, 1);
    const int pf0 = __shfl_up_sync(0xffffffffu, L.f0, 1), pf1 = __shfl_up_sync(0xffffffffu, L.f1, 1);
    const float cz = __shfl_sync(0xffffffffu, L.z0, 31);   // old entry 31 moves to entry 32
    const int cf = __shfl_sync(0xffffffffu, L.f0, 31);
    const int i0 = lane, i1 = 32 + lane;
    if (i0 == rank) { L.z0 = z; L.f0 = f; }
    else if (i0 > rank) { L.z0 = pz0; L.f0 = pf0; }
    if (i1 == rank) { L.z1 = z; L.f1 = f; }
    else if (i1 > rank) { L.z1 = lane == 0 ? cz : pz1; L.f1 = lane == 0 ? cf : pf1; }
    const float kInf = __int_as_float(0x7f800000);
    if (i0 >= K) { L.z0 = kInf; L.f0 = 0x7fffffff; }
    if (i1 >= K) { L.z1 = kInf; L.f1 = 0x7fffffff; }
    L.m = min(L.m + 1, K);
}

// K-th entry of the list (valid when m == K)
__device__ __forceinline__ void warp_list_kth(const WarpList &L, int K, float &z, int &f) {
    const int i = K - 1;
    const float a = __shfl_sync(0xffffffffu, L.z0, i & 31), b = __shfl_sync(0xffffffffu, L.z1, i & 31);
    const int fa = __shfl_sync(0xffffffffu, L.f0, i & 31), fb = __shfl_sync(0xffffffffu, L.f1, i & 31);
    z = i < 32 ? a : b;
    f = i < 32 ? fa : fb;
}

__device__ void redo_pixel(const FineArgs &a, const unsigned long long *ent, int cnt, int n, int r, int c,
                           const EvalFlags &fl) {
    const unsigned lane = threadIdx.x & 31u;
    const int K = a.K;
    const PixC p = pixel_centre(r, c, a.S);
    const float kInf = __int_as_float(0x7f800000);
    WarpList L{kInf, kInf, 0x7fffffff, 0x7fffffff, 0};
    for (int jb = 0; jb < cnt; jb += 32) {
        // every later face's depth is at least its key: stop once the K-th is in front
        if (L.m >= K) {
            float kz;
            int kf;
            warp_list_kth(L, K, kz, kf);
            if (__uint_as_float((unsigned)(ent[jb] >> 32)) > kz) break;
        }
        const int j = jb + (int)lane;
        bool hit = false;
        float z = 0.f;
        int fid = 0;
        if (j < cnt) {
            const unsigned long long v = ent[j];
            fid = (int)(unsigned)(v & 0xffffffffull);
            const float4 *src = reinterpret_cast<const float4 *>(a.rec + fid);
            FaceRec R;
            R.c = __ldg(src + kRecC);
            if (in_bbox(R, p)) {
                R.a = __ldg(src + kRecA);
                R.b = __ldg(src + kRecB);
                R.d = __ldg(src + kRecD);
                R.e = __ldg(src + kRecE);
                R.h = __ldg(src + kRecH);
                hit = face_key_nobbox(R, p, fl, z);
            }
        }
        unsigned mask = __ballot_sync(0xffffffffu, hit);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const float zz = __shfl_sync(0xffffffffu, z, src);
            const int ff = __shfl_sync(0xffffffffu, fid, src);
            bool admit = L.m < K;
            if (!admit) {
                float kz;
                int kf;
                warp_list_kth(L, K, kz, kf);
                admit = key_less(zz, ff, kz, kf);
            }
            if (admit) warp_list_insert(L, zz, ff, K);
        }
    }
    const int64_t s0 = (((int64_t)n * a.S + r) * a.S + c) * K;
    if ((int)lane < K) a.out.pix_to_face[s0 + lane] = (int)lane < L.m ? pack_key(L.z0, L.f0) : -1ll;
    if (32 + (int)lane < K) a.out.pix_to_face[s0 + 32 + lane] = 32 + (int)lane < L.m ? pack_key(L.z1, L.f1) : -1ll;
}

// ---------------------------------------------------------------------------
// the streaming fine pass
// ---------------------------------------------------------------------------
// Pixel of thread t in a BS x BS bin: each warp covers an 8 x 4 block (8
// columns, 4 rows) rather than two full rows, so that the warp's footprint is
// about as wide as tall, like the inflated face bboxes it is culled against.
template <int BS>
__device__ __forceinline__ void tile_pixel_of(int t, int &ty, int &tx) {
    const int lane = t & 31, warp = t >> 5;
    ty = (warp / (BS / 8)) * 4 + (lane >> 3);
    tx = (warp % (BS / 8)) * 8 + (lane & 7);
}

template <int BS>
__global__ void __launch_bounds__(BS *BS, BS == 16 ? 3 : 8) k_fine_stream(FineArgs a) {
    constexpr int BD = BS * BS;
    __shared__ FaceRec s_rec[BD];
    __shared__ int s_id[BD];
    __shared__ float s_key[BD];
    __shared__ int s_item, s_nredo;
    int *s_redo = s_id;  // after the walk: the pixels left for the warp redo
    // dynamic: the bin's sorted entries (sort_cap), then the rings ([slot][thread])
    extern __shared__ unsigned long long s_sort[];
    float *ring_z = reinterpret_cast<float *>(s_sort + a.sort_cap);
    int *ring_f = reinterpret_cast<int *>(ring_z + kRing * BD);
    const int tid = threadIdx.x;
    int ty, tx;
    tile_pixel_of<BS>(tid, ty, tx);
    const int lane = tid & 31, warp = tid >> 5;
    float *rz = ring_z + tid;  // ring entry j at rz[j * BD]
    int *rf = ring_f + tid;
    EvalFlags fl = a.fl;
    const int nb2 = a.nb * a.nb;
    const int K = a.K;
    const float kInf = __int_as_float(0x7f800000);
    while (true) {
        if (tid == 0) {
            s_item = (int)atomicAdd(a.queue, 1u);
            s_nredo = 0;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= a.items) break;
        const int n = item / nb2, rem = item - n * nb2;
        const int by = rem / a.nb, bx = rem - by * a.nb;
        const int r = by * BS + ty, c = bx * BS + tx;
        fl.znear = __ldg(a.cams + 16 * n + 13);
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
        const int cnt = a.eff[item];  // <= max_faces_per_bin <= sort_cap (checked on the host)
        const int off = a.offsets[item];
        sort_entries<BD>(s_sort, a.lists + off, cnt);
        const int64_t s0 = (((int64_t)n * a.S + r) * a.S + c) * K;
        int head = 0, nr = 0, nfin = 0;           // ring head, unsettled entries, settled slots
        float kth_z = kInf;                       // K-th entry while the list is full
        int kth_f = 0x7fffffff;
        bool redo = false;
        auto settle = [&](float z, int f) { a.out.pix_to_face[s0 + nfin] = pack_key(z, f); ++nfin; };
        for (int base = 0; base < cnt; base += BD) {
            const int mc = min(BD, cnt - base);
            if (tid < mc) {
                const unsigned long long v = s_sort[base + tid];
                const int fid = (int)(unsigned)(v & 0xffffffffull);
                s_id[tid] = fid;
                s_key[tid] = __uint_as_float((unsigned)(v >> 32));
                const float4 *src = reinterpret_cast<const float4 *>(a.rec + fid);
                FaceRec R;
                R.a = __ldg(src + kRecA);
                R.b = __ldg(src + kRecB);
                R.c = __ldg(src + kRecC);
                R.d = __ldg(src + kRecD);
                R.e = __ldg(src + kRecE);
                R.h = __ldg(src + kRecH);
                s_rec[tid] = R;
            }
            __syncthreads();
            bool warp_done = false;
            for (int jb = 0; jb < mc; jb += 32) {
                // a lane that is done (or invalid, or left for the redo) needs no more faces
                const bool live = valid && !redo && nfin < K;
                const float thr = !live ? 0.f : (nfin + nr >= K ? kth_z : kInf);
                const float wthr = __int_as_float(__reduce_max_sync(0xffffffffu, __float_as_int(thr)));
                if (s_key[jb] > wthr) {
                    warp_done = true;
                    break;
                }
                const int jl = jb + lane;
                bool hit = false;
                if (jl < mc) {
                    const float4 bb = s_rec[jl].c;
                    hit = bb.x <= wx1 && bb.y >= wx0 && bb.z <= wy1 && bb.w >= wy0 && !(s_key[jl] > wthr);
                }
                unsigned mask = __ballot_sync(0xffffffffu, hit);
                while (mask) {
                    const int jj = jb + __ffs(mask) - 1;
                    mask &= mask - 1;
                    if (!valid || redo || nfin >= K) continue;
                    FaceRec R;
                    R.c = s_rec[jj].c;
                    if (!in_bbox(R, p)) continue;
                    const float key = s_key[jj];
                    const bool full = nfin + nr >= K;
                    if (full && key > kth_z) continue;  // its depth is at least its key
                    R.a = s_rec[jj].a;
                    R.b = s_rec[jj].b;
                    R.d = s_rec[jj].d;
                    R.e = s_rec[jj].e;
                    R.h = s_rec[jj].h;
                    float z;
                    if (!face_key_nobbox(R, p, fl, z)) continue;
                    const int fid = s_id[jj];
                    if (full && !key_less(z, fid, kth_z, kth_f)) continue;
                    // entries in front of this face's key are settled: no later face precedes them
                    while (nr > 0) {
                        const int h = head & (kRing - 1);
                        const float fz = rz[h * BD];
                        if (!(fz < key)) break;
                        settle(fz, rf[h * BD]);
                        ++head;
                        --nr;
                    }
                    if (full) --nr;             // the K-th entry is displaced (nr >= 1: not done)
                    if (nr == kRing) {          // no room: this pixel is redone by a warp
                        redo = true;
                        continue;
                    }
                    int pos = nr;               // insertion from the tail (arrivals are nearly sorted)
                    while (pos > 0) {
                        const int hp = (head + pos - 1) & (kRing - 1);
                        const float pz = rz[hp * BD];
                        const int pf = rf[hp * BD];
                        if (!key_less(z, fid, pz, pf)) break;
                        const int hq = (head + pos) & (kRing - 1);
                        rz[hq * BD] = pz;
                        rf[hq * BD] = pf;
                        --pos;
                    }
                    const int hq = (head + pos) & (kRing - 1);
                    rz[hq * BD] = z;
                    rf[hq * BD] = fid;
                    ++nr;
                    if (nfin + nr >= K) {
                        const int hl = (head + nr - 1) & (kRing - 1);
                        kth_z = rz[hl * BD];
                        kth_f = rf[hl * BD];
                    }
                }
            }
            if (!warp_done && base + BD < cnt) {
                const bool live = valid && !redo && nfin < K;
                const float thr = !live ? 0.f : (nfin + nr >= K ? kth_z : kInf);
                const float wthr = __int_as_float(__reduce_max_sync(0xffffffffu, __float_as_int(thr)));
                warp_done = __uint_as_float((unsigned)(s_sort[base + BD] >> 32)) > wthr;
            }
            if (__syncthreads_and(warp_done)) break;
        }
        // everything left in the ring is settled; empty slots get -1
        if (valid && !redo) {
            while (nr > 0) {
                const int h = head & (kRing - 1);
                settle(rz[h * BD], rf[h * BD]);
                ++head;
                --nr;
            }
            for (int k = nfin; k < K; ++k) a.out.pix_to_face[s0 + k] = -1ll;
        }
        if (valid && redo) s_redo[atomicAdd(&s_nredo, 1)] = tid;
        __syncthreads();
        const int nredo = s_nredo;
        for (int i = warp; i < nredo; i += BD / 32) {
            int rty, rtx;
            tile_pixel_of<BS>(s_redo[i], rty, rtx);
            redo_pixel(a, s_sort, cnt, n, by * BS + rty, bx * BS + rtx, fl);
        }
        if (nredo > 0 && lane == 0 && warp == 0) atomicAdd(a.redo_count, (unsigned)nredo);
        __syncthreads();  // s_sort, s_item and s_nredo are reused by the next item
    }
}

// ---------------------------------------------------------------------------
// Fragment attributes: a block takes PB = 256 / K whole pixels, one thread per
// slot in output order (consecutive threads, consecutive slots: coalesced)
// ---------------------------------------------------------------------------
template <bool BL>
__global__ void __launch_bounds__(256) k_frag_attr(FragAttrArgs a) {
    __shared__ float s_keep[256];
    const int K = a.K, S = a.S;
    const int PB = 256 / K;
    const int t = threadIdx.x;
    const int64_t pix0 = (int64_t)blockIdx.x * PB;
    const int lp = t / K, k = t - lp * K;
    const int64_t pix = pix0 + lp;
    const bool active = lp < PB && pix < a.P;
    float keep = 1.f;
    if (active) {
        const int64_t s = pix * K + k;
        long long v = a.out.pix_to_face[s];
        // a key names a face of the batch; anything else (never written by the
        // fine pass) is reported and treated as an empty slot
        if (v >= 0 && (long long)(unsigned)(v & 0xffffffffll) >= a.F) {
            set_status(a.status, MESHRAST_ST_BAD_INDEX);
            v = -1ll;
        }
        if (v < 0) {
            a.out.pix_to_face[s] = -1ll;
            a.out.zbuf[s] = -1.f;
            a.out.bary[3 * s] = -1.f;
            a.out.bary[3 * s + 1] = -1.f;
            a.out.bary[3 * s + 2] = -1.f;
            a.out.dists[s] = -1.f;
        } else {
            const int f = (int)(unsigned)(v & 0xffffffffll);
            const float z = __uint_as_float((unsigned)((unsigned long long)v >> 32));
            const float4 *src = reinterpret_cast<const float4 *>(a.rec + f);
            FaceRec R;
            R.a = __ldg(src + kRecA);
            R.b = __ldg(src + kRecB);
            R.d = __ldg(src + kRecD);
            R.e = __ldg(src + kRecE);
            const int64_t n = pix / ((int64_t)S * S);
            const int rem = (int)(pix - n * S * S);
            const int r = rem / S, c = rem - r * S;
            float bp[3], d;
            face_fragment(R, pixel_centre(r, c, S), a.fl, bp, d);
            a.out.pix_to_face[s] = f;
            a.out.zbuf[s] = z;
            a.out.bary[3 * s] = bp[0];
            a.out.bary[3 * s + 1] = bp[1];
            a.out.bary[3 * s + 2] = bp[2];
            a.out.dists[s] = d;
            if constexpr (BL) keep = sigmoidf_(d / a.sigma);
        }
    }
    if constexpr (BL) {
        // Algorithm 1: alpha = 1 - prod_k (1 - prob_k); one warp per pixel
        // multiplies its K factors in a fixed tree order
        s_keep[t] = keep;
        __syncthreads();
        const int lane = t & 31;
        for (int q = t >> 5; q < PB; q += 8) {
            const int64_t qp = pix0 + q;
            float m = 1.f;
            if (lane < K) m = s_keep[q * K + lane];
            if (lane + 32 < K) m *= s_keep[q * K + lane + 32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m *= __shfl_xor_sync(0xffffffffu, m, o);
            if (lane == 0 && qp < a.P) reinterpret_cast<float4 *>(a.image)[qp] = make_float4(0.f, 0.f, 0.f, 1.f - m);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t fine_stream_smem(int sort_cap, int bin) { return (size_t)sort_cap * 8 + (size_t)kRing * bin * bin * 8; }

template <int BS>
static cudaError_t launch_fine_stream_t(const FineArgs &a, cudaStream_t st) {
    constexpr int BD = BS * BS;
    const size_t dyn = fine_stream_smem(a.sort_cap, BS);
    auto kern = k_fine_stream<BS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, BD, dyn);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min<int>(a.items, mr_host::num_sms() * std::max(1, bps)));
    kern<<<grid, BD, dyn, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fine_stream(const FineArgs &a, int bin, cudaStream_t st) {
    if (bin == 8) return launch_fine_stream_t<8>(a, st);
    if (bin == 16) return launch_fine_stream_t<16>(a, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_frag_attr(const FragAttrArgs &a, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    if (a.K < 1 || a.K > 64) return cudaErrorInvalidValue;
    const int PB = 256 / a.K;
    const int64_t blocks = (a.P + PB - 1) / PB;
    if (a.image) k_frag_attr<true><<<(unsigned)blocks, 256, 0, st>>>(a);
    else k_frag_attr<false><<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mr
