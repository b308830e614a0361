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
// candidates stay on chip, in a ring of kRing1 entries per pixel in shared
// memory (the settled prefix is a counter).
//
// A pixel whose unsettled candidates outgrow the ring (rare on smooth meshes;
// common on strongly deformed ones, whose tilted faces lie far behind their
// nearest corner) is queued with its 8 x 4 block; a second pass walks the
// queued blocks again for those pixels only, with a ring of 64 entries, at
// least K, which cannot overflow.  Its shared memory (64 KB per block of 4
// warps) is paid only by the blocks that need it.
//
// The fine pass writes each slot as one 64-bit key: (depth bits << 32) | face
// id, or -1 for an empty slot, into pix_to_face.  k_frag_attr, one thread per
// slot (consecutive slots on consecutive threads: coalesced), expands it into
// pix_to_face, zbuf, barycentrics and distance, and applies the silhouette
// blend (Algorithm 1) when asked.
#include <cuda_runtime.h>

#include <algorithm>

#include "bin_common.cuh"
#include "blend_common.cuh"
#include "rast_common.cuh"
#include "rast_internal.h"

namespace mr {

// unsettled candidates a pixel keeps on chip: first pass, second pass (>= K)
constexpr int kRing1 = 16, kRing2 = 64;
constexpr int kWarps1 = 8, kWarps2 = 4;  // warps per block of each pass

__device__ __forceinline__ long long pack_key(float z, int f) {
    return (long long)(((unsigned long long)__float_as_uint(z) << 32) | (unsigned)f);
}

// ---------------------------------------------------------------------------
// front-to-back order of every bin's list, sorted in place before the fine
// pass (one block per bin; small shared memory, many blocks per SM)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sort_bins(FineArgs a) {
    extern __shared__ unsigned long long s_sort[];
    for (int item = blockIdx.x; item < a.items; item += gridDim.x) {
        const int bin = a.order ? __ldg(a.order + item) : item;  // longest bins first
        const int cnt = a.eff[bin];  // <= sort_cap (checked on the host); uniform over the block
        if (cnt <= 1) continue;
        unsigned long long *list = a.lists + a.offsets[bin];
        sort_entries<256, true>(s_sort, list, cnt);
        for (int i = threadIdx.x; i < cnt; i += 256) list[i] = s_sort[i];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// the streaming fine pass: every warp works on its own, with no block
// barrier.  A work item is an 8 x 4 block of pixels of one bin (8 columns, 4
// rows: about as wide as tall, like the inflated face bboxes the warp culls
// against); the warp walks the bin's sorted list from L2 32 entries at a
// time, each lane keeping its pixel's unsettled candidates in its own ring.
// ---------------------------------------------------------------------------

// Whether no point of the rectangle [x0, x1] x [y0, y1] can be within
// sqrt(blur) of the face: the whole rectangle lies beyond the line of one of
// its edges by more than that.  The barycentric of the opposite corner is
// affine in the point, so its largest value over the rectangle is taken at a
// corner; beyond the line it is negative and the squared distance to the line
// is b^2 H.  A 10 % margin on the squared distance covers the fp32 rounding,
// and slivers (whose fp32 barycentrics are less accurate) are never rejected:
// a face this rejects is no candidate for any pixel of the rectangle.
__device__ __forceinline__ bool rect_beyond_edge(const float4 &ra, const float4 &rb, const float4 &rd,
                                                 const float4 &rh, float x0, float x1, float y0, float y1,
                                                 float blur) {
    const float ux = rb.x, uy = rb.y, wx = rb.z, wy = rb.w, iA = rd.x;
    const float sliver = (ux * ux + uy * uy + wx * wx + wy * wy) * fabsf(iA);
    const float qx = x0 - (ra.x + ra.z), qy = y0 - (ra.y + ra.w);
    const float b2 = (ux * qy - uy * qx) * iA, b1 = (qx * wy - qy * wx) * iA, b0 = 1.f - b1 - b2;
    const float dx = x1 - x0, dy = y1 - y0;
    const float g2x = -uy * iA * dx, g2y = ux * iA * dy, g1x = wy * iA * dx, g1y = -wx * iA * dy;
    const float m2 = b2 + fmaxf(g2x, 0.f) + fmaxf(g2y, 0.f);
    const float m1 = b1 + fmaxf(g1x, 0.f) + fmaxf(g1y, 0.f);
    const float m0 = b0 + fmaxf(-g1x - g2x, 0.f) + fmaxf(-g1y - g2y, 0.f);
    const float lim = blur * 1.1f;
    const bool out = (m0 < 0.f && m0 * m0 * rh.x > lim) || (m1 < 0.f && m1 * m1 * rh.y > lim) ||
                     (m2 < 0.f && m2 * m2 * rh.z > lim);
    return out && sliver <= 64.f;
}

// First pass (SECOND = false): every item, a ring of RING = 16 per pixel,
// WARPS = 8 warps per block.  Pixels whose unsettled candidates outgrow it are
// queued, per item, as a lane mask.  Second pass (SECOND = true): the queued
// items again, only their queued lanes, with a ring of RING = 64 >= K, which
// cannot overflow (a pixel never holds more than K - settled candidates).
template <int BS, int RING, int WARPS, bool SECOND>
__global__ void __launch_bounds__(WARPS * 32, SECOND ? 3 : 4) k_fine_stream(FineArgs a) {
    constexpr int SUB = BS * BS / 32;  // 8 x 4 pixel blocks per bin
    // per warp: the rings ([slot][lane]), depths then face ids
    extern __shared__ float s_ring[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float (*rz)[32] = reinterpret_cast<float (*)[32]>(s_ring + (size_t)wib * RING * 32);
    int (*rf)[32] = reinterpret_cast<int (*)[32]>(s_ring + (size_t)(WARPS + wib) * RING * 32);
    EvalFlags fl = a.fl;
    const int nb2 = a.nb * a.nb;
    const int K = a.K;
    const long long total = SECOND ? 0ll : (long long)a.items * SUB;
    const float kInf = __int_as_float(0x7f800000);
    while (true) {
        long long item = 0;
        unsigned lanes = 0xffffffffu;  // the lanes this pass takes
        if constexpr (SECOND) {
            unsigned long long e = 0ull;
            if (lane == 0) {
                const unsigned j = atomicAdd(a.redo_head, 1u);
                e = j < *a.redo_q ? a.redo_items[j] : ~0ull;
            }
            e = __shfl_sync(0xffffffffu, e, 0);
            if (e == ~0ull) break;
            item = (long long)(e >> 32);
            lanes = (unsigned)e;
        } else {
            if (lane == 0) item = (long long)atomicAdd(a.queue, 1u);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item >= total) break;
        }
        const int qb = (int)(item / SUB), sub = (int)(item - (long long)qb * SUB);
        const int bin = a.order ? __ldg(a.order + qb) : qb;  // longest bins first
        const int n = bin / nb2, rem = bin - n * nb2;
        const int by = rem / a.nb, bx = rem - by * a.nb;
        const int r = by * BS + (sub / (BS / 8)) * 4 + (lane >> 3);
        const int c = bx * BS + (sub % (BS / 8)) * 8 + (lane & 7);
        fl.znear = __ldg(a.cams + 16 * n + 13);
        const bool valid = (r < a.S) && (c < a.S) && ((lanes >> lane) & 1u);
        const PixC p = pixel_centre(r, c, a.S);
        float wx0 = 1.f, wx1 = -1.f, wy0 = 1.f, wy1 = -1.f;
        {
            const unsigned cmin = __reduce_min_sync(0xffffffffu, valid ? (unsigned)c : 0xffffffffu);
            const unsigned cmax = __reduce_max_sync(0xffffffffu, valid ? (unsigned)c : 0u);
            const unsigned rmin = __reduce_min_sync(0xffffffffu, valid ? (unsigned)r : 0xffffffffu);
            const unsigned rmax = __reduce_max_sync(0xffffffffu, valid ? (unsigned)r : 0u);
            if (cmin > cmax) continue;  // no pixel of this block lies in the image (warp-uniform)
            wx1 = pc_hi((int)cmin, a.S);
            wx0 = pc_hi((int)cmax, a.S);
            wy1 = pc_hi((int)rmin, a.S);
            wy0 = pc_hi((int)rmax, a.S);
        }
        const int cnt = a.eff[bin];
        // the bin's list, sorted front to back by k_sort_bins
        const unsigned long long *ent = a.lists + a.offsets[bin];
        const int64_t s0 = (((int64_t)n * a.S + r) * a.S + c) * K;
        int head = 0, nr = 0, nfin = 0;           // ring head, unsettled entries, settled slots
        float kth_z = kInf;                       // K-th entry while the list is full
        int kth_f = 0x7fffffff;
        bool redo = false;
        auto settle = [&](float z, int f) { a.out.pix_to_face[s0 + nfin] = pack_key(z, f); ++nfin; };
        for (int jb = 0; jb < cnt; jb += 32) {
            // a lane that is done (or invalid, or left for the redo) needs no more faces
            const bool live = valid && !redo && nfin < K;
            const float thr = !live ? 0.f : (nfin + nr >= K ? kth_z : kInf);
            const float wthr = __int_as_float(__reduce_max_sync(0xffffffffu, __float_as_int(thr)));
            const int jl = jb + lane;
            int fid = 0;
            float key = kInf;
            float4 bb = make_float4(1.f, -1.f, 1.f, -1.f);
            if (jl < cnt) {
                const unsigned long long v = __ldg(ent + jl);
                fid = (int)(unsigned)(v & 0xffffffffull);
                key = __uint_as_float((unsigned)(v >> 32));
                bb = __ldg(reinterpret_cast<const float4 *>(a.rec + fid) + kRecC);
            }
            // keys ascend along the list: once the first is behind every lane, the rest is too
            if (__shfl_sync(0xffffffffu, key, 0) > wthr) break;
            bool hit = bb.x <= wx1 && bb.y >= wx0 && bb.z <= wy1 && bb.w >= wy0 && !(key > wthr);
            if (hit) {
                // the first 64 bytes of the record, which the loop below reads
                // one face after another, come to L1 here for all faces at once
                const float4 *rp = reinterpret_cast<const float4 *>(a.rec + fid);
                const float4 ra = __ldg(rp + kRecA), rb = __ldg(rp + kRecB), rd = __ldg(rp + kRecD);
                const float4 rh = __ldg(rp + kRecH);
                asm volatile("prefetch.global.L1 [%0];" ::"l"(rp + kRecE));
                // a face whose bbox meets the block but whose blur region misses it
                if (fl.blur > 0.f && rect_beyond_edge(ra, rb, rd, rh, wx0, wx1, wy0, wy1, fl.blur)) hit = false;
            }
            unsigned mask = __ballot_sync(0xffffffffu, hit);
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const int f = __shfl_sync(0xffffffffu, fid, src);
                const float fkey = __shfl_sync(0xffffffffu, key, src);
                FaceRec R;
                R.c.x = __shfl_sync(0xffffffffu, bb.x, src);
                R.c.y = __shfl_sync(0xffffffffu, bb.y, src);
                R.c.z = __shfl_sync(0xffffffffu, bb.z, src);
                R.c.w = __shfl_sync(0xffffffffu, bb.w, src);
                if (!valid || redo || nfin >= K) continue;
                if (!in_bbox(R, p)) continue;
                const bool full = nfin + nr >= K;
                if (full && fkey > kth_z) continue;  // its depth is at least its key
                const float4 *rs = reinterpret_cast<const float4 *>(a.rec + f);
                R.a = __ldg(rs + kRecA);
                R.b = __ldg(rs + kRecB);
                R.d = __ldg(rs + kRecD);
                R.e = __ldg(rs + kRecE);
                R.h = __ldg(rs + kRecH);
                float z;
                if (!face_key_nobbox(R, p, fl, z)) continue;
                if (full && !key_less(z, f, kth_z, kth_f)) continue;
                // entries in front of this face's key are settled: no later face precedes them
                while (nr > 0) {
                    const int h = head & (RING - 1);
                    const float fz = rz[h][lane];
                    if (!(fz < fkey)) break;
                    settle(fz, rf[h][lane]);
                    ++head;
                    --nr;
                }
                if (full) --nr;             // the K-th entry is displaced (nr >= 1: not done)
                if (nr == RING) {           // no room: this pixel goes to the second pass
                    redo = true;
                    continue;
                }
                int pos = nr;               // insertion from the tail (arrivals are nearly sorted)
                while (pos > 0) {
                    const int hp = (head + pos - 1) & (RING - 1);
                    const float pz = rz[hp][lane];
                    const int pf = rf[hp][lane];
                    if (!key_less(z, f, pz, pf)) break;
                    const int hq = (head + pos) & (RING - 1);
                    rz[hq][lane] = pz;
                    rf[hq][lane] = pf;
                    --pos;
                }
                const int hq = (head + pos) & (RING - 1);
                rz[hq][lane] = z;
                rf[hq][lane] = f;
                ++nr;
                if (nfin + nr >= K) {
                    const int hl = (head + nr - 1) & (RING - 1);
                    kth_z = rz[hl][lane];
                    kth_f = rf[hl][lane];
                }
            }
        }
        // everything left in the ring is settled; empty slots get -1
        if (valid && !redo) {
            while (nr > 0) {
                const int h = head & (RING - 1);
                settle(rz[h][lane], rf[h][lane]);
                ++head;
                --nr;
            }
            for (int k = nfin; k < K; ++k) a.out.pix_to_face[s0 + k] = -1ll;
        }
        // pixels whose unsettled candidates outgrew the ring: queued for the
        // second pass (each item at most once, so the queue never fills)
        if constexpr (!SECOND) {
            const unsigned todo = __ballot_sync(0xffffffffu, valid && redo);
            if (todo && lane == 0) {
                atomicAdd(a.redo_count, (unsigned)__popc(todo));
                a.redo_items[atomicAdd(a.redo_q, 1u)] = ((unsigned long long)item << 32) | todo;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Fragment attributes: a block takes PB = 256 / K whole pixels, one thread per
// slot in output order (consecutive threads, consecutive slots: coalesced)
// ---------------------------------------------------------------------------
// q = n / d for n < 2^26 and 1 <= d <= 8192 from a 32-bit reciprocal, corrected to exact
__device__ __forceinline__ unsigned div_small(unsigned n, unsigned d, unsigned magic) {
    unsigned q = __umulhi(n, magic);
    if ((q + 1) * d <= n) ++q;
    if (q * d > n) --q;
    return q;
}

template <bool BL>
__global__ void __launch_bounds__(256, 6) k_frag_attr(FragAttrArgs a) {
    __shared__ float s_keep[256];
    const int K = a.K, S = a.S;
    const int PB = 256 / K;
    const int t = threadIdx.x;
    // grid: x = chunk of PB pixels of one image, y = image
    const unsigned SS = (unsigned)S * (unsigned)S;
    const unsigned q0 = blockIdx.x * (unsigned)PB;            // first pixel of the chunk in its image
    const int lp = (int)__fdividef((float)t + 0.5f, (float)K); // t / K (t < 256: exact)
    const int k = t - lp * K;
    const unsigned qi = q0 + (unsigned)lp;
    const int64_t pix0 = (int64_t)blockIdx.y * SS + q0;
    const int64_t pix = pix0 + lp;
    const bool active = lp < PB && qi < SS;
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
            const int r = (int)div_small(qi, (unsigned)S, a.magic_S), c = (int)qi - r * S;
            float bp[3], d;
            face_fragment(R, pixel_centre(r, c, S), a.fl, bp, d);
            a.out.pix_to_face[s] = f;
            a.out.zbuf[s] = z;
            a.out.bary[3 * s] = bp[0];
            a.out.bary[3 * s + 1] = bp[1];
            a.out.bary[3 * s + 2] = bp[2];
            a.out.dists[s] = d;
            if constexpr (BL) keep = __frcp_rn(1.f + expf(-d * a.inv_sigma));  // 1 - prob = sigmoid(d / sigma)
        }
    }
    if constexpr (BL) {
        // Algorithm 1: alpha = 1 - prod_k (1 - prob_k); one warp per pixel
        // multiplies its K factors in a fixed tree order
        s_keep[t] = keep;
        __syncthreads();
        const int lane = t & 31;
        for (int q = t >> 5; q < PB; q += 8) {
            float m = 1.f;
            if (lane < K) m = s_keep[q * K + lane];
            if (lane + 32 < K) m *= s_keep[q * K + lane + 32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m *= __shfl_xor_sync(0xffffffffu, m, o);
            if (lane == 0 && q0 + (unsigned)q < SS)
                reinterpret_cast<float4 *>(a.image)[pix0 + q] = make_float4(0.f, 0.f, 0.f, 1.f - m);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static cudaError_t launch_sort_bins(const FineArgs &a, cudaStream_t st) {
    const size_t dyn = (size_t)a.sort_cap * 8;
    cudaError_t e = cudaFuncSetAttribute(k_sort_bins, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_sort_bins, 256, dyn);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min<int>(a.items, mr_host::num_sms() * std::max(1, bps)));
    k_sort_bins<<<grid, 256, dyn, st>>>(a);
    return cudaGetLastError();
}

template <int BS>
static cudaError_t launch_fine_stream_t(const FineArgs &a, cudaStream_t st) {
    // first pass: every 8 x 4 block of every bin
    {
        auto kern = k_fine_stream<BS, kRing1, kWarps1, false>;
        const size_t dyn = (size_t)2 * kWarps1 * kRing1 * 32 * sizeof(float);  // 32 KB
        int bps = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kWarps1 * 32, dyn);
        if (e != cudaSuccess) return e;
        const long long warps = (long long)a.items * (BS * BS / 32);
        const long long need = (warps + kWarps1 - 1) / kWarps1;
        const int grid =
            (int)std::max(1LL, std::min<long long>(need, (long long)mr_host::num_sms() * std::max(1, bps)));
        kern<<<grid, kWarps1 * 32, dyn, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // second pass: the queued blocks (their count is on the device; warps stop
    // at the end of the queue)
    auto kern = k_fine_stream<BS, kRing2, kWarps2, true>;
    const size_t dyn = (size_t)2 * kWarps2 * kRing2 * 32 * sizeof(float);  // 64 KB
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kWarps2 * 32, dyn);
    if (e != cudaSuccess) return e;
    const long long need = ((long long)a.items * (BS * BS / 32) + kWarps2 - 1) / kWarps2;
    const int grid = (int)std::max(1LL, std::min<long long>(need, (long long)mr_host::num_sms() * std::max(1, bps)));
    kern<<<grid, kWarps2 * 32, dyn, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fine_stream(const FineArgs &a, int bin, cudaStream_t st) {
    cudaError_t e = launch_sort_bins(a, st);
    if (e != cudaSuccess) return e;
    if (bin == 8) return launch_fine_stream_t<8>(a, st);
    if (bin == 16) return launch_fine_stream_t<16>(a, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_frag_attr(const FragAttrArgs &a, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    if (a.K < 1 || a.K > 64) return cudaErrorInvalidValue;
    if (a.S < 1 || a.S > 8192 || a.P % ((int64_t)a.S * a.S) != 0) return cudaErrorInvalidValue;
    const int PB = 256 / a.K;
    const int64_t N = a.P / ((int64_t)a.S * a.S);
    if (N > 65535) return cudaErrorInvalidValue;
    FragAttrArgs b = a;
    b.inv_sigma = 1.f / a.sigma;
    b.magic_S = (unsigned)((0x100000000ull + (unsigned)a.S - 1) / (unsigned)a.S);
    const dim3 grid((unsigned)(((int64_t)a.S * a.S + PB - 1) / PB), (unsigned)N);
    if (a.image) k_frag_attr<true><<<grid, 256, 0, st>>>(b);
    else k_frag_attr<false><<<grid, 256, 0, st>>>(b);
    return cudaGetLastError();
}

}  // namespace mr
