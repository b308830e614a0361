// Forward rasterization kernels for sm_103a.
//
// Section 3.2 of the paper ("Rasterizer"): camera transform to NDC, a
// two-pass approach that first assigns faces to image tiles (bins) and then
// finds, per pixel, the K nearest faces along z with a priority queue, and the
// Fragment data of those faces.  Launch sequence of one binned forward:
//   k_stage     one thread per face: double-float projection, 96-byte face
//               record, warp-aggregated bin counts
//   k_scan      one block: clamp counts to capacity, exclusive scan -> offsets
//   k_fill      one thread per face: warp-aggregated atomic append into lists
//   k_fine      persistent blocks pull (image, bin) items from a global queue,
//               stage each bin's face records in shared memory, keep a
//               register-resident top-K per pixel, write the fragments
// The plain form (bin_size 0) replaces scan/fill/fine by k_naive, one launch
// per image, every pixel against every face of its image.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "rast_common.cuh"
#include "rast_internal.h"
#include "blend_common.cuh"
#include "bin_common.cuh"

namespace mr {

// ---------------------------------------------------------------------------
// staging
// ---------------------------------------------------------------------------
// Build the record of face f; returns the mesh index or -1 when culled.
__device__ int stage_face(const StageArgs &a, int64_t f, int n, FaceRec &R) {
    const float kInf = __int_as_float(0x7f800000);
    R.a = make_float4(0.f, 0.f, 0.f, 0.f);
    R.b = make_float4(0.f, 0.f, 0.f, 0.f);
    R.c = make_float4(kInf, -kInf, kInf, -kInf);
    R.d = make_float4(0.f, 1.f, 1.f, 1.f);
    R.e = make_float4(0.f, 0.f, 0.f, 0.f);
    R.h = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n < 0) return -1;
    unsigned bad = 0;
    int64_t vi[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        vi[i] = a.faces[3 * f + i];
        if (vi[i] < 0 || vi[i] >= a.V) bad |= MESHRAST_ST_BAD_INDEX;
    }
    if (bad) { set_status(a.status, bad); return -1; }
    const float *cam = a.cams + 16 * n;
    df X[3], Y[3], Z[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float px = a.verts[3 * vi[i]], py = a.verts[3 * vi[i] + 1], pz = a.verts[3 * vi[i] + 2];
        if (!(isfinite(px) && isfinite(py) && isfinite(pz))) bad |= MESHRAST_ST_NONFINITE;
        project_corner(cam, px, py, pz, X[i], Y[i], Z[i]);
    }
    if (bad) { set_status(a.status, bad); return -1; }
    const float znear = cam[13];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        // z < znear (as a double-float) culls the face
        if (Z[i].hi < znear || (Z[i].hi == znear && Z[i].lo < 0.f) || !isfinite(Z[i].hi)) return -1;
        if (!isfinite(X[i].hi) || !isfinite(Y[i].hi)) return -1;
    }
    df Ux = df_sub(X[1], X[0]), Uy = df_sub(Y[1], Y[0]);
    df Wx = df_sub(X[2], X[0]), Wy = df_sub(Y[2], Y[0]);
    // area in double-float (matches an FP64 evaluation to ~1e-14): culling and 1/A
    df Adf = df_sub(df_mul(Ux, Wy), df_mul(Uy, Wx));
    if (!(fabsf(Adf.hi) >= kCullArea)) return -1;
    const float A = __fadd_rn(Adf.hi, Adf.lo);
    float ux = Ux.hi, uy = Uy.hi, wx = Wx.hi, wy = Wy.hi;
    float r = (a.blur > 0.f) ? sqrtf(a.blur) : 0.f;
    df xmin = df_min(df_min(X[0], X[1]), X[2]), xmax = df_max(df_max(X[0], X[1]), X[2]);
    df ymin = df_min(df_min(Y[0], Y[1]), Y[2]), ymax = df_max(df_max(Y[0], Y[1]), Y[2]);
    R.a = make_float4(X[0].hi, Y[0].hi, X[0].lo, Y[0].lo);
    R.b = make_float4(ux, uy, wx, wy);
    R.c = make_float4(df_round_down(df_add(xmin, {-r, 0.f})), df_round_up(df_add(xmax, {r, 0.f})),
                      df_round_down(df_add(ymin, {-r, 0.f})), df_round_up(df_add(ymax, {r, 0.f})));
    R.d = make_float4(__fdiv_rn(1.f, A), __fdiv_rn(1.f, Z[0].hi), __fdiv_rn(1.f, Z[1].hi),
                      __fdiv_rn(1.f, Z[2].hi));
    R.e = make_float4(Ux.lo, Uy.lo, Wx.lo, Wy.lo);
    const float A2 = A * A;
    const float l0 = (wx - ux) * (wx - ux) + (wy - uy) * (wy - uy), l1 = wx * wx + wy * wy, l2 = ux * ux + uy * uy;
    R.h = make_float4(A2 / l0, A2 / l1, A2 / l2, 0.f);
    return n;
}

__global__ void __launch_bounds__(256) k_stage(StageArgs a) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    FaceRec R;
    int n = block_find_mesh(a.first_face, a.num_faces, a.N, a.F, f);
    if (f < a.F) {
        n = stage_face(a, f, n, R);
        float4 *dst = reinterpret_cast<float4 *>(a.rec + f);
        dst[kRecA] = R.a;
        dst[kRecB] = R.b;
        dst[kRecC] = R.c;
        dst[kRecD] = R.d;
        dst[kRecE] = R.e;
        dst[kRecH] = R.h;
        if (a.face_mesh) a.face_mesh[f] = n;
    }
    if (!a.do_count) return;
    // warp-aggregated bin counting; every lane of the warp takes part
    int bx0 = 1, bx1 = 0, by0 = 1, by1 = 0;
    if (n >= 0) bin_rect(R, a.S, a.bin, bx0, bx1, by0, by1);
    const int nbx = max(0, bx1 - bx0 + 1), nby = max(0, by1 - by0 + 1);
    const int cnt = nbx * nby;
    const int wmax = __reduce_max_sync(0xffffffffu, cnt);
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < wmax; ++i) {
        int key = -1;
        if (i < cnt) key = (n * a.nb + by0 + i / nbx) * a.nb + bx0 + i % nbx;
        unsigned grp = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && lane == __ffs(grp) - 1) atomicAdd(a.counts + key, __popc(grp));
    }
}

// ---------------------------------------------------------------------------
// scan: one block; clamps counts, exclusive scan, resets cursors and queue
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan(ScanArgs a) {
    __shared__ long long warp_sums[32];
    __shared__ long long carry_s;   // running sum of the clamped counts (may exceed the capacity)
    __shared__ int maxc_s;
    __shared__ unsigned long long tot_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        carry_s = 0;
        maxc_s = 0;
        tot_s = 0ull;
        *a.queue = 0u;
        // packed-layout validation of first_face / num_faces
        unsigned bad = 0;
        int64_t prev_end = 0;
        for (int n = 0; n < a.N; ++n) {
            int64_t lo = a.first_face[n], cnt = a.num_faces[n];
            if (lo < 0 || cnt < 0 || lo + cnt > a.F || lo < prev_end) bad |= MESHRAST_ST_BAD_MESH_RANGE;
            prev_end = lo + (cnt > 0 ? cnt : 0);
        }
        set_status(a.status, bad);
    }
    __syncthreads();
    bool overflow = false;
    int local_max = 0;
    unsigned long long local_tot = 0;
    for (int64_t base = 0; base < a.NB; base += 1024) {
        const int64_t b = base + tid;
        int c = (b < a.NB) ? a.counts[b] : 0;
        local_max = max(local_max, c);
        local_tot += (unsigned long long)c;
        int e = c;
        if (e > a.max_per_bin) { e = a.max_per_bin; overflow = true; }
        // block exclusive scan of e (64-bit: 1024 counts may sum past 2^31)
        long long x = e;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            long long s = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const long long carry = carry_s;
        // 64-bit position; entries past the capacity are dropped (overflow bit)
        const long long excl = carry + (wid ? warp_sums[wid - 1] : 0ll) + x - e;
        if (b < a.NB) {
            const long long room = (long long)a.capacity - excl;
            if ((long long)e > room) { e = (int)max(0ll, room); overflow = true; }
            a.offsets[b] = (int)min(excl, (long long)a.capacity);  // capacity < 2^31 (checked on the host)
            a.eff[b] = e;
            a.cursor[b] = 0;
        }
        __syncthreads();
        if (tid == 1023) carry_s = carry + warp_sums[31];
        __syncthreads();
    }
    // block totals: warp reductions first, then one shared atomic per warp
    local_max = __reduce_max_sync(0xffffffffu, local_max);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local_tot += __shfl_xor_sync(0xffffffffu, local_tot, o);
    if (lane == 0) {
        atomicMax(&maxc_s, local_max);
        atomicAdd(&tot_s, local_tot);
    }
    if (__any_sync(0xffffffffu, overflow) && lane == 0) set_status(a.status, MESHRAST_ST_BIN_OVERFLOW);
    __syncthreads();
    if (tid == 0) {
        a.offsets[a.NB] = (int)min(carry_s, (long long)a.capacity);
        *a.maxcount = maxc_s;
        *a.total = (long long)tot_s;
    }
    if (!a.order) return;
    // Queue order of the fine pass: bins by descending work class (the bit
    // length of the clamped count), a counting sort over 32 classes, so the
    // longest bins start first and the short ones fill the tail.  The order
    // within a class is whatever the atomics give: each bin's output depends
    // on that bin alone.
    __shared__ int cls_n[32];
    if (tid < 32) cls_n[tid] = 0;
    __syncthreads();
    for (int64_t base = 0; base < a.NB; base += 1024) {  // every lane takes every round
        const int64_t b = base + tid;
        const int cls = (b < a.NB) ? 32 - __clz(a.eff[b]) : -1;  // 0: empty bin; eff < 2^31
        const unsigned grp = __match_any_sync(0xffffffffu, cls);
        if (cls >= 0 && lane == __ffs(grp) - 1) atomicAdd(&cls_n[cls], __popc(grp));
    }
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int c = 31; c >= 0; --c) {
            const int n = cls_n[c];
            cls_n[c] = s;  // first position of class c
            s += n;
        }
    }
    __syncthreads();
    for (int64_t base = 0; base < a.NB; base += 1024) {
        const int64_t b = base + tid;
        const int cls = (b < a.NB) ? 32 - __clz(a.eff[b]) : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, cls);
        const int leader = __ffs(grp) - 1;
        int first = 0;
        if (cls >= 0 && lane == leader) first = atomicAdd(&cls_n[cls], __popc(grp));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (cls >= 0) a.order[first + __popc(grp & ((1u << lane) - 1u))] = (int)b;
    }
}

// ---------------------------------------------------------------------------
// fill: warp-aggregated atomic append into the per-bin lists
// ---------------------------------------------------------------------------
// Lower bound on a face's depth at any pixel where it is a candidate (nearest
// corner), valid when the depth is a convex combination of the corner depths:
// with clipping, or without blur (inside pixels only).  Slightly reduced so
// that fp32 rounding of the key can never fall below it.
__device__ __forceinline__ float face_zmin(const FaceRec &R) {
    if (!(R.c.x <= R.c.y)) return __int_as_float(0x7f800000);  // culled
    return __fdividef(1.f, fmaxf(R.d.y, fmaxf(R.d.z, R.d.w))) * (1.f - 1e-6f);
}

// Bin-list entry: nearest-corner depth (a positive float, so its bits order
// like the value) in the high word, face id in the low word; sorting entries
// as integers orders a bin's faces front to back, ties by id.
__device__ __forceinline__ unsigned long long bin_entry(float zmin, int f) {
    return ((unsigned long long)__float_as_uint(zmin) << 32) | (unsigned)f;
}

__global__ void __launch_bounds__(256) k_fill(FillArgs a) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int n = -1;
    FaceRec R;
    if (f < a.F) {
        n = a.face_mesh[f];
        if (n >= 0) {
            const float4 *src = reinterpret_cast<const float4 *>(a.rec + f);
            R.c = src[kRecC];
            R.d = src[kRecD];
        }
    }
    int bx0 = 1, bx1 = 0, by0 = 1, by1 = 0;
    if (n >= 0) bin_rect(R, a.S, a.bin, bx0, bx1, by0, by1);
    const unsigned long long entry = n >= 0 ? bin_entry(face_zmin(R), (int)f) : 0ull;
    const int nbx = max(0, bx1 - bx0 + 1), nby = max(0, by1 - by0 + 1);
    const int cnt = nbx * nby;
    const int wmax = __reduce_max_sync(0xffffffffu, cnt);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = 0; i < wmax; ++i) {
        int key = -1;
        if (i < cnt) key = (n * a.nb + by0 + i / nbx) * a.nb + bx0 + i % nbx;
        unsigned grp = __match_any_sync(0xffffffffu, key);
        int leader = __ffs(grp) - 1;
        int base = 0;
        if (key >= 0 && lane == leader) base = atomicAdd(a.cursor + key, __popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (key >= 0) {
            int slot = base + __popc(grp & lt);
            if (slot < a.eff[key]) a.lists[a.offsets[key] + slot] = entry;
        }
    }
}

// ---------------------------------------------------------------------------
// output of one pixel's K fragments
// ---------------------------------------------------------------------------
template <int KM, bool BL>
__device__ __forceinline__ void write_pixel(const FineOut &o, int64_t pix, int K, const TopK<KM> &tk,
                                            const FaceRec *rec, const PixC &p, const EvalFlags &fl,
                                            const FineBlend &bl) {
    const int64_t s0 = pix * (int64_t)K;
    FwdBlend fb;
    if constexpr (BL) fb.begin(bl, tk.f[0] != 0x7fffffff, tk.z[0]);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (k >= K) break;
        const int64_t s = s0 + k;
        const int f = tk.f[k];
        const bool store = !BL || bl.frag;
        if (f == 0x7fffffff) {
            if (store) {
                o.pix_to_face[s] = -1;
                o.zbuf[s] = -1.f;
                o.bary[3 * s] = -1.f;
                o.bary[3 * s + 1] = -1.f;
                o.bary[3 * s + 2] = -1.f;
                o.dists[s] = -1.f;
            }
        } else {
            FaceRec R;
            const float4 *src = reinterpret_cast<const float4 *>(rec + f);
            R.a = __ldg(src + kRecA);
            R.b = __ldg(src + kRecB);
            R.c = __ldg(src + kRecC);
            R.d = __ldg(src + kRecD);
            R.e = __ldg(src + kRecE);
            float bp[3], d;
            face_fragment(R, p, fl, bp, d);
            if (store) {
                o.pix_to_face[s] = f;
                o.zbuf[s] = tk.z[k];
                o.bary[3 * s] = bp[0];
                o.bary[3 * s + 1] = bp[1];
                o.bary[3 * s + 2] = bp[2];
                o.dists[s] = d;
            }
            if constexpr (BL) fb.slot(bl, f, tk.z[k], d, bp);
        }
    }
    if constexpr (BL) fb.end(bl, pix);
}

// Fragments of one pixel's K winners written directly by the owning thread,
// 16-byte vector stores when K is a multiple of 4 (ids: K/2, depths and
// distances: K/4, barycentrics: 3K/4 stores per pixel).

template <int KM, bool BL>
__device__ __forceinline__ void write_pixel_vec(const FineOut &o, int64_t pix, int K, const TopK<KM> &tk,
                                                const FaceRec *rec, const PixC &p, const EvalFlags &fl,
                                                const FineBlend &bl) {
    if (K != KM || (KM % 4) != 0) {
        write_pixel<KM, BL>(o, pix, K, tk, rec, p, fl, bl);
        return;
    }
    FwdBlend fb;
    if constexpr (BL) fb.begin(bl, tk.f[0] != 0x7fffffff, tk.z[0]);
    const bool store = !BL || bl.frag;
    const int64_t s0 = pix * KM;
    const unsigned long long pol = l2_keep_policy();
    longlong2 *ip = reinterpret_cast<longlong2 *>(o.pix_to_face + s0);
    float4 *zp = reinterpret_cast<float4 *>(o.zbuf + s0);
    float4 *dp = reinterpret_cast<float4 *>(o.dists + s0);
    float4 *bp = reinterpret_cast<float4 *>(o.bary + s0 * 3);
#pragma unroll
    for (int j = 0; j < KM / 2; ++j) {
        if (!store) break;
        longlong2 v;
        v.x = (tk.f[2 * j] == 0x7fffffff) ? -1ll : (long long)tk.f[2 * j];
        v.y = (tk.f[2 * j + 1] == 0x7fffffff) ? -1ll : (long long)tk.f[2 * j + 1];
        st_keep(ip + j, v, pol);
    }
    // four slots at a time: one float4 of depths, of distances, three of barycentrics
#pragma unroll
    for (int j = 0; j < KM / 4; ++j) {
        float bb[4][3], dd[4], zz[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = 4 * j + i;
            bb[i][0] = bb[i][1] = bb[i][2] = -1.f;
            dd[i] = -1.f;
            zz[i] = -1.f;
            if (tk.f[k] == 0x7fffffff) continue;
            FaceRec R;
            const float4 *src = reinterpret_cast<const float4 *>(rec + tk.f[k]);
            R.a = __ldg(src + kRecA);
            R.b = __ldg(src + kRecB);
            R.c = __ldg(src + kRecC);
            R.d = __ldg(src + kRecD);
            R.e = __ldg(src + kRecE);
            face_fragment(R, p, fl, bb[i], dd[i]);
            zz[i] = tk.z[k];
            if constexpr (BL) fb.slot(bl, tk.f[k], zz[i], dd[i], bb[i]);
        }
        if (!store) continue;
        st_keep(zp + j, make_float4(zz[0], zz[1], zz[2], zz[3]), pol);
        st_keep(dp + j, make_float4(dd[0], dd[1], dd[2], dd[3]), pol);
        st_keep(bp + 3 * j, make_float4(bb[0][0], bb[0][1], bb[0][2], bb[1][0]), pol);
        st_keep(bp + 3 * j + 1, make_float4(bb[1][1], bb[1][2], bb[2][0], bb[2][1]), pol);
        st_keep(bp + 3 * j + 2, make_float4(bb[2][2], bb[3][0], bb[3][1], bb[3][2]), pol);
    }
    if constexpr (BL) fb.end(bl, pix);
}

__device__ __forceinline__ void write_pixel_smem(const FineOut &o, int64_t pix, int K, const SmemTopK &tk,
                                                 const FaceRec *rec, const PixC &p, const EvalFlags &fl) {
    const int64_t s0 = pix * (int64_t)K;
    for (int k = 0; k < K; ++k) {
        const int64_t s = s0 + k;
        const int f = k < tk.n ? tk.f[k * tk.stride] : 0x7fffffff;
        if (f == 0x7fffffff) {
            o.pix_to_face[s] = -1;
            o.zbuf[s] = -1.f;
            o.bary[3 * s] = -1.f;
            o.bary[3 * s + 1] = -1.f;
            o.bary[3 * s + 2] = -1.f;
            o.dists[s] = -1.f;
        } else {
            FaceRec R;
            const float4 *src = reinterpret_cast<const float4 *>(rec + f);
            R.a = __ldg(src + kRecA);
            R.b = __ldg(src + kRecB);
            R.c = __ldg(src + kRecC);
            R.d = __ldg(src + kRecD);
            R.e = __ldg(src + kRecE);
            float bp[3], d;
            face_fragment(R, p, fl, bp, d);
            o.pix_to_face[s] = f;
            o.zbuf[s] = tk.z[k * tk.stride];
            o.bary[3 * s] = bp[0];
            o.bary[3 * s + 1] = bp[1];
            o.bary[3 * s + 2] = bp[2];
            o.dists[s] = d;
        }
    }
}

// ---------------------------------------------------------------------------
// fine pass: persistent blocks, one bin (bin x bin pixels = block) per item
// ---------------------------------------------------------------------------
template <int KM, int BS, bool BL>
__global__ void __launch_bounds__(BS *BS) k_fine(FineArgs a) {
    constexpr int BD = BS * BS;
    __shared__ FaceRec s_rec[BD];
    __shared__ int s_id[BD];
    __shared__ float s_key[BD];
    __shared__ int s_item;
    // dynamic: sort_cap bin entries; K > 16: afterwards the per-thread lists
    extern __shared__ unsigned long long s_sort[];
    const int tid = threadIdx.x;
    // K <= 16: each warp covers an 8 x 4 block of the bin (about as wide as
    // tall, like the inflated face bboxes it is culled against); K > 16: two
    // rows (the tile writer below walks slots in row order)
    const int ty = KM > 0 ? ((tid >> 5) / (BS / 8)) * 4 + ((tid & 31) >> 3) : tid / BS;
    const int tx = KM > 0 ? ((tid >> 5) % (BS / 8)) * 8 + (tid & 7) : tid % BS;
    EvalFlags fl = a.fl;
    const bool zcull = fl.clip || !(fl.blur > 0.f);
    const int nb2 = a.nb * a.nb;
    while (true) {
        if (tid == 0) s_item = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.items) break;
        const int bin = a.order ? __ldg(a.order + item) : item;  // longest bins first
        const int n = bin / nb2, rem = bin - n * nb2;
        const int by = rem / a.nb, bx = rem - by * a.nb;
        const int r = by * BS + ty, c = bx * BS + tx;
        fl.znear = __ldg(a.cams + 16 * n + 13);
        const bool valid = (r < a.S) && (c < a.S);
        const PixC p = pixel_centre(r, c, a.S);
        // rectangle spanned by the centres of this warp's valid pixels (x and y
        // decrease with the column and row index); empty when no lane is valid
        const int lane = tid & 31;
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
        const int cnt = a.eff[bin];
        const int off = a.offsets[bin];
        TopK<(KM > 0 ? KM : 1)> tk;
        SmemTopK stk;
        // The bin's list is sorted front to back in segments of up to sort_cap
        // entries (one segment unless the bin holds more faces than that).
        // K <= 16: each segment is sorted in shared memory right before it is
        // walked.  K > 16: every segment is sorted first and written back to
        // the (block-owned) list, so that the same shared memory then holds
        // the per-pixel lists.
        if constexpr (KM > 0) {
            tk.init();
        } else {
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
            // Chunks of BD faces, front to back: every lane walks the staged
            // faces in order.  Faces are culled 32 at a time for the whole
            // warp: lane j tests face jb + j against the rectangle spanned by
            // the warp's pixel centres and against the warp's largest K-th
            // depth; one ballot names the faces the warp walks pixel by pixel.
            // A face is skipped by a lane when its bbox misses the pixel or its
            // nearest corner lies behind the lane's K-th depth.  Once a warp's
            // largest K-th depth lies in front of the next face, the rest of
            // the segment is behind all its lanes, and the block stops when
            // that holds for every warp.
            for (int base = 0; base < m; base += BD) {
                const int mc = min(BD, m - base);
                if (tid < mc) {
                    const unsigned long long v = ent[base + tid];
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
                    float thr;
                    if constexpr (KM > 0) thr = tk.z[KM - 1];
                    else thr = stk.thr();
                    const float wthr =
                        __int_as_float(__reduce_max_sync(0xffffffffu, valid ? __float_as_int(thr) : 0));
                    if (zcull && s_key[jb] > wthr) {
                        warp_done = true;
                        break;
                    }
                    const int jl = jb + lane;
                    bool hit = false;
                    if (jl < mc) {
                        const float4 bb = s_rec[jl].c;
                        hit = bb.x <= wx1 && bb.y >= wx0 && bb.z <= wy1 && bb.w >= wy0 &&
                              !(zcull && s_key[jl] > wthr);
                    }
                    unsigned mask = __ballot_sync(0xffffffffu, hit);
                    while (mask) {
                        const int jj = jb + __ffs(mask) - 1;
                        mask &= mask - 1;
                        if (!valid) continue;
                        FaceRec R;
                        R.c = s_rec[jj].c;
                        if (!in_bbox(R, p)) continue;
                        if constexpr (KM > 0) thr = tk.z[KM - 1];
                        else thr = stk.thr();
                        if (zcull && s_key[jj] > thr) continue;
                        R.a = s_rec[jj].a;
                        R.b = s_rec[jj].b;
                        R.d = s_rec[jj].d;
                        R.e = s_rec[jj].e;
                        R.h = s_rec[jj].h;
                        float z;
                        if (face_key_nobbox(R, p, fl, z)) {
                            const int fid = s_id[jj];
                            if constexpr (KM > 0) {
                                if (tk.admits(z, fid)) tk.insert(z, fid);
                            } else {
                                if (stk.admits(z, fid)) stk.insert(z, fid);
                            }
                        }
                    }
                }
                if (!warp_done && zcull && base + BD < m) {
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
            if (valid) write_pixel_vec<KM, BL>(a.out, ((int64_t)n * a.S + r) * a.S + c, a.K, tk, a.rec, p, fl, a.blend);
        } else {
            // K > 16: the block writes its tile slot by slot: consecutive
            // threads take consecutive output slots of a tile row (coalesced),
            // each recomputing its slot's barycentrics and distance
            s_id[tid] = valid ? stk.n : 0;
            __syncthreads();
            const int K = a.K;
            const int rows = min(BS, a.S - by * BS), cols = min(BS, a.S - bx * BS);
            const int per_row = cols * K;
            const float *lz = reinterpret_cast<const float *>(s_sort);
            const int *lf = reinterpret_cast<const int *>(s_sort) + BD * K;
            for (int i = tid; i < rows * per_row; i += BD) {
                const int ry = i / per_row, rem = i - ry * per_row;
                const int cx = rem / K, k = rem - cx * K;
                const int t = ry * BS + cx;
                const int rr = by * BS + ry, cc = bx * BS + cx;
                const int64_t sl = (((int64_t)n * a.S + rr) * a.S + cc) * K + k;
                if (k < s_id[t]) {
                    const int f = lf[t * K + k];
                    FaceRec R;
                    const float4 *src = reinterpret_cast<const float4 *>(a.rec + f);
                    R.a = __ldg(src + kRecA);
                    R.b = __ldg(src + kRecB);
                    R.c = __ldg(src + kRecC);
                    R.d = __ldg(src + kRecD);
                    R.e = __ldg(src + kRecE);
                    float bp[3], d;
                    face_fragment(R, pixel_centre(rr, cc, a.S), fl, bp, d);
                    a.out.pix_to_face[sl] = f;
                    a.out.zbuf[sl] = lz[t * K + k];
                    a.out.bary[3 * sl] = bp[0];
                    a.out.bary[3 * sl + 1] = bp[1];
                    a.out.bary[3 * sl + 2] = bp[2];
                    a.out.dists[sl] = d;
                } else {
                    a.out.pix_to_face[sl] = -1;
                    a.out.zbuf[sl] = -1.f;
                    a.out.bary[3 * sl] = -1.f;
                    a.out.bary[3 * sl + 1] = -1.f;
                    a.out.bary[3 * sl + 2] = -1.f;
                    a.out.dists[sl] = -1.f;
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// plain form: one launch per image, every pixel against every face
// ---------------------------------------------------------------------------
template <int KM>
__global__ void __launch_bounds__(256) k_naive(NaiveArgs a, int n) {
    extern __shared__ unsigned char s_dyn[];
    const int64_t pidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = pidx < (int64_t)a.S * a.S;
    const int r = (int)(pidx / a.S), c = (int)(pidx % a.S);
    const PixC p = pixel_centre(r, c, a.S);
    EvalFlags fl = a.fl;
    fl.znear = __ldg(a.cams + 16 * n + 13);
    int64_t lo = a.first_face[n], hi = lo + a.num_faces[n];
    lo = max(lo, (int64_t)0);
    hi = min(hi, a.F);
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
    for (int64_t f = lo; f < hi; ++f) {
        FaceRec R;
        const float4 *src = reinterpret_cast<const float4 *>(a.rec + f);
        R.a = __ldg(src + kRecA);
        R.b = __ldg(src + kRecB);
        R.c = __ldg(src + kRecC);
        R.d = __ldg(src + kRecD);
        R.e = __ldg(src + kRecE);
        R.h = __ldg(src + kRecH);
        float z;
        if (face_key(R, p, fl, z)) {
            if constexpr (KM > 0) {
                if (tk.admits(z, (int)f)) tk.insert(z, (int)f);
            } else {
                if (stk.admits(z, (int)f)) stk.insert(z, (int)f);
            }
        }
    }
    const int64_t pix = (int64_t)n * a.S * a.S + pidx;
    if constexpr (KM > 0) write_pixel<KM, false>(a.out, pix, a.K, tk, a.rec, p, fl, FineBlend{});
    else write_pixel_smem(a.out, pix, a.K, stk, a.rec, p, fl);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int km_for(int K) {
    if (K <= 1) return 1;
    if (K <= 2) return 2;
    if (K <= 4) return 4;
    if (K <= 8) return 8;
    if (K <= 16) return 16;
    return 0;  // shared-memory lists
}

template <int KM, int BS, bool BL>
static cudaError_t launch_fine_t(const FineArgs &a, cudaStream_t st) {
    constexpr int BD = BS * BS;
    // the sort buffer; KM == 0: the same memory then holds the per-thread lists
    const size_t dyn = std::max((size_t)a.sort_cap * 8, (KM > 0) ? (size_t)0 : (size_t)BD * a.K * 8);
    auto kern = k_fine<KM, BS, BL>;
    cudaError_t e = cudaSuccess;
    if (dyn > 0) {  // static + dynamic above 48 KB needs the opt-in
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, BD, dyn);
    if (e != cudaSuccess) return e;
    int grid = std::max(1, std::min<int>(a.items, mr_host::num_sms() * std::max(1, bps)));
    kern<<<grid, BD, dyn, st>>>(a);
    return cudaGetLastError();
}

// The silhouette blend runs inside the fine pass for K <= 16; the softmax
// blend does not (its colour gathers cost the fine pass more than the separate
// blend kernel's pass over the fragments).
bool fine_blends(int K, bool rgb) { return km_for(K) > 0 && !rgb; }

cudaError_t launch_fine(const FineArgs &a, int bin, cudaStream_t st) {
    const int km = km_for(a.K);
    const bool bl = a.blend.on != 0;
#define MR_FINE(KM_)                                                          \
    if (km == KM_) {                                                          \
        if (bin == 8) return bl ? launch_fine_t<KM_, 8, true>(a, st)          \
                                : launch_fine_t<KM_, 8, false>(a, st);        \
        if (bin == 16) return bl ? launch_fine_t<KM_, 16, true>(a, st)        \
                                 : launch_fine_t<KM_, 16, false>(a, st);      \
    }
    MR_FINE(1) MR_FINE(2) MR_FINE(4) MR_FINE(8) MR_FINE(16)
#undef MR_FINE
    if (km == 0) {
        if (bin == 8) return launch_fine_t<0, 8, false>(a, st);
        if (bin == 16) return launch_fine_t<0, 16, false>(a, st);
    }
    return cudaErrorInvalidValue;
}

template <int KM>
static cudaError_t launch_naive_t(const NaiveArgs &a, int N, cudaStream_t st) {
    const int BD = 256;
    size_t dyn = (KM > 0) ? 0 : (size_t)BD * a.K * 8;
    auto kern = k_naive<KM>;
    if (KM == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    const int64_t P = (int64_t)a.S * a.S;
    const int grid = (int)((P + BD - 1) / BD);
    for (int n = 0; n < N; ++n) {
        kern<<<grid, BD, dyn, st>>>(a, n);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_naive(const NaiveArgs &a, int N, cudaStream_t st) {
    switch (km_for(a.K)) {
        case 1: return launch_naive_t<1>(a, N, st);
        case 2: return launch_naive_t<2>(a, N, st);
        case 4: return launch_naive_t<4>(a, N, st);
        case 8: return launch_naive_t<8>(a, N, st);
        case 16: return launch_naive_t<16>(a, N, st);
        default: return launch_naive_t<0>(a, N, st);
    }
}

cudaError_t launch_stage(const StageArgs &a, cudaStream_t st) {
    if (a.F <= 0) return cudaSuccess;
    const int grid = (int)((a.F + 255) / 256);
    k_stage<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan(const ScanArgs &a, cudaStream_t st) {
    k_scan<<<1, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fill(const FillArgs &a, cudaStream_t st) {
    if (a.F <= 0) return cudaSuccess;
    const int grid = (int)((a.F + 255) / 256);
    k_fill<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mr
