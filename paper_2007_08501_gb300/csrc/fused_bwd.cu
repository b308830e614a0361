// Fused backward for sm_103a: the blend adjoint (Algorithms 1 and 2) and the
// rasterizer adjoint (Section 3.2, backward from the cached Fragment data) in
// one pass over the fragments.
//
// blend_bwd followed by rast_mesh_bwd writes dL/d(zbuf, bary, dists) for every
// slot (20 bytes) and reads it back, together with pix_to_face, in a second
// launch.  Here each thread owns one pixel: it forms the slot's blend adjoint
// in registers and pulls it straight through the per-slot rasterizer adjoint
// (slot_corner_grads), so the fragment gradients never reach memory.  For
// every slot k the warp (2 rows x 16 pixels) groups lanes holding the same
// face once; one lane per face adds the face's colour gradients (softmax
// blend) and, through the projection Jacobian and R^T, its vertex gradients.
// The per-slot arithmetic is that of k_blend_bwd and k_rast_bwd.
#include <cuda_runtime.h>

#include "blend_common.cuh"
#include "rast_adjoint.cuh"
#include "rast_common.cuh"
#include "rast_internal.h"

namespace mr {

// bary and vertex ids of slot s (face f, already range-checked against F)
__device__ __forceinline__ void slot_vertices(const BlendArgs &a, int64_t s, int f, int64_t vi[3], float b[3]) {
    b[0] = __ldg(a.bary + 3 * s);
    b[1] = __ldg(a.bary + 3 * s + 1);
    b[2] = __ldg(a.bary + 3 * s + 2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int64_t v = __ldg(a.faces + 3 * (int64_t)f + i);
        vi[i] = (v < 0 || v >= a.V) ? -1 : v;
    }
}

__device__ __forceinline__ void load_adjoint_rec(const FaceRec *rec, int f, FaceRec &R) {
    const float4 *src = reinterpret_cast<const float4 *>(rec + f);
    R.a = __ldg(src + kRecA);
    R.b = __ldg(src + kRecB);
    R.d = __ldg(src + kRecD);
    R.e = __ldg(src + kRecE);
}

// one lane per face: colour atomics (softmax blend) and vertex atomics
template <bool RGB, int NA>
__device__ __forceinline__ void scatter_face(const BlendArgs &a, const RastBwdArgs &r, int key, bool any_live, int nf,
                                             const FaceRec &R, const int64_t vi[3], const float (&acc)[NA]) {
    if (any_live && nf >= 0) {
        const float *cam = r.cams + 16 * nf;
        const float fo = cam[12];
        const float v0x = R.a.x + R.a.z, v0y = R.a.y + R.a.w;
        const float Px[3] = {0.f, R.b.x, R.b.z}, Py[3] = {0.f, R.b.y, R.b.w};
        const float iz[3] = {R.d.y, R.d.z, R.d.w};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            // x = f x_v / z_v, y = f y_v / z_v: d/dx_v = f/z, d/dz_v = -(x dL/dx + y dL/dy)/z
            const float xn = v0x + Px[i], yn = v0y + Py[i];
            const float gxv = acc[3 * i] * fo * iz[i];
            const float gyv = acc[3 * i + 1] * fo * iz[i];
            const float gzv = acc[3 * i + 2] - (acc[3 * i] * xn + acc[3 * i + 1] * yn) * iz[i];
            const int64_t v = __ldg(r.faces + 3 * (int64_t)key + i);
            float *gv = r.grad_verts + 3 * v;
            atomicAdd(gv + 0, cam[0] * gxv + cam[3] * gyv + cam[6] * gzv);
            atomicAdd(gv + 1, cam[1] * gxv + cam[4] * gyv + cam[7] * gzv);
            atomicAdd(gv + 2, cam[2] * gxv + cam[5] * gyv + cam[8] * gzv);
        }
    }
    if constexpr (RGB) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (vi[i] < 0) continue;
            float *gcol = a.grad_colors + 3 * vi[i];
            atomicAdd(gcol, acc[9 + 3 * i]);
            atomicAdd(gcol + 1, acc[9 + 3 * i + 1]);
            atomicAdd(gcol + 2, acc[9 + 3 * i + 2]);
        }
    }
}

// Silhouette blend: only dL/d(dists) reaches the rasterizer, so a slot moves
// the x, y of its nearest edge's two corners (acc[2 i + {0, 1}] for corner
// i); one lane per face pulls them through the projection Jacobian and R^T.
__device__ __forceinline__ void scatter_face_dist(const RastBwdArgs &r, int key, int nf, const FaceRec &R,
                                                  const float (&acc)[6]) {
    const float *cam = r.cams + 16 * nf;
    const float fo = cam[12];
    const float v0x = R.a.x + R.a.z, v0y = R.a.y + R.a.w;
    const float Px[3] = {0.f, R.b.x, R.b.z}, Py[3] = {0.f, R.b.y, R.b.w};
    const float iz[3] = {R.d.y, R.d.z, R.d.w};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float ax = acc[2 * i], ay = acc[2 * i + 1];
        if (ax == 0.f && ay == 0.f) continue;  // a corner no lane's nearest edge touches
        const float xn = v0x + Px[i], yn = v0y + Py[i];
        const float gxv = ax * fo * iz[i];
        const float gyv = ay * fo * iz[i];
        const float gzv = -(ax * xn + ay * yn) * iz[i];
        const int64_t v = __ldg(r.faces + 3 * (int64_t)key + i);
        float *gv = r.grad_verts + 3 * v;
        atomicAdd(gv + 0, cam[0] * gxv + cam[3] * gyv + cam[6] * gzv);
        atomicAdd(gv + 1, cam[1] * gxv + cam[4] * gyv + cam[7] * gzv);
        atomicAdd(gv + 2, cam[2] * gxv + cam[5] * gyv + cam[8] * gzv);
    }
}

// Per-slot tail shared by both kernels: rasterizer adjoint of the slot's
// fragment gradient, warp grouping by face, one lane per face scatters.
// acc[9..17] holds the slot's colour gradients (RGB) on entry.
template <bool RGB, int NA>
__device__ __forceinline__ void slot_tail(const BlendArgs &a, const RastBwdArgs &r, const PixC &p, int f, float gz,
                                          float gd, float gb0, float gb1, float gb2, const int64_t vi[3],
                                          float (&acc)[NA], RareQueue rq = RareQueue{nullptr, nullptr},
                                          int tile = 0) {
    const int fr = (f >= 0 && (int64_t)f < r.F) ? f : -1;  // an id outside the batch contributes nothing
    const int nf = fr >= 0 ? __ldg(r.face_mesh + fr) : -1;
    const bool live = nf >= 0 && (gz != 0.f || gd != 0.f || gb0 != 0.f || gb1 != 0.f || gb2 != 0.f);
    FaceRec R;
    if constexpr (!RGB) {
        static_assert(NA == 6, "silhouette: x, y of three corners");
#pragma unroll
        for (int j = 0; j < 6; ++j) acc[j] = 0.f;
        if (live) {
            load_adjoint_rec(r.rec, fr, R);
            slot_corner_grads_dist(R, p, gd, acc);
        }
        const int key = live ? fr : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        group_sum<6>(peers, acc);
        if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) scatter_face_dist(r, key, nf, R, acc);
    } else {
        float g9[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) g9[j] = 0.f;
        if (live) {
            load_adjoint_rec(r.rec, fr, R);
            slot_corner_grads(R, p, r.fl, gz, gd, gb0, gb1, gb2, g9, rq, fr, nf, tile);
        }
#pragma unroll
        for (int j = 0; j < 9; ++j) acc[j] = g9[j];
        const int key = fr;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const unsigned lv = __ballot_sync(0xffffffffu, live);
        group_sum<NA>(peers, acc);
        if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
            const bool any_live = (lv & peers) != 0u;
            if (any_live && !live) load_adjoint_rec(r.rec, fr, R);
            scatter_face<RGB, NA>(a, r, key, any_live, nf, R, vi, acc);
        }
    }
}

// ---------------------------------------------------------------------------
// register version (KM = K in {1, 2, 4, 8, 16})
// ---------------------------------------------------------------------------
// words of shared memory per slot and thread: face id, dL/d dists, and for the
// softmax blend dL/d zbuf and dL/d c_k (3)
constexpr int fused_words(bool rgb) { return rgb ? 6 : 2; }
constexpr size_t fused_smem(int km, bool rgb) { return (size_t)fused_words(rgb) * km * 256 * sizeof(float); }
constexpr int fused_min_blocks(int km, bool rgb) { return rgb ? (km >= 16 ? 2 : 3) : 4; }

template <int KM, bool RGB>
__global__ void __launch_bounds__(256, fused_min_blocks(KM, RGB)) k_blend_rast_bwd(BlendArgs a, RastBwdArgs r) {
    constexpr int NA = RGB ? 18 : 6;
    // each warp covers an 8 x 4 block of the 16 x 16 tile: neighbouring pixels
    // share faces, so the warp's grouping by face finds more peers
    const int tx = ((threadIdx.x >> 5) & 1) * 8 + (threadIdx.x & 7), ty = (threadIdx.x >> 6) * 4 + ((threadIdx.x >> 3) & 3);
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    const bool valid = row < a.S && col < a.S;
    const int64_t pix = ((int64_t)blockIdx.z * a.S + row) * a.S + col;
    const PixC p = pixel_centre(row, col, a.S);
    const float isg = __frcp_rn(a.sigma);  // d / sigma as d * (1 / sigma) in the per-slot terms
    // softmax blend: slots whose barycentric adjoint needs double-float are
    // queued and done at the end of the block
    __shared__ RareSlot s_rare[RGB ? kRareCap : 1];
    __shared__ int s_nrare;
    if (RGB && threadIdx.x == 0) s_nrare = 0;
    if (RGB) __syncthreads();
    const RareQueue rq{RGB ? s_rare : nullptr, &s_nrare};
    SlotData<KM> S;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        load_slots<KM>(a, pix, RGB, S);
        g = reinterpret_cast<const float4 *>(a.grad_image)[pix];
    } else {
#pragma unroll
        for (int k = 0; k < KM; ++k) { S.f[k] = -1; S.d[k] = 0.f; S.z[k] = 0.f; }
    }
    float keep = 1.f;
    float zmin = __int_as_float(0x7f800000);
    bool any = false;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (S.f[k] < 0) continue;
        keep *= sigmoidf_(S.d[k] * isg);
        if (RGB) zmin = fminf(zmin, S.z[k]);
        any = true;
    }
    const int64_t s0 = pix * KM;
    // silhouette: d alpha / d d_k = -prob_k * prod_j (1 - prob_j) / sigma
    const float sil = -g.w * keep / a.sigma;
    float range = 0.f, m = 0.f, delta = 0.f, iD = 0.f;
    bool face_max = false;
    float W[RGB ? KM : 1], C[RGB ? KM : 1][3];
    if constexpr (RGB) {
        range = a.zfar - a.znear;
        const float ztop = any ? (a.zfar - zmin) / range : -__int_as_float(0x7f800000);
        face_max = any && ztop > a.eps;
        m = face_max ? ztop : a.eps;
        float den = 0.f;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            W[k] = 0.f;
            C[k][0] = C[k][1] = C[k][2] = 0.f;
            if (S.f[k] < 0) continue;
            const float arg = face_max ? (zmin - S.z[k]) / (range * a.gamma) : ((a.zfar - S.z[k]) / range - m) / a.gamma;
            W[k] = sigmoidf_(-S.d[k] * isg) * expf(arg);
            float b[3];
            int64_t vi[3];
            slot_colour(a, s0 + k, S.f[k], C[k], vi, b);
            den += W[k];
        }
        delta = expf((a.eps - m) / a.gamma);
        iD = 1.f / (den + delta);
    }
    // Phase A (unrolled, registers): the blend adjoint of every slot, parked in
    // this thread's own column of shared memory (no other thread reads it).
    extern __shared__ float fsm[];
    const int tid = threadIdx.x;
    auto at = [&](int w, int k) -> float & { return fsm[(w * KM + k) * 256 + tid]; };
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int f = S.f[k];
        float gd = 0.f, gz = 0.f, gc0 = 0.f, gc1 = 0.f, gc2 = 0.f;
        if (f >= 0) {
            const float prob = sigmoidf_(-S.d[k] * isg);
            gd = sil * prob;
            if constexpr (RGB) {
                // c_k - rgb = (sum_{j != k} w_j (c_k - c_j) + delta (c_k - bg)) / D
                float d0 = delta * (C[k][0] - a.bg0), d1 = delta * (C[k][1] - a.bg1), d2 = delta * (C[k][2] - a.bg2);
#pragma unroll
                for (int j = 0; j < KM; ++j) {
                    if (j == k) continue;
                    d0 += W[j] * (C[k][0] - C[j][0]);
                    d1 += W[j] * (C[k][1] - C[j][1]);
                    d2 += W[j] * (C[k][2] - C[j][2]);
                }
                const float gw = (g.x * d0 + g.y * d1 + g.z * d2) * iD * iD;
                const float q = sigmoidf_(S.d[k] * isg);
                const float arg = face_max ? (zmin - S.z[k]) / (range * a.gamma) : ((a.zfar - S.z[k]) / range - m) / a.gamma;
                gd = sil * prob + gw * expf(arg) * (-prob * q * isg);
                gz = gw * W[k] / a.gamma * (-1.f / range);
                gc0 = g.x * W[k] * iD;
                gc1 = g.y * W[k] * iD;
                gc2 = g.z * W[k] * iD;
            }
        }
        at(0, k) = __int_as_float(f);
        at(1, k) = gd;
        if constexpr (RGB) {
            at(2, k) = gz;
            at(3, k) = gc0;
            at(4, k) = gc1;
            at(5, k) = gc2;
        }
    }
    // Phase B (one slot per iteration, not unrolled: the rasterizer adjoint and
    // the warp grouping are large): dL/d(bary) = dL/dc_k . (vertex colours),
    // colour gradients dL/dc_k (x) bary, then the slot's rasterizer adjoint.
#pragma unroll 1
    for (int k = 0; k < KM; ++k) {
        const int f = __float_as_int(at(0, k));
        const float gd = at(1, k);
        float gz = 0.f, gb[3] = {0.f, 0.f, 0.f};
        float acc[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) acc[j] = 0.f;
        int64_t vi[3] = {-1, -1, -1};
        if constexpr (RGB) {
            gz = at(2, k);
            const float gc0 = at(3, k), gc1 = at(4, k), gc2 = at(5, k);
            if (f >= 0 && (int64_t)f < a.F) {
                float b[3];
                slot_vertices(a, s0 + k, f, vi, b);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float3 cv = vertex_colour(a, vi[i]);
                    gb[i] = gc0 * cv.x + gc1 * cv.y + gc2 * cv.z;
                    acc[9 + 3 * i] = gc0 * b[i];
                    acc[9 + 3 * i + 1] = gc1 * b[i];
                    acc[9 + 3 * i + 2] = gc2 * b[i];
                }
            }
        }
        slot_tail<RGB, NA>(a, r, p, f, gz, gd, gb[0], gb[1], gb[2], vi, acc, rq, (ty << 4) | tx);
    }
    if constexpr (RGB) flush_rare_slots(rq, r.rec, r.cams, r.faces, r.grad_verts, a.S, r.fl);
}

// ---------------------------------------------------------------------------
// generic version (any K): re-reads slots from global memory
// ---------------------------------------------------------------------------
template <bool RGB>
__global__ void __launch_bounds__(256) k_blend_rast_bwd_any(BlendArgs a, RastBwdArgs r) {
    constexpr int NA = RGB ? 18 : 6;
    // each warp covers an 8 x 4 block of the 16 x 16 tile: neighbouring pixels
    // share faces, so the warp's grouping by face finds more peers
    const int tx = ((threadIdx.x >> 5) & 1) * 8 + (threadIdx.x & 7), ty = (threadIdx.x >> 6) * 4 + ((threadIdx.x >> 3) & 3);
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    const bool valid = row < a.S && col < a.S;
    const int64_t pix = ((int64_t)blockIdx.z * a.S + row) * a.S + col;
    const PixC p = pixel_centre(row, col, a.S);
    const float isg = __frcp_rn(a.sigma);  // d / sigma as d * (1 / sigma) in the per-slot terms
    const int K = a.K;
    const int64_t s0 = pix * K;
    __shared__ RareSlot s_rare[RGB ? kRareCap : 1];
    __shared__ int s_nrare;
    if (RGB && threadIdx.x == 0) s_nrare = 0;
    if (RGB) __syncthreads();
    const RareQueue rq{RGB ? s_rare : nullptr, &s_nrare};
    const float4 g = valid ? reinterpret_cast<const float4 *>(a.grad_image)[pix] : make_float4(0.f, 0.f, 0.f, 0.f);
    float keep = 1.f, zmin = __int_as_float(0x7f800000);
    bool any = false;
    auto take = [&](long long f, float d, int k) {
        if (f < 0) return;
        keep *= sigmoidf_(d * isg);
        if (RGB) zmin = fminf(zmin, __ldg(a.zbuf + s0 + k));
        any = true;
    };
    if (valid && (K & 1) == 0) {
        // even K: slot pairs are 16-byte (ids) and 8-byte (distances) aligned
        const longlong2 *fp = reinterpret_cast<const longlong2 *>(a.pix_to_face + s0);
        const float2 *dp = reinterpret_cast<const float2 *>(a.dists + s0);
        for (int j = 0; j < K / 2; ++j) {
            const longlong2 f2 = __ldg(fp + j);
            const float2 d2 = __ldg(dp + j);
            take(f2.x, d2.x, 2 * j);
            take(f2.y, d2.y, 2 * j + 1);
        }
    } else if (valid) {
        for (int k = 0; k < K; ++k) take(__ldg(a.pix_to_face + s0 + k), __ldg(a.dists + s0 + k), k);
    }
    const float sil = -g.w * keep / a.sigma;
    float range = 0.f, m = 0.f, iD = 0.f, delta = 0.f;
    bool face_max = false;
    float Wl[RGB ? kMaxK : 1], Cl[RGB ? kMaxK : 1][3];  // per-slot weights and colours (local memory)
    if constexpr (RGB) {
        range = a.zfar - a.znear;
        const float ztop = any ? (a.zfar - zmin) / range : -__int_as_float(0x7f800000);
        face_max = any && ztop > a.eps;
        m = face_max ? ztop : a.eps;
        float den = 0.f;
        for (int k = 0; k < K; ++k) {
            Wl[k] = 0.f;
            Cl[k][0] = Cl[k][1] = Cl[k][2] = 0.f;
            if (!valid) continue;
            const int64_t s = s0 + k;
            const int f = clamp_id(a.pix_to_face[s]);
            if (f < 0) continue;
            const float z = a.zbuf[s];
            const float arg = face_max ? (zmin - z) / (range * a.gamma) : ((a.zfar - z) / range - m) / a.gamma;
            Wl[k] = sigmoidf_(-a.dists[s] * isg) * expf(arg);
            float b[3];
            int64_t vi[3];
            slot_colour(a, s, f, Cl[k], vi, b);
            den += Wl[k];
        }
        delta = expf((a.eps - m) / a.gamma);
        iD = 1.f / (den + delta);
    }
    // the next slot's id and distance are loaded one iteration ahead
    int f_next = valid ? clamp_id(__ldg(a.pix_to_face + s0)) : -1;
    float d_next = valid ? __ldg(a.dists + s0) : 0.f;
    for (int k = 0; k < K; ++k) {  // uniform trip count: every lane reaches the warp grouping
        const int64_t s = s0 + k;
        const int f = f_next;
        const float d = d_next;
        if (valid && k + 1 < K) {
            f_next = clamp_id(__ldg(a.pix_to_face + s + 1));
            d_next = __ldg(a.dists + s + 1);
        }
        float gd = 0.f, gz = 0.f, gb[3] = {0.f, 0.f, 0.f};
        float acc[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) acc[j] = 0.f;
        int64_t vi[3] = {-1, -1, -1};
        if (f >= 0) {
            const float prob = sigmoidf_(-d * isg);
            gd = sil * prob;
            if constexpr (RGB) {
                float b[3] = {0.f, 0.f, 0.f};
                if ((int64_t)f < a.F) slot_vertices(a, s, f, vi, b);
                const float z = a.zbuf[s];
                const float arg = face_max ? (zmin - z) / (range * a.gamma) : ((a.zfar - z) / range - m) / a.gamma;
                const float E = expf(arg);
                const float Wk = prob * E;
                float d0 = delta * (Cl[k][0] - a.bg0), d1 = delta * (Cl[k][1] - a.bg1), d2 = delta * (Cl[k][2] - a.bg2);
                for (int j = 0; j < K; ++j) {
                    if (j == k) continue;
                    d0 += Wl[j] * (Cl[k][0] - Cl[j][0]);
                    d1 += Wl[j] * (Cl[k][1] - Cl[j][1]);
                    d2 += Wl[j] * (Cl[k][2] - Cl[j][2]);
                }
                const float gw = (g.x * d0 + g.y * d1 + g.z * d2) * iD * iD;
                gd += gw * E * (-prob * sigmoidf_(d * isg) * isg);
                gz = gw * Wk / a.gamma * (-1.f / range);
                const float gc0 = g.x * Wk * iD, gc1 = g.y * Wk * iD, gc2 = g.z * Wk * iD;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float3 cv = vertex_colour(a, vi[i]);
                    gb[i] = gc0 * cv.x + gc1 * cv.y + gc2 * cv.z;
                    acc[9 + 3 * i] = gc0 * b[i];
                    acc[9 + 3 * i + 1] = gc1 * b[i];
                    acc[9 + 3 * i + 2] = gc2 * b[i];
                }
            }
        }
        slot_tail<RGB, NA>(a, r, p, f, gz, gd, gb[0], gb[1], gb[2], vi, acc, rq, (ty << 4) | tx);
    }
    if constexpr (RGB) flush_rare_slots(rq, r.rec, r.cams, r.faces, r.grad_verts, a.S, r.fl);
}

// ---------------------------------------------------------------------------
template <int KM, bool RGB>
static void launch_fused_t(const BlendArgs &a, const RastBwdArgs &r, dim3 grid, cudaStream_t st) {
    constexpr size_t smem = fused_smem(KM, RGB);
    // dynamic plus static shared memory may exceed the 48 KB a launch gets
    // without the opt-in
    if constexpr (smem > 32 * 1024) {
        static bool set = false;  // one attribute call per process and instantiation
        if (!set) {
            cudaFuncSetAttribute(k_blend_rast_bwd<KM, RGB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            set = true;
        }
    }
    k_blend_rast_bwd<KM, RGB><<<grid, 256, smem, st>>>(a, r);
}

template <bool RGB>
static void launch_fused_rgb(const BlendArgs &a, const RastBwdArgs &r, dim3 grid, cudaStream_t st) {
    switch (a.K) {
        case 1: launch_fused_t<1, RGB>(a, r, grid, st); break;
        case 2: launch_fused_t<2, RGB>(a, r, grid, st); break;
        case 4: launch_fused_t<4, RGB>(a, r, grid, st); break;
        case 8: launch_fused_t<8, RGB>(a, r, grid, st); break;
        case 16: launch_fused_t<16, RGB>(a, r, grid, st); break;
        default: k_blend_rast_bwd_any<RGB><<<grid, 256, 0, st>>>(a, r); break;
    }
}

cudaError_t launch_blend_rast_bwd(const BlendArgs &a, const RastBwdArgs &r, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const unsigned tiles = (unsigned)((a.S + 15) / 16);
    const dim3 grid(tiles, tiles, (unsigned)a.N);
    if (a.mode == MESHRAST_BLEND_RGB)
        launch_fused_rgb<true>(a, r, grid, st);
    else
        launch_fused_rgb<false>(a, r, grid, st);
    return cudaGetLastError();
}

}  // namespace mr
