// Soft blends for sm_103a: Algorithm 1 (silhouette) and Algorithm 2 (softmax
// rgb) of the paper, forward and hand-written adjoint, one thread per pixel.
//
//   prob_k = sigmoid(-d_k / sigma),  1 - prob_k = sigmoid(d_k / sigma)
//   alpha  = 1 - prod_k (1 - prob_k)
//   zinv_k = (zfar - z_k)/(zfar - znear),  m = max(eps, max_k zinv_k)
//   w_k    = prob_k exp((zinv_k - m)/gamma),  delta = exp((eps - m)/gamma)
//   rgb    = (sum_k w_k c_k + delta bg)/(sum_k w_k + delta)
// over the slots with pix_to_face >= 0; c_k is the per-vertex colour of the
// slot's face interpolated with its barycentrics.  When m is a face's zinv
// the exponent zinv_k - m is formed as (z_min - z_k)/(zfar - znear), which
// is the same number without the cancellation of two values near 1.  The
// adjoint treats m as a constant: rgb does not depend on it.
#include <cuda_runtime.h>

#include "rast_common.cuh"
#include "rast_internal.h"
#include "blend_common.cuh"

namespace mr {

// ---------------------------------------------------------------------------
// register version (KM = K <= 16)
// ---------------------------------------------------------------------------
template <int KM>
__global__ void __launch_bounds__(256) k_blend_fwd(BlendArgs a) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= a.P) return;
    const bool rgb = a.mode == MESHRAST_BLEND_RGB;
    SlotData<KM> S;
    load_slots<KM>(a, pix, rgb, S);
    float keep = 1.f;
    float zmin = __int_as_float(0x7f800000);
    bool any = false;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (S.f[k] < 0) continue;
        keep *= sigmoidf_(S.d[k] / a.sigma);
        if (rgb) zmin = fminf(zmin, S.z[k]);
        any = true;
    }
    float4 out = make_float4(0.f, 0.f, 0.f, 1.f - keep);
    if (rgb) {
        const float range = a.zfar - a.znear;
        const float ztop = any ? (a.zfar - zmin) / range : -__int_as_float(0x7f800000);
        const bool face_max = any && ztop > a.eps;
        const float m = face_max ? ztop : a.eps;
        float num0 = 0.f, num1 = 0.f, num2 = 0.f, den = 0.f;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            if (S.f[k] < 0) continue;
            const float arg = face_max ? (zmin - S.z[k]) / (range * a.gamma)
                                       : ((a.zfar - S.z[k]) / range - m) / a.gamma;
            const float w = sigmoidf_(-S.d[k] / a.sigma) * expf(arg);
            float c[3], b[3];
            int64_t vi[3];
            slot_colour(a, pix * KM + k, S.f[k], c, vi, b);
            num0 += w * c[0];
            num1 += w * c[1];
            num2 += w * c[2];
            den += w;
        }
        const float delta = expf((a.eps - m) / a.gamma);
        const float D = den + delta;
        out.x = (num0 + delta * a.bg0) / D;
        out.y = (num1 + delta * a.bg1) / D;
        out.z = (num2 + delta * a.bg2) / D;
    }
    reinterpret_cast<float4 *>(a.image)[pix] = out;
}

// colour-gradient contributions of one slot (3 vertices x 3 channels), summed
// over the warp's lanes that hold the same face; one lane per face adds them
__device__ __forceinline__ void scatter_colour_grads(const BlendArgs &a, int key, const int64_t vi[3],
                                                     float (&gcv)[9]) {
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    group_sum<9>(peers, gcv);
    if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (vi[i] < 0) continue;
            float *gcol = a.grad_colors + 3 * vi[i];
            atomicAdd(gcol, gcv[3 * i]);
            atomicAdd(gcol + 1, gcv[3 * i + 1]);
            atomicAdd(gcol + 2, gcv[3 * i + 2]);
        }
    }
}

template <int KM>
__global__ void __launch_bounds__(256, (KM >= 16 ? 2 : 3)) k_blend_bwd(BlendArgs a) {
    int64_t pix;
    const bool valid = tile_pixel(a, pix);
    const bool rgb = a.mode == MESHRAST_BLEND_RGB;
    SlotData<KM> S;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        load_slots<KM>(a, pix, rgb, S);
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
        keep *= sigmoidf_(S.d[k] / a.sigma);
        if (rgb) zmin = fminf(zmin, S.z[k]);
        any = true;
    }
    const int64_t s0 = pix * KM;
    // silhouette: d alpha / d d_k = -prob_k * prod_j (1 - prob_j) / sigma
    const float sil = -g.w * keep / a.sigma;
    if (!rgb) {
        if (!valid) return;
        if constexpr (KM % 4 == 0) {
            float4 *dp = reinterpret_cast<float4 *>(a.grad_dists + s0);
#pragma unroll
            for (int j = 0; j < KM / 4; ++j) {
                float v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k = 4 * j + i;
                    v[i] = (S.f[k] < 0) ? 0.f : sil * sigmoidf_(-S.d[k] / a.sigma);
                }
                dp[j] = make_float4(v[0], v[1], v[2], v[3]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < KM; ++k) a.grad_dists[s0 + k] = (S.f[k] < 0) ? 0.f : sil * sigmoidf_(-S.d[k] / a.sigma);
        }
        return;
    }
    const float range = a.zfar - a.znear;
    const float ztop = any ? (a.zfar - zmin) / range : -__int_as_float(0x7f800000);
    const bool face_max = any && ztop > a.eps;
    const float m = face_max ? ztop : a.eps;
    float W[KM], C[KM][3];
    float den = 0.f;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        W[k] = 0.f;
        C[k][0] = C[k][1] = C[k][2] = 0.f;
        if (S.f[k] < 0) continue;
        const float arg = face_max ? (zmin - S.z[k]) / (range * a.gamma) : ((a.zfar - S.z[k]) / range - m) / a.gamma;
        W[k] = sigmoidf_(-S.d[k] / a.sigma) * expf(arg);
        float b[3];
        int64_t vi[3];
        slot_colour(a, s0 + k, S.f[k], C[k], vi, b);
        den += W[k];
    }
    const float delta = expf((a.eps - m) / a.gamma);
    const float iD = 1.f / (den + delta);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int64_t s = s0 + k;
        float gcv[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) gcv[j] = 0.f;
        int64_t vi[3] = {-1, -1, -1};
        int key = -1;
        if (S.f[k] < 0) {
            if (valid) {
                a.grad_dists[s] = 0.f;
                a.grad_zbuf[s] = 0.f;
                a.grad_bary[3 * s] = 0.f;
                a.grad_bary[3 * s + 1] = 0.f;
                a.grad_bary[3 * s + 2] = 0.f;
            }
        } else {
            key = S.f[k];
            float c[3], b[3];
            slot_colour(a, s, S.f[k], c, vi, b);
            // c_k - rgb = (sum_{j != k} w_j (c_k - c_j) + delta (c_k - bg)) / D: exact for the
            // dominant face, where c_k - rgb would otherwise be lost to cancellation
            float d0 = delta * (C[k][0] - a.bg0), d1 = delta * (C[k][1] - a.bg1), d2 = delta * (C[k][2] - a.bg2);
#pragma unroll
            for (int j = 0; j < KM; ++j) {
                if (j == k) continue;
                d0 += W[j] * (C[k][0] - C[j][0]);
                d1 += W[j] * (C[k][1] - C[j][1]);
                d2 += W[j] * (C[k][2] - C[j][2]);
            }
            const float gw = (g.x * d0 + g.y * d1 + g.z * d2) * iD * iD;
            const float prob = sigmoidf_(-S.d[k] / a.sigma);
            const float q = sigmoidf_(S.d[k] / a.sigma);
            const float arg = face_max ? (zmin - S.z[k]) / (range * a.gamma) : ((a.zfar - S.z[k]) / range - m) / a.gamma;
            a.grad_dists[s] = sil * prob + gw * expf(arg) * (-prob * q / a.sigma);
            a.grad_zbuf[s] = gw * W[k] / a.gamma * (-1.f / range);
            const float gc0 = g.x * W[k] * iD, gc1 = g.y * W[k] * iD, gc2 = g.z * W[k] * iD;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float3 col = vertex_colour(a, vi[i]);
                a.grad_bary[3 * s + i] = gc0 * col.x + gc1 * col.y + gc2 * col.z;
                gcv[3 * i] = gc0 * b[i];
                gcv[3 * i + 1] = gc1 * b[i];
                gcv[3 * i + 2] = gc2 * b[i];
            }
        }
        scatter_colour_grads(a, key, vi, gcv);
    }
}

// ---------------------------------------------------------------------------
// generic version (any K): re-reads slots from global memory
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_blend_fwd_any(BlendArgs a) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= a.P) return;
    const bool rgb = a.mode == MESHRAST_BLEND_RGB;
    const int K = a.K;
    const int64_t s0 = pix * K;
    float keep = 1.f, zmin = __int_as_float(0x7f800000);
    bool any = false;
    auto take = [&](long long f, float d, int k) {
        if (f < 0) return;
        keep *= sigmoidf_(d / a.sigma);
        if (rgb) zmin = fminf(zmin, __ldg(a.zbuf + s0 + k));
        any = true;
    };
    if ((K & 1) == 0) {
        // even K: slot pairs are 16-byte (ids) and 8-byte (distances) aligned
        const longlong2 *fp = reinterpret_cast<const longlong2 *>(a.pix_to_face + s0);
        const float2 *dp = reinterpret_cast<const float2 *>(a.dists + s0);
        for (int j = 0; j < K / 2; ++j) {
            const longlong2 f2 = __ldg(fp + j);
            const float2 d2 = __ldg(dp + j);
            take(f2.x, d2.x, 2 * j);
            take(f2.y, d2.y, 2 * j + 1);
        }
    } else {
        for (int k = 0; k < K; ++k) take(__ldg(a.pix_to_face + s0 + k), __ldg(a.dists + s0 + k), k);
    }
    float4 out = make_float4(0.f, 0.f, 0.f, 1.f - keep);
    if (rgb) {
        const float range = a.zfar - a.znear;
        const float ztop = any ? (a.zfar - zmin) / range : -__int_as_float(0x7f800000);
        const bool face_max = any && ztop > a.eps;
        const float m = face_max ? ztop : a.eps;
        float num0 = 0.f, num1 = 0.f, num2 = 0.f, den = 0.f;
        for (int k = 0; k < K; ++k) {
            const int64_t s = s0 + k;
            const int64_t f = a.pix_to_face[s];
            if (f < 0) continue;
            const float z = a.zbuf[s];
            const float arg = face_max ? (zmin - z) / (range * a.gamma) : ((a.zfar - z) / range - m) / a.gamma;
            const float w = sigmoidf_(-a.dists[s] / a.sigma) * expf(arg);
            float c[3], b[3];
            int64_t vi[3];
            slot_colour(a, s, f, c, vi, b);
            num0 += w * c[0];
            num1 += w * c[1];
            num2 += w * c[2];
            den += w;
        }
        const float delta = expf((a.eps - m) / a.gamma);
        const float D = den + delta;
        out.x = (num0 + delta * a.bg0) / D;
        out.y = (num1 + delta * a.bg1) / D;
        out.z = (num2 + delta * a.bg2) / D;
    }
    reinterpret_cast<float4 *>(a.image)[pix] = out;
}

__global__ void __launch_bounds__(256) k_blend_bwd_any(BlendArgs a) {
    int64_t pix;
    const bool valid = tile_pixel(a, pix);
    const bool rgb = a.mode == MESHRAST_BLEND_RGB;
    const int K = a.K;
    const int64_t s0 = pix * K;
    const float4 g = valid ? reinterpret_cast<const float4 *>(a.grad_image)[pix] : make_float4(0.f, 0.f, 0.f, 0.f);
    float keep = 1.f, zmin = __int_as_float(0x7f800000);
    bool any = false;
    for (int k = 0; valid && k < K; ++k) {
        if (a.pix_to_face[s0 + k] < 0) continue;
        keep *= sigmoidf_(a.dists[s0 + k] / a.sigma);
        if (rgb) zmin = fminf(zmin, a.zbuf[s0 + k]);
        any = true;
    }
    float range = 0.f, m = 0.f, iD = 0.f, delta = 0.f;
    bool face_max = false;
    float Wl[kMaxK], Cl[kMaxK][3];  // per-slot weights and colours (local memory)
    if (rgb) {
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
            const int64_t f = a.pix_to_face[s];
            if (f < 0) continue;
            const float z = a.zbuf[s];
            const float arg = face_max ? (zmin - z) / (range * a.gamma) : ((a.zfar - z) / range - m) / a.gamma;
            Wl[k] = sigmoidf_(-a.dists[s] / a.sigma) * expf(arg);
            float b[3];
            int64_t vi[3];
            slot_colour(a, s, f, Cl[k], vi, b);
            den += Wl[k];
        }
        delta = expf((a.eps - m) / a.gamma);
        iD = 1.f / (den + delta);
    }
    for (int k = 0; k < K; ++k) {  // uniform trip count: every lane reaches the warp aggregation
        const int64_t s = s0 + k;
        const int64_t f = valid ? a.pix_to_face[s] : -1;
        float gcv[9];
        for (int j = 0; j < 9; ++j) gcv[j] = 0.f;
        int64_t vi[3] = {-1, -1, -1};
        int key = -1;
        if (valid) {
            if (f < 0) {
                a.grad_dists[s] = 0.f;
                if (rgb) {
                    a.grad_zbuf[s] = 0.f;
                    a.grad_bary[3 * s] = a.grad_bary[3 * s + 1] = a.grad_bary[3 * s + 2] = 0.f;
                }
            } else {
                const float d = a.dists[s];
                const float prob = sigmoidf_(-d / a.sigma);
                float gd = g.w * (-prob * keep / a.sigma);
                if (rgb) {
                    key = clamp_id(f);
                    const float z = a.zbuf[s];
                    const float arg = face_max ? (zmin - z) / (range * a.gamma)
                                               : ((a.zfar - z) / range - m) / a.gamma;
                    const float E = expf(arg);
                    const float W = prob * E;
                    float c[3], b[3];
                    slot_colour(a, s, f, c, vi, b);
                    float d0 = delta * (Cl[k][0] - a.bg0), d1 = delta * (Cl[k][1] - a.bg1),
                          d2 = delta * (Cl[k][2] - a.bg2);
                    for (int j = 0; j < K; ++j) {
                        if (j == k) continue;
                        d0 += Wl[j] * (Cl[k][0] - Cl[j][0]);
                        d1 += Wl[j] * (Cl[k][1] - Cl[j][1]);
                        d2 += Wl[j] * (Cl[k][2] - Cl[j][2]);
                    }
                    const float gw = (g.x * d0 + g.y * d1 + g.z * d2) * iD * iD;
                    gd += gw * E * (-prob * sigmoidf_(d / a.sigma) / a.sigma);
                    a.grad_zbuf[s] = gw * W / a.gamma * (-1.f / range);
                    const float gc0 = g.x * W * iD, gc1 = g.y * W * iD, gc2 = g.z * W * iD;
                    for (int i = 0; i < 3; ++i) {
                        const float3 col = vertex_colour(a, vi[i]);
                        a.grad_bary[3 * s + i] = gc0 * col.x + gc1 * col.y + gc2 * col.z;
                        gcv[3 * i] = gc0 * b[i];
                        gcv[3 * i + 1] = gc1 * b[i];
                        gcv[3 * i + 2] = gc2 * b[i];
                    }
                }
                a.grad_dists[s] = gd;
            }
        }
        if (rgb) scatter_colour_grads(a, key, vi, gcv);
    }
}

// ---------------------------------------------------------------------------
template <int KM>
static void launch_fwd_t(const BlendArgs &a, int grid, cudaStream_t st) {
    k_blend_fwd<KM><<<grid, 256, 0, st>>>(a);
}
template <int KM>
static void launch_bwd_t(const BlendArgs &a, dim3 grid, cudaStream_t st) {
    k_blend_bwd<KM><<<grid, 256, 0, st>>>(a);
}

cudaError_t launch_blend_fwd(const BlendArgs &a, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const int grid = (int)((a.P + 255) / 256);
    switch (a.K) {
        case 1: launch_fwd_t<1>(a, grid, st); break;
        case 2: launch_fwd_t<2>(a, grid, st); break;
        case 4: launch_fwd_t<4>(a, grid, st); break;
        case 8: launch_fwd_t<8>(a, grid, st); break;
        case 16: launch_fwd_t<16>(a, grid, st); break;
        default: k_blend_fwd_any<<<grid, 256, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const BlendArgs &a, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    const unsigned tiles = (unsigned)((a.S + 15) / 16);
    const dim3 grid(tiles, tiles, (unsigned)a.N);
    switch (a.K) {
        case 1: launch_bwd_t<1>(a, grid, st); break;
        case 2: launch_bwd_t<2>(a, grid, st); break;
        case 4: launch_bwd_t<4>(a, grid, st); break;
        case 8: launch_bwd_t<8>(a, grid, st); break;
        case 16: launch_bwd_t<16>(a, grid, st); break;
        default: k_blend_bwd_any<<<grid, 256, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace mr
