// Device helpers shared by the blend kernels and the fused backward: the
// sigmoid, slot loads, per-slot interpolated colours and the 16 x 16 pixel
// tiling of the backward launches.
#pragma once

#include "rast_common.cuh"
#include "rast_internal.h"

namespace mr {

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

// face ids as int: negative -> -1 (empty), beyond int range -> INT_MAX (no colour)
__device__ __forceinline__ int clamp_id(long long v) { return v < 0 ? -1 : (v > 0x7fffffffLL ? 0x7fffffff : (int)v); }

template <int KM>
struct SlotData {
    float z[KM], d[KM];
    int f[KM];
};

// load the K slots of pixel `pix` (KM == K)
template <int KM>
__device__ __forceinline__ void load_slots(const BlendArgs &a, int64_t pix, bool rgb, SlotData<KM> &S) {
    const int64_t s0 = pix * KM;
    if constexpr (KM % 4 == 0) {
        const float4 *dp = reinterpret_cast<const float4 *>(a.dists + s0);
#pragma unroll
        for (int j = 0; j < KM / 4; ++j) {
            float4 v = __ldg(dp + j);
            S.d[4 * j] = v.x; S.d[4 * j + 1] = v.y; S.d[4 * j + 2] = v.z; S.d[4 * j + 3] = v.w;
        }
        if (rgb) {
            const float4 *zp = reinterpret_cast<const float4 *>(a.zbuf + s0);
#pragma unroll
            for (int j = 0; j < KM / 4; ++j) {
                float4 v = __ldg(zp + j);
                S.z[4 * j] = v.x; S.z[4 * j + 1] = v.y; S.z[4 * j + 2] = v.z; S.z[4 * j + 3] = v.w;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            S.d[k] = __ldg(a.dists + s0 + k);
            if (rgb) S.z[k] = __ldg(a.zbuf + s0 + k);
        }
    }
    if constexpr (KM % 2 == 0) {
        const longlong2 *fp = reinterpret_cast<const longlong2 *>(a.pix_to_face + s0);
#pragma unroll
        for (int j = 0; j < KM / 2; ++j) {
            longlong2 v = __ldg(fp + j);
            S.f[2 * j] = clamp_id(v.x);
            S.f[2 * j + 1] = clamp_id(v.y);
        }
    } else {
#pragma unroll
        for (int k = 0; k < KM; ++k) S.f[k] = clamp_id(__ldg(a.pix_to_face + s0 + k));
    }
}

__device__ __forceinline__ void slot_colour(const BlendArgs &a, int64_t s, int64_t f, float c[3], int64_t vi[3],
                                            float b[3]) {
    b[0] = __ldg(a.bary + 3 * s);
    b[1] = __ldg(a.bary + 3 * s + 1);
    b[2] = __ldg(a.bary + 3 * s + 2);
    c[0] = c[1] = c[2] = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        vi[i] = -1;
        if (f >= a.F) continue;  // ids outside the batch contribute no colour
        const int64_t v = __ldg(a.faces + 3 * (int64_t)f + i);
        if (v < 0 || v >= a.V) continue;
        vi[i] = v;
        const float *col = a.colors + 3 * v;
        c[0] += b[i] * __ldg(col);
        c[1] += b[i] * __ldg(col + 1);
        c[2] += b[i] * __ldg(col + 2);
    }
}

__device__ __forceinline__ float3 vertex_colour(const BlendArgs &a, int64_t v) {
    if (v < 0) return make_float3(0.f, 0.f, 0.f);
    const float *col = a.colors + 3 * v;
    return make_float3(__ldg(col), __ldg(col + 1), __ldg(col + 2));
}

// Algorithms 1-2 accumulated slot by slot while the fine pass writes a pixel's
// fragments (slots in output order, sorted by depth, so the first valid slot
// holds the smallest depth).  The arithmetic and its order are those of
// k_blend_fwd.
struct FwdBlend {
    float keep, zmin, range, m, num0, num1, num2, den;
    bool face_max;
    __device__ __forceinline__ void begin(const FineBlend &b, bool any, float zfirst) {
        keep = 1.f;
        num0 = num1 = num2 = den = 0.f;
        zmin = any ? zfirst : __int_as_float(0x7f800000);
        range = b.zfar - b.znear;
        const float ztop = any ? (b.zfar - zmin) / range : -__int_as_float(0x7f800000);
        face_max = any && ztop > b.eps;
        m = face_max ? ztop : b.eps;
    }
    __device__ __forceinline__ void slot(const FineBlend &b, int f, float z, float d, const float bb[3]) {
        keep *= sigmoidf_(d / b.sigma);
        if (!b.rgb) return;
        const float arg = face_max ? (zmin - z) / (range * b.gamma) : ((b.zfar - z) / range - m) / b.gamma;
        const float w = sigmoidf_(-d / b.sigma) * expf(arg);
        float c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if ((int64_t)f >= b.F) continue;
            const int64_t v = __ldg(b.faces + 3 * (int64_t)f + i);
            if (v < 0 || v >= b.V) continue;
            const float *col = b.colors + 3 * v;
            c0 += bb[i] * __ldg(col);
            c1 += bb[i] * __ldg(col + 1);
            c2 += bb[i] * __ldg(col + 2);
        }
        num0 += w * c0;
        num1 += w * c1;
        num2 += w * c2;
        den += w;
    }
    __device__ __forceinline__ void end(const FineBlend &b, int64_t pix) const {
        float4 out = make_float4(0.f, 0.f, 0.f, 1.f - keep);
        if (b.rgb) {
            const float delta = expf((b.eps - m) / b.gamma);
            const float D = den + delta;
            out.x = (num0 + delta * b.bg0) / D;
            out.y = (num1 + delta * b.bg1) / D;
            out.z = (num2 + delta * b.bg2) / D;
        }
        reinterpret_cast<float4 *>(b.image)[pix] = out;
    }
};

// pixel of a thread in the 16 x 16 tiled launch used by the backward kernels
__device__ __forceinline__ bool tile_pixel(const BlendArgs &a, int64_t &pix) {
    // each warp covers an 8 x 4 block of the 16 x 16 tile
    const int tx = ((threadIdx.x >> 5) & 1) * 8 + (threadIdx.x & 7), ty = (threadIdx.x >> 6) * 4 + ((threadIdx.x >> 3) & 3);
    const int r = blockIdx.y * 16 + ty, c = blockIdx.x * 16 + tx;
    pix = ((int64_t)blockIdx.z * a.S + r) * a.S + c;
    return r < a.S && c < a.S;
}

}  // namespace mr
