// Lit shading of mesh fragments for sm_103a (Section 3.2 of the paper,
// "Shaders": flat, Gouraud and Phong shading with per-vertex colours, blended
// by hard assignment or softmax), forward and hand-written adjoint, with the
// C ABI of include/meshrast.h (shade_fwd, shade_bwd).
//
// One thread per pixel.  The reflection model (one point light, world space,
// E the camera centre of the pixel's image):
//   m = n/|n|, l = (L - x)/|L - x|, v = (E - x)/|E - x|, c = m . l,
//   r = 2 c m - l, s = r . v,
//   phi = a * (ambient + diffuse * max(c, 0)) + specular * (c > 0 and s > 0 ? s^sh : 0)
// Softmax blending is Algorithm 2 on the shaded colours (with the same
// cancellation-free forms as the unlit blend); hard blending takes slot 0.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "meshrast.h"
#include "rast_common.cuh"
#include "rast_internal.h"

namespace mr {

struct ShadeArgs {
    int64_t P;  // pixels
    int N, S, K;
    int64_t F, V;
    const int64_t *p2f, *faces;
    const float *zbuf, *bary, *dists, *verts, *normals, *colors, *cams;
    float sigma, gamma, znear, zfar, eps, bg[3];
    float L[3], amb[3], dif[3], spec[3], sh;
    int shading, blend;
    float *image;
    const float *grad_image;
    float *grad_zbuf, *grad_bary, *grad_dists, *grad_verts, *grad_normals, *grad_colors;
};

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 ld3(const float *p, int64_t i) {
    return {__ldg(p + 3 * i), __ldg(p + 3 * i + 1), __ldg(p + 3 * i + 2)};
}

// phi(x, n, a); with G (the upstream colour gradient) also its adjoint into gx, gn, ga
template <bool ADJ>
__device__ __forceinline__ V3 phi(const ShadeArgs &s, V3 E, V3 x, V3 n, V3 a, V3 G, V3 &gx, V3 &gn, V3 &ga) {
    const V3 u = v3(s.L[0], s.L[1], s.L[2]) - x, w = E - x;
    const float iu = rsqrtf(dot(u, u)), iw = rsqrtf(dot(w, w)), in = rsqrtf(dot(n, n));
    const V3 l = iu * u, v = iw * w, m = in * n;
    const float c = dot(m, l);
    const float D = fmaxf(c, 0.f);
    const V3 r = (2.f * c) * m - l;
    const float sv = dot(r, v);
    const bool spec_on = c > 0.f && sv > 0.f;
    const float Sp = spec_on ? powf(sv, s.sh) : 0.f;
    const V3 out = v3(a.x * (s.amb[0] + s.dif[0] * D) + s.spec[0] * Sp, a.y * (s.amb[1] + s.dif[1] * D) + s.spec[1] * Sp,
                      a.z * (s.amb[2] + s.dif[2] * D) + s.spec[2] * Sp);
    if constexpr (ADJ) {
        ga = ga + v3(G.x * (s.amb[0] + s.dif[0] * D), G.y * (s.amb[1] + s.dif[1] * D), G.z * (s.amb[2] + s.dif[2] * D));
        const float gD = G.x * a.x * s.dif[0] + G.y * a.y * s.dif[1] + G.z * a.z * s.dif[2];
        const float gSp = G.x * s.spec[0] + G.y * s.spec[1] + G.z * s.spec[2];
        float gc = c > 0.f ? gD : 0.f;
        V3 gm = v3(0.f, 0.f, 0.f), gl = v3(0.f, 0.f, 0.f), gv = v3(0.f, 0.f, 0.f);
        if (spec_on) {
            const float gs = gSp * s.sh * powf(sv, s.sh - 1.f);
            gv = gs * r;                       // s = r . v
            gm = (2.f * c * gs) * v;           // r = 2 c m - l
            gl = (-gs) * v;
            gc += 2.f * gs * dot(m, v);
        }
        gm = gm + gc * l;                      // c = m . l
        gl = gl + gc * m;
        gn = gn + in * (gm - dot(m, gm) * m);  // m = n / |n|
        gx = gx - iu * (gl - dot(l, gl) * l) - iw * (gv - dot(v, gv) * v);
    }
    return out;
}

// Shaded colour of one slot; with ADJ also the adjoint for colour gradient G:
// gb (3), and the corners' position, normal and colour gradients (gP, gN, gA)
template <bool ADJ>
__device__ __forceinline__ V3 slot_shade(const ShadeArgs &s, V3 E, const int64_t vi[3], const float b[3], V3 G,
                                         float gb[3], V3 gP[3], V3 gN[3], V3 gA[3]) {
    V3 P[3], Nn[3], A[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        P[i] = ld3(s.verts, vi[i]);
        Nn[i] = ld3(s.normals, vi[i]);
        A[i] = ld3(s.colors, vi[i]);
    }
    V3 out = v3(0.f, 0.f, 0.f);
    if (s.shading == MESHRAST_SHADE_GOURAUD) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const V3 c = phi<ADJ>(s, E, P[i], Nn[i], A[i], b[i] * G, gP[i], gN[i], gA[i]);
            out = out + b[i] * c;
            if constexpr (ADJ) gb[i] += dot(G, c);
        }
        return out;
    }
    const V3 x = b[0] * P[0] + b[1] * P[1] + b[2] * P[2];
    const V3 a = b[0] * A[0] + b[1] * A[1] + b[2] * A[2];
    const V3 e1 = P[1] - P[0], e2 = P[2] - P[0];
    const V3 n = (s.shading == MESHRAST_SHADE_PHONG) ? b[0] * Nn[0] + b[1] * Nn[1] + b[2] * Nn[2] : cross(e1, e2);
    V3 gx = v3(0.f, 0.f, 0.f), gn = v3(0.f, 0.f, 0.f), ga = v3(0.f, 0.f, 0.f);
    out = phi<ADJ>(s, E, x, n, a, G, gx, gn, ga);
    if constexpr (ADJ) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gb[i] += dot(gx, P[i]) + dot(ga, A[i]);
            gP[i] = gP[i] + b[i] * gx;
            gA[i] = gA[i] + b[i] * ga;
        }
        if (s.shading == MESHRAST_SHADE_PHONG) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                gb[i] += dot(gn, Nn[i]);
                gN[i] = gN[i] + b[i] * gn;
            }
        } else {
            // n = e1 x e2: d/de1 = e2 x gn, d/de2 = gn x e1
            const V3 g1 = cross(e2, gn), g2 = cross(gn, e1);
            gP[1] = gP[1] + g1;
            gP[2] = gP[2] + g2;
            gP[0] = gP[0] - g1 - g2;
        }
    }
    return out;
}

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }

// face corners (range-checked: -1 when the face or a vertex is out of range)
__device__ __forceinline__ bool slot_face(const ShadeArgs &s, int64_t f, int64_t vi[3]) {
    if (f < 0 || f >= s.F) return false;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        vi[i] = __ldg(s.faces + 3 * f + i);
        if (vi[i] < 0 || vi[i] >= s.V) return false;
    }
    return true;
}

__global__ void __launch_bounds__(256) k_shade_fwd(ShadeArgs s) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= s.P) return;
    const int n = (int)(pix / ((int64_t)s.S * s.S));
    const V3 E = ld3(s.cams + 16 * (int64_t)n + 9, 0);
    const V3 dummy = v3(0.f, 0.f, 0.f);  // colour gradient (unused without the adjoint)
    float gbd[3];
    V3 gP[3], gN[3], gA[3];
    float4 out;
    if (s.blend == MESHRAST_SHADE_HARD) {
        int64_t vi[3];
        const int64_t f = __ldg(s.p2f + pix * s.K);
        if (!slot_face(s, f, vi)) {
            out = make_float4(s.bg[0], s.bg[1], s.bg[2], 0.f);
        } else {
            const float b[3] = {__ldg(s.bary + 3 * pix * s.K), __ldg(s.bary + 3 * pix * s.K + 1),
                                __ldg(s.bary + 3 * pix * s.K + 2)};
            const V3 c = slot_shade<false>(s, E, vi, b, dummy, gbd, gP, gN, gA);
            out = make_float4(c.x, c.y, c.z, 1.f);
        }
        reinterpret_cast<float4 *>(s.image)[pix] = out;
        return;
    }
    float keep = 1.f, zmin = __int_as_float(0x7f800000);
    bool any = false;
    for (int k = 0; k < s.K; ++k) {
        const int64_t q = pix * s.K + k;
        if (__ldg(s.p2f + q) < 0) continue;
        keep *= sigm(__ldg(s.dists + q) / s.sigma);
        zmin = fminf(zmin, __ldg(s.zbuf + q));
        any = true;
    }
    const float range = s.zfar - s.znear;
    const float ztop = any ? (s.zfar - zmin) / range : -__int_as_float(0x7f800000);
    const bool face_max = any && ztop > s.eps;
    const float m = face_max ? ztop : s.eps;
    V3 num = v3(0.f, 0.f, 0.f);
    float den = 0.f;
    for (int k = 0; k < s.K; ++k) {
        const int64_t q = pix * s.K + k;
        int64_t vi[3];
        if (!slot_face(s, __ldg(s.p2f + q), vi)) continue;
        const float z = __ldg(s.zbuf + q);
        const float arg = face_max ? (zmin - z) / (range * s.gamma) : ((s.zfar - z) / range - m) / s.gamma;
        const float w = sigm(-__ldg(s.dists + q) / s.sigma) * expf(arg);
        const float b[3] = {__ldg(s.bary + 3 * q), __ldg(s.bary + 3 * q + 1), __ldg(s.bary + 3 * q + 2)};
        num = num + w * slot_shade<false>(s, E, vi, b, dummy, gbd, gP, gN, gA);
        den += w;
    }
    const float delta = expf((s.eps - m) / s.gamma);
    const float D = den + delta;
    out = make_float4((num.x + delta * s.bg[0]) / D, (num.y + delta * s.bg[1]) / D, (num.z + delta * s.bg[2]) / D,
                      1.f - keep);
    reinterpret_cast<float4 *>(s.image)[pix] = out;
}

// corners' gradients of one slot summed over the warp's lanes holding the same
// face; one lane per face adds them
__device__ __forceinline__ void scatter_corners(const ShadeArgs &s, int key, const int64_t vi[3], V3 gP[3], V3 gN[3],
                                                V3 gA[3]) {
    float acc[27];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        acc[9 * i + 0] = gP[i].x; acc[9 * i + 1] = gP[i].y; acc[9 * i + 2] = gP[i].z;
        acc[9 * i + 3] = gN[i].x; acc[9 * i + 4] = gN[i].y; acc[9 * i + 5] = gN[i].z;
        acc[9 * i + 6] = gA[i].x; acc[9 * i + 7] = gA[i].y; acc[9 * i + 8] = gA[i].z;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    group_sum<27>(peers, acc);
    if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                atomicAdd(s.grad_verts + 3 * vi[i] + j, acc[9 * i + j]);
                atomicAdd(s.grad_normals + 3 * vi[i] + j, acc[9 * i + 3 + j]);
                atomicAdd(s.grad_colors + 3 * vi[i] + j, acc[9 * i + 6 + j]);
            }
        }
    }
}

// One thread per pixel of a 16 x 16 tile.  The K shaded colours and weights
// live in local arrays (K <= 64).
__global__ void __launch_bounds__(256) k_shade_bwd(ShadeArgs s) {
    // each warp covers an 8 x 4 block of the 16 x 16 tile: neighbouring pixels
    // share faces, so the warp's grouping by face finds more peers
    const int tx = ((threadIdx.x >> 5) & 1) * 8 + (threadIdx.x & 7), ty = (threadIdx.x >> 6) * 4 + ((threadIdx.x >> 3) & 3);
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    const bool valid = row < s.S && col < s.S;
    const int n = blockIdx.z;
    const int64_t pix = ((int64_t)n * s.S + row) * s.S + col;
    const V3 E = ld3(s.cams + 16 * (int64_t)n + 9, 0);
    const float4 g = valid ? reinterpret_cast<const float4 *>(s.grad_image)[pix] : make_float4(0.f, 0.f, 0.f, 0.f);
    const V3 grgb = v3(g.x, g.y, g.z);
    float gbd[3];
    const V3 dummy = v3(0.f, 0.f, 0.f);
    if (s.blend == MESHRAST_SHADE_HARD) {
        for (int k = 0; k < s.K; ++k) {  // uniform trip count: every lane reaches the warp grouping
            const int64_t q = pix * s.K + k;
            int64_t vi[3] = {-1, -1, -1};
            float gb[3] = {0.f, 0.f, 0.f};
            V3 gP[3], gN[3], gA[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) gP[i] = gN[i] = gA[i] = v3(0.f, 0.f, 0.f);
            int key = -1;
            if (valid && k == 0 && slot_face(s, __ldg(s.p2f + q), vi)) {
                const float b[3] = {__ldg(s.bary + 3 * q), __ldg(s.bary + 3 * q + 1), __ldg(s.bary + 3 * q + 2)};
                (void)slot_shade<true>(s, E, vi, b, grgb, gb, gP, gN, gA);
                key = (int)__ldg(s.p2f + q);
            }
            if (valid) {
                s.grad_zbuf[q] = 0.f;
                s.grad_dists[q] = 0.f;
                s.grad_bary[3 * q] = gb[0];
                s.grad_bary[3 * q + 1] = gb[1];
                s.grad_bary[3 * q + 2] = gb[2];
            }
            if (k == 0) scatter_corners(s, key, vi, gP, gN, gA);
        }
        return;
    }
    float keep = 1.f, zmin = __int_as_float(0x7f800000);
    bool any = false;
    for (int k = 0; valid && k < s.K; ++k) {
        const int64_t q = pix * s.K + k;
        if (__ldg(s.p2f + q) < 0) continue;
        keep *= sigm(__ldg(s.dists + q) / s.sigma);
        zmin = fminf(zmin, __ldg(s.zbuf + q));
        any = true;
    }
    const float range = s.zfar - s.znear;
    const float ztop = any ? (s.zfar - zmin) / range : -__int_as_float(0x7f800000);
    const bool face_max = any && ztop > s.eps;
    const float m = face_max ? ztop : s.eps;
    float Wl[kMaxK];
    V3 Cl[kMaxK];
    float den = 0.f;
    for (int k = 0; k < s.K; ++k) {
        const int64_t q = pix * s.K + k;
        Wl[k] = 0.f;
        Cl[k] = v3(0.f, 0.f, 0.f);
        int64_t vi[3];
        if (!valid || !slot_face(s, __ldg(s.p2f + q), vi)) continue;
        const float z = __ldg(s.zbuf + q);
        const float arg = face_max ? (zmin - z) / (range * s.gamma) : ((s.zfar - z) / range - m) / s.gamma;
        Wl[k] = sigm(-__ldg(s.dists + q) / s.sigma) * expf(arg);
        const float b[3] = {__ldg(s.bary + 3 * q), __ldg(s.bary + 3 * q + 1), __ldg(s.bary + 3 * q + 2)};
        V3 gP[3], gN[3], gA[3];
        Cl[k] = slot_shade<false>(s, E, vi, b, dummy, gbd, gP, gN, gA);
        den += Wl[k];
    }
    const float delta = expf((s.eps - m) / s.gamma);
    const float iD = 1.f / (den + delta);
    const V3 bgv = v3(s.bg[0], s.bg[1], s.bg[2]);
    for (int k = 0; k < s.K; ++k) {  // uniform trip count: every lane reaches the warp grouping
        const int64_t q = pix * s.K + k;
        int64_t vi[3] = {-1, -1, -1};
        float gb[3] = {0.f, 0.f, 0.f};
        V3 gP[3], gN[3], gA[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) gP[i] = gN[i] = gA[i] = v3(0.f, 0.f, 0.f);
        int key = -1;
        float gd = 0.f, gz = 0.f;
        if (valid && slot_face(s, __ldg(s.p2f + q), vi)) {
            key = (int)__ldg(s.p2f + q);
            const float d = __ldg(s.dists + q);
            const float prob = sigm(-d / s.sigma);
            gd = g.w * (-prob * keep / s.sigma);
            // c_k - rgb = (sum_{j != k} w_j (c_k - c_j) + delta (c_k - bg)) / D (no cancellation)
            V3 diff = delta * (Cl[k] - bgv);
            for (int j = 0; j < s.K; ++j)
                if (j != k) diff = diff + Wl[j] * (Cl[k] - Cl[j]);
            const float gw = dot(grgb, diff) * iD * iD;
            const float z = __ldg(s.zbuf + q);
            const float arg = face_max ? (zmin - z) / (range * s.gamma) : ((s.zfar - z) / range - m) / s.gamma;
            gd += gw * expf(arg) * (-prob * sigm(d / s.sigma) / s.sigma);
            gz = gw * Wl[k] / s.gamma * (-1.f / range);
            const float b[3] = {__ldg(s.bary + 3 * q), __ldg(s.bary + 3 * q + 1), __ldg(s.bary + 3 * q + 2)};
            (void)slot_shade<true>(s, E, vi, b, (Wl[k] * iD) * grgb, gb, gP, gN, gA);
        }
        if (valid) {
            s.grad_dists[q] = gd;
            s.grad_zbuf[q] = gz;
            s.grad_bary[3 * q] = gb[0];
            s.grad_bary[3 * q + 1] = gb[1];
            s.grad_bary[3 * q + 2] = gb[2];
        }
        scatter_corners(s, key, vi, gP, gN, gA);
    }
}

static int fill_shade(ShadeArgs &a, const blend_params *bp, const shade_params *sp, int64_t N, int64_t S, int64_t K,
                      const int64_t *p2f, const float *zbuf, const float *bary, const float *dists,
                      const int64_t *faces, int64_t F, const float *verts, const float *normals, const float *colors,
                      int64_t V, const float *cams) {
    if (!bp || !sp) return MESHRAST_ERR_INVALID_ARG;
    if (N < 0 || N > 65535 || S < 0 || S > 8192 || K < 1) return MESHRAST_ERR_INVALID_ARG;
    if (K > kMaxK) return MESHRAST_ERR_UNSUPPORTED;
    if (!(bp->sigma > 0.f) || !(bp->gamma > 0.f) || !(bp->zfar > bp->znear)) return MESHRAST_ERR_INVALID_ARG;
    if (sp->shading < 0 || sp->shading > 2 || sp->blend < 0 || sp->blend > 1 || sp->reserved != 0 ||
        !(sp->shininess > 0.f))
        return MESHRAST_ERR_INVALID_ARG;
    if (F < 0 || V < 0) return MESHRAST_ERR_INVALID_ARG;
    std::memset(&a, 0, sizeof(a));
    a.P = N * S * S;
    a.N = (int)N;
    a.S = (int)S;
    a.K = (int)K;
    a.F = F;
    a.V = V;
    a.p2f = p2f;
    a.faces = faces;
    a.zbuf = zbuf;
    a.bary = bary;
    a.dists = dists;
    a.verts = verts;
    a.normals = normals;
    a.colors = colors;
    a.cams = cams;
    a.sigma = bp->sigma;
    a.gamma = bp->gamma;
    a.znear = bp->znear;
    a.zfar = bp->zfar;
    a.eps = bp->eps;
    for (int j = 0; j < 3; ++j) {
        a.bg[j] = bp->bg[j];
        a.L[j] = sp->light[j];
        a.amb[j] = sp->ambient[j];
        a.dif[j] = sp->diffuse[j];
        a.spec[j] = sp->specular[j];
    }
    a.sh = sp->shininess;
    a.shading = sp->shading;
    a.blend = sp->blend;
    if (a.P > 0 && (!p2f || !zbuf || !bary || !dists || !faces || !verts || !normals || !colors || !cams))
        return MESHRAST_ERR_INVALID_ARG;
    return MESHRAST_OK;
}

}  // namespace mr

extern "C" {

int shade_fwd(const blend_params *bp, const shade_params *sp, int64_t N, int64_t S, int64_t K,
              const int64_t *pix_to_face, const float *zbuf, const float *bary, const float *dists,
              const int64_t *faces, int64_t F, const float *verts, const float *normals, const float *vert_colors,
              int64_t V, const float *cams, float *image, void *stream) {
    mr::ShadeArgs a;
    int rc = mr::fill_shade(a, bp, sp, N, S, K, pix_to_face, zbuf, bary, dists, faces, F, verts, normals, vert_colors,
                            V, cams);
    if (rc) return rc;
    if (a.P == 0) return MESHRAST_OK;
    if (!image || ((uintptr_t)image & 15u) != 0) return MESHRAST_ERR_INVALID_ARG;
    a.image = image;
    mr::k_shade_fwd<<<(unsigned)((a.P + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

int shade_bwd(const blend_params *bp, const shade_params *sp, int64_t N, int64_t S, int64_t K,
              const int64_t *pix_to_face, const float *zbuf, const float *bary, const float *dists,
              const int64_t *faces, int64_t F, const float *verts, const float *normals, const float *vert_colors,
              int64_t V, const float *cams, const float *grad_image, float *grad_zbuf, float *grad_bary,
              float *grad_dists, float *grad_verts, float *grad_normals, float *grad_vert_colors, void *stream) {
    mr::ShadeArgs a;
    int rc = mr::fill_shade(a, bp, sp, N, S, K, pix_to_face, zbuf, bary, dists, faces, F, verts, normals, vert_colors,
                            V, cams);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (V > 0) {
        if (!grad_verts || !grad_normals || !grad_vert_colors) return MESHRAST_ERR_INVALID_ARG;
        const size_t bytes = (size_t)V * 3 * sizeof(float);
        if (cudaMemsetAsync(grad_verts, 0, bytes, st) != cudaSuccess ||
            cudaMemsetAsync(grad_normals, 0, bytes, st) != cudaSuccess ||
            cudaMemsetAsync(grad_vert_colors, 0, bytes, st) != cudaSuccess)
            return MESHRAST_ERR_CUDA;
    }
    if (a.P == 0) return MESHRAST_OK;
    if (!grad_image || !grad_zbuf || !grad_bary || !grad_dists || ((uintptr_t)grad_image & 15u) != 0)
        return MESHRAST_ERR_INVALID_ARG;
    a.grad_image = grad_image;
    a.grad_zbuf = grad_zbuf;
    a.grad_bary = grad_bary;
    a.grad_dists = grad_dists;
    a.grad_verts = grad_verts;
    a.grad_normals = grad_normals;
    a.grad_colors = grad_vert_colors;
    const unsigned tiles = (unsigned)((S + 15) / 16);
    mr::k_shade_bwd<<<dim3(tiles, tiles, (unsigned)N), 256, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

}  // extern "C"
