// Shared device code of the sm_103a mesh rasterizer: the staged face record,
// double-float helpers, pixel centres and the per-(pixel, face) evaluation
// used by the fine pass, the plain per-image pass and the backward pass.
//
// Geometry follows Section 3.2 of the paper ("Rasterizer"): perspective
// camera to NDC, per-pixel K nearest faces along z, Fragment data (face id,
// barycentrics, z, signed xy distance).  The conventions are the ones stated
// in include/meshrast.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "meshrast.h"

namespace mr {

constexpr float kCullArea = 1e-12f;
constexpr int kMaxK = 64;

// Bin entries the fine pass sorts at a time: the bin capacity rounded up to a
// power of two, at least 256 (one per thread of the largest block), at most
// 8192 (64 KB of shared memory).  When the per-pixel lists live in shared
// memory too (K > 16) the sort reuses their space, so the cap is also kept
// within it (BD threads x K entries x 8 bytes), but never below 2048.
inline int fine_sort_cap(int max_per_bin, int K, int BD) {
    int lim = 8192;
    if (K > 16) {
        int fit = 2048;
        while (fit * 2 <= BD * K && fit * 2 <= 8192) fit <<= 1;
        lim = fit;
    }
    int c = 256;
    while (c < max_per_bin && c < lim) c <<= 1;
    return c;
}

// ---------------------------------------------------------------------------
// Staged face record: 96 bytes, six float4, written once per face by the
// staging kernel and read by the fine, plain and backward kernels.  In memory
// the float4s are stored in the order a, b, d, e, c, h (indices kRec*): the
// four the per-slot passes read (attributes, adjoints) fill the first 64 bytes,
// two 32-byte sectors, of the record.
//   a = (v0x_hi, v0y_hi, v0x_lo, v0y_lo)   corner 0 in NDC as a double-float
//   b = (ux, uy, wx, wy)                   u = v1 - v0, w = v2 - v0 (NDC), high parts
//   c = (xmin, xmax, ymin, ymax)           bbox inflated by sqrt(blur), rounded outward;
//                                          culled faces have xmin = +inf, xmax = -inf
//   d = (1/A, 1/z0, 1/z1, 1/z2)            A = cross(u, w) from the double-float edges,
//                                          z_i = view depth of corner i
//   e = (ux_lo, uy_lo, wx_lo, wy_lo)       low parts of the edges
//   h = (H0, H1, H2, 0)                    H_i = (A / |edge opposite corner i|)^2: the squared
//                                          distance from a point to that edge's line is b_i^2 H_i
// Corner 0 as hi + lo and the edges as hi + lo keep the geometry exact to
// ~1e-14.  The face loop decides coverage with the fp32 high parts (a sign
// test, robust to ~3e-8 of the edge length); barycentrics that are output or
// feed an extrapolated depth are evaluated in double-float, so they stay
// within ~1e-7 of FP64 even for slivers seen edge-on.
// ---------------------------------------------------------------------------
struct __align__(16) FaceRec {
    float4 a, b, c, d, e, h;
};
static_assert(sizeof(FaceRec) == 96, "face record is 96 bytes");
// float4 index of each field in a record in global memory
constexpr int kRecA = 0, kRecB = 1, kRecD = 2, kRecE = 3, kRecC = 4, kRecH = 5;

// Stores that ask L2 to keep their lines ahead of other data (evict_last):
// Fragment data that the blend and the backward read back right away.
__device__ __forceinline__ unsigned long long l2_keep_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(float4 *p, float4 v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_keep(longlong2 *p, longlong2 v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v2.s64 [%0], {%1, %2}, %3;" ::"l"(p), "l"(v.x), "l"(v.y), "l"(pol)
                 : "memory");
}

// ---------------------------------------------------------------------------
// double-float (unevaluated sum hi + lo) arithmetic, error-free transforms
// of Knuth (two-sum) and Dekker (two-product via fma).
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    float lo = __fadd_rn(s.lo, t.hi);
    df u = quick_two_sum(s.hi, lo);
    return quick_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    return quick_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, lo);
}
__device__ __forceinline__ df df_div(df a, df b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    df r = df_sub(a, df_mul_f(b, q1));
    float q2 = __fdiv_rn(r.hi, b.hi);
    df q = quick_two_sum(q1, q2);
    r = df_sub(a, df_mul(b, q));
    return df_add(q, {__fdiv_rn(r.hi, b.hi), 0.f});
}
// rounding a double-float down / up to a float (outward rounding of bboxes)
__device__ __forceinline__ float df_round_down(df a) { return (a.lo < 0.f) ? nextafterf(a.hi, -INFINITY) : a.hi; }
__device__ __forceinline__ float df_round_up(df a) { return (a.lo > 0.f) ? nextafterf(a.hi, INFINITY) : a.hi; }

// ---------------------------------------------------------------------------
// pixel centres: x = 1 - (2c+1)/S = (S - 2c - 1)/S, as a double-float
// ---------------------------------------------------------------------------
struct PixC {
    float xh, xl, yh, yl;
};
__device__ __forceinline__ void pix_coord(int i, int S, float &h, float &l) {
    float num = (float)(S - 2 * i - 1);  // exact for S < 2^24
    if ((S & (S - 1)) == 0) {
        // S = 2^m: the quotient num * 2^-m is exact, the same value the
        // correctly rounded division gives, and the remainder is 0
        h = __fmul_rn(num, __int_as_float((127 - (31 - __clz(S))) << 23));
        l = 0.f;
        return;
    }
    float Sf = (float)S;
    h = __fdiv_rn(num, Sf);
    l = __fdiv_rn(__fmaf_rn(-h, Sf, num), Sf);
}
__device__ __forceinline__ PixC pixel_centre(int r, int c, int S) {
    PixC p;
    pix_coord(c, S, p.xh, p.xl);
    pix_coord(r, S, p.yh, p.yl);
    return p;
}

// ---------------------------------------------------------------------------
// per-(pixel, face) evaluation
// ---------------------------------------------------------------------------
struct EvalFlags {
    int persp, clip;
    float blur, znear;
};

__device__ __forceinline__ bool in_bbox(const FaceRec &r, const PixC &p) {
    return p.xh >= r.c.x && p.xh <= r.c.y && p.yh >= r.c.z && p.yh <= r.c.w;
}

// pixel position relative to corner 0
__device__ __forceinline__ void local_q(const FaceRec &r, const PixC &p, float &qx, float &qy) {
    qx = __fadd_rn(__fsub_rn(p.xh, r.a.x), __fsub_rn(p.xl, r.a.z));
    qy = __fadd_rn(__fsub_rn(p.yh, r.a.y), __fsub_rn(p.yl, r.a.w));
}

// screen barycentrics from the edge functions
//   e0 = cross(v2 - v1, p - v1), e1 = cross(v0 - v2, p - v2), e2 = cross(v1 - v0, p - v0)
// in corner-0-relative coordinates (v0 = 0, v1 = u, v2 = w, p = q).
__device__ __forceinline__ void screen_bary(const FaceRec &r, float qx, float qy, float &b0, float &b1,
                                            float &b2) {
    const float ux = r.b.x, uy = r.b.y, wx = r.b.z, wy = r.b.w;
    float e2 = __fmaf_rn(ux, qy, -__fmul_rn(uy, qx));
    float e1 = __fmaf_rn(qx, wy, -__fmul_rn(qy, wx));
    float ax = __fsub_rn(wx, ux), ay = __fsub_rn(wy, uy);
    float rx = __fsub_rn(qx, ux), ry = __fsub_rn(qy, uy);
    float e0 = __fmaf_rn(ax, ry, -__fmul_rn(ay, rx));
    b0 = __fmul_rn(e0, r.d.x);
    b1 = __fmul_rn(e1, r.d.x);
    b2 = __fmul_rn(e2, r.d.x);
}

// cross(a, b) = ax by - ay bx in full double-float arithmetic
__device__ __forceinline__ df df_cross(df ax, df ay, df bx, df by) {
    return df_sub(df_mul(ax, by), df_mul(ay, bx));
}

// Double-float difference a - b with the rounding error of the high parts
// kept exactly (two-sum) and the low parts added to it: not renormalised, good
// to ~1e-14 relative, which is all the cross products below need.
__device__ __forceinline__ df df_sub_fast(df a, df b) {
    const df s = two_sum(a.hi, -b.hi);
    return {s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo))};
}

// cross(a, b) = ax by - ay bx of double-float vectors, rounded once: the
// products of the high parts and their difference are exact (fma, two-sum),
// the low parts enter to first order.  ~17 instructions.
__device__ __forceinline__ float df_cross_f(df ax, df ay, df bx, df by) {
    const float p = __fmul_rn(ax.hi, by.hi), pe = __fmaf_rn(ax.hi, by.hi, -p);
    const float r = __fmul_rn(ay.hi, bx.hi), re = __fmaf_rn(ay.hi, bx.hi, -r);
    const df d = two_sum(p, -r);
    const float lo = __fmaf_rn(ax.hi, by.lo, __fmaf_rn(ax.lo, by.hi, -__fmaf_rn(ay.hi, bx.lo, __fmul_rn(ay.lo, bx.hi))));
    return __fadd_rn(d.hi, __fadd_rn(d.lo, __fadd_rn(__fsub_rn(pe, re), lo)));
}

// pixel minus corner 0, as a double-float
__device__ __forceinline__ void local_q_df(const FaceRec &r, const PixC &p, df &qx, df &qy) {
    qx = df_sub_fast({p.xh, p.xl}, {r.a.x, r.a.z});
    qy = df_sub_fast({p.yh, p.yl}, {r.a.y, r.a.w});
}

// Screen barycentrics from edge functions of the double-float corners and
// pixel (q = p - v0, u, w), each edge function rounded once, then scaled by
// 1/A: every component keeps ~1e-7 relative accuracy, even near zero and on
// slivers seen edge-on.
__device__ __forceinline__ void screen_bary_df(const FaceRec &r, const PixC &p, float &b0, float &b1, float &b2) {
    df qx, qy;
    local_q_df(r, p, qx, qy);
    const df ux = {r.b.x, r.e.x}, uy = {r.b.y, r.e.y}, wx = {r.b.z, r.e.z}, wy = {r.b.w, r.e.w};
    const float e2 = df_cross_f(ux, uy, qx, qy);
    const float e1 = df_cross_f(qx, qy, wx, wy);
    const float e0 = df_cross_f(df_sub_fast(wx, ux), df_sub_fast(wy, uy), df_sub_fast(qx, ux), df_sub_fast(qy, uy));
    b0 = __fmul_rn(e0, r.d.x);
    b1 = __fmul_rn(e1, r.d.x);
    b2 = __fmul_rn(e2, r.d.x);
}

// The same from two edge functions: b1, b2 as above and b0 = 1 - b1 - b2
// (the three sum to 1).  b0 then carries an absolute error of ~6e-8 (1 + |b1|
// + |b2|) instead of a relative one, which is all a clipped fragment needs:
// clipping divides by the sum of the positive (perspective-corrected)
// barycentrics, which is 1 plus the magnitudes of the negative ones and so at
// least the largest magnitude among them: every clipped component keeps ~2e-7
// absolute (times the ratio of the corner depths).
__device__ __forceinline__ void screen_bary_df2(const FaceRec &r, const PixC &p, float &b0, float &b1, float &b2) {
    df qx, qy;
    local_q_df(r, p, qx, qy);
    const df ux = {r.b.x, r.e.x}, uy = {r.b.y, r.e.y}, wx = {r.b.z, r.e.z}, wy = {r.b.w, r.e.w};
    b2 = __fmul_rn(df_cross_f(ux, uy, qx, qy), r.d.x);
    b1 = __fmul_rn(df_cross_f(qx, qy, wx, wy), r.d.x);
    b0 = __fsub_rn(__fsub_rn(1.f, b1), b2);
}

// squared distance from (qx,qy) to segment a + t e, t in [0,1]; returns s, t
__device__ __forceinline__ float seg_dist2(float ax, float ay, float ex, float ey, float qx, float qy,
                                           float &t) {
    float l2 = __fmaf_rn(ex, ex, __fmul_rn(ey, ey));
    float px = __fsub_rn(qx, ax), py = __fsub_rn(qy, ay);
    float dot = __fmaf_rn(px, ex, __fmul_rn(py, ey));
    // s is stationary in t at the interior minimum, so a ~2 ulp quotient is enough
    t = (l2 > 0.f) ? __fdividef(dot, l2) : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    float rx = __fsub_rn(px, __fmul_rn(t, ex)), ry = __fsub_rn(py, __fmul_rn(t, ey));
    return __fmaf_rn(rx, rx, __fmul_rn(ry, ry));
}

// nearest edge segment (0: v0v1, 1: v1v2, 2: v2v0; ties to the lower index)
__device__ __forceinline__ float nearest_edge(const FaceRec &r, float qx, float qy, int &edge, float &t) {
    const float ux = r.b.x, uy = r.b.y, wx = r.b.z, wy = r.b.w;
    float t0, t1, t2;
    float s0 = seg_dist2(0.f, 0.f, ux, uy, qx, qy, t0);
    float s1 = seg_dist2(ux, uy, __fsub_rn(wx, ux), __fsub_rn(wy, uy), qx, qy, t1);
    float s2 = seg_dist2(wx, wy, -wx, -wy, qx, qy, t2);
    float s = s0;
    edge = 0;
    t = t0;
    if (s1 < s) { s = s1; edge = 1; t = t1; }
    if (s2 < s) { s = s2; edge = 2; t = t2; }
    return s;
}

// Depth of a face at a pixel and final barycentrics, in the order
// perspective correction -> clipping -> z = sum b'_i z_i.
// With perspective correction 1/z is affine in the pixel position:
// T = sum b_i / z_i = iz0 + b1 (iz1 - iz0) + b2 (iz2 - iz0), which keeps its
// accuracy when extrapolated outside the face.  A clipped depth is formed as
// z_j + sum_i c_i (z_i - z_j) / sum c with j the largest weight, so a pixel
// clipped to a shared vertex gets exactly that vertex's depth from every face.
template <bool FAST>
__device__ __forceinline__ float rcp_(float x) {
    if constexpr (FAST) return __fdividef(1.f, x);
    else return __fdiv_rn(1.f, x);
}

template <bool FAST>
__device__ __forceinline__ float clipped_depth(float c0, float c1, float c2, const float z[3], float *bp,
                                               bool want) {
    float cs = __fadd_rn(__fadd_rn(c0, c1), c2);
    float ic = rcp_<FAST>(cs);
    float w0 = __fmul_rn(c0, ic), w1 = __fmul_rn(c1, ic), w2 = __fmul_rn(c2, ic);
    if (want) { bp[0] = w0; bp[1] = w1; bp[2] = w2; }
    if (c0 >= c1 && c0 >= c2)
        return __fadd_rn(z[0], __fadd_rn(__fmul_rn(w1, __fsub_rn(z[1], z[0])), __fmul_rn(w2, __fsub_rn(z[2], z[0]))));
    if (c1 >= c2)
        return __fadd_rn(z[1], __fadd_rn(__fmul_rn(w0, __fsub_rn(z[0], z[1])), __fmul_rn(w2, __fsub_rn(z[2], z[1]))));
    return __fadd_rn(z[2], __fadd_rn(__fmul_rn(w0, __fsub_rn(z[0], z[2])), __fmul_rn(w1, __fsub_rn(z[1], z[2]))));
}

// FAST selects approximate (~1 ulp) reciprocals: used for the sort key in the
// face loop, whose value is also the zbuf output.
template <bool WANT_BARY, bool FAST = false>
__device__ __forceinline__ float face_depth(const FaceRec &r, int persp, int clip, bool inside, float b0,
                                            float b1, float b2, float *bp) {
    if (persp) {
        const float T = __fadd_rn(r.d.y, __fadd_rn(__fmul_rn(b1, __fsub_rn(r.d.z, r.d.y)),
                                                   __fmul_rn(b2, __fsub_rn(r.d.w, r.d.y))));
        const float iT = rcp_<FAST>(T);
        if (!clip || inside) {
            // b~ = (b_i / z_i) / T; z = 1 / T
            if (WANT_BARY) {
                bp[0] = __fmul_rn(__fmul_rn(b0, r.d.y), iT);
                bp[1] = __fmul_rn(__fmul_rn(b1, r.d.z), iT);
                bp[2] = __fmul_rn(__fmul_rn(b2, r.d.w), iT);
            }
            return iT;
        }
        const float t0 = __fmul_rn(__fmul_rn(b0, r.d.y), iT);
        const float t1 = __fmul_rn(__fmul_rn(b1, r.d.z), iT);
        const float t2 = __fmul_rn(__fmul_rn(b2, r.d.w), iT);
        const float z[3] = {rcp_<FAST>(r.d.y), rcp_<FAST>(r.d.z), rcp_<FAST>(r.d.w)};
        return clipped_depth<FAST>(fmaxf(t0, 0.f), fmaxf(t1, 0.f), fmaxf(t2, 0.f), z, bp, WANT_BARY);
    }
    const float z[3] = {rcp_<FAST>(r.d.y), rcp_<FAST>(r.d.z), rcp_<FAST>(r.d.w)};
    if (!clip || inside) {
        if (WANT_BARY) { bp[0] = b0; bp[1] = b1; bp[2] = b2; }
        return __fadd_rn(z[0], __fadd_rn(__fmul_rn(b1, __fsub_rn(z[1], z[0])), __fmul_rn(b2, __fsub_rn(z[2], z[0]))));
    }
    return clipped_depth<FAST>(fmaxf(b0, 0.f), fmaxf(b1, 0.f), fmaxf(b2, 0.f), z, bp, WANT_BARY);
}

// Division-free "squared distance to segment a + t e (t in [0,1]) < blur":
// in the interior of the segment the squared distance times |e|^2 is
// |p - a|^2 |e|^2 - ((p - a).e)^2.
__device__ __forceinline__ bool seg_within(float ax, float ay, float ex, float ey, float qx, float qy,
                                           float blur) {
    const float px = qx - ax, py = qy - ay;
    const float dot = px * ex + py * ey;
    const float l2 = ex * ex + ey * ey;
    const float pa2 = px * px + py * py;
    const float bx = px - ex, by = py - ey;
    const float end2 = (dot <= 0.f) ? pa2 : bx * bx + by * by;
    const bool mid = (dot > 0.f) && (dot < l2);
    return mid ? (pa2 * l2 - dot * dot < blur * l2) : (end2 < blur);
}

__device__ __forceinline__ bool within_blur(const FaceRec &r, float qx, float qy, float blur) {
    const float ux = r.b.x, uy = r.b.y, wx = r.b.z, wy = r.b.w;
    return seg_within(0.f, 0.f, ux, uy, qx, qy, blur) || seg_within(ux, uy, wx - ux, wy - uy, qx, qy, blur) ||
           seg_within(wx, wy, -wx, -wy, qx, qy, blur);
}

// Candidate test + sort key for the K-nearest pass (the bbox test is done by
// the caller).  Returns true and the depth when the face is a candidate.
__device__ __forceinline__ bool face_key_nobbox(const FaceRec &r, const PixC &p, const EvalFlags &fl, float &z) {
    float qx, qy;
    local_q(r, p, qx, qy);
    float b0, b1, b2;
    screen_bary(r, qx, qy, b0, b1, b2);
    const bool inside = (b0 >= 0.f) && (b1 >= 0.f) && (b2 >= 0.f);
    if (!inside) {
        if (!(fl.blur > 0.f)) return false;
        // farther than sqrt(blur) from the line of a violated edge: not a candidate
        const float lim = fl.blur * 1.0001f;
        if ((b0 < 0.f && b0 * b0 * r.h.x > lim) || (b1 < 0.f && b1 * b1 * r.h.y > lim) ||
            (b2 < 0.f && b2 * b2 * r.h.z > lim))
            return false;
        if (!within_blur(r, qx, qy, fl.blur)) return false;
        // Outside the face the barycentrics grow with the distance over the
        // face's height.  Unclipped extrapolation, or a sliver (edge^2 / area
        // large, where rounding moves fp32 barycentrics by ~6e-8 edge^2/area),
        // takes the depth from the double-float barycentrics.
        const float sliver = (r.b.x * r.b.x + r.b.y * r.b.y + r.b.z * r.b.z + r.b.w * r.b.w) * fabsf(r.d.x);
        if (!fl.clip || sliver > 64.f) screen_bary_df(r, p, b0, b1, b2);
    }
    z = face_depth<false, true>(r, fl.persp, fl.clip, inside, b0, b1, b2, nullptr);
    return isfinite(z) && z >= fl.znear;
}

__device__ __forceinline__ bool face_key(const FaceRec &r, const PixC &p, const EvalFlags &fl, float &z) {
    if (!in_bbox(r, p)) return false;
    return face_key_nobbox(r, p, fl, z);
}

// Full fragment (for a face already known to be a candidate).
__device__ __forceinline__ void face_fragment(const FaceRec &r, const PixC &p, const EvalFlags &fl, float *bp,
                                              float &dist) {
    float qx, qy;
    local_q(r, p, qx, qy);
    float b0, b1, b2;
    screen_bary(r, qx, qy, b0, b1, b2);
    // coverage from the same fp32 sign test as the face loop
    bool inside = (b0 >= 0.f) && (b1 >= 0.f) && (b2 >= 0.f);
    // unclipped extrapolation outputs the barycentrics themselves: each keeps
    // its relative accuracy there
    if (fl.clip) screen_bary_df2(r, p, b0, b1, b2);
    else screen_bary_df(r, p, b0, b1, b2);
    int e;
    float t;
    float s = nearest_edge(r, qx, qy, e, t);
    dist = inside ? -s : s;
    // approximate (~2 ulp) reciprocals: the barycentrics keep ~3e-7 relative
    (void)face_depth<true, true>(r, fl.persp, fl.clip, inside, b0, b1, b2, bp);
}

// strict total order on (depth, face id)
__device__ __forceinline__ bool key_less(float za, int fa, float zb, int fb) {
    return za < zb || (za == zb && fa < fb);
}

// Register-resident top-K (KM slots, sorted ascending).  Slots beyond the
// runtime K are kept too: the first K of the top KM are the top K.
template <int KM>
struct TopK {
    float z[KM];
    int f[KM];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int k = 0; k < KM; ++k) { z[k] = __int_as_float(0x7f800000); f[k] = 0x7fffffff; }
    }
    __device__ __forceinline__ bool admits(float zz, int ff) const { return key_less(zz, ff, z[KM - 1], f[KM - 1]); }
    __device__ __forceinline__ void insert(float zz, int ff) {
        z[KM - 1] = zz;
        f[KM - 1] = ff;
#pragma unroll
        for (int k = KM - 1; k > 0; --k) {
            bool sw = key_less(z[k], f[k], z[k - 1], f[k - 1]);
            float tz = z[k - 1];
            int tf = f[k - 1];
            z[k - 1] = sw ? z[k] : tz;
            f[k - 1] = sw ? f[k] : tf;
            z[k] = sw ? tz : z[k];
            f[k] = sw ? tf : f[k];
        }
    }
};

// ---------------------------------------------------------------------------
// warp aggregation by key: lanes with equal keys form a group (peers); the
// sum of each group's values ends in the group's lowest lane.  Tree over the
// group's ranks: each round a lane adds the value of its next remaining peer,
// then lanes of odd rank leave.  Every lane of the warp must call this.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void group_sum(unsigned peers, float (&x)[NV]) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned rem = peers & ~((2u << lane) - 1u);   // peers above this lane
    unsigned rank = __popc(peers & ((1u << lane) - 1u));
    while (__any_sync(0xffffffffu, rem != 0u)) {
        const int next = __ffs(rem);               // 1-based lane of the next peer, 0 if none
        const int src = next ? next - 1 : (int)lane;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const float t = __shfl_sync(0xffffffffu, x[j], src);
            if (next) x[j] += t;
        }
        const bool done = rank & 1u;
        rem &= __ballot_sync(0xffffffffu, !done);
        rank >>= 1;
    }
}

__device__ __forceinline__ void set_status(unsigned *status, unsigned bits) {
    if (bits) atomicOr(status, bits);
}

// ---------------------------------------------------------------------------
// workspace layout (host and device agree through this struct)
// ---------------------------------------------------------------------------
struct WsLayout {
    size_t status;      // uint32 status word
    size_t queue;       // uint32 work-queue head of the fine pass
    size_t total;       // int64 sum of raw bin counts
    size_t maxcount;    // int32 largest raw bin count
    size_t redo;        // uint32 pixels the large-K streaming fine pass handed to its second pass
    size_t redo_q;      // uint32 blocks queued for that second pass
    size_t redo_head;   // uint32 the second pass's position in its queue
    size_t redo_items;  // (K > 16) uint64 per 8 x 4 pixel block of every bin: the queue
    size_t records;     // F x FaceRec
    size_t face_mesh;   // F x int32
    size_t counts;      // NB x int32 raw counts
    size_t eff;         // NB x int32 counts clamped to capacity
    size_t offsets;     // (NB + 1) x int32
    size_t cursor;      // NB x int32
    size_t order;       // NB x int32 bins in the fine pass's queue order
    size_t lists;       // capacity x uint64 entries (depth key << 32 | face id)
    int64_t nb;         // bins per side
    int64_t NB;         // N * nb * nb
    int64_t capacity;   // entries in lists
    size_t bytes;       // total
};

}  // namespace mr

// host-side helpers shared by the translation units
namespace mr_host {
bool ws_layout(const rast_params *p, int64_t V, int64_t F, mr::WsLayout *L);
int num_sms();
}
