// Per-slot adjoint of the rasterizer shared by rast_mesh_bwd and the fused
// backward: dL/d(bary, zbuf, dists) of one fragment -> dL/d(NDC corners).
#pragma once

#include "rast_common.cuh"

namespace mr {

// Pixel minus its nearest point on edge `edge` (0: v0v1, 1: v1v2, 2: v2v0) at
// segment parameter t, for the gradient of the squared distance.  Near the
// edge this residual is a difference of nearly equal coordinates, so it is
// formed in double-float from the record's hi + lo corners: in the interior
// of the segment as the perpendicular part cross(e, p - a) e_perp / |e|^2
// (the cross product is the edge function, exact to ~1e-14), at a clamped end
// as p minus that corner.  Its relative error stays ~1e-7 however close the
// pixel is to the edge.
__device__ __forceinline__ void corner_df(const FaceRec &R, int i, df &x, df &y) {
    // corner i relative to corner 0, as a double-float (selects, no indexing)
    x = (i == 0) ? df{0.f, 0.f} : (i == 1) ? df{R.b.x, R.e.x} : df{R.b.z, R.e.z};
    y = (i == 0) ? df{0.f, 0.f} : (i == 1) ? df{R.b.y, R.e.y} : df{R.b.w, R.e.w};
}

__device__ __forceinline__ void edge_residual(const FaceRec &R, const PixC &p, int edge, float t, float &rx,
                                              float &ry) {
    df qx, qy;
    local_q_df(R, p, qx, qy);
    const int ia = edge, ib = (edge == 2) ? 0 : edge + 1;
    if (t <= 0.f || t >= 1.f) {
        df cx, cy;
        corner_df(R, (t <= 0.f) ? ia : ib, cx, cy);
        const df dx = df_sub_fast(qx, cx), dy = df_sub_fast(qy, cy);
        rx = __fadd_rn(dx.hi, dx.lo);
        ry = __fadd_rn(dy.hi, dy.lo);
        return;
    }
    df axd, ayd, bxd, byd;
    corner_df(R, ia, axd, ayd);
    corner_df(R, ib, bxd, byd);
    const df ex = df_sub_fast(bxd, axd), ey = df_sub_fast(byd, ayd);
    const float c = df_cross_f(ex, ey, df_sub_fast(qx, axd), df_sub_fast(qy, ayd));
    const float exf = __fadd_rn(ex.hi, ex.lo), eyf = __fadd_rn(ey.hi, ey.lo);
    const float s = __fdividef(c, __fmaf_rn(exf, exf, __fmul_rn(eyf, eyf)));
    rx = -eyf * s;
    ry = exf * s;
}

// Gradient of the squared distance to the nearest edge segment, s = |r|^2 with
// r = p - a - t (b - a): ds/da = -2 r (1 - t), ds/db = -2 r t (the t-derivative
// vanishes at the nearest point).  gs = dL/ds; adds to the corners' x, y.
__device__ __forceinline__ void dist_corner_grads(const FaceRec &R, const PixC &p, int edge, float tseg, float gs,
                                                  float (&gx)[3], float (&gy)[3]) {
    float rx, ry;
    edge_residual(R, p, edge, tseg, rx, ry);
    const int ia = edge, ib = (edge == 2) ? 0 : edge + 1;
    const float wa = -2.f * gs * (1.f - tseg), wb = -2.f * gs * tseg;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float w = (i == ia) ? wa : (i == ib) ? wb : 0.f;
        gx[i] += w * rx;
        gy[i] += w * ry;
    }
}

// Corner gradients of a slot whose only upstream gradient is dL/d(dists) (the
// silhouette blend): the barycentrics and the depth do not enter.
// g[2*i + {0,1}] = dL/d(x_i, y_i) of corner i; the depths get nothing.
__device__ __forceinline__ void slot_corner_grads_dist(const FaceRec &R, const PixC &p, float gd, float (&g)[6]) {
    float qx, qy;
    local_q(R, p, qx, qy);
    float b0, b1, b2;
    screen_bary(R, qx, qy, b0, b1, b2);
    const bool inside = (b0 >= 0.f) && (b1 >= 0.f) && (b2 >= 0.f);  // the forward's sign test
    int edge;
    float tseg;
    (void)nearest_edge(R, qx, qy, edge, tseg);
    float gx[3] = {0.f, 0.f, 0.f}, gy[3] = {0.f, 0.f, 0.f};
    dist_corner_grads(R, p, edge, tseg, inside ? -gd : gd, gx, gy);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g[2 * i] = gx[i];
        g[2 * i + 1] = gy[i];
    }
}

template <typename T>
__device__ __forceinline__ T rcp_t(T x) {
    if constexpr (sizeof(T) == 4) return __fdividef(1.f, x);
    else return 1.0 / x;
}

// Barycentric part of one slot's adjoint: dL/d(bary', zbuf) -> dL/d(x, y, z) of
// the three corners (corner-0-relative: P0 = 0, P1 = u, P2 = w), in the
// order perspective correction -> clipping -> z.  With p = sum_k b_k P_k
// held fixed, d b_k / d P_j = -b_j grad_p(b_k), so corner j's (x, y) gradient
// is -b_j G with
//   G = sum_k gb_k grad(b_k) = (gb_1 - gb_0) grad(b_1) + (gb_2 - gb_0) grad(b_2)
// (the three gradients sum to zero): no 1/A-sized terms cancel.  The
// weighted-mean subtractions of the normalisation adjoints are formed from
// pairwise differences, and depth differences from 1/z differences.
template <typename T>
__device__ __forceinline__ void bary_adjoint(const T (&b)[3], const T (&iz)[3], T ux, T uy, T wx, T wy, T invA,
                                             int persp, int clip, bool inside, const T (&gbp)[3], T gz,
                                             T (&gx)[3], T (&gy)[3], T (&gZ)[3]) {
    const T zc[3] = {rcp_t(iz[0]), rcp_t(iz[1]), rcp_t(iz[2])};
    T bt[3], iT = T(1);
    if (persp) {
        // 1/z is affine in the pixel position: T = iz0 + b1 (iz1 - iz0) + b2 (iz2 - iz0)
        iT = rcp_t(iz[0] + b[1] * (iz[1] - iz[0]) + b[2] * (iz[2] - iz[0]));
        for (int i = 0; i < 3; ++i) bt[i] = b[i] * iz[i] * iT;
    } else {
        for (int i = 0; i < 3; ++i) bt[i] = b[i];
    }
    T bp[3], ics = T(1);
    if (clip) {
        T cc[3];
        for (int i = 0; i < 3; ++i) cc[i] = bt[i] > T(0) ? bt[i] : T(0);
        ics = rcp_t(cc[0] + cc[1] + cc[2]);
        for (int i = 0; i < 3; ++i) bp[i] = cc[i] * ics;
    } else {
        for (int i = 0; i < 3; ++i) bp[i] = bt[i];
    }
    const T g1x = wy * invA, g1y = -wx * invA;   // grad b_1 = (wy, -wx) / A
    const T g2x = -uy * invA, g2y = ux * invA;   // grad b_2 = (-uy, ux) / A
    T d1, d2;                                    // gb_1 - gb_0, gb_2 - gb_0
    // z_i - z_j = (1/z_j - 1/z_i) z_i z_j
    auto zdiff = [&](int i, int j) { return (iz[j] - iz[i]) * zc[i] * zc[j]; };
    if (clip && !inside) {
        // clipped barycentrics, z = sum_i b'_i z_i
        T gbt[3], gb[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gZ[i] = gz * bp[i];
            T acc = T(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) acc += bp[j] * ((gbp[i] - gbp[j]) + gz * zdiff(i, j));
            gbt[i] = (bt[i] > T(0)) ? acc * ics : T(0);
        }
        if (persp) {
            // b~_i = t_i / T, t_i = b_i / z_i
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T acc = T(0);
#pragma unroll
                for (int j = 0; j < 3; ++j) acc += bt[j] * (gbt[i] - gbt[j]);
                const T gt = acc * iT;
                gb[i] = gt * iz[i];
                gZ[i] -= gt * b[i] * iz[i] * iz[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) gb[i] = gbt[i];
        }
        d1 = gb[1] - gb[0];
        d2 = gb[2] - gb[0];
    } else if (persp) {
        // b' = b~ = t / T and z = 1/T: dL/dT from the depth, s = -gz z^2, is
        // shared by every t_i
        T N[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T acc = T(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) acc += bt[j] * (gbp[i] - gbp[j]);
            N[i] = acc * iT;
        }
        const T s = -gz * iT * iT;
#pragma unroll
        for (int i = 0; i < 3; ++i) gZ[i] = -(N[i] + s) * b[i] * iz[i] * iz[i];
        d1 = (N[1] * iz[1] - N[0] * iz[0]) + s * (iz[1] - iz[0]);
        d2 = (N[2] * iz[2] - N[0] * iz[0]) + s * (iz[2] - iz[0]);
    } else {
        // affine: b' = b, z = sum_i b_i z_i
#pragma unroll
        for (int i = 0; i < 3; ++i) gZ[i] = gz * b[i];
        d1 = (gbp[1] - gbp[0]) + gz * zdiff(1, 0);
        d2 = (gbp[2] - gbp[0]) + gz * zdiff(2, 0);
    }
    const T Gx = d1 * g1x + d2 * g2x, Gy = d1 * g1y + d2 * g2y;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gx[i] = -b[i] * Gx;
        gy[i] = -b[i] * Gy;
    }
}

// The same in FP64 for the slots whose barycentric gradient is ill-conditioned
// in fp32 (slivers, far-extrapolated barycentrics: ~1 % of the slots of a
// sphere seen edge-on near its silhouette).  Every input is taken at full
// accuracy: the corners and the pixel as double-float sums, the barycentrics
// from edge functions of those.
static __device__ __noinline__ void bary_adjoint_f64(const FaceRec &R, const PixC &p, int persp, int clip, bool inside,
                                              float gbp0, float gbp1, float gbp2, float gz, float (&gx)[3],
                                              float (&gy)[3], float (&gZ)[3]) {
    const double qx = ((double)p.xh - (double)R.a.x) + ((double)p.xl - (double)R.a.z);
    const double qy = ((double)p.yh - (double)R.a.y) + ((double)p.yl - (double)R.a.w);
    const double ux = (double)R.b.x + (double)R.e.x, uy = (double)R.b.y + (double)R.e.y;
    const double wx = (double)R.b.z + (double)R.e.z, wy = (double)R.b.w + (double)R.e.w;
    const double A = ux * wy - uy * wx, invA = 1.0 / A;
    const double e2 = ux * qy - uy * qx, e1 = qx * wy - qy * wx;
    const double e0 = (wx - ux) * (qy - uy) - (wy - uy) * (qx - ux);
    const double b[3] = {e0 * invA, e1 * invA, e2 * invA};
    const double iz[3] = {(double)R.d.y, (double)R.d.z, (double)R.d.w};
    const double gbp[3] = {(double)gbp0, (double)gbp1, (double)gbp2};
    double dx[3], dy[3], dZ[3];
    bary_adjoint<double>(b, iz, ux, uy, wx, wy, invA, persp, clip, inside, gbp, (double)gz, dx, dy, dZ);
    for (int i = 0; i < 3; ++i) {
        gx[i] = (float)dx[i];
        gy[i] = (float)dy[i];
        gZ[i] = (float)dZ[i];
    }
}

// NDC-space corner gradients of one slot: g[3*i + {0,1,2}] = dL/d(x_i, y_i, z_i)
// of corner i (NDC x, NDC y, view depth).  Uses the record's a, b, d and e.
__device__ __forceinline__ void slot_corner_grads(const FaceRec &R, const PixC &p, const EvalFlags &fl, float gz,
                                                  float gd, float gbp0, float gbp1, float gbp2, float (&g)[9]) {
    float qx, qy;
    local_q(R, p, qx, qy);
    float b[3];
    screen_bary(R, qx, qy, b[0], b[1], b[2]);
    // coverage from the fp32 sign test of the forward
    const bool inside = (b[0] >= 0.f) && (b[1] >= 0.f) && (b[2] >= 0.f);
    int edge;
    float tseg;
    (void)nearest_edge(R, qx, qy, edge, tseg);
    float gx[3] = {0.f, 0.f, 0.f}, gy[3] = {0.f, 0.f, 0.f}, gZ[3] = {0.f, 0.f, 0.f};
    if (gz != 0.f || gbp0 != 0.f || gbp1 != 0.f || gbp2 != 0.f) {
        // fp32 unless the face is a sliver (edge^2 / area large) or the pixel
        // lies far outside it (|b| large): there the barycentric gradient
        // is a near-cancellation of large terms, and FP64 keeps it to ~1e-7
        const float sliver = (R.b.x * R.b.x + R.b.y * R.b.y + R.b.z * R.b.z + R.b.w * R.b.w) * fabsf(R.d.x);
        const float bmax = fmaxf(fabsf(b[0]), fmaxf(fabsf(b[1]), fabsf(b[2])));
        if (sliver > 64.f || bmax > 4.f) {
            bary_adjoint_f64(R, p, fl.persp, fl.clip, inside, gbp0, gbp1, gbp2, gz, gx, gy, gZ);
        } else {
            // near a clip kink the forward's clamped component has the sign of
            // the double-float barycentrics: take those
            const float bmin = fminf(fabsf(b[0]), fminf(fabsf(b[1]), fabsf(b[2])));
            if (bmin < 1e-5f * fmaxf(1.f, sliver)) screen_bary_df(R, p, b[0], b[1], b[2]);
            const float iz[3] = {R.d.y, R.d.z, R.d.w};
            const float gbp[3] = {gbp0, gbp1, gbp2};
            bary_adjoint<float>(b, iz, R.b.x, R.b.y, R.b.z, R.b.w, R.d.x, fl.persp, fl.clip, inside, gbp, gz, gx,
                                gy, gZ);
        }
    }
    // distance to the nearest segment
    const float gs = inside ? -gd : gd;
    if (gs != 0.f) dist_corner_grads(R, p, edge, tseg, gs, gx, gy);
    for (int i = 0; i < 3; ++i) {
        g[3 * i] = gx[i];
        g[3 * i + 1] = gy[i];
        g[3 * i + 2] = gZ[i];
    }
}

}  // namespace mr
