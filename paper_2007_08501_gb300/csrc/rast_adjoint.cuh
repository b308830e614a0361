// Per-slot adjoint of the rasterizer shared by rast_mesh_bwd and the fused
// backward: dL/d(bary, zbuf, dists) of one fragment -> dL/d(NDC corners).
#pragma once

#include "rast_common.cuh"

namespace mr {

// gradient of e(p; a, b) = cross(b - a, p - a) with respect to a and b
__device__ __forceinline__ void edge_grad(float ax, float ay, float bx, float by, float px, float py, float g,
                                          float &gax, float &gay, float &gbx, float &gby) {
    gax += g * (by - py);
    gay += g * (px - bx);
    gbx += g * (py - ay);
    gby += g * (ax - px);
}

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
    const df qx = df_add(two_sum(p.xh, -R.a.x), two_sum(p.xl, -R.a.z));
    const df qy = df_add(two_sum(p.yh, -R.a.y), two_sum(p.yl, -R.a.w));
    const int ia = edge, ib = (edge == 2) ? 0 : edge + 1;
    if (t <= 0.f || t >= 1.f) {
        df cx, cy;
        corner_df(R, (t <= 0.f) ? ia : ib, cx, cy);
        const df dx = df_sub(qx, cx), dy = df_sub(qy, cy);
        rx = __fadd_rn(dx.hi, dx.lo);
        ry = __fadd_rn(dy.hi, dy.lo);
        return;
    }
    df axd, ayd, bxd, byd;
    corner_df(R, ia, axd, ayd);
    corner_df(R, ib, bxd, byd);
    const df ex = df_sub(bxd, axd), ey = df_sub(byd, ayd);
    const df cr = df_cross(ex, ey, df_sub(qx, axd), df_sub(qy, ayd));
    const float c = __fadd_rn(cr.hi, cr.lo);
    const float exf = __fadd_rn(ex.hi, ex.lo), eyf = __fadd_rn(ey.hi, ey.lo);
    const float s = __fdiv_rn(c, __fmaf_rn(exf, exf, __fmul_rn(eyf, eyf)));
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

// NDC-space corner gradients of one slot: g[3*i + {0,1,2}] = dL/d(x_i, y_i, z_i)
// of corner i (NDC x, NDC y, view depth).  Uses the record's a, b, d and e.
__device__ __forceinline__ void slot_corner_grads(const FaceRec &R, const PixC &p, const EvalFlags &fl, float gz,
                                                  float gd, float gbp0, float gbp1, float gbp2, float (&g)[9]) {
    // ---- forward recompute (corner-0-relative coordinates) ----
    float qx, qy;
    local_q(R, p, qx, qy);
    float b[3];
    screen_bary(R, qx, qy, b[0], b[1], b[2]);
    // Coverage from the fp32 sign test of the forward.  The forward output the
    // double-float barycentrics; fp32 ones are off by ~6e-8 edge^2/area, which
    // near zero (a clip kink) or on a sliver can flip the sign of a clamped
    // component, so those cases take the double-float values.
    const bool inside = (b[0] >= 0.f) && (b[1] >= 0.f) && (b[2] >= 0.f);
    {
        const float sliver = (R.b.x * R.b.x + R.b.y * R.b.y + R.b.z * R.b.z + R.b.w * R.b.w) * fabsf(R.d.x);
        const float bmin = fminf(fabsf(b[0]), fminf(fabsf(b[1]), fabsf(b[2])));
        if (sliver > 64.f || bmin < 1e-5f * fmaxf(1.f, sliver)) screen_bary_df(R, p, b[0], b[1], b[2]);
    }
    int edge;
    float tseg;
    (void)nearest_edge(R, qx, qy, edge, tseg);
    const float iz[3] = {R.d.y, R.d.z, R.d.w};
    const float zc[3] = {__fdividef(1.f, iz[0]), __fdividef(1.f, iz[1]), __fdividef(1.f, iz[2])};
    float bt[3], iT = 1.f;
    if (fl.persp) {
        // 1/z is affine in the pixel position: T = iz0 + b1 (iz1 - iz0) + b2 (iz2 - iz0)
        iT = __fdividef(1.f, iz[0] + b[1] * (iz[1] - iz[0]) + b[2] * (iz[2] - iz[0]));
        for (int i = 0; i < 3; ++i) bt[i] = b[i] * iz[i] * iT;
    } else {
        for (int i = 0; i < 3; ++i) bt[i] = b[i];
    }
    float bp[3], ics = 1.f;
    if (fl.clip) {
        float cc[3];
        for (int i = 0; i < 3; ++i) cc[i] = fmaxf(bt[i], 0.f);
        ics = __fdividef(1.f, cc[0] + cc[1] + cc[2]);
        for (int i = 0; i < 3; ++i) bp[i] = cc[i] * ics;
    } else {
        for (int i = 0; i < 3; ++i) bp[i] = bt[i];
    }

    // ---- adjoint ----
    float gbp[3] = {gbp0, gbp1, gbp2};
    float gZ[3];
    for (int i = 0; i < 3; ++i) {  // z = sum b'_i z_i
        gbp[i] += gz * zc[i];
        gZ[i] = gz * bp[i];
    }
    float gbt[3];
    if (fl.clip) {
        const float dot = gbp[0] * bp[0] + gbp[1] * bp[1] + gbp[2] * bp[2];
        for (int i = 0; i < 3; ++i) gbt[i] = (bt[i] > 0.f) ? (gbp[i] - dot) * ics : 0.f;
    } else {
        for (int i = 0; i < 3; ++i) gbt[i] = gbp[i];
    }
    float gb[3];
    if (fl.persp) {
        // t_i = b_i / z_i, b~_i = t_i / T:  dt_i/db_i = iz_i, dt_i/dz_i = -b_i iz_i^2
        const float dot = gbt[0] * bt[0] + gbt[1] * bt[1] + gbt[2] * bt[2];
        for (int i = 0; i < 3; ++i) {
            const float gt = (gbt[i] - dot) * iT;
            gb[i] = gt * iz[i];
            gZ[i] -= gt * b[i] * iz[i] * iz[i];
        }
    } else {
        for (int i = 0; i < 3; ++i) gb[i] = gbt[i];
    }
    const float invA = R.d.x;
    float gA = 0.f, ge[3];
    for (int i = 0; i < 3; ++i) {
        ge[i] = gb[i] * invA;
        gA -= gb[i] * b[i] * invA;
    }
    // local corner positions: P0 = 0, P1 = u, P2 = w; pixel = q
    const float Px[3] = {0.f, R.b.x, R.b.z}, Py[3] = {0.f, R.b.y, R.b.w};
    float gx[3] = {0.f, 0.f, 0.f}, gy[3] = {0.f, 0.f, 0.f};
    // e0 = e(p; P1, P2), e1 = e(p; P2, P0), e2 = e(p; P0, P1)
    edge_grad(Px[1], Py[1], Px[2], Py[2], qx, qy, ge[0], gx[1], gy[1], gx[2], gy[2]);
    edge_grad(Px[2], Py[2], Px[0], Py[0], qx, qy, ge[1], gx[2], gy[2], gx[0], gy[0]);
    edge_grad(Px[0], Py[0], Px[1], Py[1], qx, qy, ge[2], gx[0], gy[0], gx[1], gy[1]);
    // A = e(P2; P0, P1)
    edge_grad(Px[0], Py[0], Px[1], Py[1], Px[2], Py[2], gA, gx[0], gy[0], gx[1], gy[1]);
    gx[2] += gA * (Py[0] - Py[1]);
    gy[2] += gA * (Px[1] - Px[0]);
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
