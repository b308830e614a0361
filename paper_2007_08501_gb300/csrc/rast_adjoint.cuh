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
    if (gs != 0.f) {
        const int ia = edge, ib = (edge == 2) ? 0 : edge + 1;
        const float rx = qx - (Px[ia] + tseg * (Px[ib] - Px[ia]));
        const float ry = qy - (Py[ia] + tseg * (Py[ib] - Py[ia]));
        gx[ia] += gs * (-2.f * rx * (1.f - tseg));
        gy[ia] += gs * (-2.f * ry * (1.f - tseg));
        gx[ib] += gs * (-2.f * rx * tseg);
        gy[ib] += gs * (-2.f * ry * tseg);
    }
    for (int i = 0; i < 3; ++i) {
        g[3 * i] = gx[i];
        g[3 * i + 1] = gy[i];
        g[3 * i + 2] = gZ[i];
    }
}

}  // namespace mr
