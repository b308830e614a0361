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

// A double-float number (~44-bit significand) for the few slots whose
// barycentric adjoint is ill-conditioned in fp32: GB300's FP64 rate is a
// small fraction of its FP32 rate, fp32 pairs are several times cheaper.
struct dfv {
    df v;
    dfv() = default;
    __device__ __forceinline__ dfv(df x) : v(x) {}
    __device__ __forceinline__ dfv(float x) : v{x, 0.f} {}
    __device__ __forceinline__ dfv(int x) : v{(float)x, 0.f} {}
    __device__ __forceinline__ float f() const { return __fadd_rn(v.hi, v.lo); }
};
__device__ __forceinline__ dfv operator+(dfv a, dfv b) { return dfv(df_add(a.v, b.v)); }
__device__ __forceinline__ dfv operator-(dfv a, dfv b) { return dfv(df_sub(a.v, b.v)); }
__device__ __forceinline__ dfv operator-(dfv a) { return dfv(df_neg(a.v)); }
__device__ __forceinline__ dfv operator*(dfv a, dfv b) { return dfv(df_mul(a.v, b.v)); }
__device__ __forceinline__ dfv &operator+=(dfv &a, dfv b) { return a = a + b; }
__device__ __forceinline__ dfv &operator-=(dfv &a, dfv b) { return a = a - b; }
__device__ __forceinline__ bool operator>(dfv a, dfv b) {
    const df d = df_sub(a.v, b.v);
    return d.hi > 0.f || (d.hi == 0.f && d.lo > 0.f);
}

__device__ __forceinline__ float rcp_t(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ dfv rcp_t(dfv x) { return dfv(df_div({1.f, 0.f}, x.v)); }

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
        // clipped barycentrics: b'_i = t_i / U over the unclipped set (b~_i > 0),
        // U = sum of t_j there, t_i = b_i / z_i (b_i when affine): T cancels in
        // the renormalisation, so the adjoint is taken through t directly;
        // z = sum_i b'_i z_i
        T t[3], Ut = T(0);
        for (int i = 0; i < 3; ++i) {
            t[i] = persp ? b[i] * iz[i] : b[i];
            if (bt[i] > T(0)) Ut += t[i];   // the t of the unclipped set share T's sign
        }
        const T iU = rcp_t(Ut);
        T gb[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gZ[i] = gz * bp[i];
            T gt = T(0);
            if (bt[i] > T(0)) {
                T acc = T(0);
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (bt[j] > T(0)) acc += bp[j] * ((gbp[i] - gbp[j]) + gz * zdiff(i, j));
                gt = acc * iU;
            }
            if (persp) {
                gb[i] = gt * iz[i];
                gZ[i] -= gt * b[i] * iz[i] * iz[i];
            } else {
                gb[i] = gt;
            }
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

// The same in double-float for the slots whose barycentric gradient is
// ill-conditioned in fp32 (slivers seen far outside: ~1 % of the slots of a
// sphere near its silhouette).  Every input is taken at full accuracy: the
// corners and the pixel as double-float sums, the barycentrics from
// double-float edge functions of those.
static __device__ __noinline__ void bary_adjoint_df(const FaceRec &R, const PixC &p, int persp, int clip, bool inside,
                                                    float gbp0, float gbp1, float gbp2, float gz, float (&gx)[3],
                                                    float (&gy)[3], float (&gZ)[3]) {
    const df qx = df_add(two_sum(p.xh, -R.a.x), two_sum(p.xl, -R.a.z));
    const df qy = df_add(two_sum(p.yh, -R.a.y), two_sum(p.yl, -R.a.w));
    const df ux = {R.b.x, R.e.x}, uy = {R.b.y, R.e.y}, wx = {R.b.z, R.e.z}, wy = {R.b.w, R.e.w};
    const df A = df_cross(ux, uy, wx, wy);
    const df invA = df_div({1.f, 0.f}, A);
    const df e2 = df_cross(ux, uy, qx, qy);
    const df e1 = df_cross(qx, qy, wx, wy);
    const df e0 = df_cross(df_sub(wx, ux), df_sub(wy, uy), df_sub(qx, ux), df_sub(qy, uy));
    const dfv b[3] = {dfv(df_mul(e0, invA)), dfv(df_mul(e1, invA)), dfv(df_mul(e2, invA))};
    const dfv iz[3] = {dfv(R.d.y), dfv(R.d.z), dfv(R.d.w)};
    const dfv gbp[3] = {dfv(gbp0), dfv(gbp1), dfv(gbp2)};
    dfv dx[3], dy[3], dZ[3];
    bary_adjoint<dfv>(b, iz, dfv(ux), dfv(uy), dfv(wx), dfv(wy), dfv(invA), persp, clip, inside, gbp, dfv(gz), dx,
                      dy, dZ);
    for (int i = 0; i < 3; ++i) {
        gx[i] = dx[i].f();
        gy[i] = dy[i].f();
        gZ[i] = dZ[i].f();
    }
}

// Slots whose barycentric adjoint needs double-float are put aside in a
// per-block queue in shared memory and done at the end of the block, one
// thread per slot: done in line, one such lane would hold up the other 31 of
// its warp for the whole double-float evaluation.
constexpr int kRareCap = 256;   // ~1 % of a 16 x 16 tile's slots need it at K = 8
struct RareSlot {
    int f, nf, tile;       // face, its image, the slot's pixel in the block's 16 x 16 tile (row << 4 | column)
    float gz, gb0, gb1, gb2;
};
struct RareQueue {
    RareSlot *e;
    int *n;
};

// NDC corner gradients g[9] of face R (corner-0-relative record) through the
// projection Jacobian and R^T of camera cam to world space: atomics into
// grad_verts at the face's three vertices.
__device__ __forceinline__ void scatter_corner_grads(const FaceRec &R, const float *cam, const int64_t *faces,
                                                     int64_t f, const float (&g)[9], float *grad_verts) {
    const float fo = cam[12];
    const float v0x = R.a.x + R.a.z, v0y = R.a.y + R.a.w;
    const float Px[3] = {0.f, R.b.x, R.b.z}, Py[3] = {0.f, R.b.y, R.b.w};
    const float iz[3] = {R.d.y, R.d.z, R.d.w};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        // x = f x_v / z_v, y = f y_v / z_v: d/dx_v = f/z, d/dz_v = -(x dL/dx + y dL/dy)/z
        const float xn = v0x + Px[i], yn = v0y + Py[i];
        const float gxv = g[3 * i] * fo * iz[i];
        const float gyv = g[3 * i + 1] * fo * iz[i];
        const float gzv = g[3 * i + 2] - (g[3 * i] * xn + g[3 * i + 1] * yn) * iz[i];
        const int64_t vi = __ldg(faces + 3 * f + i);
        float *gv = grad_verts + 3 * vi;
        atomicAdd(gv + 0, cam[0] * gxv + cam[3] * gyv + cam[6] * gzv);
        atomicAdd(gv + 1, cam[1] * gxv + cam[4] * gyv + cam[7] * gzv);
        atomicAdd(gv + 2, cam[2] * gxv + cam[5] * gyv + cam[8] * gzv);
    }
}

// The queued slots of a block whose threads own the pixels of a 16 x 16 tile
// (thread t: row blockIdx.y * 16 + t / 16, column blockIdx.x * 16 + t % 16).
// Every thread of the block must call it, after its last slot.
__device__ __forceinline__ void flush_rare_slots(const RareQueue &q, const FaceRec *rec, const float *cams,
                                                 const int64_t *faces, float *grad_verts, int S, const EvalFlags &fl) {
    __syncthreads();
    const int cnt = min(*q.n, kRareCap);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const RareSlot e = q.e[i];
        const int r = blockIdx.y * 16 + (e.tile >> 4), c = blockIdx.x * 16 + (e.tile & 15);
        const PixC p = pixel_centre(r, c, S);
        FaceRec R;
        const float4 *src = reinterpret_cast<const float4 *>(rec + e.f);
        R.a = __ldg(src + kRecA);
        R.b = __ldg(src + kRecB);
        R.d = __ldg(src + kRecD);
        R.e = __ldg(src + kRecE);
        float qx, qy, b[3];
        local_q(R, p, qx, qy);
        screen_bary(R, qx, qy, b[0], b[1], b[2]);
        const bool inside = (b[0] >= 0.f) && (b[1] >= 0.f) && (b[2] >= 0.f);
        float gx[3], gy[3], gZ[3], g[9];
        bary_adjoint_df(R, p, fl.persp, fl.clip, inside, e.gb0, e.gb1, e.gb2, e.gz, gx, gy, gZ);
        for (int j = 0; j < 3; ++j) {
            g[3 * j] = gx[j];
            g[3 * j + 1] = gy[j];
            g[3 * j + 2] = gZ[j];
        }
        scatter_corner_grads(R, cams + 16 * e.nf, faces, e.f, g, grad_verts);
    }
}

// NDC-space corner gradients of one slot: g[3*i + {0,1,2}] = dL/d(x_i, y_i, z_i)
// of corner i (NDC x, NDC y, view depth).  Uses the record's a, b, d and e.
// With a queue (q.e non-NULL), a slot whose barycentric part needs
// double-float leaves that part to flush_rare_slots (face f of image nf) while
// there is room; without one it is evaluated in fp32.
__device__ __forceinline__ void slot_corner_grads(const FaceRec &R, const PixC &p, const EvalFlags &fl, float gz,
                                                  float gd, float gbp0, float gbp1, float gbp2, float (&g)[9],
                                                  RareQueue q = RareQueue{nullptr, nullptr}, int f = 0, int nf = 0,
                                                  int tile = 0) {
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
        // fp32 unless the face is a sliver (edge^2 / area large) and the pixel
        // lies far outside it (|b| large): there the barycentric gradient is a
        // near-cancellation of large terms, and double-float keeps it to
        // ~1e-7 (about 1 % of the slots of a sphere seen near its silhouette)
        const float sliver = (R.b.x * R.b.x + R.b.y * R.b.y + R.b.z * R.b.z + R.b.w * R.b.w) * fabsf(R.d.x);
        const float bmax = fmaxf(fabsf(b[0]), fmaxf(fabsf(b[1]), fabsf(b[2])));
        // (a full queue leaves the slot to the fp32 evaluation below: the same
        // formula, at fp32 accuracy)
        const int i = (sliver > 64.f && bmax > 8.f && q.e) ? atomicAdd(q.n, 1) : kRareCap;
        if (i < kRareCap) {
            q.e[i] = RareSlot{f, nf, tile, gz, gbp0, gbp1, gbp2};
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
