// Backward rasterization for sm_103a.
//
// Section 3.2 of the paper: the backward pass reuses the Fragment data (the
// face id of each slot) instead of recomputing face-pixel intersections.  For
// every non-empty slot this kernel recomputes the fragment of that face at
// that pixel from the staged face record and pulls dL/d(bary, zbuf, dists)
// back through clipping, perspective correction, the edge functions and the
// nearest-segment distance to the three NDC corners, then through the
// projection Jacobian and R^T to world-space vertices (atomic scatter).
#include <cuda_runtime.h>

#include "rast_common.cuh"
#include "rast_internal.h"

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
// of corner i (NDC x, NDC y, view depth).  Returns false for an empty slot.
__device__ __forceinline__ void slot_corner_grads(const FaceRec &R, const PixC &p, const EvalFlags &fl, float gz,
                                                  float gd, float gbp0, float gbp1, float gbp2, float (&g)[9]) {
    // ---- forward recompute (corner-0-relative coordinates) ----
    float qx, qy;
    local_q(R, p, qx, qy);
    float b[3];
    screen_bary(R, qx, qy, b[0], b[1], b[2]);
    const bool inside = (b[0] >= 0.f) && (b[1] >= 0.f) && (b[2] >= 0.f);
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

// One block = a 16 x 16 pixel tile of one image; each thread loops over its
// pixel's K slots.  For every k the warp (2 rows x 16 pixels) sums the corner
// gradients of lanes that hold the same face, and one lane per face applies
// the projection Jacobian and R^T and issues the atomics.
__global__ void __launch_bounds__(256) k_rast_bwd(RastBwdArgs a) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int n = blockIdx.z;
    const int r = blockIdx.y * 16 + ty, c = blockIdx.x * 16 + tx;
    const bool valid = (r < a.S) && (c < a.S);
    const PixC p = pixel_centre(r, c, a.S);
    const int64_t pix = ((int64_t)n * a.S + r) * a.S + c;
    for (int k = 0; k < a.K; ++k) {
        const int64_t s = pix * a.K + k;
        int64_t f = valid ? a.pix_to_face[s] : -1;
        if (f >= a.F) f = -1;  // an id outside the batch contributes nothing
        int nf = (f >= 0) ? a.face_mesh[f] : -1;
        if (nf < 0) f = -1;
        float g[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) g[j] = 0.f;
        FaceRec R;
        if (f >= 0) {
            const float4 *src = reinterpret_cast<const float4 *>(a.rec + f);
            R.a = __ldg(src);
            R.b = __ldg(src + 1);
            R.c = __ldg(src + 2);
            R.d = __ldg(src + 3);
            R.e = __ldg(src + 4);
            const float gz = a.grad_zbuf ? a.grad_zbuf[s] : 0.f;
            const float gd = a.grad_dists ? a.grad_dists[s] : 0.f;
            float gb0 = 0.f, gb1 = 0.f, gb2 = 0.f;
            if (a.grad_bary) {
                gb0 = a.grad_bary[3 * s];
                gb1 = a.grad_bary[3 * s + 1];
                gb2 = a.grad_bary[3 * s + 2];
            }
            if (gz != 0.f || gd != 0.f || gb0 != 0.f || gb1 != 0.f || gb2 != 0.f)
                slot_corner_grads(R, p, a.fl, gz, gd, gb0, gb1, gb2, g);
            else
                f = -1;
        }
        const int key = (int)f;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        group_sum<9>(peers, g);
        if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
            // NDC -> view -> world, once per face and warp
            const float *cam = a.cams + 16 * nf;
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
                const int64_t vi = a.faces[3 * f + i];
                float *gv = a.grad_verts + 3 * vi;
                atomicAdd(gv + 0, cam[0] * gxv + cam[3] * gyv + cam[6] * gzv);
                atomicAdd(gv + 1, cam[1] * gxv + cam[4] * gyv + cam[7] * gzv);
                atomicAdd(gv + 2, cam[2] * gxv + cam[5] * gyv + cam[8] * gzv);
            }
        }
    }
}

cudaError_t launch_rast_bwd(const RastBwdArgs &a, int N, cudaStream_t st) {
    if (a.slots <= 0 || N <= 0) return cudaSuccess;
    const unsigned tiles = (unsigned)((a.S + 15) / 16);
    k_rast_bwd<<<dim3(tiles, tiles, (unsigned)N), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mr
