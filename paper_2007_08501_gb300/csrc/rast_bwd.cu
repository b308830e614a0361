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
#include "rast_adjoint.cuh"

namespace mr {

// One block = a 16 x 16 pixel tile of one image; each thread loops over its
// pixel's K slots.  For every k the warp (2 rows x 16 pixels) sums the corner
// gradients of lanes that hold the same face, and one lane per face applies
// the projection Jacobian and R^T and issues the atomics.
__global__ void __launch_bounds__(256) k_rast_bwd(RastBwdArgs a) {
    // each warp covers an 8 x 4 block of the 16 x 16 tile: neighbouring pixels
    // share faces, so the warp's grouping by face finds more peers
    const int tx = ((threadIdx.x >> 5) & 1) * 8 + (threadIdx.x & 7), ty = (threadIdx.x >> 6) * 4 + ((threadIdx.x >> 3) & 3);
    const int n = blockIdx.z;
    const int r = blockIdx.y * 16 + ty, c = blockIdx.x * 16 + tx;
    const bool valid = (r < a.S) && (c < a.S);
    const PixC p = pixel_centre(r, c, a.S);
    const int64_t pix = ((int64_t)n * a.S + r) * a.S + c;
    __shared__ RareSlot s_rare[kRareCap];
    __shared__ int s_nrare;
    if (threadIdx.x == 0) s_nrare = 0;
    __syncthreads();
    const RareQueue rq{s_rare, &s_nrare};
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
            R.a = __ldg(src + kRecA);
            R.b = __ldg(src + kRecB);
            R.c = __ldg(src + kRecC);
            R.d = __ldg(src + kRecD);
            R.e = __ldg(src + kRecE);
            const float gz = a.grad_zbuf ? a.grad_zbuf[s] : 0.f;
            const float gd = a.grad_dists ? a.grad_dists[s] : 0.f;
            float gb0 = 0.f, gb1 = 0.f, gb2 = 0.f;
            if (a.grad_bary) {
                gb0 = a.grad_bary[3 * s];
                gb1 = a.grad_bary[3 * s + 1];
                gb2 = a.grad_bary[3 * s + 2];
            }
            if (gz != 0.f || gd != 0.f || gb0 != 0.f || gb1 != 0.f || gb2 != 0.f)
                slot_corner_grads(R, p, a.fl, gz, gd, gb0, gb1, gb2, g, rq, (int)f, nf, (ty << 4) | tx);
            else
                f = -1;
        }
        const int key = (int)f;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        group_sum<9>(peers, g);
        if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
            scatter_corner_grads(R, a.cams + 16 * nf, a.faces, f, g, a.grad_verts);  // once per face and warp
    }
    flush_rare_slots(rq, a.rec, a.cams, a.faces, a.grad_verts, a.S, a.fl);
}

cudaError_t launch_rast_bwd(const RastBwdArgs &a, int N, cudaStream_t st) {
    if (a.slots <= 0 || N <= 0) return cudaSuccess;
    const unsigned tiles = (unsigned)((a.S + 15) / 16);
    k_rast_bwd<<<dim3(tiles, tiles, (unsigned)N), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mr
