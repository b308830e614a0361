// Kernel argument blocks and host launchers shared between the translation
// units of libmeshrast (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rast_common.cuh"

namespace mr {

struct StageArgs {
    const float *verts;
    int64_t V;
    const int64_t *faces;
    int64_t F;
    const int64_t *first_face;
    const int64_t *num_faces;
    int N;
    const float *cams;
    float blur;
    int S, bin, nb, do_count;
    FaceRec *rec;
    int *face_mesh;
    int *counts;
    unsigned *status;
};

struct ScanArgs {
    const int *counts;
    int *eff, *offsets, *cursor;
    int *order;  // non-NULL: bins by descending work class, for the fine pass's queue
    int64_t NB, capacity;
    int max_per_bin;
    unsigned *queue, *status;
    long long *total;
    int *maxcount;
    const int64_t *first_face, *num_faces;
    int N;
    int64_t F;
};

struct FillArgs {
    const FaceRec *rec;
    const int *face_mesh;
    int64_t F;
    int S, bin, nb;
    int *cursor;
    const int *eff, *offsets;
    unsigned long long *lists;  // (nearest-corner depth bits << 32) | face id
};

struct FineOut {
    int64_t *pix_to_face;
    float *zbuf, *bary, *dists;
};

// Blend (Algorithm 1; the fields of Algorithm 2 are kept for FwdBlend) applied
// by the fine pass to each pixel's fragments as it writes them (register path,
// K <= 16): same arithmetic as blend_fwd.
struct FineBlend {
    int on, rgb;
    int frag;   // 0: blend only, no Fragment data written (silhouette, fine-pass blend)
    float sigma, gamma, znear, zfar, eps, bg0, bg1, bg2;
    const int64_t *faces;
    const float *colors;
    int64_t F, V;
    float *image;
};

struct FineArgs {
    const FaceRec *rec;
    const float *cams;
    unsigned long long *lists;  // K > 16: each block sorts its bins' lists in place
    const int *eff, *offsets;
    const int *order;           // queue position -> bin (bins by descending work class)
    unsigned *queue;
    unsigned *redo_count;       // large-K streaming pass: pixels handed to its second pass
    unsigned *redo_q;           // queued 8 x 4 blocks (item << 32 | lane mask) and their count,
    unsigned long long *redo_items;  //   written by the first pass
    unsigned *redo_head;        // the second pass's position in that queue
    int items, nb, S, K;
    int sort_cap;  // bin entries sorted at a time (power of two)
    EvalFlags fl;
    FineOut out;
    FineBlend blend;
};

// Fragment attributes after the large-K streaming fine pass: pix_to_face holds
// (depth bits << 32) | face id per slot (-1: empty) on entry.
struct FragAttrArgs {
    const FaceRec *rec;
    FineOut out;
    int64_t F;        // faces in the batch (a key's face id must be below)
    unsigned *status;
    int64_t P;        // pixels
    int S, K;
    EvalFlags fl;
    float sigma;
    float *image;     // non-NULL: silhouette blend (Algorithm 1) into (P, 4)
    unsigned magic_S; // ceil(2^32 / S), set by the launcher
    float inv_sigma;  // 1 / sigma, set by the launcher
};

struct NaiveArgs {
    const FaceRec *rec;
    const float *cams;
    const int64_t *first_face, *num_faces;
    int64_t F;
    int S, K;
    EvalFlags fl;
    FineOut out;
};

struct RastBwdArgs {
    const FaceRec *rec;
    const int *face_mesh;
    const int64_t *faces;
    const float *verts;
    const float *cams;
    const int64_t *pix_to_face;
    const float *grad_zbuf, *grad_bary, *grad_dists;
    float *grad_verts;
    int64_t F, V;
    int64_t slots;  // N * S * S * K
    int S, K;
    EvalFlags fl;
};

struct BlendArgs {
    int64_t P;  // pixels
    int64_t F, V;
    int N, S;
    int K;
    const int64_t *pix_to_face;
    const float *zbuf, *bary, *dists;
    const int64_t *faces;
    const float *colors;
    float sigma, gamma, znear, zfar, eps;
    float bg0, bg1, bg2;
    int mode;
    float *image;
    const float *grad_image;
    float *grad_zbuf, *grad_bary, *grad_dists, *grad_colors;
};

cudaError_t launch_stage(const StageArgs &a, cudaStream_t st);
cudaError_t launch_scan(const ScanArgs &a, cudaStream_t st);
cudaError_t launch_fill(const FillArgs &a, cudaStream_t st);
cudaError_t launch_fine(const FineArgs &a, int bin, cudaStream_t st);
bool fine_blends(int K, bool rgb);  // whether launch_fine applies FineArgs::blend
cudaError_t launch_naive(const NaiveArgs &a, int N, cudaStream_t st);
// large K: front-to-back streaming fine pass + attribute pass (fine_stream.cu)
cudaError_t launch_fine_stream(const FineArgs &a, int bin, cudaStream_t st);
cudaError_t launch_frag_attr(const FragAttrArgs &a, cudaStream_t st);
cudaError_t launch_rast_bwd(const RastBwdArgs &a, int N, cudaStream_t st);
cudaError_t launch_blend_fwd(const BlendArgs &a, cudaStream_t st);
cudaError_t launch_blend_bwd(const BlendArgs &a, cudaStream_t st);
cudaError_t launch_blend_rast_bwd(const BlendArgs &a, const RastBwdArgs &r, cudaStream_t st);

}  // namespace mr
