/*
 * meshrast.h -- C ABI of the GB300 (sm_103a) packed-mesh rasterizer and its
 * soft blends.
 *
 * The operations are those of Section 3.2 of "Accelerating 3D Deep Learning
 * with PyTorch3D" (Ravi et al., 2020), "Differentiable mesh renderer":
 *   - the rasterizer maps meshes from world to view coordinates with a
 *     camera, finds for every pixel the K nearest faces along z (per-pixel
 *     priority queues), works in two passes (image tiles first, then pixels),
 *     and returns Fragment data: face id, barycentric coordinates, z distance
 *     and signed xy distance ("Rasterizer");
 *   - shaders blend the K fragments of a pixel: Algorithm 1 (silhouette) and
 *     Algorithm 2 (softmax) ("Shaders");
 *   - the backward pass reuses the cached Fragment data instead of
 *     recomputing face-pixel intersections.
 * Conventions the paper leaves open are fixed here and restated per call.
 *
 * General rules
 *   - Every pointer argument is DEVICE memory of the current CUDA device,
 *     contiguous, row-major, owned by the caller.  The library never
 *     allocates, never synchronises inside a forward/backward call and never
 *     runs anything on the host CPU: the calls only enqueue kernels (and
 *     cudaMemsetAsync) on `stream` (a cudaStream_t; NULL = legacy default
 *     stream), so a sequence of them can be captured in a CUDA graph.
 *   - Return value: 0 on success, a negative MESHRAST_ERR_* code for a
 *     synchronous argument error (nothing was enqueued) or a launch failure.
 *   - Asynchronous problems found by the kernels set bits (MESHRAST_ST_*) in
 *     a status word inside the workspace; outputs are then undefined.  Read
 *     it with rast_query_status() after the stream (or graph) has run.
 *   - Sizes are int64_t; face indices and pix_to_face are int64_t; all
 *     floating point data is float32.
 *
 * Packed mesh batch (Section 3, "3D data structures": list/packed/padded)
 *   verts      (V, 3)  world positions
 *   faces      (F, 3)  vertex indices into verts; any face may use any vertex
 *                      (several images may share vertices)
 *   first_face (N,)    image n rasterizes faces [first_face[n], first_face[n] + num_faces[n]);
 *   num_faces  (N,)    first_face must be non-decreasing and the ranges disjoint
 *   cams       (N, 16) per image: R (3x3 row-major, world->view), C (camera
 *                      centre), f = 1/tan(fov/2), znear, 0, 0.
 *                      p_view = R (p_world - C); NDC x = f x/z, y = f y/z;
 *                      the depth is the view z.  View +X is image-left,
 *                      +Y image-up, +Z into the screen.
 * Image: S x S pixels; pixel (row r, col c) has its centre at NDC
 *   (1 - (2c+1)/S, 1 - (2r+1)/S); row 0 is the top row.
 * Fragments, shape (N, S, S, K[, 3]), slot-major within a pixel:
 *   pix_to_face  global packed face id of the k-th nearest face, or -1
 *   zbuf         view depth at the pixel (-1 when empty)
 *   bary         barycentrics (b0, b1, b2) after optional perspective
 *                correction then optional clipping (-1 when empty)
 *   dists        signed squared NDC distance from the pixel centre to the
 *                face's nearest edge segment: negative inside (-1 when empty)
 *   A face is a candidate for a pixel when the pixel lies in it (closed), or
 *   blur_radius > 0 and the squared distance is < blur_radius; and its depth
 *   there is finite and >= znear.  The K candidates with the smallest
 *   (depth, face id) are kept in that order.  Faces with a corner nearer than
 *   znear, or with |NDC double area| < 1e-12, are culled.  Both windings are
 *   rasterized.
 */
#ifndef MESHRAST_H
#define MESHRAST_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MESHRAST_API __attribute__((visibility("default")))
#else
#define MESHRAST_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define MESHRAST_OK                 0
#define MESHRAST_ERR_INVALID_ARG   (-1)   /* bad size, NULL pointer, bad flag */
#define MESHRAST_ERR_WORKSPACE     (-2)   /* workspace too small or not 256-byte aligned */
#define MESHRAST_ERR_UNSUPPORTED   (-3)   /* K > 64, bin_size not in {0, 8, 16}, or a binned layout
                                             with N * nb^2 >= 2^31 - 1 bins or > 2^31 - 1 list entries */
#define MESHRAST_ERR_CUDA          (-4)   /* a kernel launch or memset failed */
#define MESHRAST_ERR_STATIC_TOO_LARGE (-5) /* rast_mesh_fwd_static: the call needs more workspace
                                              than MESHRAST_STATIC_WORKSPACE_BYTES */

/* ---- status bits (asynchronous, in the workspace) -------------------- */
#define MESHRAST_ST_BIN_OVERFLOW    1u    /* a bin held more than max_faces_per_bin faces,
                                             or all bins together more than max_bin_entries */
#define MESHRAST_ST_BAD_INDEX       2u    /* a face used a vertex index outside [0, V) */
#define MESHRAST_ST_BAD_MESH_RANGE  4u    /* first_face / num_faces outside [0, F] or not packed */
#define MESHRAST_ST_NONFINITE       8u    /* a face had a non-finite corner (face culled) */

/* Rasterizer parameters (Section 3.2 "Rasterizer"). */
typedef struct {
    int32_t N;                    /* images (= meshes) in the batch, 0 .. 65535 */
    int32_t image_size;           /* S, 1 .. 8192 */
    int32_t faces_per_pixel;      /* K, 1 .. 64 */
    int32_t bin_size;             /* 0: plain form, one unbinned launch per image;
                                     8 or 16: coarse-to-fine with bins of bin_size^2 pixels */
    int32_t max_faces_per_bin;    /* binned mode: capacity of one bin (> 0) */
    int32_t perspective_correct;  /* 0/1: barycentrics of the 3D point on the face */
    int32_t clip_barycentric_coords; /* 0/1: clamp at 0 and renormalise (after perspective) */
    int32_t reserved;             /* must be 0 */
    float   blur_radius;          /* >= 0, squared NDC units (same units as dists) */
    float   reserved_f;           /* must be 0 */
    int64_t max_bin_entries;      /* binned mode: capacity of all bin lists together;
                                     0 means N * nb * nb * max_faces_per_bin, nb = ceil(S / bin_size).
                                     Bins (N * nb * nb) and this capacity must stay below 2^31 - 1
                                     (32-bit device counters), else MESHRAST_ERR_UNSUPPORTED */
} rast_params;

/* Blend parameters (Algorithms 1 and 2; zfar, znear, sigma, gamma are the
 * user hyper-parameters the paper names). */
#define MESHRAST_BLEND_SIL 0      /* alpha only (Algorithm 1); rgb written as 0 */
#define MESHRAST_BLEND_RGB 1      /* softmax rgb (Algorithm 2) + silhouette alpha */
typedef struct {
    float sigma;                  /* > 0 */
    float gamma;                  /* > 0 */
    float znear, zfar;            /* zfar > znear */
    float bg[3];                  /* background colour of the softmax blend */
    float eps;                    /* background depth term, e.g. 1e-10 */
    int32_t mode;                 /* MESHRAST_BLEND_SIL or MESHRAST_BLEND_RGB */
    int32_t reserved;             /* must be 0 */
} blend_params;

/* Bytes of device workspace that rast_mesh_fwd / rast_mesh_bwd need for
 * these parameters and sizes (a multiple of 256).  Returns 0 for invalid
 * parameters.  The workspace must be 256-byte aligned. */
MESHRAST_API size_t rast_workspace_bytes(const rast_params *p, int64_t V, int64_t F);

/* Forward rasterization (Section 3.2 "Rasterizer": camera transform, coarse
 * binning into image tiles, per-pixel K nearest faces, Fragment data).
 * Outputs (all overwritten, every slot written):
 *   pix_to_face (N,S,S,K) int64, zbuf (N,S,S,K), bary (N,S,S,K,3), dists (N,S,S,K).
 * Clears the workspace status word, then ORs MESHRAST_ST_* bits into it. */
MESHRAST_API int rast_mesh_fwd(const rast_params *p,
                  const float *verts, int64_t V,
                  const int64_t *faces, int64_t F,
                  const int64_t *first_face, const int64_t *num_faces,
                  const float *cams,
                  int64_t *pix_to_face, float *zbuf, float *bary, float *dists,
                  void *workspace, size_t workspace_bytes, void *stream);

/* Backward rasterization: dL/dverts from dL/d(zbuf, bary, dists), holding
 * the face selection pix_to_face fixed.  Barycentrics, depth and distance of
 * every non-empty slot are recomputed from pix_to_face and the geometry (the
 * forward's bary/zbuf/dists are not needed).  grad_zbuf, grad_bary and
 * grad_dists may each be NULL (taken as zero).  grad_verts (V, 3) is
 * overwritten.  Gradients reach only the vertices (not the cameras).
 * Leaves the status word as it is and ORs new bits into it. */
MESHRAST_API int rast_mesh_bwd(const rast_params *p,
                  const float *verts, int64_t V,
                  const int64_t *faces, int64_t F,
                  const int64_t *first_face, const int64_t *num_faces,
                  const float *cams,
                  const int64_t *pix_to_face,
                  const float *grad_zbuf, const float *grad_bary, const float *grad_dists,
                  float *grad_verts,
                  void *workspace, size_t workspace_bytes, void *stream);

/* Blend forward (Algorithm 1; Algorithm 2 when mode == MESHRAST_BLEND_RGB).
 *   prob_k = sigmoid(-dists_k / sigma) over slots with pix_to_face >= 0;
 *   alpha  = 1 - prod_k (1 - prob_k);
 *   zinv_k = (zfar - zbuf_k)/(zfar - znear); m = max(eps, max_k zinv_k);
 *   w_k = prob_k exp((zinv_k - m)/gamma); delta = exp((eps - m)/gamma);
 *   rgb = (sum_k w_k c_k + delta bg)/(sum_k w_k + delta), where c_k is the
 *   per-vertex colour of face pix_to_face_k interpolated with bary_k.
 * image (N,S,S,4) = (r, g, b, alpha), overwritten.
 * In MESHRAST_BLEND_SIL mode zbuf, bary, faces and vert_colors may be NULL. */
MESHRAST_API int blend_fwd(const blend_params *bp, int64_t N, int64_t S, int64_t K,
              const int64_t *pix_to_face, const float *zbuf, const float *bary,
              const float *dists,
              const int64_t *faces, int64_t F, const float *vert_colors, int64_t V,
              float *image, void *stream);

/* Forward rasterization and blend in one call: what rast_mesh_fwd followed by
 * blend_fwd on its fragments computes (Section 3.2 "Rasterizer" and
 * "Shaders", Algorithms 1-2), same arithmetic in the same order.  In
 * MESHRAST_BLEND_SIL mode with bin_size 8 or 16 and K <= 16 the fine pass
 * blends each pixel's fragments while it writes them (no second pass over
 * the fragments); otherwise the blend runs as a separate kernel inside this
 * call.
 * Outputs (all overwritten): the Fragments as in rast_mesh_fwd, and image
 * (N,S,S,4) as in blend_fwd; N, S, K come from p.  vert_colors may be NULL in
 * MESHRAST_BLEND_SIL mode.  image, pix_to_face, dists (and zbuf) must be
 * 16-byte aligned.  Status word as in rast_mesh_fwd.
 * Silhouette without Fragment data: in MESHRAST_BLEND_SIL mode with
 * bin_size 8 or 16 and K <= 16, pix_to_face, zbuf, bary and dists may all be
 * NULL; the fine pass then writes only the image (the same values as with
 * the Fragments written), and nothing is left for a backward pass.  NULL
 * Fragment pointers in any other case are MESHRAST_ERR_INVALID_ARG. */
MESHRAST_API int rast_blend_fwd(const rast_params *p, const blend_params *bp,
                  const float *verts, int64_t V,
                  const int64_t *faces, int64_t F,
                  const int64_t *first_face, const int64_t *num_faces,
                  const float *cams, const float *vert_colors,
                  int64_t *pix_to_face, float *zbuf, float *bary, float *dists,
                  float *image,
                  void *workspace, size_t workspace_bytes, void *stream);

/* Blend backward: adjoint of blend_fwd for upstream grad_image (N,S,S,4).
 * grad_dists (N,S,S,K) is overwritten.  In MESHRAST_BLEND_RGB mode
 * grad_zbuf (N,S,S,K), grad_bary (N,S,S,K,3) and grad_vert_colors (V,3) are
 * overwritten; in MESHRAST_BLEND_SIL mode they may be NULL (and are not
 * touched when given). */
MESHRAST_API int blend_bwd(const blend_params *bp, int64_t N, int64_t S, int64_t K,
              const int64_t *pix_to_face, const float *zbuf, const float *bary,
              const float *dists,
              const int64_t *faces, int64_t F, const float *vert_colors, int64_t V,
              const float *grad_image,
              float *grad_zbuf, float *grad_bary, float *grad_dists, float *grad_vert_colors,
              void *stream);

/* Fused backward of blend_fwd over the output of rast_mesh_fwd: the blend
 * adjoint (Algorithms 1 and 2) pulled straight through the rasterizer
 * adjoint (Section 3.2, backward from the cached Fragment data), without
 * materialising dL/d(zbuf, bary, dists).
 * Computes what blend_bwd followed by rast_mesh_bwd computes (the latter
 * given blend_bwd's grad_zbuf, grad_bary, grad_dists; in
 * MESHRAST_BLEND_SIL mode only grad_dists), up to float rounding order:
 *   grad_verts (V,3)            overwritten: dL/dverts
 *   grad_vert_colors (V,3)      overwritten in MESHRAST_BLEND_RGB mode
 *                               (may be NULL in MESHRAST_BLEND_SIL mode)
 * p and the geometry are those of the forward; N, S, K come from p.
 * pix_to_face, zbuf, bary, dists are the forward's Fragments (zbuf, bary and
 * vert_colors may be NULL in MESHRAST_BLEND_SIL mode); grad_image (N,S,S,4)
 * is dL/d(image of blend_fwd).  The fragments and grad_image must be
 * 16-byte aligned.  Uses the workspace like rast_mesh_bwd (the face records
 * are rebuilt; the status word is left as it is, new bits are ORed in). */
MESHRAST_API int blend_rast_bwd(const rast_params *p, const blend_params *bp,
                  const float *verts, int64_t V,
                  const int64_t *faces, int64_t F,
                  const int64_t *first_face, const int64_t *num_faces,
                  const float *cams,
                  const int64_t *pix_to_face, const float *zbuf, const float *bary,
                  const float *dists, const float *vert_colors,
                  const float *grad_image,
                  float *grad_verts, float *grad_vert_colors,
                  void *workspace, size_t workspace_bytes, void *stream);

/* ---- lit shading (Section 3.2 "Shaders": flat, Gouraud and Phong shading
 * with per-vertex colours, blended by hard assignment or softmax) ----------
 * One point light and the textbook Phong reflection model, all in world
 * space, E the camera centre of the pixel's image (cams row, entries 9..11):
 *   m = n/|n|, l = (light - x)/|light - x|, v = (E - x)/|E - x|, c = m . l,
 *   r = 2 c m - l, s = r . v,
 *   phi(x, n, a) = a * (ambient + diffuse * max(c, 0))
 *                  + specular * (c > 0 and s > 0 ? s^shininess : 0)
 *   FLAT:    n = (P1 - P0) x (P2 - P0) (the face's winding), x = sum b_i P_i,
 *            a = sum b_i A_i
 *   GOURAUD: colour = sum b_i phi(P_i, N_i, A_i)
 *   PHONG:   x = sum b_i P_i, n = sum b_i N_i, a = sum b_i A_i
 * with P, N, A the face's vertex positions, normals and colours and b the
 * fragment's barycentrics.  SOFTMAX blends the shaded colours with
 * Algorithm 2 (alpha of Algorithm 1, as blend_fwd in MESHRAST_BLEND_RGB mode);
 * HARD takes the nearest fragment's colour (bg where the pixel has none) and
 * alpha 1 where covered. */
#define MESHRAST_SHADE_FLAT    0
#define MESHRAST_SHADE_GOURAUD 1
#define MESHRAST_SHADE_PHONG   2
#define MESHRAST_SHADE_SOFTMAX 0
#define MESHRAST_SHADE_HARD    1
typedef struct {
    float light[3];               /* point light position (world) */
    float ambient[3];
    float diffuse[3];
    float specular[3];
    float shininess;              /* > 0 */
    int32_t shading;              /* MESHRAST_SHADE_FLAT / _GOURAUD / _PHONG */
    int32_t blend;                /* MESHRAST_SHADE_SOFTMAX / _HARD */
    int32_t reserved;             /* must be 0 */
} shade_params;

/* Shaded image (N,S,S,4) = (r, g, b, alpha) of the Fragments (as from
 * rast_mesh_fwd), overwritten.  bp gives sigma, gamma, znear, zfar, bg and
 * eps (its mode is ignored).  verts, normals, vert_colors (V,3); cams (N,16).
 * pix_to_face, dists and image must be 16-byte aligned. */
MESHRAST_API int shade_fwd(const blend_params *bp, const shade_params *sp, int64_t N, int64_t S, int64_t K,
              const int64_t *pix_to_face, const float *zbuf, const float *bary, const float *dists,
              const int64_t *faces, int64_t F, const float *verts, const float *normals,
              const float *vert_colors, int64_t V, const float *cams, float *image, void *stream);

/* Adjoint of shade_fwd for upstream grad_image (N,S,S,4): grad_zbuf,
 * grad_dists (N,S,S,K) and grad_bary (N,S,S,K,3) are overwritten (feed them
 * to rast_mesh_bwd); grad_verts (the lighting's direct dependence on the
 * positions, to add to rast_mesh_bwd's), grad_normals and grad_vert_colors
 * (V,3) are overwritten. */
MESHRAST_API int shade_bwd(const blend_params *bp, const shade_params *sp, int64_t N, int64_t S, int64_t K,
              const int64_t *pix_to_face, const float *zbuf, const float *bary, const float *dists,
              const int64_t *faces, int64_t F, const float *verts, const float *normals,
              const float *vert_colors, int64_t V, const float *cams, const float *grad_image,
              float *grad_zbuf, float *grad_bary, float *grad_dists, float *grad_verts,
              float *grad_normals, float *grad_vert_colors, void *stream);

/* Waits for `stream`, then copies the workspace status word to *status
 * (host memory).  Returns MESHRAST_ERR_CUDA if the stream failed. */
MESHRAST_API int rast_query_status(const void *workspace, uint32_t *status, void *stream);

/* Waits for `stream`, then reports the bin occupancy of the last binned
 * forward that ran on this workspace: the largest per-bin face count and the
 * sum of all counts (both before any capacity clamp).  Used to size
 * max_faces_per_bin and max_bin_entries. */
MESHRAST_API int rast_bin_occupancy(const rast_params *p, int64_t V, int64_t F, const void *workspace,
                       int32_t *max_count, int64_t *total_entries, void *stream);

/* Where a forward leaves its coarse-binning result in the workspace, for
 * callers that inspect the bin assignment (the first pass of Section 3.2's
 * two-pass rasterizer).  Pure host computation; byte offsets from the start of
 * the workspace, valid for binned parameters (bin_size 8 or 16):
 *   counts   int32[NB]    faces whose inflated bbox meets bin b (before any clamp)
 *   eff      int32[NB]    entries stored for bin b (counts clamped to the capacities)
 *   offsets  int32[NB+1]  first list entry of bin b
 *   lists    uint64[capacity]  entries of bin b at lists[offsets[b] .. offsets[b] + eff[b]):
 *            (float bits of the face's nearest-corner view depth << 32) | face id
 *            (order within a bin unspecified)
 * Bin b = (n * nb + by) * nb + bx for image n, bin row by, bin column bx;
 * bin (by, bx) holds the pixel rows by*bin_size .. and columns bx*bin_size ...
 * Returns MESHRAST_ERR_INVALID_ARG / _UNSUPPORTED as rast_workspace_bytes
 * would return 0, or when out is NULL or the parameters are not binned. */
typedef struct {
    int64_t counts, eff, offsets, lists;   /* byte offsets */
    int64_t nb;                            /* bins per image side, ceil(S / bin_size) */
    int64_t NB;                            /* N * nb * nb */
    int64_t capacity;                      /* entries lists can hold */
    int64_t bytes;                         /* = rast_workspace_bytes */
    int64_t redo;                          /* uint32 at this byte offset: pixels the large-K (K > 16)
                                              fine pass handed to its second pass (their unsettled
                                              candidates outgrew the 16-entry per-pixel ring) */
    int64_t order;                         /* int32[NB] at this byte offset: the order in which
                                              the block fine pass takes the bins, a permutation
                                              of 0 .. NB-1 with the bit length of eff[b]
                                              non-increasing (longest bins first); written by
                                              every binned forward except the large-K streaming
                                              pass, which takes the bins in index order */
} rast_bin_layout;
MESHRAST_API int rast_workspace_bin_layout(const rast_params *p, int64_t V, int64_t F, rast_bin_layout *out);

/* ---- forward without a caller-supplied workspace -------------------------
 * Not part of the paper's method; it exists for callers that cannot allocate
 * device memory at all -- for example a plugin inside a host application
 * that owns every device allocation and exposes no allocator, or a
 * real-time loop that must not allocate once it is running -- and so cannot
 * provide the workspace rast_mesh_fwd asks for.
 *
 * rast_mesh_fwd_static computes exactly what rast_mesh_fwd computes, with
 * the same arguments minus the workspace.  Its workspace is one array of
 * MESHRAST_STATIC_WORKSPACE_BYTES (16 MiB) built into the library, which
 * every GPU that loads the library keeps until the process exits; the call
 * itself allocates nothing.
 *   - A call whose rast_workspace_bytes() would exceed that size returns
 *     MESHRAST_ERR_STATIC_TOO_LARGE and enqueues nothing.  As a guide, a
 *     batch of 8 x 5,120 faces at 256x256 with bins of 16 and
 *     max_faces_per_bin = 256 needs about 8 MiB.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before capturing any stream on that device.  A failed lookup is not
 *     remembered (the next call tries again); a successful one is kept for
 *     the life of the context, so after cudaDeviceReset() the process must
 *     not call this entry point again (the kept address would be stale).
 *   - All calls share the one array, and each call starts by resetting what
 *     it needs.  Calls that overlap on the GPU (two streams, or several host
 *     threads) race on it: order them on one stream.
 *   - Outputs follow the same rules as rast_mesh_fwd; the status word the
 *     call leaves in the array (MESHRAST_ST_* bits, e.g. a bin overflow) is
 *     read with rast_query_static_status. */
#define MESHRAST_STATIC_WORKSPACE_BYTES (16u << 20)
MESHRAST_API int rast_mesh_fwd_static(const rast_params *p,
                                      const float *verts, int64_t V,
                                      const int64_t *faces, int64_t F,
                                      const int64_t *first_face, const int64_t *num_faces,
                                      const float *cams,
                                      int64_t *pix_to_face, float *zbuf, float *bary, float *dists,
                                      void *stream);

/* Status word (MESHRAST_ST_* bits) of the last rast_mesh_fwd_static call on
 * the current device, like rast_query_status for a caller-owned workspace:
 * synchronises `stream` (the one the call ran on), then copies the word to
 * *status.  The word belongs to the shared array, so a later static call
 * resets it.  Returns MESHRAST_ERR_INVALID_ARG for a NULL status pointer and
 * MESHRAST_ERR_CUDA when the stream or the copy fails. */
MESHRAST_API int rast_query_static_status(uint32_t *status, void *stream);

/* ---- measurement -----------------------------------------------------
 * FP32 FMA throughput probe (no counterpart in the paper: it measures the
 * denominator of the ALU rooflines).  Enqueues `blocks` blocks of 256 threads;
 * each thread runs 8 independent chains of iters * 16 fused multiply-adds
 * and writes one float to out[block * 256 + thread] (out holds blocks * 256
 * floats).  FLOPs per launch = blocks * 256 * 8 * 16 * iters * 2; time it
 * with CUDA events on `stream`.  MESHRAST_ERR_INVALID_ARG for a NULL out,
 * blocks outside 1 .. 2^20 or iters < 1. */
MESHRAST_API int meshrast_fma_probe(float *out, int64_t blocks, int32_t iters, void *stream);

/* Static text for a MESHRAST_ERR_* code. */
MESHRAST_API const char *rast_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* MESHRAST_H */
