/*
 * points.h -- C ABI of the GB300 (sm_103a) point-cloud rasterizer and its
 * compositing, beside the mesh rasterizer of meshrast.h (same library, same
 * conventions, return codes and status bits).
 *
 * The operations are those of Section 3.2 of "Accelerating 3D Deep Learning
 * with PyTorch3D" (Ravi et al., 2020), "Differentiable point cloud renderer":
 *   - each point is splatted to a circular region of radius r in screen
 *     space; the rasterizer finds, per pixel, the K nearest points along z
 *     whose regions overlap the pixel (same two-pass design as the mesh
 *     rasterizer: image tiles first, then pixels);
 *   - the opacity of a point at a pixel decreases away from the region's
 *     centre; read here as alpha = 1 - d / r^2, d the squared NDC distance
 *     from the pixel centre to the projected point;
 *   - Alpha compositing f = sum_i alpha_i prod_{j<i} (1 - alpha_j) f_i over
 *     the pixel's points in increasing z, and Norm compositing
 *     f = (sum_i alpha_i f_i) / (sum_i alpha_i), with gradients to point
 *     features and, through the opacities, to point positions.
 *
 * Packed point-cloud batch (device memory, row-major, caller-owned):
 *   points      (P, 3)  world positions
 *   first_point (N,)    image n rasterizes points [first_point[n], first_point[n] + num_points[n]);
 *   num_points  (N,)    first_point non-decreasing, ranges disjoint
 *   cams        (N, 16) as in meshrast.h: R (world->view), C, f, znear, 0, 0
 *   features    (P, D)  per-point features, 1 <= D <= 8
 * A point nearer than znear (or not finite) is culled.  A point overlaps a
 * pixel when d < r^2 (strict).  The K overlapping points with the smallest
 * (depth, point id) are kept in that order.
 * Fragments (N, S, S, K): idx (global point id, -1 empty) int64, zbuf (view
 * depth, -1 empty), dists (d, -1 empty).
 * The workspace has the layout rules of meshrast.h (256-byte aligned, status
 * word first: rast_query_status reads it).
 */
#ifndef MESHRAST_POINTS_H
#define MESHRAST_POINTS_H

#include "meshrast.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t N;                   /* images (= clouds), 0 .. 65535 */
    int32_t image_size;          /* S, 1 .. 8192 */
    int32_t points_per_pixel;    /* K, 1 .. 64 */
    int32_t bin_size;            /* 0: plain form (one launch per image, every pixel against
                                    every point of its cloud); 8 or 16: coarse-to-fine */
    int32_t max_points_per_bin;  /* binned mode: capacity of one bin (> 0) */
    int32_t reserved;            /* must be 0 */
    float   radius;              /* splat radius r in NDC units, > 0 */
    float   reserved_f;          /* must be 0 */
    int64_t max_bin_entries;     /* binned mode: capacity of all bin lists together;
                                    0 means N * nb * nb * max_points_per_bin */
} pts_params;

#define PTS_COMPOSITE_ALPHA 0
#define PTS_COMPOSITE_NORM  1

/* Bytes of device workspace pts_rasterize_fwd / pts_rasterize_bwd need (a
 * multiple of 256); 0 for invalid parameters. */
MESHRAST_API size_t pts_workspace_bytes(const pts_params *p, int64_t P);

/* Forward rasterization of points (Section 3.2, point cloud renderer:
 * K nearest points along z whose splats overlap each pixel).
 * idx, zbuf, dists (N,S,S,K) are overwritten, every slot.  Clears the status
 * word, then ORs MESHRAST_ST_* bits into it (BAD_MESH_RANGE for bad
 * first_point / num_points, BIN_OVERFLOW, NONFINITE). */
MESHRAST_API int pts_rasterize_fwd(const pts_params *p, const float *points, int64_t P,
                                   const int64_t *first_point, const int64_t *num_points,
                                   const float *cams, int64_t *idx, float *zbuf, float *dists,
                                   void *workspace, size_t workspace_bytes, void *stream);

/* Backward rasterization: dL/dpoints (P,3) (overwritten) from dL/dzbuf and
 * dL/ddists (either may be NULL), holding idx fixed; the distance and depth
 * of every non-empty slot are recomputed from idx and the points (an id
 * outside its image's range contributes nothing).  The workspace is checked
 * as for pts_rasterize_fwd but not written. */
MESHRAST_API int pts_rasterize_bwd(const pts_params *p, const float *points, int64_t P,
                                   const int64_t *first_point, const int64_t *num_points,
                                   const float *cams, const int64_t *idx,
                                   const float *grad_zbuf, const float *grad_dists, float *grad_points,
                                   void *workspace, size_t workspace_bytes, void *stream);

/* Compositing (mode PTS_COMPOSITE_ALPHA or PTS_COMPOSITE_NORM) of the
 * fragments into image (N,S,S,D) (overwritten; a pixel without points is 0).
 * N, S, K and r come from p; features (P, D).  Slots with idx outside
 * [0, P) are skipped. */
MESHRAST_API int pts_composite_fwd(const pts_params *p, int32_t mode, const int64_t *idx, const float *dists,
                                   const float *features, int64_t P, int32_t D, float *image, void *stream);

/* Adjoint of pts_composite_fwd for upstream grad_image (N,S,S,D):
 * grad_dists (N,S,S,K) and grad_features (P,D) are overwritten. */
MESHRAST_API int pts_composite_bwd(const pts_params *p, int32_t mode, const int64_t *idx, const float *dists,
                                   const float *features, int64_t P, int32_t D, const float *grad_image,
                                   float *grad_dists, float *grad_features, void *stream);

/* Waits for the stream, then reports the bin occupancy of the last binned
 * pts_rasterize_fwd on this workspace (largest bin count, sum of counts). */
MESHRAST_API int pts_bin_occupancy(const pts_params *p, int64_t P, const void *workspace, int32_t *max_count,
                                   int64_t *total_entries, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MESHRAST_POINTS_H */
