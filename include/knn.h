/*
 * knn.h -- C ABI of exact K nearest neighbours and the Chamfer loss on packed
 * heterogeneous batches of point clouds, on GB300 (sm_103a); same library,
 * return codes and conventions as meshrast.h.
 *
 * The operations are those of Section 3.1 of "Accelerating 3D Deep Learning
 * with PyTorch3D" (Ravi et al., 2020), "3D operators":
 *   - K Nearest Neighbors: exact KNN of D-dimensional points (D <= 4,
 *     K <= 32), heterogeneous batches handled natively, one kernel
 *     specialisation per (D, K) range;
 *   - Chamfer loss (Eq. 1): for clouds P and Q, the mean over p in P of the
 *     squared distance to its nearest neighbour in Q plus the mean over q in
 *     Q of the squared distance to its nearest neighbour in P, computed from
 *     the neighbours found by KNN instead of a |P| x |Q| distance matrix.
 *
 * Packed batches (device memory, row-major, caller-owned):
 *   p1 (P1, D), first1 (N,), len1 (N,)   query clouds: cloud i is rows
 *                                        first1[i] .. first1[i] + len1[i] - 1
 *   p2 (P2, D), first2 (N,), len2 (N,)   candidate clouds, same form
 * Query cloud i only sees candidate cloud i.  In each batch, first is
 * non-decreasing and the ranges are disjoint and inside the array;
 * len2[i] < 2^31.  Coordinates must be finite.
 *
 * Distance and ranking: the squared Euclidean distance evaluated in fp32 as
 * s = dx_0 * dx_0, then s = fma(dx_c, dx_c, s) for c = 1 .. D-1 with
 * dx_c = p1_c - p2_c, every step rounded to nearest even (no other
 * contraction or reassociation), so results are reproducible bit for bit.
 * Neighbours are ranked by ascending distance, equal distances by ascending
 * candidate row.
 *
 * Return value: MESHRAST_OK, or MESHRAST_ERR_INVALID_ARG (NULL pointer with
 * a non-zero size, D outside 1..4, K outside 1..32, N < 0),
 * MESHRAST_ERR_WORKSPACE (too small / not 256-byte aligned) or
 * MESHRAST_ERR_CUDA (a launch failed).  Everything is enqueued on `stream`
 * (a cudaStream_t, NULL = legacy default stream); no call synchronises, and
 * every call can be captured in a CUDA graph.
 */
#ifndef MESHRAST_KNN_H
#define MESHRAST_KNN_H

#include "meshrast.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bytes of device workspace knn_points / chamfer_fwd need for N clouds (a
 * multiple of 256; 256-byte aligned base).  Contents need not persist. */
MESHRAST_API size_t knn_workspace_bytes(int64_t N);

/* K nearest neighbours (Section 3.1, "K Nearest Neighbors").
 * idx (P1, K) int64: the global row in p2 of the k-th nearest candidate of
 * each query row, -1 where the candidate cloud has fewer than k + 1 points;
 * dists (P1, K) float: its squared distance (+infinity where idx is -1).
 * Rows of p1 outside every cloud are left untouched. */
MESHRAST_API int knn_points(const float *p1, int64_t P1, const int64_t *first1, const int64_t *len1,
                            const float *p2, int64_t P2, const int64_t *first2, const int64_t *len2,
                            int64_t N, int32_t D, int32_t K, int64_t *idx, float *dists,
                            void *workspace, size_t workspace_bytes, void *stream);

/* Adjoint of the distances of knn_points with idx held fixed: for upstream
 * grad_dists (P1, K), grad_p1 (P1, D) and grad_p2 (P2, D) are overwritten
 * with sum_k 2 g_k (p1 - p2[idx_k]) and its negative scattered to the
 * neighbours.  Slots with idx outside [0, P2) contribute nothing. */
MESHRAST_API int knn_points_bwd(const float *p1, int64_t P1, const float *p2, int64_t P2, int32_t D,
                                int32_t K, const int64_t *idx, const float *grad_dists, float *grad_p1,
                                float *grad_p2, void *stream);

/* Chamfer loss (Eq. 1) of each pair of clouds (P_i = cloud i of p, Q_i =
 * cloud i of q).  Writes the nearest neighbours both ways, idx_pq (P1,) with
 * d_pq (P1,) and idx_qp (P2,) with d_qp (P2,) (as knn_points with K = 1),
 * the per-pair losses loss_per_pair (N,) and their mean loss (1,).  An empty
 * cloud contributes 0 to both terms of its pair; loss is 0 when N = 0.
 * Sums are taken in fp32 in a fixed order (deterministic). */
MESHRAST_API int chamfer_fwd(const float *p, int64_t P1, const int64_t *first1, const int64_t *len1,
                             const float *q, int64_t P2, const int64_t *first2, const int64_t *len2,
                             int64_t N, int32_t D, int64_t *idx_pq, float *d_pq, int64_t *idx_qp,
                             float *d_qp, float *loss_per_pair, float *loss, void *workspace,
                             size_t workspace_bytes, void *stream);

/* Adjoint of chamfer_fwd with the neighbours held fixed.  The upstream
 * gradient of pair i is grad_per_pair[i] + grad_loss[0] / N (either pointer
 * may be NULL, read as 0).  grad_p (P1, D) and grad_q (P2, D) are
 * overwritten. */
MESHRAST_API int chamfer_bwd(const float *p, int64_t P1, const int64_t *first1, const int64_t *len1,
                             const float *q, int64_t P2, const int64_t *first2, const int64_t *len2,
                             int64_t N, int32_t D, const int64_t *idx_pq, const int64_t *idx_qp,
                             const float *grad_loss, const float *grad_per_pair, float *grad_p, float *grad_q,
                             void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MESHRAST_KNN_H */
