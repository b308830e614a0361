/*
 * CPU oracle of exact K nearest neighbours on packed heterogeneous batches of
 * point clouds (Sec. 3.1, "K Nearest Neighbors": exact KNN for D-dimensional
 * points, D <= 4, K <= 32, heterogeneous batches handled natively).
 *
 * TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU-baseline leg are
 * the only callers.  Nothing in the product package links or loads this file.
 *
 * Packed layout: cloud i of the query batch is rows first1[i] .. first1[i] +
 * len1[i] - 1 of p1 (row-major, D floats per point); cloud i of the candidate
 * batch is rows first2[i] .. first2[i] + len2[i] - 1 of p2.  A query only
 * looks at the candidates of the cloud with the same index i.
 *
 * Distance: the squared Euclidean distance.  Which points are the K nearest is
 * an integer decision, so it is taken in fp32 -- the precision of the kernel --
 * with one fixed evaluation order: dx_c = p1_c - p2_c (fp32), then
 * s = dx_0 * dx_0 and s = fma(dx_c, dx_c, s) for c = 1 .. D-1, every step
 * rounded to nearest.  Ranking: ascending distance, equal distances by
 * ascending candidate index.  Results: the global row of the neighbour in p2
 * and its fp32 distance; slots beyond the size of the candidate cloud hold
 * index -1 and distance +infinity.
 *
 * Compiled without FMA contraction (-ffp-contract=off), so that only the
 * explicit fmaf calls fuse.
 */
#include <math.h>
#include <stdint.h>

static float sqdist(const float *a, const float *b, int D) {
    float d0 = a[0] - b[0];
    float s = d0 * d0;
    for (int c = 1; c < D; ++c) {
        float dc = a[c] - b[c];
        s = fmaf(dc, dc, s);
    }
    return s;
}

/* (d, j) before (e, k) in the ranking */
static int ranks_before(float d, int64_t j, float e, int64_t k) { return d < e || (d == e && j < k); }

/* cloud of query row r: the i with first1[i] <= r < first1[i] + len1[i], or -1 */
static int64_t cloud_of(int64_t r, const int64_t *first1, const int64_t *len1, int64_t N) {
    for (int64_t i = 0; i < N; ++i)
        if (r >= first1[i] && r < first1[i] + len1[i]) return i;
    return -1;
}

/*
 * K nearest candidates of each query row listed in rows[0 .. nrows-1] (all
 * rows 0 .. P1-1 when rows is NULL).  Output row t (of K slots) belongs to
 * rows[t].  Every candidate of the cloud is visited in index order and kept
 * in a list sorted by the ranking above, truncated to K entries.
 */
void okn_knn(const float *p1, int64_t P1, const int64_t *first1, const int64_t *len1, const float *p2,
             const int64_t *first2, const int64_t *len2, int64_t N, int D, int K, const int64_t *rows,
             int64_t nrows, int64_t *idx, float *dists) {
    if (!rows) nrows = P1;
    for (int64_t t = 0; t < nrows; ++t) {
        const int64_t r = rows ? rows[t] : t;
        int64_t *oi = idx + t * K;
        float *od = dists + t * K;
        int n = 0;
        const int64_t i = cloud_of(r, first1, len1, N);
        if (i >= 0) {
            for (int64_t j = first2[i]; j < first2[i] + len2[i]; ++j) {
                const float d = sqdist(p1 + r * D, p2 + j * D, D);
                if (n == K && !ranks_before(d, j, od[K - 1], oi[K - 1])) continue;
                int pos = n < K ? n : K - 1;   /* the last kept entry drops out when full */
                while (pos > 0 && ranks_before(d, j, od[pos - 1], oi[pos - 1])) {
                    od[pos] = od[pos - 1];
                    oi[pos] = oi[pos - 1];
                    --pos;
                }
                od[pos] = d;
                oi[pos] = j;
                if (n < K) ++n;
            }
        }
        for (int k = n; k < K; ++k) {
            oi[k] = -1;
            od[k] = INFINITY;
        }
    }
}
