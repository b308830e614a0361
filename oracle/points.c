/*
 * FP64 CPU oracle for the point-cloud rasterizer and its two compositing
 * rules.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links or calls this
 * file; only the tests and the benchmark's CPU-baseline leg do.  It shares no
 * code with the CUDA kernels (nor with oracle.c).
 *
 * What each function follows (Section 3.2 of the paper, "Differentiable point
 * cloud renderer"):
 *   - the same world -> view -> NDC camera as the mesh renderer;
 *   - each point is splatted to a circular region of radius r in screen
 *     space; a pixel takes the K nearest points along z whose regions
 *     overlap it (here: all overlapping points, sorted by (z, point id));
 *   - the opacity decreases away from the region's centre: read here as
 *     alpha = 1 - d / r^2 with d the squared NDC distance from the pixel
 *     centre to the projected point (1 at the centre, 0 on the rim);
 *   - Alpha compositing: f = sum_i alpha_i prod_{j<i} (1 - alpha_j) f_i over
 *     the pixel's points in increasing z;
 *   - Norm compositing: f = (sum_i alpha_i f_i) / (sum_i alpha_i);
 *   - gradients reach point features and, through the opacities, the point
 *     positions (the order along z is held fixed).
 * Conventions the paper leaves open (NDC axes, pixel centres, units of r,
 * the opacity profile, strict inclusion d < r^2, culling nearer than znear,
 * empty pixels composite to 0) follow one documented reading; each is
 * restated at the function that applies it.
 *
 * Parity pins: tests/test_oracle_points.py checks every function here against
 * closed forms, brute-force enumeration and central finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

/* cam row (16 doubles): R (3x3 row-major, world->view), C (centre), f, znear.
 * view = R (p - C); x_ndc = f x/z, y_ndc = f y/z; depth = z_view. */
static void orp_view(const double *cam, const double *pw, double v[3]) {
    const double *R = cam, *C = cam + 9;
    double d0 = pw[0] - C[0], d1 = pw[1] - C[1], d2 = pw[2] - C[2];
    v[0] = R[0] * d0 + R[1] * d1 + R[2] * d2;
    v[1] = R[3] * d0 + R[4] * d1 + R[5] * d2;
    v[2] = R[6] * d0 + R[7] * d1 + R[8] * d2;
}

/* pixel (row r, col c) of an S x S image: centre (1 - (2c+1)/S, 1 - (2r+1)/S) */
static double orp_pix(int64_t i, int64_t S) { return 1.0 - (2.0 * (double)i + 1.0) / (double)S; }

/* Projected point: returns 0 when culled (nearer than znear, or not finite). */
static int orp_project(const double *cam, const double *pw, double *x, double *y, double *z) {
    double v[3];
    orp_view(cam, pw, v);
    if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2]) || !(v[2] >= cam[13])) return 0;
    *x = cam[12] * v[0] / v[2];
    *y = cam[12] * v[1] / v[2];
    *z = v[2];
    return 1;
}

typedef struct {
    double z;
    int64_t i;
} orp_key;

static int orp_key_cmp(const void *a, const void *b) {
    const orp_key *x = (const orp_key *)a, *y = (const orp_key *)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    if (x->i < y->i) return -1;
    if (x->i > y->i) return 1;
    return 0;
}

static int orp_range(const int64_t *first, const int64_t *num, int64_t n, int64_t P, int64_t *lo, int64_t *hi) {
    *lo = first[n] < 0 ? 0 : first[n];
    *hi = first[n] + num[n];
    if (*hi > P) *hi = P;
    return *hi > *lo;
}

/* All points of cloud n overlapping pixel (r, c), sorted by (z, id); returns
 * their number (only cap are written). A point overlaps when the squared NDC
 * distance d from the pixel centre to the projected point is < r^2. */
static int64_t orp_candidates(const double *points, int64_t P, const int64_t *first, const int64_t *num,
                              const double *cams, int64_t S, double radius, int64_t n, int64_t r, int64_t c,
                              orp_key *keys) {
    int64_t lo, hi;
    if (!orp_range(first, num, n, P, &lo, &hi)) return 0;
    const double *cam = cams + 16 * n;
    const double px = orp_pix(c, S), py = orp_pix(r, S), r2 = radius * radius;
    int64_t m = 0;
    for (int64_t i = lo; i < hi; i++) {
        double x, y, z;
        if (!orp_project(cam, points + 3 * i, &x, &y, &z)) continue;
        const double dx = px - x, dy = py - y, d = dx * dx + dy * dy;
        if (!(d < r2)) continue;
        keys[m].z = z;
        keys[m].i = i;
        m++;
    }
    qsort(keys, (size_t)m, sizeof(orp_key), orp_key_cmp);
    return m;
}

/* Fragments for npix pixels (pixels[p] = (n, row, col)); pixels == NULL means
 * all N*S*S pixels in (n, row, col) order.  Per pixel K slots: idx (global
 * point id or -1), zbuf (view depth, -1 empty), dists (squared NDC distance,
 * -1 empty). */
int orp_rasterize(const double *points, int64_t P, const int64_t *first, const int64_t *num, int64_t N,
                  const double *cams, int64_t S, int64_t K, double radius, const int64_t *pixels, int64_t npix,
                  int64_t *idx, double *zbuf, double *dists) {
    if (!pixels) npix = N * S * S;
    orp_key *keys = (orp_key *)malloc(sizeof(orp_key) * (size_t)(P + 1));
    for (int64_t p = 0; p < npix; p++) {
        int64_t n, r, c;
        if (pixels) { n = pixels[3 * p]; r = pixels[3 * p + 1]; c = pixels[3 * p + 2]; }
        else { n = p / (S * S); r = (p / S) % S; c = p % S; }
        const int64_t m = orp_candidates(points, P, first, num, cams, S, radius, n, r, c, keys);
        const double *cam = cams + 16 * n;
        const double px = orp_pix(c, S), py = orp_pix(r, S);
        for (int64_t k = 0; k < K; k++) {
            const int64_t s = p * K + k;
            if (k < m) {
                double x, y, z;
                orp_project(cam, points + 3 * keys[k].i, &x, &y, &z);
                idx[s] = keys[k].i;
                zbuf[s] = z;
                dists[s] = (px - x) * (px - x) + (py - y) * (py - y);
            } else {
                idx[s] = -1;
                zbuf[s] = -1.0;
                dists[s] = -1.0;
            }
        }
    }
    free(keys);
    return 0;
}

/* Flag bits per pixel:
 *  1  some point's rim passes within eps of the centre: |sqrt(d) - r| < eps
 *  2  two of the first K+1 sorted candidates have depths within eps
 *  4  some point's depth within eps of znear */
int orp_margins(const double *points, int64_t P, const int64_t *first, const int64_t *num, int64_t N,
                const double *cams, int64_t S, int64_t K, double radius, const int64_t *pixels, int64_t npix,
                double eps, uint8_t *flags) {
    if (!pixels) npix = N * S * S;
    orp_key *keys = (orp_key *)malloc(sizeof(orp_key) * (size_t)(P + 1));
    for (int64_t p = 0; p < npix; p++) {
        int64_t n, r, c;
        if (pixels) { n = pixels[3 * p]; r = pixels[3 * p + 1]; c = pixels[3 * p + 2]; }
        else { n = p / (S * S); r = (p / S) % S; c = p % S; }
        uint8_t fl = 0;
        int64_t lo, hi;
        if (orp_range(first, num, n, P, &lo, &hi)) {
            const double *cam = cams + 16 * n;
            const double px = orp_pix(c, S), py = orp_pix(r, S);
            for (int64_t i = lo; i < hi; i++) {
                double v[3];
                orp_view(cam, points + 3 * i, v);
                if (isfinite(v[2]) && fabs(v[2] - cam[13]) < eps) fl |= 4;
                double x, y, z;
                if (!orp_project(cam, points + 3 * i, &x, &y, &z)) continue;
                const double d = (px - x) * (px - x) + (py - y) * (py - y);
                if (fabs(sqrt(d) - radius) < eps) fl |= 1;
            }
            const int64_t m = orp_candidates(points, P, first, num, cams, S, radius, n, r, c, keys);
            for (int64_t k = 0; k + 1 < m && k < K; k++)
                if (keys[k + 1].z - keys[k].z < eps) fl |= 2;
        }
        flags[p] = fl;
    }
    free(keys);
    return 0;
}

/* Opacity of a valid slot: alpha = 1 - d / r^2. */
static double orp_alpha(double d, double radius) { return 1.0 - d / (radius * radius); }

/* Compositing of npix pixels' K slots with D-channel point features
 * (features (P, D)); mode 0: Alpha, 1: Norm.  Only slots with idx >= 0 take
 * part, in slot order (increasing z).  A pixel without points gets 0. */
int orp_composite_fwd(int64_t npix, int64_t K, const int64_t *idx, const double *dists, const double *features,
                      int64_t D, double radius, int mode, double *out) {
    for (int64_t p = 0; p < npix; p++) {
        double *o = out + p * D;
        for (int64_t c = 0; c < D; c++) o[c] = 0.0;
        double T = 1.0, asum = 0.0;
        for (int64_t k = 0; k < K; k++) {
            const int64_t i = idx[p * K + k];
            if (i < 0) continue;
            const double a = orp_alpha(dists[p * K + k], radius);
            const double w = (mode == 0) ? a * T : a;
            for (int64_t c = 0; c < D; c++) o[c] += w * features[i * D + c];
            T *= 1.0 - a;
            asum += a;
        }
        if (mode == 1 && asum > 0.0)
            for (int64_t c = 0; c < D; c++) o[c] /= asum;
    }
    return 0;
}

/* Adjoint of orp_composite_fwd for upstream grad_out (npix, D): grad_dists
 * (npix, K) (0 on empty slots) and grad_features (P, D) (accumulated, the
 * caller zeroes it).  grad_features_abs and grad_dists_abs (either may be
 * NULL) receive the magnitudes of the terms that form each component. */
int orp_composite_bwd(int64_t npix, int64_t K, const int64_t *idx, const double *dists, const double *features,
                      int64_t D, double radius, int mode, const double *grad_out, double *grad_dists,
                      double *grad_features, double *grad_features_abs, double *grad_dists_abs) {
    const double r2 = radius * radius;
    double *a = (double *)malloc(sizeof(double) * (size_t)K);
    double *T = (double *)malloc(sizeof(double) * (size_t)K);
    double *S = (double *)malloc(sizeof(double) * (size_t)D);
    double *out = (double *)malloc(sizeof(double) * (size_t)D);
    for (int64_t p = 0; p < npix; p++) {
        const double *g = grad_out + p * D;
        double Tc = 1.0, asum = 0.0;
        for (int64_t c = 0; c < D; c++) out[c] = 0.0;
        for (int64_t k = 0; k < K; k++) {
            const int64_t i = idx[p * K + k];
            grad_dists[p * K + k] = 0.0;
            if (grad_dists_abs) grad_dists_abs[p * K + k] = 0.0;
            if (i < 0) { a[k] = 0.0; T[k] = Tc; continue; }
            a[k] = orp_alpha(dists[p * K + k], radius);
            T[k] = Tc;
            for (int64_t c = 0; c < D; c++) out[c] += a[k] * features[i * D + c];
            Tc *= 1.0 - a[k];
            asum += a[k];
        }
        if (mode == 1) {
            if (!(asum > 0.0)) continue;
            for (int64_t c = 0; c < D; c++) out[c] /= asum;
            /* f = sum a f_i / sum a: df/df_i = a_i / A, df/da_i = (f_i - f) / A */
            for (int64_t k = 0; k < K; k++) {
                const int64_t i = idx[p * K + k];
                if (i < 0) continue;
                double ga = 0.0, gabs = 0.0;
                for (int64_t c = 0; c < D; c++) {
                    const double t = a[k] / asum * g[c];
                    grad_features[i * D + c] += t;
                    if (grad_features_abs) grad_features_abs[i * D + c] += fabs(t);
                    ga += g[c] * (features[i * D + c] - out[c]) / asum;
                    gabs += fabs(g[c]) * (fabs(features[i * D + c]) + fabs(out[c])) / asum;
                }
                grad_dists[p * K + k] = -ga / r2;
                if (grad_dists_abs) grad_dists_abs[p * K + k] = gabs / r2;
            }
        } else {
            /* f = P_k + T_k (a_k f_k + (1 - a_k) S_k), S_k the composite of the slots after
             * k on their own: df/da_k = T_k (f_k - S_k), df/df_k = a_k T_k. */
            for (int64_t c = 0; c < D; c++) S[c] = 0.0;
            for (int64_t k = K - 1; k >= 0; k--) {
                const int64_t i = idx[p * K + k];
                if (i < 0) continue;
                double ga = 0.0, gabs = 0.0;
                for (int64_t c = 0; c < D; c++) {
                    const double fc = features[i * D + c];
                    const double t = a[k] * T[k] * g[c];
                    grad_features[i * D + c] += t;
                    if (grad_features_abs) grad_features_abs[i * D + c] += fabs(t);
                    ga += g[c] * T[k] * (fc - S[c]);
                    gabs += fabs(g[c]) * T[k] * (fabs(fc) + fabs(S[c]));
                    S[c] = a[k] * fc + (1.0 - a[k]) * S[c];
                }
                grad_dists[p * K + k] = -ga / r2;
                if (grad_dists_abs) grad_dists_abs[p * K + k] = gabs / r2;
            }
        }
    }
    free(a);
    free(T);
    free(S);
    free(out);
    return 0;
}

/* Adjoint of orp_rasterize conditioned on idx: dL/dpoints (P, 3) (accumulated;
 * the caller zeroes it) from grad_zbuf and grad_dists (either may be NULL).
 * d = (px - x)^2 + (py - y)^2 with x = f x_v / z_v, y = f y_v / z_v, and
 * zbuf = z_v; view = R (p - C).  grad_points_abs (may be NULL) accumulates
 * the magnitudes of the terms. */
int orp_rast_bwd(const double *points, int64_t P, const int64_t *first, const int64_t *num, int64_t N,
                 const double *cams, int64_t S, int64_t K, const int64_t *idx, const double *grad_zbuf,
                 const double *grad_dists, const int64_t *pixels, int64_t npix, double *grad_points,
                 double *grad_points_abs) {
    (void)first;
    (void)num;
    if (!pixels) npix = N * S * S;
    for (int64_t p = 0; p < npix; p++) {
        int64_t n, r, c;
        if (pixels) { n = pixels[3 * p]; r = pixels[3 * p + 1]; c = pixels[3 * p + 2]; }
        else { n = p / (S * S); r = (p / S) % S; c = p % S; }
        const double *cam = cams + 16 * n;
        const double px = orp_pix(c, S), py = orp_pix(r, S), f = cam[12];
        for (int64_t k = 0; k < K; k++) {
            const int64_t i = idx[p * K + k];
            if (i < 0 || i >= P) continue;
            const double gd = grad_dists ? grad_dists[p * K + k] : 0.0;
            const double gz = grad_zbuf ? grad_zbuf[p * K + k] : 0.0;
            double v[3];
            orp_view(cam, points + 3 * i, v);
            const double x = f * v[0] / v[2], y = f * v[1] / v[2];
            /* dd/dx = -2 (px - x), dd/dy = -2 (py - y) */
            const double gx = gd * -2.0 * (px - x), gy = gd * -2.0 * (py - y);
            /* x = f xv / zv: dx/dxv = f / zv, dx/dzv = -x / zv */
            const double gxv = gx * f / v[2], gyv = gy * f / v[2];
            const double gzv = gz - (gx * x + gy * y) / v[2];
            const double *R = cam;
            for (int j = 0; j < 3; j++) {
                grad_points[3 * i + j] += R[j] * gxv + R[3 + j] * gyv + R[6 + j] * gzv;
                if (grad_points_abs)
                    grad_points_abs[3 * i + j] += fabs(R[j] * gxv) + fabs(R[3 + j] * gyv) +
                                                  fabs(R[6 + j]) * (fabs(gz) + fabs(gx * x / v[2]) +
                                                                    fabs(gy * y / v[2]));
            }
        }
    }
    return 0;
}
