/*
 * FP64 CPU oracle for the packed-mesh rasterizer and its soft blends.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links or calls this
 * file; only the tests, the package's smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code with the CUDA kernels.
 *
 * It is deliberately plain: every pixel is compared with every face of its
 * mesh, every candidate is kept, the candidates are sorted, and the gradients
 * are a hand-written adjoint of the same FP64 formulas.  Inputs are upcast to
 * double by the caller.
 *
 * What each function follows (Section 3.2 of the paper, "Differentiable mesh
 * renderer"):
 *   - world -> view -> NDC camera transform ("Rasterizer": the camera maps
 *     meshes from world to view coordinates, perspective cameras);
 *   - K nearest faces along z per pixel, found by a per-pixel priority queue
 *     in the paper; here: all candidates, sorted by (z, face id);
 *   - Fragment data: face id, barycentric coordinates, z distance and signed
 *     xy distance of the pixel to the face;
 *   - faces influence a pixel inside the face and, softened, within a blur
 *     radius outside it (following the SoftRas relaxation the paper adopts);
 *   - coarse binning into image tiles (two-pass approach, Laine & Karras);
 *   - Algorithm 1 (silhouette blending) and Algorithm 2 (softmax blending).
 * Conventions the paper leaves open (NDC axes, pixel centres, units of the
 * distance, culling, the background term of the softmax blend) follow one
 * documented reading; each is restated at the function that applies it.
 *
 * Parity pins: every function here is checked in tests/test_oracle_*.py
 * against closed forms, brute force, linear-algebra solves or central
 * finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CULL_AREA 1e-12

/* ---------------------------------------------------------------------- */
/* camera: world -> view -> NDC                                            */
/* ---------------------------------------------------------------------- */
/* cam row (16 doubles): R (3x3 row-major, world->view), C (centre), f, znear.
 * p_view = R (p_world - C);  x_ndc = f x/z,  y_ndc = f y/z,  depth = z_view. */
static void orc_project(const double *cam, const double *pw, double out[3]) {
    const double *R = cam, *C = cam + 9;
    double d0 = pw[0] - C[0], d1 = pw[1] - C[1], d2 = pw[2] - C[2];
    double x = R[0] * d0 + R[1] * d1 + R[2] * d2;
    double y = R[3] * d0 + R[4] * d1 + R[5] * d2;
    double z = R[6] * d0 + R[7] * d1 + R[8] * d2;
    double f = cam[12];
    out[0] = f * x / z;
    out[1] = f * y / z;
    out[2] = z;
}

static void orc_view(const double *cam, const double *pw, double out[3]) {
    const double *R = cam, *C = cam + 9;
    double d0 = pw[0] - C[0], d1 = pw[1] - C[1], d2 = pw[2] - C[2];
    out[0] = R[0] * d0 + R[1] * d1 + R[2] * d2;
    out[1] = R[3] * d0 + R[4] * d1 + R[5] * d2;
    out[2] = R[6] * d0 + R[7] * d1 + R[8] * d2;
}

/* Pixel (row r, col c) of an S x S image has its centre at
 * (1 - (2c+1)/S, 1 - (2r+1)/S): row 0 is the top, col 0 the left, +X left. */
static double orc_pix(int64_t i, int64_t S) { return 1.0 - (2.0 * (double)i + 1.0) / (double)S; }

/* ---------------------------------------------------------------------- */
/* one face against one pixel                                              */
/* ---------------------------------------------------------------------- */
typedef struct {
    double P[3][3];     /* corners: x_ndc, y_ndc, z_view */
    double A;           /* signed double area in NDC */
    int culled;
} orc_face;

/* Corners of face f under camera cam.  Culled when any corner is nearer than
 * znear or the NDC double area is below 1e-12 in magnitude; both windings are
 * kept (no back-face culling). */
static void orc_setup_face(const double *verts, int64_t V, const int64_t *faces, int64_t f,
                           const double *cam, orc_face *F) {
    F->culled = 0;
    for (int i = 0; i < 3; i++) {
        int64_t vi = faces[3 * f + i];
        if (vi < 0 || vi >= V) { F->culled = 1; return; }
        orc_project(cam, verts + 3 * vi, F->P[i]);
    }
    double znear = cam[13];
    for (int i = 0; i < 3; i++)
        if (!(F->P[i][2] >= znear)) F->culled = 1;
    F->A = (F->P[1][0] - F->P[0][0]) * (F->P[2][1] - F->P[0][1]) -
           (F->P[1][1] - F->P[0][1]) * (F->P[2][0] - F->P[0][0]);
    if (!(fabs(F->A) >= ORC_CULL_AREA)) F->culled = 1;
}

/* e(p; a, b) = (x_b - x_a)(y_p - y_a) - (y_b - y_a)(x_p - x_a) */
static double orc_edge(const double *a, const double *b, double px, double py) {
    return (b[0] - a[0]) * (py - a[1]) - (b[1] - a[1]) * (px - a[0]);
}

/* squared distance from p to segment ab; *t_out gets the clamped parameter */
static double orc_seg_dist2(const double *a, const double *b, double px, double py, double *t_out) {
    double ex = b[0] - a[0], ey = b[1] - a[1];
    double l2 = ex * ex + ey * ey;
    double t = 0.0;
    if (l2 > 0.0) t = ((px - a[0]) * ex + (py - a[1]) * ey) / l2;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double rx = px - (a[0] + t * ex), ry = py - (a[1] + t * ey);
    if (t_out) *t_out = t;
    return rx * rx + ry * ry;
}

typedef struct {
    double b[3];        /* screen barycentrics */
    double bt[3];       /* after perspective correction */
    double bp[3];       /* final (after clipping) */
    double z;           /* depth */
    double s;           /* squared distance to the nearest edge segment */
    double d;           /* signed: -s inside, +s outside */
    int inside;
    int edge;           /* nearest edge: 0 = v0v1, 1 = v1v2, 2 = v2v0 */
    double t;           /* segment parameter on that edge */
    double s_all[3];
    double t_all[3];
    int candidate;
} orc_frag;

/* Fragment of face F at pixel (px, py).
 *   b0 = e(p; v1, v2)/A, b1 = e(p; v2, v0)/A, b2 = e(p; v0, v1)/A; inside iff min b >= 0.
 *   s  = min over the segments (v0v1, v1v2, v2v0) of the squared distance; d = -s inside, +s outside.
 *   perspective correction: b~_i = (b_i/z_i) / sum_j (b_j/z_j)
 *   clipping (after perspective correction): b'_i = max(b~_i, 0) / sum_j max(b~_j, 0)
 *   z = sum_i b'_i z_i.
 * Candidate iff (inside or (blur > 0 and d < blur)) and z is finite and >= znear. */
static void orc_fragment(const orc_face *F, double px, double py, double blur, int persp, int clip,
                         double znear, orc_frag *o) {
    const double *v0 = F->P[0], *v1 = F->P[1], *v2 = F->P[2];
    o->b[0] = orc_edge(v1, v2, px, py) / F->A;
    o->b[1] = orc_edge(v2, v0, px, py) / F->A;
    o->b[2] = orc_edge(v0, v1, px, py) / F->A;
    o->inside = (o->b[0] >= 0.0 && o->b[1] >= 0.0 && o->b[2] >= 0.0);
    double t01, t12, t20;
    o->s_all[0] = orc_seg_dist2(v0, v1, px, py, &t01);
    o->s_all[1] = orc_seg_dist2(v1, v2, px, py, &t12);
    o->s_all[2] = orc_seg_dist2(v2, v0, px, py, &t20);
    o->t_all[0] = t01; o->t_all[1] = t12; o->t_all[2] = t20;
    o->edge = 0; o->s = o->s_all[0]; o->t = t01;
    if (o->s_all[1] < o->s) { o->edge = 1; o->s = o->s_all[1]; o->t = t12; }
    if (o->s_all[2] < o->s) { o->edge = 2; o->s = o->s_all[2]; o->t = t20; }
    o->d = o->inside ? -o->s : o->s;

    if (persp) {
        double t0 = o->b[0] / v0[2], t1 = o->b[1] / v1[2], t2 = o->b[2] / v2[2];
        double T = t0 + t1 + t2;
        o->bt[0] = t0 / T; o->bt[1] = t1 / T; o->bt[2] = t2 / T;
    } else {
        for (int i = 0; i < 3; i++) o->bt[i] = o->b[i];
    }
    if (clip) {
        double c0 = o->bt[0] > 0.0 ? o->bt[0] : 0.0;
        double c1 = o->bt[1] > 0.0 ? o->bt[1] : 0.0;
        double c2 = o->bt[2] > 0.0 ? o->bt[2] : 0.0;
        double cs = c0 + c1 + c2;
        o->bp[0] = c0 / cs; o->bp[1] = c1 / cs; o->bp[2] = c2 / cs;
    } else {
        for (int i = 0; i < 3; i++) o->bp[i] = o->bt[i];
    }
    o->z = o->bp[0] * v0[2] + o->bp[1] * v1[2] + o->bp[2] * v2[2];
    int near = o->inside || (blur > 0.0 && o->d < blur);
    o->candidate = near && isfinite(o->z) && o->z >= znear;
}

/* ---------------------------------------------------------------------- */
/* forward: brute force K nearest                                          */
/* ---------------------------------------------------------------------- */
typedef struct { double z; int64_t f; } orc_key;

static int orc_key_cmp(const void *a, const void *b) {
    const orc_key *x = (const orc_key *)a, *y = (const orc_key *)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    if (x->f < y->f) return -1;
    if (x->f > y->f) return 1;
    return 0;
}

static int orc_mesh_range(const int64_t *first_face, const int64_t *num_faces, int64_t n, int64_t F,
                          int64_t *lo, int64_t *hi) {
    *lo = first_face[n];
    *hi = first_face[n] + num_faces[n];
    if (*lo < 0) *lo = 0;
    if (*hi > F) *hi = F;
    return *hi > *lo;
}

/* All candidates of mesh n at pixel (r, c), sorted by (z, face id).  Returns
 * the number found (may exceed cap; only cap entries are written). */
int64_t orc_pixel_candidates(const double *verts, int64_t V, const int64_t *faces, int64_t F,
                             const int64_t *first_face, const int64_t *num_faces,
                             const double *cams, int64_t S, double blur, int persp, int clip,
                             int64_t n, int64_t r, int64_t c, int64_t *out_faces, double *out_z,
                             int64_t cap) {
    int64_t lo, hi;
    if (!orc_mesh_range(first_face, num_faces, n, F, &lo, &hi)) return 0;
    const double *cam = cams + 16 * n;
    double px = orc_pix(c, S), py = orc_pix(r, S);
    orc_key *keys = (orc_key *)malloc(sizeof(orc_key) * (size_t)(hi - lo));
    int64_t m = 0;
    for (int64_t f = lo; f < hi; f++) {
        orc_face Fc;
        orc_setup_face(verts, V, faces, f, cam, &Fc);
        if (Fc.culled) continue;
        orc_frag o;
        orc_fragment(&Fc, px, py, blur, persp, clip, cam[13], &o);
        if (!o.candidate) continue;
        keys[m].z = o.z; keys[m].f = f; m++;
    }
    qsort(keys, (size_t)m, sizeof(orc_key), orc_key_cmp);
    for (int64_t i = 0; i < m && i < cap; i++) {
        out_faces[i] = keys[i].f;
        if (out_z) out_z[i] = keys[i].z;
    }
    free(keys);
    return m;
}

/* Fragments for P pixels (pixels[p] = (n, row, col)); pixels == NULL means all
 * N*S*S pixels in (n, row, col) order.  Outputs per pixel K slots:
 * pix_to_face (global face id or -1), zbuf, bary (3), dists; empty slots hold -1. */
int orc_rasterize(const double *verts, int64_t V, const int64_t *faces, int64_t F,
                  const int64_t *first_face, const int64_t *num_faces, int64_t N,
                  const double *cams, int64_t S, int64_t K, double blur, int persp, int clip,
                  const int64_t *pixels, int64_t P,
                  int64_t *pix_to_face, double *zbuf, double *bary, double *dists) {
    if (!pixels) P = N * S * S;
    int64_t *cf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(F + 1));
    for (int64_t p = 0; p < P; p++) {
        int64_t n, r, c;
        if (pixels) { n = pixels[3 * p]; r = pixels[3 * p + 1]; c = pixels[3 * p + 2]; }
        else { n = p / (S * S); r = (p / S) % S; c = p % S; }
        int64_t m = orc_pixel_candidates(verts, V, faces, F, first_face, num_faces, cams, S, blur,
                                         persp, clip, n, r, c, cf, NULL, F + 1);
        const double *cam = cams + 16 * n;
        double px = orc_pix(c, S), py = orc_pix(r, S);
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            if (k < m) {
                orc_face Fc;
                orc_setup_face(verts, V, faces, cf[k], cam, &Fc);
                orc_frag o;
                orc_fragment(&Fc, px, py, blur, persp, clip, cam[13], &o);
                pix_to_face[s] = cf[k];
                zbuf[s] = o.z;
                bary[3 * s] = o.bp[0]; bary[3 * s + 1] = o.bp[1]; bary[3 * s + 2] = o.bp[2];
                dists[s] = o.d;
            } else {
                pix_to_face[s] = -1;
                zbuf[s] = -1.0;
                bary[3 * s] = bary[3 * s + 1] = bary[3 * s + 2] = -1.0;
                dists[s] = -1.0;
            }
        }
    }
    free(cf);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* margins: pixels whose selection is decided by FP rounding               */
/* ---------------------------------------------------------------------- */
/* Flag bits per pixel (eps in Euclidean NDC units, or z units for depth):
 *  1  blur == 0 and some face's boundary passes within eps of the centre
 *  2  blur  > 0 and some face's blur boundary (distance sqrt(blur)) within eps
 *  4  some face's |A| within eps (relative) of the cull threshold
 *  8  two of the first K+1 sorted candidates have depths within eps
 * 16  some face's corner depth, or a candidate's z, within eps of znear
 * 32  (gradient) a top-K face whose two nearest edge segments are within eps in distance
 *     but reach different points (a shared corner is not a tie)
 * 64  (gradient) a top-K face with a perspective-corrected barycentric within eps of 0 (clip kink)
 * 128 a top-(K+1) candidate outside its face without clipping whose extrapolation is
 *     ill-conditioned: kappa * max(|z|, max_i |b~_i|) > 50, kappa = sum |b_i w_i| / |sum b_i w_i|
 *     with w_i = 1/z_i (perspective) or z_i (affine), so an fp32 evaluation (~1.5e-7 relative
 *     error in the barycentrics) can miss the depth or the barycentrics by more than 1e-5 */
int orc_margins(const double *verts, int64_t V, const int64_t *faces, int64_t F,
                const int64_t *first_face, const int64_t *num_faces, int64_t N,
                const double *cams, int64_t S, int64_t K, double blur, int persp, int clip,
                const int64_t *pixels, int64_t P, double eps, uint8_t *flags) {
    if (!pixels) P = N * S * S;
    int64_t *cf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(F + 1));
    double *cz = (double *)malloc(sizeof(double) * (size_t)(F + 1));
    double rb = sqrt(blur > 0.0 ? blur : 0.0);
    for (int64_t p = 0; p < P; p++) {
        int64_t n, r, c;
        if (pixels) { n = pixels[3 * p]; r = pixels[3 * p + 1]; c = pixels[3 * p + 2]; }
        else { n = p / (S * S); r = (p / S) % S; c = p % S; }
        uint8_t fl = 0;
        const double *cam = cams + 16 * n;
        double px = orc_pix(c, S), py = orc_pix(r, S), znear = cam[13];
        int64_t lo, hi;
        if (orc_mesh_range(first_face, num_faces, n, F, &lo, &hi)) {
            for (int64_t f = lo; f < hi; f++) {
                orc_face Fc;
                orc_setup_face(verts, V, faces, f, cam, &Fc);
                int bad = 0;
                for (int i = 0; i < 3; i++) {
                    int64_t vi = faces[3 * f + i];
                    if (vi < 0 || vi >= V) bad = 1;
                }
                if (bad) continue;
                for (int i = 0; i < 3; i++)
                    if (fabs(Fc.P[i][2] - znear) < eps) fl |= 16;
                if (fabs(fabs(Fc.A) - ORC_CULL_AREA) < eps * ORC_CULL_AREA) fl |= 4;
                if (Fc.culled) continue;
                orc_frag o;
                orc_fragment(&Fc, px, py, blur, persp, clip, znear, &o);
                double dist = sqrt(o.s);
                if (blur == 0.0 && dist < eps) fl |= 1;
                if (blur > 0.0 && !o.inside && fabs(dist - rb) < eps) fl |= 2;
                if (o.candidate && fabs(o.z - znear) < eps) fl |= 16;
            }
            int64_t m = orc_pixel_candidates(verts, V, faces, F, first_face, num_faces, cams, S,
                                             blur, persp, clip, n, r, c, cf, cz, F + 1);
            for (int64_t i = 0; i + 1 < m && i < K; i++)
                if (fabs(cz[i + 1] - cz[i]) < eps) fl |= 8;
            for (int64_t i = 0; i < m && i <= K; i++) {
                if (clip) break;
                orc_face Fc;
                orc_setup_face(verts, V, faces, cf[i], cam, &Fc);
                orc_frag o;
                orc_fragment(&Fc, px, py, blur, persp, clip, znear, &o);
                if (o.inside) continue;
                double num = 0.0, den = 0.0;
                for (int a = 0; a < 3; a++) {
                    double wa = persp ? 1.0 / Fc.P[a][2] : Fc.P[a][2];
                    num += fabs(o.b[a] * wa);
                    den += o.b[a] * wa;
                }
                double mag = fabs(o.z);
                for (int a = 0; a < 3; a++)
                    if (fabs(o.bt[a]) > mag) mag = fabs(o.bt[a]);
                if (num / fabs(den) * mag > 50.0) fl |= 128;
            }
            for (int64_t i = 0; i < m && i < K; i++) {
                orc_face Fc;
                orc_setup_face(verts, V, faces, cf[i], cam, &Fc);
                orc_frag o;
                orc_fragment(&Fc, px, py, blur, persp, clip, znear, &o);
                double dd[3] = {sqrt(o.s_all[0]), sqrt(o.s_all[1]), sqrt(o.s_all[2])};
                double nx[3], ny[3];   /* nearest point on each segment */
                for (int a = 0; a < 3; a++) {
                    const double *pa = Fc.P[a], *pb = Fc.P[(a + 1) % 3];
                    nx[a] = pa[0] + o.t_all[a] * (pb[0] - pa[0]);
                    ny[a] = pa[1] + o.t_all[a] * (pb[1] - pa[1]);
                }
                /* a tie only matters when the tied segments reach different points
                   (two segments meeting at their shared corner give the same gradient) */
                for (int a = 0; a < 3; a++)
                    if (a != o.edge && fabs(dd[a] - dd[o.edge]) < eps &&
                        hypot(nx[a] - nx[o.edge], ny[a] - ny[o.edge]) > eps)
                        fl |= 32;
                if (clip)
                    for (int a = 0; a < 3; a++)
                        if (fabs(o.bt[a]) < eps) fl |= 64;
            }
        }
        flags[p] = fl;
    }
    free(cf);
    free(cz);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* coarse binning                                                          */
/* ---------------------------------------------------------------------- */
/* Face f (of image n) is in bin (n, by, bx) iff its screen bounding box,
 * inflated by r = sqrt(blur) on every side, meets the closed rectangle spanned
 * by the centres of the bin's pixels.  counts has N*nb*nb entries (nb =
 * ceil(S/bin)); when offsets != NULL the lists are also filled (ascending face
 * id within a bin) and amb[j] = 1 marks a membership decided within eps of a
 * boundary. */
int orc_bins(const double *verts, int64_t V, const int64_t *faces, int64_t F,
             const int64_t *first_face, const int64_t *num_faces, int64_t N,
             const double *cams, int64_t S, int64_t bin, double blur, double eps,
             int64_t *counts, const int64_t *offsets, int64_t *lists, uint8_t *amb) {
    int64_t nb = (S + bin - 1) / bin;
    double r = sqrt(blur > 0.0 ? blur : 0.0);
    int64_t *cursor = NULL;
    if (offsets) {
        cursor = (int64_t *)calloc((size_t)(N * nb * nb), sizeof(int64_t));
    } else {
        memset(counts, 0, sizeof(int64_t) * (size_t)(N * nb * nb));
    }
    for (int64_t n = 0; n < N; n++) {
        int64_t lo, hi;
        if (!orc_mesh_range(first_face, num_faces, n, F, &lo, &hi)) continue;
        const double *cam = cams + 16 * n;
        for (int64_t f = lo; f < hi; f++) {
            orc_face Fc;
            orc_setup_face(verts, V, faces, f, cam, &Fc);
            if (Fc.culled) continue;
            double xmin = Fc.P[0][0], xmax = Fc.P[0][0], ymin = Fc.P[0][1], ymax = Fc.P[0][1];
            for (int i = 1; i < 3; i++) {
                if (Fc.P[i][0] < xmin) xmin = Fc.P[i][0];
                if (Fc.P[i][0] > xmax) xmax = Fc.P[i][0];
                if (Fc.P[i][1] < ymin) ymin = Fc.P[i][1];
                if (Fc.P[i][1] > ymax) ymax = Fc.P[i][1];
            }
            xmin -= r; xmax += r; ymin -= r; ymax += r;
            for (int64_t by = 0; by < nb; by++) {
                int64_t r0 = by * bin, r1 = (by + 1) * bin - 1;
                if (r1 > S - 1) r1 = S - 1;
                /* rows go down, y goes down: centres span [pix(r1), pix(r0)] */
                double ylo = orc_pix(r1, S), yhi = orc_pix(r0, S);
                for (int64_t bx = 0; bx < nb; bx++) {
                    int64_t c0 = bx * bin, c1 = (bx + 1) * bin - 1;
                    if (c1 > S - 1) c1 = S - 1;
                    double xlo = orc_pix(c1, S), xhi = orc_pix(c0, S);
                    int in = (xmin <= xhi) && (xmax >= xlo) && (ymin <= yhi) && (ymax >= ylo);
                    int a = fabs(xmin - xhi) < eps || fabs(xmax - xlo) < eps ||
                            fabs(ymin - yhi) < eps || fabs(ymax - ylo) < eps;
                    if (!in) continue;
                    int64_t b = (n * nb + by) * nb + bx;
                    if (offsets) {
                        int64_t j = offsets[b] + cursor[b]++;
                        lists[j] = f;
                        amb[j] = (uint8_t)a;
                    } else {
                        counts[b]++;
                    }
                }
            }
        }
    }
    free(cursor);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* blends (Algorithm 1: silhouette; Algorithm 2: softmax rgb)              */
/* ---------------------------------------------------------------------- */
/* prob = sigmoid(-d/sigma); alpha = 1 - prod_valid (1 - prob).  1 - prob is
 * evaluated as sigmoid(d/sigma), the same number without the cancellation. */
static double orc_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Softmax blend (Algorithm 2), with the background term:
 *   zinv_k   = (zfar - z_k)/(zfar - znear)
 *   zinv_max = max(eps, max_valid zinv_k)
 *   w_k      = prob_k exp((zinv_k - zinv_max)/gamma)
 *   delta    = exp((eps - zinv_max)/gamma)
 *   rgb      = (sum w_k c_k + delta bg) / (sum w_k + delta)
 * with c_k = sum_i b'_{k,i} color[v_i] (per-vertex colours interpolated by the
 * slot's barycentrics).  Only slots with pix_to_face >= 0 take part.
 * mode 0: silhouette only (rgb written as 0); mode 1: rgb + silhouette alpha.
 * rgba: P x 4. */
int orc_blend_fwd(int64_t P, int64_t K, const int64_t *pix_to_face, const double *zbuf,
                  const double *bary, const double *dists, const int64_t *faces,
                  const double *colors, double sigma, double gamma, double znear, double zfar,
                  const double *bg, int mode, double eps, double *rgba) {
    for (int64_t p = 0; p < P; p++) {
        double keep = 1.0;
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            if (pix_to_face[s] < 0) continue;
            keep *= orc_sigmoid(dists[s] / sigma);
        }
        rgba[4 * p + 3] = 1.0 - keep;
        if (mode == 0) {
            rgba[4 * p] = rgba[4 * p + 1] = rgba[4 * p + 2] = 0.0;
            continue;
        }
        double zmax = eps;
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            if (pix_to_face[s] < 0) continue;
            double zi = (zfar - zbuf[s]) / (zfar - znear);
            if (zi > zmax) zmax = zi;
        }
        double num[3] = {0, 0, 0}, den = 0.0;
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            int64_t f = pix_to_face[s];
            if (f < 0) continue;
            double prob = orc_sigmoid(-dists[s] / sigma);
            double zi = (zfar - zbuf[s]) / (zfar - znear);
            double w = prob * exp((zi - zmax) / gamma);
            for (int ch = 0; ch < 3; ch++) {
                double col = 0.0;
                for (int i = 0; i < 3; i++) col += bary[3 * s + i] * colors[3 * faces[3 * f + i] + ch];
                num[ch] += w * col;
            }
            den += w;
        }
        double delta = exp((eps - zmax) / gamma);
        for (int ch = 0; ch < 3; ch++) rgba[4 * p + ch] = (num[ch] + delta * bg[ch]) / (den + delta);
    }
    return 0;
}

/* Adjoint of orc_blend_fwd.  Outputs are overwritten: grad_zbuf, grad_dists
 * (P x K), grad_bary (P x K x 3); grad_colors (V x 3) is ACCUMULATED into
 * (caller zeroes it); grad_colors_abs (optional) accumulates the absolute
 * values of the same contributions (the scale of each sum, for tolerances).
 * slot_abs (optional, P x K x 5: dists, zbuf, bary0..2) receives the same
 * per-slot gradients evaluated with every additive term replaced by its
 * absolute value -- the scale against which their rounding is judged.  zinv_max is treated as a constant: rgb does not depend
 * on it (it cancels between numerator and denominator). */
int orc_blend_bwd(int64_t P, int64_t K, const int64_t *pix_to_face, const double *zbuf,
                  const double *bary, const double *dists, const int64_t *faces,
                  const double *colors, double sigma, double gamma, double znear, double zfar,
                  const double *bg, int mode, double eps, const double *grad_rgba,
                  double *grad_zbuf, double *grad_bary, double *grad_dists, double *grad_colors,
                  double *grad_colors_abs, double *slot_abs) {
    double *q = (double *)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
    for (int64_t p = 0; p < P; p++) {
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            grad_zbuf[s] = 0.0; grad_dists[s] = 0.0;
            grad_bary[3 * s] = grad_bary[3 * s + 1] = grad_bary[3 * s + 2] = 0.0;
            if (slot_abs) for (int j = 0; j < 5; j++) slot_abs[5 * s + j] = 0.0;
            q[k] = (pix_to_face[s] >= 0) ? orc_sigmoid(dists[s] / sigma) : 1.0;   /* 1 - prob */
        }
        /* silhouette: alpha = 1 - prod q_k; d alpha / d prob_k = prod_{j != k} q_j */
        double ga = grad_rgba[4 * p + 3];
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            if (pix_to_face[s] < 0) continue;
            double others = 1.0;
            for (int64_t j = 0; j < K; j++)
                if (j != k) others *= q[j];
            double prob = orc_sigmoid(-dists[s] / sigma);
            /* d prob / d dist = -prob (1 - prob) / sigma */
            grad_dists[s] += ga * others * (-prob * q[k] / sigma);
            if (slot_abs) slot_abs[5 * s] += fabs(ga * others * (-prob * q[k] / sigma));
        }
        if (mode == 0) continue;
        double zmax = eps;
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            if (pix_to_face[s] < 0) continue;
            double zi = (zfar - zbuf[s]) / (zfar - znear);
            if (zi > zmax) zmax = zi;
        }
        double num[3] = {0, 0, 0}, den = 0.0;
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            int64_t f = pix_to_face[s];
            if (f < 0) continue;
            double prob = orc_sigmoid(-dists[s] / sigma);
            double zi = (zfar - zbuf[s]) / (zfar - znear);
            double w = prob * exp((zi - zmax) / gamma);
            for (int ch = 0; ch < 3; ch++) {
                double col = 0.0;
                for (int i = 0; i < 3; i++) col += bary[3 * s + i] * colors[3 * faces[3 * f + i] + ch];
                num[ch] += w * col;
            }
            den += w;
        }
        double delta = exp((eps - zmax) / gamma);
        double D = den + delta;
        double rgb[3];
        for (int ch = 0; ch < 3; ch++) rgb[ch] = (num[ch] + delta * bg[ch]) / D;
        const double *g = grad_rgba + 4 * p;
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            int64_t f = pix_to_face[s];
            if (f < 0) continue;
            double prob = orc_sigmoid(-dists[s] / sigma);
            double zi = (zfar - zbuf[s]) / (zfar - znear);
            double E = exp((zi - zmax) / gamma);
            double w = prob * E;
            double col[3], gw = 0.0, gw_abs = 0.0;
            for (int ch = 0; ch < 3; ch++) {
                col[ch] = 0.0;
                for (int i = 0; i < 3; i++) col[ch] += bary[3 * s + i] * colors[3 * faces[3 * f + i] + ch];
                /* rgb_ch = (sum w c + delta bg)/D: d/dw_k = (c_k - rgb)/D, d/dc_k = w_k/D */
                gw += g[ch] * (col[ch] - rgb[ch]) / D;
                gw_abs += fabs(g[ch]) * (fabs(col[ch]) + fabs(rgb[ch])) / D;
            }
            for (int ch = 0; ch < 3; ch++) {
                double gc = g[ch] * w / D;
                for (int i = 0; i < 3; i++) {
                    int64_t v = faces[3 * f + i];
                    grad_bary[3 * s + i] += gc * colors[3 * v + ch];
                    if (slot_abs) slot_abs[5 * s + 2 + i] += fabs(gc * colors[3 * v + ch]);
                    grad_colors[3 * v + ch] += gc * bary[3 * s + i];
                    if (grad_colors_abs) grad_colors_abs[3 * v + ch] += fabs(gc * bary[3 * s + i]);
                }
            }
            /* w = prob E: d/dprob = E, d/dzinv = w/gamma, dzinv/dz = -1/(zfar - znear) */
            double gprob = gw * E;
            grad_dists[s] += gprob * (-prob * q[k] / sigma);
            grad_zbuf[s] += gw * w / gamma * (-1.0 / (zfar - znear));
            if (slot_abs) {
                slot_abs[5 * s] += gw_abs * E * prob * q[k] / sigma;
                slot_abs[5 * s + 1] += gw_abs * w / gamma / (zfar - znear);
            }
        }
    }
    free(q);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* rasterizer adjoint, conditioned on a given pix_to_face                  */
/* ---------------------------------------------------------------------- */
/* gradient of e(p; a, b) with respect to a, b (2D each) */
static void orc_edge_grad(const double *a, const double *b, double px, double py, double g,
                          double *ga, double *gb) {
    ga[0] += g * (b[1] - py);
    ga[1] += g * (px - b[0]);
    gb[0] += g * (py - a[1]);
    gb[1] += g * (-(px - a[0]));
}

/* For every slot with pix_to_face >= 0: the fragment of that face at that
 * pixel is recomputed in FP64 and dL/d(bary, zbuf, dists) is pulled back
 * through clipping, perspective correction, the edge functions and the
 * segment distance to the three NDC corners, then through the projection
 * Jacobian and R^T to world-space vertex positions.  grad_zbuf, grad_bary,
 * grad_dists may be NULL (zero).  grad_verts (V x 3) is ACCUMULATED into;
 * grad_verts_abs (optional) accumulates, per component, the magnitudes of the terms
 * that the projection Jacobian and R^T combine into each contribution (the scale
 * against which an fp32 evaluation of the sum is judged). */
int orc_rast_bwd(const double *verts, int64_t V, const int64_t *faces, int64_t F,
                 const int64_t *first_face, const int64_t *num_faces, int64_t N,
                 const double *cams, int64_t S, int64_t K, double blur, int persp, int clip,
                 const int64_t *pixels, int64_t P, const int64_t *pix_to_face,
                 const double *grad_zbuf, const double *grad_bary, const double *grad_dists,
                 double *grad_verts, double *grad_verts_abs) {
    (void)first_face; (void)num_faces; (void)F;
    if (!pixels) P = N * S * S;
    for (int64_t p = 0; p < P; p++) {
        int64_t n, r, c;
        if (pixels) { n = pixels[3 * p]; r = pixels[3 * p + 1]; c = pixels[3 * p + 2]; }
        else { n = p / (S * S); r = (p / S) % S; c = p % S; }
        const double *cam = cams + 16 * n;
        double px = orc_pix(c, S), py = orc_pix(r, S);
        for (int64_t k = 0; k < K; k++) {
            int64_t s = p * K + k;
            int64_t f = pix_to_face[s];
            if (f < 0) continue;
            orc_face Fc;
            orc_setup_face(verts, V, faces, f, cam, &Fc);
            if (Fc.culled) continue;
            orc_frag o;
            orc_fragment(&Fc, px, py, blur, persp, clip, cam[13], &o);
            double gz = grad_zbuf ? grad_zbuf[s] : 0.0;
            double gd = grad_dists ? grad_dists[s] : 0.0;
            double gbp[3] = {0, 0, 0};
            if (grad_bary) for (int i = 0; i < 3; i++) gbp[i] = grad_bary[3 * s + i];
            double gP[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};   /* d/d(x_ndc, y_ndc, z) */
            /* z = sum b'_i z_i */
            for (int i = 0; i < 3; i++) {
                gbp[i] += gz * Fc.P[i][2];
                gP[i][2] += gz * o.bp[i];
            }
            /* clipping */
            double gbt[3];
            if (clip) {
                double cs = 0.0;
                for (int i = 0; i < 3; i++) cs += (o.bt[i] > 0.0 ? o.bt[i] : 0.0);
                double dot = gbp[0] * o.bp[0] + gbp[1] * o.bp[1] + gbp[2] * o.bp[2];
                for (int i = 0; i < 3; i++) gbt[i] = (o.bt[i] > 0.0) ? (gbp[i] - dot) / cs : 0.0;
            } else {
                for (int i = 0; i < 3; i++) gbt[i] = gbp[i];
            }
            /* perspective correction */
            double gb[3];
            if (persp) {
                double t[3], T = 0.0;
                for (int i = 0; i < 3; i++) { t[i] = o.b[i] / Fc.P[i][2]; T += t[i]; }
                double dot = gbt[0] * o.bt[0] + gbt[1] * o.bt[1] + gbt[2] * o.bt[2];
                for (int i = 0; i < 3; i++) {
                    double gt = (gbt[i] - dot) / T;
                    gb[i] = gt / Fc.P[i][2];
                    gP[i][2] += -gt * o.b[i] / (Fc.P[i][2] * Fc.P[i][2]);
                }
            } else {
                for (int i = 0; i < 3; i++) gb[i] = gbt[i];
            }
            /* b_i = e_i / A */
            double gA = 0.0, ge[3];
            for (int i = 0; i < 3; i++) { ge[i] = gb[i] / Fc.A; gA += -gb[i] * o.b[i] / Fc.A; }
            double g2[3][2] = {{0, 0}, {0, 0}, {0, 0}};
            orc_edge_grad(Fc.P[1], Fc.P[2], px, py, ge[0], g2[1], g2[2]);
            orc_edge_grad(Fc.P[2], Fc.P[0], px, py, ge[1], g2[2], g2[0]);
            orc_edge_grad(Fc.P[0], Fc.P[1], px, py, ge[2], g2[0], g2[1]);
            /* A = e(v2; v0, v1): its dependence on v2 enters through the "pixel" slot */
            orc_edge_grad(Fc.P[0], Fc.P[1], Fc.P[2][0], Fc.P[2][1], gA, g2[0], g2[1]);
            g2[2][0] += gA * (-(Fc.P[1][1] - Fc.P[0][1]));
            g2[2][1] += gA * (Fc.P[1][0] - Fc.P[0][0]);
            /* distance: s = |p - a - t(b - a)|^2 at the nearest segment */
            double gs = o.inside ? -gd : gd;
            if (gs != 0.0) {
                int ia = o.edge, ib = (o.edge + 1) % 3;
                const double *a = Fc.P[ia], *b = Fc.P[ib];
                double rx = px - (a[0] + o.t * (b[0] - a[0]));
                double ry = py - (a[1] + o.t * (b[1] - a[1]));
                g2[ia][0] += gs * (-2.0 * rx * (1.0 - o.t));
                g2[ia][1] += gs * (-2.0 * ry * (1.0 - o.t));
                g2[ib][0] += gs * (-2.0 * rx * o.t);
                g2[ib][1] += gs * (-2.0 * ry * o.t);
            }
            for (int i = 0; i < 3; i++) { gP[i][0] += g2[i][0]; gP[i][1] += g2[i][1]; }
            /* NDC -> view -> world */
            const double *R = cam;
            double fo = cam[12];
            for (int i = 0; i < 3; i++) {
                int64_t vi = faces[3 * f + i];
                double pv[3];
                orc_view(cam, verts + 3 * vi, pv);
                double gxv = gP[i][0] * fo / pv[2];
                double gyv = gP[i][1] * fo / pv[2];
                double gzv = gP[i][2] - gP[i][0] * fo * pv[0] / (pv[2] * pv[2])
                                      - gP[i][1] * fo * pv[1] / (pv[2] * pv[2]);
                /* magnitudes of the terms combined by the projection Jacobian and R^T */
                double axv = fabs(gxv), ayv = fabs(gyv);
                double azv = fabs(gP[i][2]) + fabs(gP[i][0] * fo * pv[0] / (pv[2] * pv[2])) +
                             fabs(gP[i][1] * fo * pv[1] / (pv[2] * pv[2]));
                for (int j = 0; j < 3; j++) {
                    double c = R[j] * gxv + R[3 + j] * gyv + R[6 + j] * gzv;
                    grad_verts[3 * vi + j] += c;
                    if (grad_verts_abs)
                        grad_verts_abs[3 * vi + j] += fabs(R[j]) * axv + fabs(R[3 + j]) * ayv + fabs(R[6 + j]) * azv;
                }
            }
        }
    }
    return 0;
}
