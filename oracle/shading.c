/*
 * FP64 CPU oracle for lit shading of mesh fragments (flat, Gouraud, Phong)
 * followed by the softmax blend (Algorithm 2) or a hard assignment.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links or calls this
 * file; only the tests do.  It shares no code with the CUDA kernels (nor with
 * oracle.c).
 *
 * What it follows (Section 3.2 of the paper, "Shaders"): shaders fetch
 * per-face data by face id, interpolate per-vertex data with the barycentric
 * coordinates, and blend the K fragments of a pixel; flat, Gouraud and Phong
 * shading with per-vertex colours, blended by hard assignment or by softmax.
 * The paper names the models without their formulas; the reading here is the
 * textbook Phong reflection model with one point light:
 *   m = n / |n|, l = (L - x) / |L - x|, v = (E - x) / |E - x|, c = m . l,
 *   r = 2 c m - l, s = r . v,
 *   phi(x, n, a) = a * (ambient + diffuse * max(c, 0))
 *                  + specular * (c > 0 and s > 0 ? s^shininess : 0)
 * with x the surface point, n its normal, a its colour, L the light position
 * and E the camera centre (all in world space).
 *   flat:    n = (P1 - P0) x (P2 - P0), x = sum b_i P_i, a = sum b_i A_i
 *   Gouraud: colour = sum b_i phi(P_i, N_i, A_i)        (lit at the vertices)
 *   Phong:   x = sum b_i P_i, n = sum b_i N_i, a = sum b_i A_i, colour = phi(x, n, a)
 * Softmax blend: Algorithm 2 on the shaded colours (same background term and
 * alpha as the unlit blend).  Hard blend: the nearest fragment's colour (the
 * background where the pixel has none), alpha 1 where covered.
 *
 * Parity pins: tests/test_oracle_shading.py (closed forms of the reflection
 * model, reduction to the unlit blend, finite differences of every adjoint).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* light: L[3], ambient[3], diffuse[3], specular[3], shininess */
typedef struct {
    double L[3], amb[3], dif[3], spec[3], sh;
} ors_light;

static void ors_unpack(const double *lp, ors_light *o) {
    memcpy(o->L, lp, 3 * sizeof(double));
    memcpy(o->amb, lp + 3, 3 * sizeof(double));
    memcpy(o->dif, lp + 6, 3 * sizeof(double));
    memcpy(o->spec, lp + 9, 3 * sizeof(double));
    o->sh = lp[12];
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* phi(x, n, a) and, when g != NULL, its adjoint: gx, gn, ga += d(g . phi)/d(x, n, a) */
static void ors_phi(const ors_light *Lt, const double *E, const double *x, const double *n, const double *a,
                    double out[3], const double *g, double *gx, double *gn, double *ga) {
    double u[3], w[3], m[3], l[3], v[3];
    for (int j = 0; j < 3; j++) { u[j] = Lt->L[j] - x[j]; w[j] = E[j] - x[j]; }
    const double lu = sqrt(dot3(u, u)), lw = sqrt(dot3(w, w)), nn = sqrt(dot3(n, n));
    for (int j = 0; j < 3; j++) { l[j] = u[j] / lu; v[j] = w[j] / lw; m[j] = n[j] / nn; }
    const double c = dot3(m, l);
    const double D = c > 0.0 ? c : 0.0;
    double r[3];
    for (int j = 0; j < 3; j++) r[j] = 2.0 * c * m[j] - l[j];
    const double s = dot3(r, v);
    const int spec_on = c > 0.0 && s > 0.0;
    const double Sp = spec_on ? pow(s, Lt->sh) : 0.0;
    for (int ch = 0; ch < 3; ch++) out[ch] = a[ch] * (Lt->amb[ch] + Lt->dif[ch] * D) + Lt->spec[ch] * Sp;
    if (!g) return;
    double gD = 0.0, gSp = 0.0;
    for (int ch = 0; ch < 3; ch++) {
        ga[ch] += g[ch] * (Lt->amb[ch] + Lt->dif[ch] * D);
        gD += g[ch] * a[ch] * Lt->dif[ch];
        gSp += g[ch] * Lt->spec[ch];
    }
    double gc = c > 0.0 ? gD : 0.0;
    double gm[3] = {0, 0, 0}, gl[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
    if (spec_on) {
        const double gs = gSp * Lt->sh * pow(s, Lt->sh - 1.0);
        /* s = r . v, r = 2 c m - l */
        for (int j = 0; j < 3; j++) {
            gv[j] += gs * r[j];
            gm[j] += 2.0 * c * gs * v[j];
            gl[j] -= gs * v[j];
        }
        gc += 2.0 * gs * dot3(m, v);
    }
    for (int j = 0; j < 3; j++) { gm[j] += gc * l[j]; gl[j] += gc * m[j]; }
    const double mg = dot3(m, gm), lg = dot3(l, gl), vg = dot3(v, gv);
    for (int j = 0; j < 3; j++) {
        gn[j] += (gm[j] - m[j] * mg) / nn;
        gx[j] -= (gl[j] - l[j] * lg) / lu;   /* u = L - x */
        gx[j] -= (gv[j] - v[j] * vg) / lw;   /* w = E - x */
    }
}

/* Shaded colour of slot s (face f, barycentrics b) and, with g != NULL, the
 * adjoint: gb (3), and per corner gP[9], gN[9], gA[9] (accumulated).  agb
 * (3, may be NULL) accumulates the magnitudes of the terms that form gb (an
 * fp32 evaluation of gb carries rounding of that size). */
static void ors_slot_colour(int shading, const ors_light *Lt, const double *E, const double *verts,
                            const double *normals, const double *colors, const int64_t *fv, const double *b,
                            double out[3], const double *g, double *gb, double *gP, double *gN, double *gA,
                            double *agb) {
    const double *P[3], *Nn[3], *A[3];
    for (int i = 0; i < 3; i++) { P[i] = verts + 3 * fv[i]; Nn[i] = normals + 3 * fv[i]; A[i] = colors + 3 * fv[i]; }
    if (shading == 1) {  /* Gouraud */
        out[0] = out[1] = out[2] = 0.0;
        for (int i = 0; i < 3; i++) {
            double phi[3], gi[3];
            if (g) for (int ch = 0; ch < 3; ch++) gi[ch] = b[i] * g[ch];
            ors_phi(Lt, E, P[i], Nn[i], A[i], phi, g ? gi : NULL, gP + 3 * i, gN + 3 * i, gA + 3 * i);
            for (int ch = 0; ch < 3; ch++) out[ch] += b[i] * phi[ch];
            if (g) gb[i] += dot3(g, phi);
            if (g && agb) agb[i] += fabs(dot3(g, phi));
        }
        return;
    }
    double x[3] = {0, 0, 0}, n[3] = {0, 0, 0}, a[3] = {0, 0, 0};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) { x[j] += b[i] * P[i][j]; a[j] += b[i] * A[i][j]; }
    double e1[3], e2[3];
    if (shading == 2) {  /* Phong */
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) n[j] += b[i] * Nn[i][j];
    } else {             /* flat: the face normal */
        for (int j = 0; j < 3; j++) { e1[j] = P[1][j] - P[0][j]; e2[j] = P[2][j] - P[0][j]; }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    }
    if (!g) {
        ors_phi(Lt, E, x, n, a, out, NULL, NULL, NULL, NULL);
        return;
    }
    double gx[3] = {0, 0, 0}, gn[3] = {0, 0, 0}, ga[3] = {0, 0, 0};
    ors_phi(Lt, E, x, n, a, out, g, gx, gn, ga);
    for (int i = 0; i < 3; i++) {
        gb[i] += dot3(gx, P[i]) + dot3(ga, A[i]);
        if (agb) agb[i] += fabs(dot3(gx, P[i])) + fabs(dot3(ga, A[i]));
        for (int j = 0; j < 3; j++) { gP[3 * i + j] += b[i] * gx[j]; gA[3 * i + j] += b[i] * ga[j]; }
    }
    if (shading == 2) {
        for (int i = 0; i < 3; i++) {
            gb[i] += dot3(gn, Nn[i]);
            if (agb) agb[i] += fabs(dot3(gn, Nn[i]));
            for (int j = 0; j < 3; j++) gN[3 * i + j] += b[i] * gn[j];
        }
    } else {
        /* n = e1 x e2: d/de1 = e2 x gn, d/de2 = gn x e1 */
        const double g1[3] = {e2[1] * gn[2] - e2[2] * gn[1], e2[2] * gn[0] - e2[0] * gn[2], e2[0] * gn[1] - e2[1] * gn[0]};
        const double g2[3] = {gn[1] * e1[2] - gn[2] * e1[1], gn[2] * e1[0] - gn[0] * e1[2], gn[0] * e1[1] - gn[1] * e1[0]};
        for (int j = 0; j < 3; j++) {
            gP[3 + j] += g1[j];
            gP[6 + j] += g2[j];
            gP[j] -= g1[j] + g2[j];
        }
    }
}

static double ors_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* blend: sigma, gamma, znear, zfar, eps, bg[3] (8 doubles) */
/* Shaded RGBA of npix pixels: image[p] = n of pixel p (selects the camera
 * centre E = cams[16 n + 9 .. 11]).  blend 0: softmax (Algorithm 2, alpha of
 * Algorithm 1); 1: hard.  Fragments (npix, K[, 3]) as from the rasterizer. */
int ors_shade_fwd(int64_t npix, int64_t K, const int64_t *image, const int64_t *p2f, const double *zbuf,
                  const double *bary, const double *dists, const int64_t *faces, const double *verts,
                  const double *normals, const double *colors, const double *cams, const double *light,
                  const double *blend, int shading, int blend_mode, double *rgba) {
    ors_light Lt;
    ors_unpack(light, &Lt);
    const double sigma = blend[0], gamma = blend[1], znear = blend[2], zfar = blend[3], eps = blend[4];
    const double *bg = blend + 5;
    for (int64_t p = 0; p < npix; p++) {
        const double *E = cams + 16 * image[p] + 9;
        double *o = rgba + 4 * p;
        if (blend_mode == 1) {
            const int64_t f = p2f[p * K];
            if (f < 0) {
                o[0] = bg[0]; o[1] = bg[1]; o[2] = bg[2]; o[3] = 0.0;
            } else {
                ors_slot_colour(shading, &Lt, E, verts, normals, colors, faces + 3 * f, bary + 3 * p * K, o,
                                NULL, NULL, NULL, NULL, NULL, NULL);
                o[3] = 1.0;
            }
            continue;
        }
        double keep = 1.0, zmax = eps;
        for (int64_t k = 0; k < K; k++) {
            const int64_t s = p * K + k;
            if (p2f[s] < 0) continue;
            keep *= ors_sigmoid(dists[s] / sigma);
            const double zi = (zfar - zbuf[s]) / (zfar - znear);
            if (zi > zmax) zmax = zi;
        }
        double num[3] = {0, 0, 0}, den = 0.0;
        for (int64_t k = 0; k < K; k++) {
            const int64_t s = p * K + k;
            const int64_t f = p2f[s];
            if (f < 0) continue;
            const double w = ors_sigmoid(-dists[s] / sigma) * exp(((zfar - zbuf[s]) / (zfar - znear) - zmax) / gamma);
            double c[3];
            ors_slot_colour(shading, &Lt, E, verts, normals, colors, faces + 3 * f, bary + 3 * s, c, NULL, NULL,
                            NULL, NULL, NULL, NULL);
            for (int ch = 0; ch < 3; ch++) num[ch] += w * c[ch];
            den += w;
        }
        const double delta = exp((eps - zmax) / gamma);
        for (int ch = 0; ch < 3; ch++) o[ch] = (num[ch] + delta * bg[ch]) / (den + delta);
        o[3] = 1.0 - keep;
    }
    return 0;
}

/* Adjoint of ors_shade_fwd for grad_rgba (npix, 4).  grad_zbuf, grad_dists
 * (npix, K) and grad_bary (npix, K, 3) are overwritten; grad_verts (the
 * direct dependence of the lighting on positions), grad_normals and
 * grad_colors (V, 3) are accumulated (the caller zeroes them).  abs_vnc (may
 * be NULL; 3 x V x 3: verts, normals, colours) accumulates the magnitudes of
 * the per-slot contributions to those sums. */
static void ors_scatter(const int64_t *fv, const double *gP, const double *gN, const double *gA, double *grad_verts,
                        double *grad_normals, double *grad_colors, double *abs_vnc, int64_t V) {
    for (int i = 0; i < 3; i++) {
        const int64_t vi = fv[i];
        for (int j = 0; j < 3; j++) {
            grad_verts[3 * vi + j] += gP[3 * i + j];
            grad_normals[3 * vi + j] += gN[3 * i + j];
            grad_colors[3 * vi + j] += gA[3 * i + j];
            if (abs_vnc) {
                abs_vnc[3 * vi + j] += fabs(gP[3 * i + j]);
                abs_vnc[3 * V + 3 * vi + j] += fabs(gN[3 * i + j]);
                abs_vnc[6 * V + 3 * vi + j] += fabs(gA[3 * i + j]);
            }
        }
    }
}

int ors_shade_bwd(int64_t npix, int64_t K, const int64_t *image, const int64_t *p2f, const double *zbuf,
                  const double *bary, const double *dists, const int64_t *faces, const double *verts,
                  const double *normals, const double *colors, const double *cams, const double *light,
                  const double *blend, int shading, int blend_mode, const double *grad_rgba, double *grad_zbuf,
                  double *grad_bary, double *grad_dists, double *grad_verts, double *grad_normals,
                  double *grad_colors, double *abs_vnc, int64_t V, double *abs_bary) {
    ors_light Lt;
    ors_unpack(light, &Lt);
    const double sigma = blend[0], gamma = blend[1], znear = blend[2], zfar = blend[3], eps = blend[4];
    const double *bg = blend + 5;
    for (int64_t s = 0; s < npix * K; s++) {
        grad_zbuf[s] = grad_dists[s] = 0.0;
        grad_bary[3 * s] = grad_bary[3 * s + 1] = grad_bary[3 * s + 2] = 0.0;
        if (abs_bary) abs_bary[3 * s] = abs_bary[3 * s + 1] = abs_bary[3 * s + 2] = 0.0;
    }
    for (int64_t p = 0; p < npix; p++) {
        const double *E = cams + 16 * image[p] + 9;
        const double *g = grad_rgba + 4 * p;
        double gc_all[64 * 3], cols[64 * 3], wts[64];
        int64_t kk = K > 64 ? 64 : K;
        if (blend_mode == 1) {
            const int64_t f = p2f[p * K];
            if (f < 0) continue;
            double c[3], gP[9] = {0}, gN[9] = {0}, gA[9] = {0};
            ors_slot_colour(shading, &Lt, E, verts, normals, colors, faces + 3 * f, bary + 3 * p * K, c, g,
                            grad_bary + 3 * p * K, gP, gN, gA, abs_bary ? abs_bary + 3 * p * K : NULL);
            ors_scatter(faces + 3 * f, gP, gN, gA, grad_verts, grad_normals, grad_colors, abs_vnc, V);
            continue;
        }
        double keep = 1.0, zmax = eps;
        for (int64_t k = 0; k < kk; k++) {
            const int64_t s = p * K + k;
            if (p2f[s] < 0) continue;
            keep *= ors_sigmoid(dists[s] / sigma);
            const double zi = (zfar - zbuf[s]) / (zfar - znear);
            if (zi > zmax) zmax = zi;
        }
        double den = 0.0, num[3] = {0, 0, 0};
        for (int64_t k = 0; k < kk; k++) {
            const int64_t s = p * K + k;
            const int64_t f = p2f[s];
            wts[k] = 0.0;
            if (f < 0) continue;
            wts[k] = ors_sigmoid(-dists[s] / sigma) * exp(((zfar - zbuf[s]) / (zfar - znear) - zmax) / gamma);
            ors_slot_colour(shading, &Lt, E, verts, normals, colors, faces + 3 * f, bary + 3 * s, cols + 3 * k,
                            NULL, NULL, NULL, NULL, NULL, NULL);
            for (int ch = 0; ch < 3; ch++) num[ch] += wts[k] * cols[3 * k + ch];
            den += wts[k];
        }
        const double delta = exp((eps - zmax) / gamma), D = den + delta;
        double rgb[3];
        for (int ch = 0; ch < 3; ch++) rgb[ch] = (num[ch] + delta * bg[ch]) / D;
        for (int64_t k = 0; k < kk; k++) {
            const int64_t s = p * K + k;
            const int64_t f = p2f[s];
            if (f < 0) continue;
            const double prob = ors_sigmoid(-dists[s] / sigma);
            /* alpha = 1 - prod(1 - prob): d/d dists_k = -prob_k keep / sigma */
            double gd = g[3] * (-prob * keep / sigma);
            /* rgb = (sum w c + delta bg) / D: dw_k -> (c_k - rgb) / D; dc_k -> w_k / D */
            const double gw = (g[0] * (cols[3 * k] - rgb[0]) + g[1] * (cols[3 * k + 1] - rgb[1]) +
                               g[2] * (cols[3 * k + 2] - rgb[2])) / D;
            const double E_k = wts[k] / prob;
            gd += gw * E_k * (-prob * (1.0 - prob) / sigma);
            grad_dists[s] = gd;
            grad_zbuf[s] = gw * wts[k] / gamma * (-1.0 / (zfar - znear));
            for (int ch = 0; ch < 3; ch++) gc_all[3 * k + ch] = g[ch] * wts[k] / D;
            double c[3], gP[9] = {0}, gN[9] = {0}, gA[9] = {0};
            ors_slot_colour(shading, &Lt, E, verts, normals, colors, faces + 3 * f, bary + 3 * s, c, gc_all + 3 * k,
                            grad_bary + 3 * s, gP, gN, gA, abs_bary ? abs_bary + 3 * s : NULL);
            ors_scatter(faces + 3 * f, gP, gN, gA, grad_verts, grad_normals, grad_colors, abs_vnc, V);
        }
    }
    return 0;
}

/* Kink margins of the reflection model: for each pixel, the smallest of |c|
 * (the diffuse and specular terms switch on at c = 0) and, where c > 0, |s|
 * (the specular term switches on at s = 0), over every evaluation of phi the
 * pixel's blend uses (one per slot, three per slot for Gouraud; slot 0 only
 * for the hard blend).  Gradients are discontinuous there. */
static double ors_phi_margin(const ors_light *Lt, const double *E, const double *x, const double *n) {
    double u[3], w[3], m[3], l[3], v[3];
    for (int j = 0; j < 3; j++) { u[j] = Lt->L[j] - x[j]; w[j] = E[j] - x[j]; }
    const double lu = sqrt(dot3(u, u)), lw = sqrt(dot3(w, w)), nn = sqrt(dot3(n, n));
    for (int j = 0; j < 3; j++) { l[j] = u[j] / lu; v[j] = w[j] / lw; m[j] = n[j] / nn; }
    const double c = dot3(m, l);
    double r[3];
    for (int j = 0; j < 3; j++) r[j] = 2.0 * c * m[j] - l[j];
    const double sv = dot3(r, v);
    double mg = fabs(c);
    if (c > 0.0 && fabs(sv) < mg) mg = fabs(sv);
    return mg;
}

int ors_shade_margins(int64_t npix, int64_t K, const int64_t *image, const int64_t *p2f, const double *bary,
                      const int64_t *faces, const double *verts, const double *normals, const double *cams,
                      const double *light, int shading, int blend_mode, double *margin) {
    ors_light Lt;
    ors_unpack(light, &Lt);
    for (int64_t p = 0; p < npix; p++) {
        const double *E = cams + 16 * image[p] + 9;
        double mg = 1e300;
        const int64_t kk = blend_mode == 1 ? 1 : K;
        for (int64_t k = 0; k < kk; k++) {
            const int64_t s = p * K + k;
            const int64_t f = p2f[s];
            if (f < 0) continue;
            const int64_t *fv = faces + 3 * f;
            const double *b = bary + 3 * s;
            const double *P[3] = {verts + 3 * fv[0], verts + 3 * fv[1], verts + 3 * fv[2]};
            const double *Nn[3] = {normals + 3 * fv[0], normals + 3 * fv[1], normals + 3 * fv[2]};
            if (shading == 1) {
                for (int i = 0; i < 3; i++) {
                    const double m1 = ors_phi_margin(&Lt, E, P[i], Nn[i]);
                    if (m1 < mg) mg = m1;
                }
                continue;
            }
            double x[3] = {0, 0, 0}, n[3] = {0, 0, 0};
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) x[j] += b[i] * P[i][j];
            if (shading == 2) {
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) n[j] += b[i] * Nn[i][j];
            } else {
                double e1[3], e2[3];
                for (int j = 0; j < 3; j++) { e1[j] = P[1][j] - P[0][j]; e2[j] = P[2][j] - P[0][j]; }
                n[0] = e1[1] * e2[2] - e1[2] * e2[1];
                n[1] = e1[2] * e2[0] - e1[0] * e2[2];
                n[2] = e1[0] * e2[1] - e1[1] * e2[0];
            }
            const double m1 = ors_phi_margin(&Lt, E, x, n);
            if (m1 < mg) mg = m1;
        }
        margin[p] = mg;
    }
    return 0;
}
