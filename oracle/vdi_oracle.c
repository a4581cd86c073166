/*
 * vdi_oracle.c -- plain, slow FP64 CPU oracle for VDI raycasting.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes (arXiv 2206.08660, "Efficient Raycasting of Volumetric
 * Depth Images ..."):
 *
 *  A VDI (Section 2.3) stores, for every pixel i of the original view V_O, a
 *  depth-sorted list L_i of supersegments S_ij with front/back depth f_ij,
 *  b_ij and classified colour/opacity.  Depths are V_O NDC z (Section 4.1:
 *  lists are cuboids of a regular w x h grid in V_O's NDC cube, Fig. 3).
 *  The stored alpha is the opacity per length unit u and the stored colour is
 *  premultiplied (C = chat * alpha), so a ray piece of world length l inside
 *  S_ij contributes opacity 1 - (1 - alpha)^(l/u) (Eq. 2) with colour chat.
 *
 *  Rendering from a new view V_N (Section 4) is therefore the exact
 *  front-to-back integral of a piecewise-constant emission-absorption field.
 *  The oracle evaluates that definition directly instead of the paper's
 *  traversal: it collects every ray parameter where the ray crosses a list
 *  boundary or a supersegment face and composites the maximal constant pieces
 *  (orc_render_exact).  Consecutive pieces of one supersegment compose
 *  exactly because (1-a)^l1 (1-a)^l2 = (1-a)^(l1+l2).
 *
 *  Other entry points: brute-force midpoint sampling along the ray
 *  (orc_render_sampled), direct per-list compositing at V_O
 *  (orc_render_direct), the supersegment-count grid of Section 4.3
 *  (orc_grid_*), the ray-subsampled preview D_R of Section 4.4
 *  (orc_render_preview), bilinear upsampling for the image-space preview D_I
 *  (Section 4.4, Fig. 7 caption) and the first-supersegment contract of
 *  Algorithm 2 (orc_first_index).
 *
 * Conventions (readings where the paper is silent):
 *  - matrices are OpenGL column-major double[16], clip = P * V * x_world;
 *  - pixel (px, py) of a W x H image has NDC centre
 *    x = 2 (px + 1/2) / W - 1,  y = 1 - 2 (py + 1/2) / H  (row 0 = top);
 *  - list i = iy * w + ix covers NDC x in [-1 + 2 ix / w, -1 + 2 (ix+1) / w]
 *    and rows from the top;
 *  - a new-view ray runs from V_N's near plane to its far plane and is clipped
 *    to V_O's frustum (-w <= x, y, z <= w in clip space) and the volume box
 *    (Section 4.1, Fig. 2a);
 *  - background is transparent black; output is premultiplied RGBA.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

typedef struct {
    int w, h, ns;
    double view_o[16], proj_o[16];
    double bmin[3], bmax[3];
    double u;              /* opacity length unit (world units) */
    const float *rgba;     /* [h][w][ns][4] premultiplied */
    const float *depth;    /* [h][w][ns][2] NDC z front, back */
    const int32_t *counts; /* [h][w] or NULL: leading slots with finite front depth */
} orc_vdi;

typedef struct {
    double view[16], proj[16];
    int W, H;
} orc_view;

/* ------------------------------------------------------------------ */
/* small linear algebra (column-major)                                 */
/* ------------------------------------------------------------------ */

static double el(const double *m, int r, int c) { return m[c * 4 + r]; }

static void mat_mul(const double *A, const double *B, double *C) {
    double T[16];
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
            double s = 0.0;
            for (int k = 0; k < 4; k++) s += el(A, r, k) * el(B, k, c);
            T[c * 4 + r] = s;
        }
    memcpy(C, T, sizeof T);
}

static void mat_vec(const double *A, const double v[4], double out[4]) {
    for (int r = 0; r < 4; r++) {
        double s = 0.0;
        for (int k = 0; k < 4; k++) s += el(A, r, k) * v[k];
        out[r] = s;
    }
}

/* Gauss-Jordan elimination with partial pivoting; returns 0 if singular. */
int orc__mat_inv(const double *A, double *out);
static int mat_inv(const double *A, double *out) { return orc__mat_inv(A, out); }
int orc__mat_inv(const double *A, double *out) {
    double a[4][8];
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
            a[r][c] = el(A, r, c);
            a[r][c + 4] = (r == c) ? 1.0 : 0.0;
        }
    for (int col = 0; col < 4; col++) {
        int piv = col;
        for (int r = col + 1; r < 4; r++)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return 0;
        if (piv != col)
            for (int c = 0; c < 8; c++) {
                double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        double inv = 1.0 / a[col][col];
        for (int c = 0; c < 8; c++) a[col][c] *= inv;
        for (int r = 0; r < 4; r++) {
            if (r == col) continue;
            double f = a[r][col];
            if (f != 0.0)
                for (int c = 0; c < 8; c++) a[r][c] -= f * a[col][c];
        }
    }
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) out[c * 4 + r] = a[r][c + 4];
    return 1;
}

static int cmp_double(const void *x, const void *y) {
    double a = *(const double *)x, b = *(const double *)y;
    return (a < b) ? -1 : (a > b) ? 1 : 0;
}

/* ------------------------------------------------------------------ */
/* VDI access                                                          */
/* ------------------------------------------------------------------ */

static int list_count(const orc_vdi *V, int i) {
    if (V->counts) return V->counts[i];
    int n = 0;
    while (n < V->ns && isfinite(V->depth[((size_t)i * V->ns + n) * 2])) n++;
    return n;
}
static double seg_f(const orc_vdi *V, int i, int j) { return V->depth[((size_t)i * V->ns + j) * 2 + 0]; }
static double seg_b(const orc_vdi *V, int i, int j) { return V->depth[((size_t)i * V->ns + j) * 2 + 1]; }
static const float *seg_rgba(const orc_vdi *V, int i, int j) { return V->rgba + ((size_t)i * V->ns + j) * 4; }

/* Add the piece with opacity alpha (per unit u) over world length l, Eq. 2. */
static void composite(double acc[4], const float *rgba, double l, double u) {
    double a = rgba[3];
    if (a <= 0.0 || l <= 0.0) return;
    double at = 1.0 - pow(1.0 - a, l / u);
    double T = 1.0 - acc[3];
    for (int c = 0; c < 3; c++) acc[c] += T * ((double)rgba[c] / a) * at;
    acc[3] += T * at;
}

/* ------------------------------------------------------------------ */
/* new-view ray in V_O clip space                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    double a[4], b[4]; /* h(t) = a + t b : V_O clip coordinates, t in [0,1] near->far of V_N */
    double len;        /* world length of the unclipped ray (t from 0 to 1) */
    double t0, t1;     /* clipped parameter range */
} oray;

typedef struct {
    double M[16];    /* P_O V_O */
    double invN[16]; /* inverse(P_N V_N) */
} oview;

static int make_oview(const orc_vdi *V, const orc_view *N, oview *ov) {
    double PV[16];
    mat_mul(V->proj_o, V->view_o, ov->M);
    mat_mul(N->proj, N->view, PV);
    return mat_inv(PV, ov->invN);
}

/* keep the part of [t0,t1] where c0 + t c1 >= 0 */
static void clip_lin(double c0, double c1, double *t0, double *t1) {
    if (c1 > 0.0) {
        double t = -c0 / c1;
        if (t > *t0) *t0 = t;
    } else if (c1 < 0.0) {
        double t = -c0 / c1;
        if (t < *t1) *t1 = t;
    } else if (c0 < 0.0) {
        *t1 = -INFINITY;
    }
}

static int setup_ray(const orc_vdi *V, const oview *ov, double x, double y, oray *r) {
    double qn[4] = {x, y, -1.0, 1.0}, qf[4] = {x, y, 1.0, 1.0}, hn[4], hf[4];
    mat_vec(ov->invN, qn, hn);
    mat_vec(ov->invN, qf, hf);
    double pn[4], d[4];
    for (int k = 0; k < 3; k++) {
        pn[k] = hn[k] / hn[3];
        d[k] = hf[k] / hf[3] - pn[k];
    }
    pn[3] = 1.0;
    d[3] = 0.0;
    mat_vec(ov->M, pn, r->a);
    mat_vec(ov->M, d, r->b);
    r->len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double t0 = 0.0, t1 = 1.0;
    for (int c = 0; c < 3; c++) {
        clip_lin(r->a[3] + r->a[c], r->b[3] + r->b[c], &t0, &t1);
        clip_lin(r->a[3] - r->a[c], r->b[3] - r->b[c], &t0, &t1);
    }
    for (int k = 0; k < 3; k++) {
        clip_lin(pn[k] - V->bmin[k], d[k], &t0, &t1);
        clip_lin(V->bmax[k] - pn[k], -d[k], &t0, &t1);
    }
    r->t0 = t0;
    r->t1 = t1;
    return t0 < t1;
}

static void ndc_at(const oray *r, double t, double p[3]) {
    double w = r->a[3] + t * r->b[3];
    for (int c = 0; c < 3; c++) p[c] = (r->a[c] + t * r->b[c]) / w;
}

/* t where NDC coordinate c equals X (the Moebius map NDC(t) inverted) */
static int cross_t(const oray *r, int c, double X, double *t) {
    double den = r->b[c] - X * r->b[3];
    if (den == 0.0) return 0;
    *t = -(r->a[c] - X * r->a[3]) / den;
    return 1;
}

static void pixel_ndc(int px, int py, int W, int H, double *x, double *y) {
    *x = 2.0 * (px + 0.5) / W - 1.0;
    *y = 1.0 - 2.0 * (py + 0.5) / H;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static double frac_dist(double g) { return fabs(g - floor(g + 0.5)); }

/* grid coordinates of an NDC point: gx in [0,w], gy in [0,h] (rows from the top) */
static void grid_xy(const orc_vdi *V, const double p[3], double *gx, double *gy) {
    *gx = (p[0] + 1.0) * 0.5 * V->w;
    *gy = (1.0 - p[1]) * 0.5 * V->h;
}

/* is the interior grid line nearest to g (lines 1..n-1) closer than eps? */
static int near_interior_line(double g, int n, double eps) {
    double k = floor(g + 0.5);
    if (k <= 0.0 || k >= n) return 0;
    return fabs(g - k) < eps;
}

#define EPS_GRID 2e-3 /* list widths */
#define EPS_Z 2e-6    /* NDC depth */

/* ------------------------------------------------------------------ */
/* O-exact: the render as an exact piecewise-constant integral         */
/* ------------------------------------------------------------------ */

static void exact_pixel(const orc_vdi *V, const oview *ov, double x, double y, double *tb_buf,
                        double *zb_buf, double out[4], int32_t *n_lists, int32_t *n_segs,
                        uint8_t *flag) {
    oray r;
    double acc[4] = {0, 0, 0, 0};
    int nl = 0, nsg = 0, fl = 0;
    if (setup_ray(V, ov, x, y, &r)) {
        double p0[3], p1[3], g0x, g0y, g1x, g1y;
        ndc_at(&r, r.t0, p0);
        ndc_at(&r, r.t1, p1);
        grid_xy(V, p0, &g0x, &g0y);
        grid_xy(V, p1, &g1x, &g1y);
        if (near_interior_line(g0x, V->w, EPS_GRID) || near_interior_line(g0y, V->h, EPS_GRID) ||
            near_interior_line(g1x, V->w, EPS_GRID) || near_interior_line(g1y, V->h, EPS_GRID))
            fl = 1;
        int nb = 0;
        tb_buf[nb++] = r.t0;
        tb_buf[nb++] = r.t1;
        /* list boundaries in x: NDC x = -1 + 2k/w, interior lines crossed */
        double lo = fmin(g0x, g1x), hi = fmax(g0x, g1x);
        for (int k = (int)floor(lo) + 1; k < hi && k < V->w; k++) {
            if (k <= 0 || (double)k <= lo) continue;
            double t;
            if (cross_t(&r, 0, -1.0 + 2.0 * k / V->w, &t) && t > r.t0 && t < r.t1) {
                double p[3], gx, gy;
                ndc_at(&r, t, p);
                grid_xy(V, p, &gx, &gy);
                if (near_interior_line(gy, V->h, EPS_GRID)) fl = 1;
                tb_buf[nb++] = t;
            }
        }
        lo = fmin(g0y, g1y);
        hi = fmax(g0y, g1y);
        for (int k = (int)floor(lo) + 1; k < hi && k < V->h; k++) {
            if (k <= 0 || (double)k <= lo) continue;
            double t;
            if (cross_t(&r, 1, 1.0 - 2.0 * k / V->h, &t) && t > r.t0 && t < r.t1) {
                double p[3], gx, gy;
                ndc_at(&r, t, p);
                grid_xy(V, p, &gx, &gy);
                if (near_interior_line(gx, V->w, EPS_GRID)) fl = 1;
                tb_buf[nb++] = t;
            }
        }
        qsort(tb_buf, nb, sizeof(double), cmp_double);
        for (int q = 0; q + 1 < nb; q++) {
            double ta = tb_buf[q], tb = tb_buf[q + 1];
            if (!(tb > ta)) continue;
            double pm[3], gx, gy, pa[3], pb[3];
            ndc_at(&r, 0.5 * (ta + tb), pm);
            grid_xy(V, pm, &gx, &gy);
            int ix = clampi((int)floor(gx), 0, V->w - 1);
            int iy = clampi((int)floor(gy), 0, V->h - 1);
            int li = iy * V->w + ix;
            int n = list_count(V, li);
            nl++;
            ndc_at(&r, ta, pa);
            ndc_at(&r, tb, pb);
            /* supersegment faces crossed inside this list */
            int nz = 0;
            zb_buf[nz++] = ta;
            zb_buf[nz++] = tb;
            for (int j = 0; j < n; j++) {
                double Z[2] = {seg_f(V, li, j), seg_b(V, li, j)};
                for (int e = 0; e < 2; e++) {
                    if (fabs(Z[e] - pa[2]) < EPS_Z || fabs(Z[e] - pb[2]) < EPS_Z) fl = 1;
                    double t;
                    if (cross_t(&r, 2, Z[e], &t) && t > ta && t < tb) zb_buf[nz++] = t;
                }
            }
            qsort(zb_buf, nz, sizeof(double), cmp_double);
            for (int s = 0; s + 1 < nz; s++) {
                double ua = zb_buf[s], ub = zb_buf[s + 1];
                if (!(ub > ua)) continue;
                double pz[3];
                ndc_at(&r, 0.5 * (ua + ub), pz);
                for (int j = 0; j < n; j++) {
                    if (seg_f(V, li, j) <= pz[2] && pz[2] <= seg_b(V, li, j)) {
                        nsg++;
                        composite(acc, seg_rgba(V, li, j), r.len * (ub - ua), V->u);
                        break;
                    }
                }
            }
        }
    }
    memcpy(out, acc, sizeof acc);
    if (n_lists) *n_lists = nl;
    if (n_segs) *n_segs = nsg;
    if (flag) *flag = (uint8_t)fl;
}

static int pixel_of(const int32_t *pix, int q, int W, int *px, int *py) {
    int idx = pix ? pix[q] : q;
    *px = idx % W;
    *py = idx / W;
    return idx;
}

ORC_EXPORT int orc_render_exact(const orc_vdi *V, const orc_view *N, const int32_t *pix, int npix,
                                double *out, int32_t *n_lists, int32_t *n_segs, uint8_t *flags,
                                int nthreads) {
    oview ov;
    if (!make_oview(V, N, &ov)) return 1;
    if (!pix) npix = N->W * N->H;
    int bufn = V->w + V->h + 8, zbn = 2 * V->ns + 4;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double *tb = malloc(sizeof(double) * bufn);
        double *zb = malloc(sizeof(double) * zbn);
#pragma omp for schedule(dynamic, 64)
        for (int q = 0; q < npix; q++) {
            int px, py;
            pixel_of(pix, q, N->W, &px, &py);
            double x, y;
            pixel_ndc(px, py, N->W, N->H, &x, &y);
            exact_pixel(V, &ov, x, y, tb, zb, out + (size_t)q * 4, n_lists ? n_lists + q : NULL,
                        n_segs ? n_segs + q : NULL, flags ? flags + q : NULL);
        }
        free(tb);
        free(zb);
    }
    return 0;
}

/* The exact render of rays through explicit V_N NDC points (x, y) = xy[2q],
 * xy[2q+1]: a pixel centre moved by a small offset is a ray the rounding of
 * a finite-precision renderer can stand for, so it gives the other valid
 * values of a ray that runs along a list boundary. */
ORC_EXPORT int orc_render_exact_ndc(const orc_vdi *V, const orc_view *N, const double *xy, int n, double *out,
                                    int32_t *n_lists, int32_t *n_segs, uint8_t *flags, int nthreads) {
    oview ov;
    if (!make_oview(V, N, &ov) || !xy) return 1;
    int bufn = V->w + V->h + 8, zbn = 2 * V->ns + 4;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double *tb = malloc(sizeof(double) * bufn);
        double *zb = malloc(sizeof(double) * zbn);
#pragma omp for schedule(dynamic, 64)
        for (int q = 0; q < n; q++)
            exact_pixel(V, &ov, xy[2 * q], xy[2 * q + 1], tb, zb, out + (size_t)q * 4, n_lists ? n_lists + q : NULL,
                        n_segs ? n_segs + q : NULL, flags ? flags + q : NULL);
        free(tb);
        free(zb);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Bytes-touched replay (the roofline numerator's access rule)          */
/*                                                                      */
/* Which VDI values an exact render reads, by the rule the method's    */
/* traversal defines (Section 4.2, Algorithm 2): per list the ray       */
/* passes through with positive length, its depth range (front of the   */
/* first and back of the last supersegment: a ray that meets neither    */
/* reads nothing else there); Algorithm 2's seed probe reads two        */
/* depths (the seed rounded to the odd slot q, so b_{q-1}, b_q for      */
/* depth increasing along the ray; the even slot q and f_q, f_{q+1}     */
/* when it decreases), each binary-search probe one depth (b_mid, or    */
/* f_mid); each supersegment walked its front and back depth; each      */
/* piece of positive length its colour.  The seed is carried from list  */
/* to list (the last supersegment met, else the search's answer); the   */
/* first list has seed 0 when depth increases along the ray and none    */
/* (plain binary search) when it decreases.  Compositing stops once     */
/* transmittance <= 2^-12.  Lists hold nsp slots (N_S rounded up to     */
/* even); slots past a list's count read as +inf.                       */
/*                                                                      */
/* Output: per list li, slot j: depth_mask[(li*nsp + j)*2 + (0 front,   */
/* 1 back)], colour_mask[li*nsp + j], range_mask[li]; the union over    */
/* the rays of pix.  flags[q] marks a ray whose reads turn on a         */
/* decision within rounding distance of a tie (the exact render's       */
/* flags, or a transmittance within 1e-3 of the termination bound).    */
/* ------------------------------------------------------------------ */

static double slot_f(const orc_vdi *V, int li, int j) { return j < list_count(V, li) ? seg_f(V, li, j) : INFINITY; }
static double slot_b(const orc_vdi *V, int li, int j) { return j < list_count(V, li) ? seg_b(V, li, j) : INFINITY; }

ORC_EXPORT int orc_touch_exact(const orc_vdi *V, const orc_view *N, const int32_t *pix, int npix, int nsp,
                               uint8_t *depth_mask, uint8_t *colour_mask, uint8_t *range_mask, uint8_t *flags) {
    oview ov;
    if (!make_oview(V, N, &ov) || nsp < V->ns || (nsp & 1)) return 1;
    if (!pix) npix = N->W * N->H;
    const double T_end = 1.0 / 4096.0;
    double *tb = malloc(sizeof(double) * (V->w + V->h + 8));
    for (int q = 0; q < npix; q++) {
        int px, py;
        pixel_of(pix, q, N->W, &px, &py);
        double x, y;
        pixel_ndc(px, py, N->W, N->H, &x, &y);
        /* the exact render's own flags for this ray */
        double zb_unused[2 * 64 + 4], acc_unused[4];
        uint8_t fl = 0;
        if (V->ns <= 64) exact_pixel(V, &ov, x, y, tb, zb_unused, acc_unused, NULL, NULL, &fl);
        oray r;
        if (setup_ray(V, &ov, x, y, &r)) {
            double p0[3], p1[3], g0x, g0y, g1x, g1y;
            ndc_at(&r, r.t0, p0);
            ndc_at(&r, r.t1, p1);
            grid_xy(V, p0, &g0x, &g0y);
            grid_xy(V, p1, &g1x, &g1y);
            const int inc = p1[2] - p0[2] >= 0.0;
            if (fabs(p1[2] - p0[2]) < 1e-6) fl = 1; /* depth direction itself near a tie */
            /* the ray's pieces in list order, as in the exact render */
            int nb = 0;
            tb[nb++] = r.t0;
            tb[nb++] = r.t1;
            double lo = fmin(g0x, g1x), hi = fmax(g0x, g1x);
            for (int k = (int)floor(lo) + 1; k < hi && k < V->w; k++) {
                double t;
                if (k > 0 && (double)k > lo && cross_t(&r, 0, -1.0 + 2.0 * k / V->w, &t) && t > r.t0 && t < r.t1)
                    tb[nb++] = t;
            }
            lo = fmin(g0y, g1y);
            hi = fmax(g0y, g1y);
            for (int k = (int)floor(lo) + 1; k < hi && k < V->h; k++) {
                double t;
                if (k > 0 && (double)k > lo && cross_t(&r, 1, 1.0 - 2.0 * k / V->h, &t) && t > r.t0 && t < r.t1)
                    tb[nb++] = t;
            }
            qsort(tb, nb, sizeof(double), cmp_double);
            double acc[4] = {0, 0, 0, 0};
            int p = inc ? 0 : -1, done = 0;
            for (int s = 0; s + 1 < nb && !done; s++) {
                double ta = tb[s], tbb = tb[s + 1];
                if (!(tbb > ta)) continue;
                double pm[3], pa[3], pb[3], gx, gy;
                ndc_at(&r, 0.5 * (ta + tbb), pm);
                grid_xy(V, pm, &gx, &gy);
                int li = clampi((int)floor(gy), 0, V->h - 1) * V->w + clampi((int)floor(gx), 0, V->w - 1);
                ndc_at(&r, ta, pa);
                ndc_at(&r, tbb, pb);
                double d_in = pa[2], d_out = pb[2];
                int n = list_count(V, li);
                range_mask[li] = 1;
                double rf = n > 0 ? seg_f(V, li, 0) : INFINITY, rb = n > 0 ? seg_b(V, li, n - 1) : -INFINITY;
                if (fmax(d_in, d_out) < rf || fmin(d_in, d_out) > rb) continue; /* nothing met in this list */
#define MARK_D(j, which) (depth_mask[((size_t)li * nsp + (j)) * 2 + (which)] = 1)
                int first;
                if (inc) {
                    /* first = min{ j : b_j >= d_in } over [0, nsp), nsp if none */
                    int a = 0, b = nsp;
                    if (p >= 0) {
                        int qq = p | 1;
                        if (qq >= nsp) qq = nsp - 1;
                        MARK_D(qq - 1, 1);
                        MARK_D(qq, 1);
                        int ge = (slot_b(V, li, qq) >= d_in) + (slot_b(V, li, qq - 1) >= d_in);
                        if (ge == 1) a = b = qq;
                        else if (ge == 2) { a = 0; b = qq - 1; }
                        else { a = qq + 1; b = nsp; }
                    }
                    while (a < b) {
                        int mid = (a + b) / 2;
                        MARK_D(mid, 1);
                        if (slot_b(V, li, mid) >= d_in) b = mid; else a = mid + 1;
                    }
                    first = a;
                } else {
                    /* first = max{ j : f_j <= d_in } over [0, nsp), -1 if none */
                    int a = -1, b = nsp - 1;
                    if (p >= 0) {
                        int qq = p & ~1;
                        if (qq >= nsp) qq = nsp - 2;
                        MARK_D(qq, 0);
                        MARK_D(qq + 1, 0);
                        int le = (slot_f(V, li, qq) <= d_in) + (slot_f(V, li, qq + 1) <= d_in);
                        if (le == 1) a = b = qq;
                        else if (le == 2) { a = qq + 1; b = nsp - 1; }
                        else { a = -1; b = qq - 1; }
                    }
                    while (a < b) {
                        int mid = (a + b + 1) / 2;
                        MARK_D(mid, 0);
                        if (slot_f(V, li, mid) <= d_in) a = mid; else b = mid - 1;
                    }
                    first = a;
                }
                /* walk the supersegments in the ray's depth order */
                int last = -1;
                for (int j = first; j >= 0 && j < nsp; j += inc ? 1 : -1) {
                    double f = slot_f(V, li, j), b = slot_b(V, li, j);
                    MARK_D(j, 0);
                    MARK_D(j, 1);
                    if (inc ? (f > d_out) : (b < d_out)) break;
                    last = j;
                    /* overlap of [f, b] with the piece's depth range, as ray parameters */
                    double za = inc ? fmax(f, d_in) : fmin(b, d_in), zbb = inc ? fmin(b, d_out) : fmax(f, d_out);
                    if (inc ? (zbb > za) : (zbb < za)) {
                        double tza, tzb;
                        if (!cross_t(&r, 2, za, &tza)) tza = ta;
                        if (!cross_t(&r, 2, zbb, &tzb)) tzb = tbb;
                        tza = fmin(fmax(tza, ta), tbb);
                        tzb = fmin(fmax(tzb, ta), tbb);
                        colour_mask[(size_t)li * nsp + j] = 1;
                        composite(acc, seg_rgba(V, li, j), r.len * fabs(tzb - tza), V->u);
                        double Tr = 1.0 - acc[3];
                        if (fabs(Tr - T_end) < 1e-3 * T_end) fl = 1;
                        if (Tr <= T_end) {
                            done = 1;
                            break;
                        }
                    }
                    if (inc ? (b > d_out) : (f < d_out)) break;
                }
#undef MARK_D
                p = (last >= 0) ? last : first;
                if (p < 0) p = 0;
            }
        }
        if (flags) flags[q] = fl;
    }
    free(tb);
    return 0;
}

/* ------------------------------------------------------------------ */
/* O-sampled: brute-force midpoint sampling at world step ~h           */
/* ------------------------------------------------------------------ */

ORC_EXPORT int orc_render_sampled(const orc_vdi *V, const orc_view *N, double h_world,
                                  const int32_t *pix, int npix, double *out, int nthreads) {
    oview ov;
    if (!make_oview(V, N, &ov) || !(h_world > 0.0)) return 1;
    if (!pix) npix = N->W * N->H;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
    for (int q = 0; q < npix; q++) {
        int px, py;
        pixel_of(pix, q, N->W, &px, &py);
        double x, y, acc[4] = {0, 0, 0, 0};
        pixel_ndc(px, py, N->W, N->H, &x, &y);
        oray r;
        if (setup_ray(V, &ov, x, y, &r)) {
            double L = r.len * (r.t1 - r.t0);
            long K = (long)ceil(L / h_world);
            if (K < 1) K = 1;
            double hs = L / (double)K;
            for (long k = 0; k < K; k++) {
                double t = r.t0 + (r.t1 - r.t0) * ((double)k + 0.5) / (double)K;
                double p[3], gx, gy;
                ndc_at(&r, t, p);
                grid_xy(V, p, &gx, &gy);
                int ix = clampi((int)floor(gx), 0, V->w - 1);
                int iy = clampi((int)floor(gy), 0, V->h - 1);
                int li = iy * V->w + ix, n = list_count(V, li);
                for (int j = 0; j < n; j++)
                    if (seg_f(V, li, j) <= p[2] && p[2] <= seg_b(V, li, j)) {
                        composite(acc, seg_rgba(V, li, j), hs, V->u);
                        break;
                    }
            }
        }
        memcpy(out + (size_t)q * 4, acc, sizeof acc);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* O-direct: render at V_O (W = w, H = h) by compositing each list      */
/* along its own pixel-centre ray, using view-space depth (no traversal) */
/* ------------------------------------------------------------------ */

/* view-space distance in front of the camera of NDC depth Z under projection P */
static double view_depth_of_ndc(const double *P, double Z) {
    /* Z = (P22 ze + P23) / (P32 ze + P33), depth = -ze */
    double ze = (P[3 * 4 + 2] - Z * P[3 * 4 + 3]) / (Z * P[2 * 4 + 3] - P[2 * 4 + 2]);
    return -ze;
}

ORC_EXPORT int orc_render_direct(const orc_vdi *V, double *out) {
    double invP[16], invV[16];
    if (!mat_inv(V->proj_o, invP) || !mat_inv(V->view_o, invV)) return 1;
    for (int iy = 0; iy < V->h; iy++)
        for (int ix = 0; ix < V->w; ix++) {
            double x, y;
            pixel_ndc(ix, iy, V->w, V->h, &x, &y);
            double qn[4] = {x, y, -1, 1}, qf[4] = {x, y, 1, 1}, en[4], ef[4], wn[4], wf[4];
            mat_vec(invP, qn, en);
            mat_vec(invP, qf, ef);
            for (int k = 0; k < 4; k++) {
                en[k] /= (k < 3) ? en[3] : 1.0;
                ef[k] /= (k < 3) ? ef[3] : 1.0;
            }
            en[3] = ef[3] = 1.0;
            mat_vec(invV, en, wn);
            mat_vec(invV, ef, wf);
            double dn = -en[2], df = -ef[2]; /* view depths of the near and far points */
            double dw[3], L = 0.0;
            for (int k = 0; k < 3; k++) {
                dw[k] = wf[k] - wn[k];
                L += dw[k] * dw[k];
            }
            L = sqrt(L);
            /* lambda in [0,1] from near to far point; clip to the box */
            double l0 = 0.0, l1 = 1.0;
            for (int k = 0; k < 3; k++) {
                clip_lin(wn[k] - V->bmin[k], dw[k], &l0, &l1);
                clip_lin(V->bmax[k] - wn[k], -dw[k], &l0, &l1);
            }
            double acc[4] = {0, 0, 0, 0};
            int li = iy * V->w + ix, n = list_count(V, li);
            if (l0 < l1)
                for (int j = 0; j < n; j++) {
                    double la = (view_depth_of_ndc(V->proj_o, seg_f(V, li, j)) - dn) / (df - dn);
                    double lb = (view_depth_of_ndc(V->proj_o, seg_b(V, li, j)) - dn) / (df - dn);
                    la = fmax(la, l0);
                    lb = fmin(lb, l1);
                    if (lb > la) composite(acc, seg_rgba(V, li, j), L * (lb - la), V->u);
                }
            memcpy(out + ((size_t)iy * V->w + ix) * 4, acc, sizeof acc);
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Supersegment-count grid (Section 4.3)                               */
/* cells: T x T lists by nz slabs of equal V_O view-depth extent       */
/* ------------------------------------------------------------------ */

/* Slab edges: view depths near + k (far - near) / nz mapped to NDC z in
 * FP64 and rounded to FP32 (the comparisons against stored FP32 depths are
 * then exact).  The outer edges are forced to -1 and +1. */
ORC_EXPORT int orc_grid_edges(const orc_vdi *V, int nz, float *edges) {
    const double *P = V->proj_o;
    double dn = view_depth_of_ndc(P, -1.0), df = view_depth_of_ndc(P, 1.0);
    for (int k = 0; k <= nz; k++) {
        double d = dn + (df - dn) * (double)k / (double)nz;
        double ze = -d;
        double Z = (P[2 * 4 + 2] * ze + P[3 * 4 + 2]) / (P[2 * 4 + 3] * ze + P[3 * 4 + 3]);
        edges[k] = (float)Z;
    }
    edges[0] = -1.0f;
    edges[nz] = 1.0f;
    return 0;
}

/* does [f,b] overlap slab [zlo, zhi)?  (zero-length pieces: zlo <= f < zhi) */
static int overlaps_slab(float f, float b, float zlo, float zhi) {
    if (f == b) return zlo <= f && f < zhi;
    return f < zhi && b > zlo;
}

ORC_EXPORT int orc_grid_counts(const orc_vdi *V, int T, int nz, uint32_t *grid) {
    float *edges = malloc(sizeof(float) * (nz + 1));
    orc_grid_edges(V, nz, edges);
    int gw = (V->w + T - 1) / T, gh = (V->h + T - 1) / T;
    memset(grid, 0, sizeof(uint32_t) * (size_t)gw * gh * nz);
    for (int iy = 0; iy < V->h; iy++)
        for (int ix = 0; ix < V->w; ix++) {
            int li = iy * V->w + ix, n = list_count(V, li);
            for (int j = 0; j < n; j++) {
                float f = (float)seg_f(V, li, j), b = (float)seg_b(V, li, j);
                for (int k = 0; k < nz; k++)
                    if (overlaps_slab(f, b, edges[k], edges[k + 1]))
                        grid[((size_t)k * gh + iy / T) * gw + ix / T] += 1;
            }
        }
    free(edges);
    return 0;
}

/* ------------------------------------------------------------------ */
/* D_R preview (Section 4.4): per grid cell the ray crosses, place      */
/* n = ceil((c / lists_in_cell) (l_c / dz_cell) / D_R) samples at equal */
/* world spacing; each sample takes the colour of the supersegment that */
/* contains it and opacity corrected by the spacing (Eq. 2).            */
/* ------------------------------------------------------------------ */

#define EPS_SAMPLE_Z 5e-6
#define EPS_COUNT 1e-4

typedef struct {
    int T, nz, gw, gh, d_r;
    const uint32_t *grid;
    const float *edges;
    double dz_cell; /* view-depth extent of one slab */
} preview_grid;

/* Decision number k of a ray (counted in the order the ray meets them) takes
 * its other side when bit k of `alt` is set. */
static int take_other(unsigned alt, int k) { return k < 32 && ((alt >> k) & 1u); }

/* One D_R preview ray through V_N NDC (x, y).  Decisions that sit within
 * rounding distance of a tie are counted in *n_tie: a sample count
 * (c/F)(l_c/dz)/D_R within EPS_COUNT of an integer (other side: the
 * neighbouring count), a sample within EPS_GRID list widths of an interior
 * list boundary (other side: the list across it), a sample within
 * EPS_SAMPLE_Z of a supersegment face of its list (other side: the
 * containment test just across that face).  With alt = 0 every decision is
 * the plain rule.  *flag also marks cell boundaries crossed close together or
 * close to a ray end (pieces of vanishing length; they move the result
 * continuously). */
static void preview_pixel(const orc_vdi *V, const oview *ov, const preview_grid *G, double x, double y,
                          unsigned alt, double *tb, double acc[4], int *n_tie, uint8_t *flag) {
    const int T = G->T, nz = G->nz;
    const float *edges = G->edges;
    int fl = 0, tie = 0;
    acc[0] = acc[1] = acc[2] = acc[3] = 0.0;
    oray r;
    if (setup_ray(V, ov, x, y, &r)) {
        int nb = 0;
        tb[nb++] = r.t0;
        tb[nb++] = r.t1;
        double p0[3], p1[3];
        ndc_at(&r, r.t0, p0);
        ndc_at(&r, r.t1, p1);
        /* cell boundaries in x (every T lists), y (every T rows), z (slab edges) */
        for (int k = 1; k * T < V->w; k++) {
            double X = -1.0 + 2.0 * (k * T) / V->w, t;
            if ((p0[0] - X) * (p1[0] - X) < 0.0 && cross_t(&r, 0, X, &t) && t > r.t0 && t < r.t1) tb[nb++] = t;
        }
        for (int k = 1; k * T < V->h; k++) {
            double Y = 1.0 - 2.0 * (k * T) / V->h, t;
            if ((p0[1] - Y) * (p1[1] - Y) < 0.0 && cross_t(&r, 1, Y, &t) && t > r.t0 && t < r.t1) tb[nb++] = t;
        }
        for (int k = 1; k < nz; k++) {
            double Z = edges[k], t;
            if ((p0[2] - Z) * (p1[2] - Z) < 0.0 && cross_t(&r, 2, Z, &t) && t > r.t0 && t < r.t1) tb[nb++] = t;
        }
        qsort(tb, nb, sizeof(double), cmp_double);
        /* flag: a cell boundary crossing close to another cell boundary */
        for (int s = 0; s < nb; s++) {
            double p[3], gx, gy;
            ndc_at(&r, tb[s], p);
            grid_xy(V, p, &gx, &gy);
            double cx = gx / T, cy = gy / T;
            int nearx = near_interior_line(gx, V->w, EPS_GRID) && frac_dist(cx) * T < EPS_GRID;
            int neary = near_interior_line(gy, V->h, EPS_GRID) && frac_dist(cy) * T < EPS_GRID;
            int nearz = 0;
            for (int k = 1; k < nz; k++)
                if (fabs(p[2] - edges[k]) < EPS_SAMPLE_Z) nearz = 1;
            if (nearx + neary + nearz >= 2) fl = 1;
            if ((s == 0 || s == nb - 1) && (nearx || neary || nearz)) fl = 1;
        }
        for (int s = 0; s + 1 < nb; s++) {
            double ta = tb[s], tbb = tb[s + 1];
            if (!(tbb > ta)) continue;
            double pm[3], gx, gy;
            ndc_at(&r, 0.5 * (ta + tbb), pm);
            grid_xy(V, pm, &gx, &gy);
            int ix = clampi((int)floor(gx), 0, V->w - 1);
            int iy = clampi((int)floor(gy), 0, V->h - 1);
            int cz = 0;
            while (cz + 1 < nz && pm[2] >= edges[cz + 1]) cz++;
            int cx = ix / T, cy = iy / T;
            uint32_t c = G->grid[((size_t)cz * G->gh + cy) * G->gw + cx];
            if (c == 0) continue;
            int fx = ((cx + 1) * T < V->w ? T : V->w - cx * T);
            int fy = ((cy + 1) * T < V->h ? T : V->h - cy * T);
            double lc = r.len * (tbb - ta);
            double want = ((double)c / (double)(fx * fy)) * (lc / G->dz_cell) / (double)G->d_r;
            long n = (long)ceil(want);
            if (fabs(want - floor(want + 0.5)) < EPS_COUNT * fmax(1.0, want)) {
                fl = 1;
                if (take_other(alt, tie++)) {
                    long k = (long)floor(want + 0.5);
                    n = (n == k) ? k + 1 : k;
                }
            }
            if (n < 1) n = 1;
            double spacing = lc / (double)n;
            for (long k = 0; k < n; k++) {
                double t = ta + (tbb - ta) * ((double)k + 0.5) / (double)n;
                double p[3], sx, sy;
                ndc_at(&r, t, p);
                grid_xy(V, p, &sx, &sy);
                int jx = clampi((int)floor(sx), 0, V->w - 1);
                int jy = clampi((int)floor(sy), 0, V->h - 1);
                if (near_interior_line(sx, V->w, EPS_GRID)) {
                    fl = 1;
                    if (take_other(alt, tie++)) {
                        int L = (int)floor(sx + 0.5);
                        jx = (jx >= L) ? L - 1 : L;
                    }
                }
                if (near_interior_line(sy, V->h, EPS_GRID)) {
                    fl = 1;
                    if (take_other(alt, tie++)) {
                        int L = (int)floor(sy + 0.5);
                        jy = (jy >= L) ? L - 1 : L;
                    }
                }
                int li = jy * V->w + jx, nn = list_count(V, li);
                /* the face of this list nearest to the sample, if within EPS_SAMPLE_Z */
                double z = p[2], best = EPS_SAMPLE_Z, face = 0.0;
                int face_kind = -1; /* 0 front, 1 back */
                for (int j = 0; j < nn; j++) {
                    double f = seg_f(V, li, j), b = seg_b(V, li, j);
                    if (fabs(z - f) < best) {
                        best = fabs(z - f);
                        face = f;
                        face_kind = 0;
                    }
                    if (fabs(z - b) < best) {
                        best = fabs(z - b);
                        face = b;
                        face_kind = 1;
                    }
                }
                if (face_kind >= 0) {
                    fl = 1;
                    if (take_other(alt, tie++)) {
                        /* inside a front face means z >= f, inside a back face z <= b */
                        const double step = 1e-12;
                        if (face_kind == 0)
                            z = (z >= face) ? face - step : face + step;
                        else
                            z = (z <= face) ? face + step : face - step;
                    }
                }
                int hit = -1;
                for (int j = 0; j < nn && hit < 0; j++)
                    if (seg_f(V, li, j) <= z && z <= seg_b(V, li, j)) hit = j;
                if (hit >= 0) composite(acc, seg_rgba(V, li, hit), spacing, V->u);
            }
        }
    }
    if (n_tie) *n_tie = tie;
    if (flag) *flag = (uint8_t)fl;
}

static int preview_setup(const orc_vdi *V, int d_r, int T, int nz, const uint32_t *grid, preview_grid *G) {
    if (d_r < 1 || T < 1 || nz < 1 || !grid) return 0;
    float *edges = malloc(sizeof(float) * (nz + 1));
    orc_grid_edges(V, nz, edges);
    G->T = T;
    G->nz = nz;
    G->d_r = d_r;
    G->gw = (V->w + T - 1) / T;
    G->gh = (V->h + T - 1) / T;
    G->grid = grid;
    G->edges = edges;
    double dn = view_depth_of_ndc(V->proj_o, -1.0), df = view_depth_of_ndc(V->proj_o, 1.0);
    G->dz_cell = (df - dn) / nz;
    return 1;
}

/* The D_R preview of every pixel (or of the listed ones), with per-pixel
 * flags for rays that meet a tie (see preview_pixel). */
ORC_EXPORT int orc_render_preview(const orc_vdi *V, const orc_view *N, int d_r, int T, int nz,
                                  const uint32_t *grid, const int32_t *pix, int npix, double *out,
                                  uint8_t *flags, int nthreads) {
    oview ov;
    preview_grid G;
    if (!make_oview(V, N, &ov) || !preview_setup(V, d_r, T, nz, grid, &G)) return 1;
    if (!pix) npix = N->W * N->H;
    int bufn = (V->w / T + V->h / T + nz) + 16;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double *tb = malloc(sizeof(double) * bufn);
#pragma omp for schedule(dynamic, 16)
        for (int q = 0; q < npix; q++) {
            int px, py;
            pixel_of(pix, q, N->W, &px, &py);
            double x, y;
            pixel_ndc(px, py, N->W, N->H, &x, &y);
            preview_pixel(V, &ov, &G, x, y, 0u, tb, out + (size_t)q * 4, NULL, flags ? flags + q : NULL);
        }
        free(tb);
    }
    free((void *)G.edges);
    return 0;
}

/* The D_R preview of the listed pixels with near-tie decisions flipped: pixel
 * q flips the decisions whose bits are set in alt[q]; n_ties[q] returns how
 * many tie decisions its ray met.  Every such result is a valid limit of the
 * preview under rounding (the GPU decides each tie in FP32). */
ORC_EXPORT int orc_render_preview_alt(const orc_vdi *V, const orc_view *N, int d_r, int T, int nz,
                                      const uint32_t *grid, const int32_t *pix, int npix, const uint32_t *alt,
                                      double *out, int32_t *n_ties, int nthreads) {
    oview ov;
    preview_grid G;
    if (!make_oview(V, N, &ov) || !preview_setup(V, d_r, T, nz, grid, &G) || !pix || !alt) return 1;
    int bufn = (V->w / T + V->h / T + nz) + 16;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double *tb = malloc(sizeof(double) * bufn);
#pragma omp for schedule(dynamic, 16)
        for (int q = 0; q < npix; q++) {
            int px, py;
            pixel_of(pix, q, N->W, &px, &py);
            double x, y;
            pixel_ndc(px, py, N->W, N->H, &x, &y);
            int nt = 0;
            preview_pixel(V, &ov, &G, x, y, alt[q], tb, out + (size_t)q * 4, &nt, NULL);
            if (n_ties) n_ties[q] = nt;
        }
        free(tb);
    }
    free((void *)G.edges);
    return 0;
}

/* ------------------------------------------------------------------ */
/* D_I preview: bilinear upsampling with half-pixel centres, clamp to   */
/* edge (Fig. 7 caption: images rendered with fewer rays are upsampled) */
/* ------------------------------------------------------------------ */

ORC_EXPORT void orc_upsample(const double *lo, int w0, int h0, double *hi, int W, int H) {
    for (int Y = 0; Y < H; Y++)
        for (int X = 0; X < W; X++) {
            double u = (X + 0.5) * w0 / (double)W - 0.5;
            double v = (Y + 0.5) * h0 / (double)H - 0.5;
            int i0 = (int)floor(u), j0 = (int)floor(v);
            double fu = u - i0, fv = v - j0;
            int i1 = clampi(i0 + 1, 0, w0 - 1), j1 = clampi(j0 + 1, 0, h0 - 1);
            i0 = clampi(i0, 0, w0 - 1);
            j0 = clampi(j0, 0, h0 - 1);
            for (int c = 0; c < 4; c++) {
                double a = lo[((size_t)j0 * w0 + i0) * 4 + c], b = lo[((size_t)j0 * w0 + i1) * 4 + c];
                double d = lo[((size_t)j1 * w0 + i0) * 4 + c], e = lo[((size_t)j1 * w0 + i1) * 4 + c];
                double top = a + (b - a) * fu, bot = d + (e - d) * fu;
                hi[((size_t)Y * W + X) * 4 + c] = top + (bot - top) * fv;
            }
        }
}

/* ------------------------------------------------------------------ */
/* First supersegment of a list on a ray (Algorithm 2's result, by     */
/* definition): for depth increasing along the ray, the smallest j with */
/* b_j >= d_entry, rejected if f_j > d_exit; for decreasing depth, the  */
/* largest j with f_j <= d_entry, rejected if b_j < d_exit.  -1: none.  */
/* ------------------------------------------------------------------ */

ORC_EXPORT int orc_first_index(const float *f, const float *b, int n, float d_entry, float d_exit,
                               int increasing) {
    if (increasing) {
        for (int j = 0; j < n; j++)
            if (b[j] >= d_entry) return (f[j] > d_exit) ? -1 : j;
        return -1;
    }
    for (int j = n - 1; j >= 0; j--)
        if (f[j] <= d_entry) return (b[j] < d_exit) ? -1 : j;
    return -1;
}
