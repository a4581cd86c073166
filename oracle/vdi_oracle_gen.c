/*
 * vdi_oracle_gen.c -- oracle for VDI generation (Section 3, Eq. 1 with a
 * fixed sensitivity gamma = tau, or the ray-adaptive gamma of Algorithm 3)
 * and for direct volume rendering at the same samples.  TEST INFRASTRUCTURE, NOT PRODUCT (see vdi_oracle.c).
 *
 * Readings where the paper is silent:
 *  - the V_O projection is an OpenGL perspective frustum; the pixel-centre
 *    ray is parameterised by V_O view depth t, so NDC z = P23 / t - P22;
 *  - samples sit at the midpoints of equal world-length intervals of `step`
 *    from the ray's entry into the box (clipped to V_O's near/far planes); the
 *    last partial interval is not sampled;
 *  - the volume fills the box with voxel centres at (index + 1/2) / n and is
 *    interpolated trilinearly (clamp to edge); u8/u16 values are divided by
 *    255/65535;
 *  - the transfer function is piecewise linear between knots; its alpha is
 *    the opacity per length unit u, so a sample of length step gets
 *    a' = 1 - (1 - alpha)^(step/u) (the paper's "length-adjusted opacity");
 *  - a ray stops once its transmittance falls to 2^-12;
 *  - a supersegment stores depth of the front of its first sample interval
 *    and the back of its last, colour chat = composite / composite opacity
 *    and alpha = 1 - (1 - composite opacity)^(u / world length), so that a
 *    render at V_O reproduces the composite exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

int orc__mat_inv(const double *A, double *out);

typedef struct {
    int nx, ny, nz, dtype; /* dtype 0 = u8, 1 = u16, 2 = f32 */
    const void *data;      /* [nz][ny][nx] */
    double bmin[3], bmax[3];
} orc_volume;

#define REAL double
#define SUFFIX _d
#include "gen_body.inc"
#undef REAL
#undef SUFFIX

#define REAL float
#define SUFFIX _f
#include "gen_body.inc"
#undef REAL
#undef SUFFIX

static double pe(const double *m, int r, int c) { return m[c * 4 + r]; }

/* ray constants of the V_O pixel-centre rays, in FP64 */
static int gen_constants(const orc_volume *vol, const float *knots, int nk, const double *view, const double *proj,
                         double tau, double step, double u, gen_consts_d *g) {
    const double *P = proj;
    if (!(pe(P, 3, 0) == 0 && pe(P, 3, 1) == 0 && pe(P, 3, 2) == -1 && pe(P, 3, 3) == 0 && pe(P, 2, 0) == 0 &&
          pe(P, 2, 1) == 0 && pe(P, 0, 1) == 0 && pe(P, 1, 0) == 0 && pe(P, 0, 3) == 0 && pe(P, 1, 3) == 0))
        return 1;
    if (nk < 2 || nk > 16) return 1;
    double Vi[16];
    if (!orc__mat_inv(view, Vi)) return 1;
    double dv0[3] = {pe(P, 0, 2) / pe(P, 0, 0), pe(P, 1, 2) / pe(P, 1, 1), -1.0};
    double dvx[3] = {1.0 / pe(P, 0, 0), 0.0, 0.0}, dvy[3] = {0.0, 1.0 / pe(P, 1, 1), 0.0};
    for (int r = 0; r < 3; r++) {
        g->E[r] = pe(Vi, r, 3) / pe(Vi, 3, 3);
        g->D0[r] = g->Dx[r] = g->Dy[r] = 0.0;
        for (int c = 0; c < 3; c++) {
            g->D0[r] += pe(Vi, r, c) * dv0[c];
            g->Dx[r] += pe(Vi, r, c) * dvx[c];
            g->Dy[r] += pe(Vi, r, c) * dvy[c];
        }
        g->bmin[r] = vol->bmin[r];
        g->bmax[r] = vol->bmax[r];
    }
    g->P22 = pe(P, 2, 2);
    g->P23 = pe(P, 2, 3);
    g->t_near = g->P23 / (g->P22 - 1.0);
    g->t_far = g->P23 / (g->P22 + 1.0);
    g->step = step;
    g->u = u;
    g->tau = tau;
    g->nk = nk;
    for (int k = 0; k < nk; k++) {
        g->kv[k] = knots[k * 5];
        for (int c = 0; c < 4; c++) g->kc[k][c] = knots[k * 5 + 1 + c];
    }
    return 0;
}

static void to_float(const gen_consts_d *d, gen_consts_f *f) {
    for (int r = 0; r < 3; r++) {
        f->E[r] = (float)d->E[r];
        f->D0[r] = (float)d->D0[r];
        f->Dx[r] = (float)d->Dx[r];
        f->Dy[r] = (float)d->Dy[r];
        f->bmin[r] = (float)d->bmin[r];
        f->bmax[r] = (float)d->bmax[r];
    }
    f->t_near = (float)d->t_near;
    f->t_far = (float)d->t_far;
    f->P22 = (float)d->P22;
    f->P23 = (float)d->P23;
    f->step = (float)d->step;
    f->u = (float)d->u;
    f->tau = (float)d->tau;
    f->nk = d->nk;
    for (int k = 0; k < d->nk; k++) {
        f->kv[k] = (float)d->kv[k];
        for (int c = 0; c < 4; c++) f->kc[k][c] = (float)d->kc[k][c];
    }
}

/* mode 0: FP64 arithmetic; mode 1: FP32 arithmetic (IEEE, no contraction).
 * adaptive != 0: each list picks its own gamma by Algorithm 3 (tau unused);
 * tau_out (nullable) receives the gamma each list used. */
ORC_EXPORT int orc_generate(const orc_volume *vol, const float *knots, int nk, const double *view, const double *proj,
                            int w, int h, int ns, double tau, double step, double u, int mode, int adaptive,
                            float *rgba, float *depth, int32_t *counts, float *tau_out, int nthreads) {
    gen_consts_d gd;
    gen_consts_f gf;
    if (gen_constants(vol, knots, nk, view, proj, tau, step, u, &gd)) return 1;
    to_float(&gd, &gf);
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1)
    for (int li = 0; li < w * h; li++) {
        float *rg = rgba + (size_t)li * ns * 4;
        float *dp = depth + (size_t)li * ns * 2;
        for (int j = 0; j < ns; j++) {
            rg[j * 4 + 0] = rg[j * 4 + 1] = rg[j * 4 + 2] = rg[j * 4 + 3] = 0.0f;
            dp[j * 2 + 0] = dp[j * 2 + 1] = INFINITY;
        }
        const int px = li % w, py = li / w;
        int n;
        double t_used = tau;
        if (mode) {
            const float t = adaptive ? adaptive_tau_f(vol, &gf, px, py, w, h, ns) : gf.tau;
            n = gen_list_tau_f(vol, &gf, px, py, w, h, ns, t, rg, dp);
            t_used = t;
        } else {
            const double t = adaptive ? adaptive_tau_d(vol, &gd, px, py, w, h, ns) : gd.tau;
            n = gen_list_tau_d(vol, &gd, px, py, w, h, ns, t, rg, dp);
            t_used = t;
        }
        counts[li] = n;
        if (tau_out) tau_out[li] = (float)t_used;
    }
    return 0;
}

ORC_EXPORT int orc_dvr(const orc_volume *vol, const float *knots, int nk, const double *view, const double *proj,
                       int w, int h, double step, double u, int mode, double *out, uint8_t *flags, int nthreads) {
    gen_consts_d gd;
    gen_consts_f gf;
    if (gen_constants(vol, knots, nk, view, proj, 0.0, step, u, &gd)) return 1;
    to_float(&gd, &gf);
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1)
    for (int li = 0; li < w * h; li++) {
        if (mode)
            dvr_list_f(vol, &gf, li % w, li / w, w, h, out + (size_t)li * 4, flags ? flags + li : NULL);
        else
            dvr_list_d(vol, &gd, li % w, li / w, w, h, out + (size_t)li * 4, flags ? flags + li : NULL);
    }
    return 0;
}
