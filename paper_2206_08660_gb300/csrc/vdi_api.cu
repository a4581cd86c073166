// vdi_api.cu -- host side of the C ABI declared in include/vdi.h: contexts,
// VDI objects, the FP64 per-view constants of the ray setup and the render
// entry points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <mutex>
#include <new>

#include "../../include/vdi.h"
#include "vdi_api_internal.h"
#include "vdi_internal.cuh"
#include "vdi_march.cuh"

#define VDI_API extern "C" __attribute__((visibility("default")))

namespace vdi {

cudaError_t launch_touch(const ViewConsts &c, const DevVdi &v, uint32_t *bm, cudaStream_t st);
cudaError_t launch_upsample(const float4 *lo, int w0, int h0, void *out, int out_fmt, int W, int H,
                            cudaStream_t st);
cudaError_t launch_search(const DevVdi &v, int li, int search, const float *de, const float *dx,
                          const int32_t *seed, const int32_t *inc, int32_t *res, int n, cudaStream_t st);
cudaError_t launch_count_leading(const float *depth, int ns, long long nl, int32_t *counts, cudaStream_t st);
cudaError_t launch_convert(int fmt, const float *rgba, const float *depth, const int32_t *counts, int ns,
                           int nsp, long long nl, float4 *dpair, void *colour, unsigned *err, cudaStream_t st);
cudaError_t launch_grid(const DevVdi &v, uint32_t *grid, cudaStream_t st);
cudaError_t launch_range(const float *depth, const int32_t *counts, int ns, long long nl, float2 *range,
                         cudaStream_t st);
cudaError_t launch_download(const DevVdi &v, int ns, float *rgba, float *depth, int32_t *counts,
                            cudaStream_t st);
cudaError_t launch_count_totals(const uint32_t *lists, const uint32_t *segs, long long n, unsigned long long *totals,
                                int sm_count, cudaStream_t st);

static thread_local char g_err[512];

vdi_status fail(vdi_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

vdi_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky-free error so later calls start clean
    return fail(e == cudaErrorMemoryAllocation ? VDI_ERR_OOM : VDI_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// 4x4 helpers, column-major (element (r, c) at m[c * 4 + r])
// ---------------------------------------------------------------------------
static inline double at(const double *m, int r, int c) { return m[c * 4 + r]; }

void mat4_mul(const double *A, const double *B, double *C) {
    double T[16];
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r)
            T[c * 4 + r] = at(A, r, 0) * at(B, 0, c) + at(A, r, 1) * at(B, 1, c) + at(A, r, 2) * at(B, 2, c) +
                           at(A, r, 3) * at(B, 3, c);
    memcpy(C, T, sizeof T);
}

static double det3(const double *m, int r0, int r1, int r2, int c0, int c1, int c2) {
    return at(m, r0, c0) * (at(m, r1, c1) * at(m, r2, c2) - at(m, r1, c2) * at(m, r2, c1)) -
           at(m, r0, c1) * (at(m, r1, c0) * at(m, r2, c2) - at(m, r1, c2) * at(m, r2, c0)) +
           at(m, r0, c2) * (at(m, r1, c0) * at(m, r2, c1) - at(m, r1, c1) * at(m, r2, c0));
}

// inverse by the adjugate: inv(r, c) = (-1)^(r+c) det(minor without row c, col r) / det
bool mat4_inv(const double *m, double *out) {
    double cof[4][4];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            int rr[3], cc[3], a = 0, b = 0;
            for (int k = 0; k < 4; ++k) {
                if (k != r) rr[a++] = k;
                if (k != c) cc[b++] = k;
            }
            const double d = det3(m, rr[0], rr[1], rr[2], cc[0], cc[1], cc[2]);
            cof[r][c] = ((r + c) & 1) ? -d : d;
        }
    double det = 0.0;
    for (int c = 0; c < 4; ++c) det += at(m, 0, c) * cof[0][c];
    if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) out[c * 4 + r] = cof[c][r] / det;
    return true;
}

static void mat4_apply(const double *m, const double v[4], double o[4]) {
    for (int r = 0; r < 4; ++r) o[r] = at(m, r, 0) * v[0] + at(m, r, 1) * v[1] + at(m, r, 2) * v[2] + at(m, r, 3) * v[3];
}

// view-space distance in front of the camera whose NDC depth under P is Z
double ndc_to_view_depth(const double *P, double Z) {
    return -(at(P, 2, 3) - Z * at(P, 3, 3)) / (Z * at(P, 3, 2) - at(P, 2, 2));
}

static bool finite16(const double *m) {
    for (int k = 0; k < 16; ++k)
        if (!isfinite(m[k])) return false;
    return true;
}

// ---------------------------------------------------------------------------
// layout
// ---------------------------------------------------------------------------
vdi_status check_desc(const vdi_desc *d, vdi_layout *L) {
    if (!d) return fail(VDI_ERR_INVALID_ARG, "desc is NULL");
    if (d->w < 1 || d->h < 1 || d->w > 32768 || d->h > 32768)
        return fail(VDI_ERR_INVALID_ARG, "list grid %dx%d out of range", d->w, d->h);
    if (d->n_s < 1 || d->n_s > kMaxNs) return fail(VDI_ERR_INVALID_ARG, "n_s=%d outside 1..%d", d->n_s, kMaxNs);
    if (d->colour_fmt != VDI_F32 && d->colour_fmt != VDI_F16)
        return fail(VDI_ERR_INVALID_ARG, "colour_fmt=%d", d->colour_fmt);
    if (!(d->length_unit > 0.0) || !isfinite(d->length_unit))
        return fail(VDI_ERR_INVALID_ARG, "length_unit must be positive");
    const int T = d->grid_tile ? d->grid_tile : 8, nz = d->grid_nz ? d->grid_nz : 20;
    if (T < 1 || T > 256 || nz < 1 || nz > kMaxNz)
        return fail(VDI_ERR_INVALID_ARG, "grid_tile=%d grid_nz=%d out of range", T, nz);
    for (int k = 0; k < 3; ++k)
        if (!(d->bbox_min[k] < d->bbox_max[k])) return fail(VDI_ERR_INVALID_ARG, "empty bbox");
    if (!finite16(d->orig.view) || !finite16(d->orig.proj))
        return fail(VDI_ERR_INVALID_ARG, "non-finite V_O matrices");
    const size_t nl = (size_t)d->w * d->h;
    const int nsp = (d->n_s + 1) & ~1;
    if (nl * (size_t)nsp >= ((size_t)1 << 31))
        return fail(VDI_ERR_UNSUPPORTED, "%dx%d lists x %d slots exceed 2^31 slot records", d->w, d->h, nsp);
    L->n_s_stored = nsp;
    L->depth_bytes = nl * nsp * 2 * sizeof(float);
    L->colour_bytes = nl * nsp * (d->colour_fmt == VDI_F32 ? 16 : 8);
    L->grid_w = div_up(d->w, T);
    L->grid_h = div_up(d->h, T);
    L->grid_nz = nz;
    L->grid_bytes = (size_t)L->grid_w * L->grid_h * nz * sizeof(uint32_t);
    L->list_bytes = nl * 2 * sizeof(float) + (size_t)div_up(d->w, kB) * div_up(d->h, kB) * 2 * sizeof(float);
    L->total_bytes = L->depth_bytes + L->colour_bytes + L->grid_bytes + L->list_bytes;
    L->paper_bytes = nl * (size_t)d->n_s * 24;
    return VDI_OK;
}

// slab edges of the count grid: equal V_O view-depth steps between the near
// and far planes (Section 4.3), mapped to NDC z in FP64 and rounded to FP32
void grid_edges(const double *P, int nz, float *edges) {
    const double dn = ndc_to_view_depth(P, -1.0), df = ndc_to_view_depth(P, 1.0);
    for (int k = 0; k <= nz; ++k) {
        const double d = dn + (df - dn) * (double)k / (double)nz;
        const double ze = -d;
        const double Z = (at(P, 2, 2) * ze + at(P, 2, 3)) / (at(P, 3, 2) * ze + at(P, 3, 3));
        edges[k] = (float)Z;
    }
    edges[0] = -1.0f;
    edges[nz] = 1.0f;
}

// ---------------------------------------------------------------------------
// per-view constants of the ray setup (FP64 on the host)
// ---------------------------------------------------------------------------
vdi_status make_view_consts(const vdi_t *v, const vdi_camera *cam, int W, int H, int d_r, ViewConsts *c) {
    if (!cam) return fail(VDI_ERR_INVALID_ARG, "view is NULL");
    if (!finite16(cam->view) || !finite16(cam->proj)) return fail(VDI_ERR_INVALID_ARG, "non-finite V_N matrices");
    double PV[16], Q[16];
    mat4_mul(cam->proj, cam->view, PV);
    if (!mat4_inv(PV, Q)) return fail(VDI_ERR_INVALID_ARG, "V_N projection*view is singular");
    // near/far points of pixel NDC (x, y) are affine in (x, y) when the
    // homogeneous w of the unprojection does not depend on x, y
    const double wscale = fabs(at(Q, 3, 2)) + fabs(at(Q, 3, 3));
    if (fabs(at(Q, 3, 0)) > 1e-12 * wscale || fabs(at(Q, 3, 1)) > 1e-12 * wscale)
        return fail(VDI_ERR_UNSUPPORTED, "V_N projection is neither perspective nor orthographic");
    const double wn = at(Q, 3, 3) - at(Q, 3, 2), wf = at(Q, 3, 3) + at(Q, 3, 2);
    if (!(wn != 0.0) || !(wf != 0.0) || (wn > 0) != (wf > 0))
        return fail(VDI_ERR_INVALID_ARG, "V_N near/far planes are degenerate");
    double O0[3], Ox[3], Oy[3], D0[3], Dx[3], Dy[3];
    for (int k = 0; k < 3; ++k) {
        O0[k] = (at(Q, k, 3) - at(Q, k, 2)) / wn;
        Ox[k] = at(Q, k, 0) / wn;
        Oy[k] = at(Q, k, 1) / wn;
        D0[k] = (at(Q, k, 3) + at(Q, k, 2)) / wf - O0[k];
        Dx[k] = at(Q, k, 0) / wf - Ox[k];
        Dy[k] = at(Q, k, 1) / wf - Oy[k];
    }
    double t_lo = 0.0, t_hi = 1.0;
    int a_aff = 1, b_aff = 1;
    const double *P = cam->proj;
    const bool persp = at(P, 3, 0) == 0.0 && at(P, 3, 1) == 0.0 && at(P, 3, 2) < 0.0 && at(P, 3, 3) == 0.0;
    const bool ortho = at(P, 3, 0) == 0.0 && at(P, 3, 1) == 0.0 && at(P, 3, 2) == 0.0 && at(P, 3, 3) != 0.0;
    if (persp) {
        // p(t) = E + t D(x, y) with the eye E: the near point is E + tau0 D
        double Vi[16];
        if (mat4_inv(cam->view, Vi)) {
            const double E[3] = {at(Vi, 0, 3) / at(Vi, 3, 3), at(Vi, 1, 3) / at(Vi, 3, 3), at(Vi, 2, 3) / at(Vi, 3, 3)};
            const double n = ndc_to_view_depth(P, -1.0), f = ndc_to_view_depth(P, 1.0);
            const double tau0 = n / (f - n);
            double err = 0.0, scale = 0.0;
            for (int k = 0; k < 3; ++k) {
                err = fmax(err, fabs(O0[k] - (E[k] + tau0 * D0[k])));
                err = fmax(err, fabs(Ox[k] - tau0 * Dx[k]));
                err = fmax(err, fabs(Oy[k] - tau0 * Dy[k]));
                scale = fmax(scale, fabs(O0[k]) + fabs(E[k]) + fabs(D0[k]));
            }
            if (isfinite(tau0) && tau0 > 0.0 && err <= 1e-9 * scale) {
                for (int k = 0; k < 3; ++k) {
                    O0[k] = E[k];
                    Ox[k] = Oy[k] = 0.0;
                }
                t_lo = tau0;
                t_hi = tau0 + 1.0;
                a_aff = 0;
            }
        }
    } else if (ortho) {
        double dmax = 0.0, scale = 0.0;
        for (int k = 0; k < 3; ++k) {
            dmax = fmax(dmax, fmax(fabs(Dx[k]), fabs(Dy[k])));
            scale = fmax(scale, fabs(D0[k]));
        }
        if (dmax <= 1e-12 * scale) {
            for (int k = 0; k < 3; ++k) Dx[k] = Dy[k] = 0.0;
            b_aff = 0;
        }
    }
    const double *M = v->M;
    double e0[4] = {O0[0], O0[1], O0[2], 1.0}, ex[4] = {Ox[0], Ox[1], Ox[2], 0.0}, ey[4] = {Oy[0], Oy[1], Oy[2], 0.0};
    double f0[4] = {D0[0], D0[1], D0[2], 0.0}, fx[4] = {Dx[0], Dx[1], Dx[2], 0.0}, fy[4] = {Dy[0], Dy[1], Dy[2], 0.0};
    double A0[4], Ax[4], Ay[4], B0[4], Bx[4], By[4];
    mat4_apply(M, e0, A0);
    mat4_apply(M, ex, Ax);
    mat4_apply(M, ey, Ay);
    mat4_apply(M, f0, B0);
    mat4_apply(M, fx, Bx);
    mat4_apply(M, fy, By);
    // fold the pixel-centre map x = (px + 1/2) 2/W - 1, y = 1 - (py + 1/2) 2/H into
    // affine forms of the integer pixel indices: a = A0' + px Ax' + py Ay'
    const double sx = 2.0 / W, sy = 2.0 / H;
    double a0[4], ax[4], ay[4], b0[4], bx[4], by[4];
    for (int k = 0; k < 4; ++k) {
        a0[k] = A0[k] + (0.5 * sx - 1.0) * Ax[k] + (1.0 - 0.5 * sy) * Ay[k];
        ax[k] = sx * Ax[k];
        ay[k] = -sy * Ay[k];
        b0[k] = B0[k] + (0.5 * sx - 1.0) * Bx[k] + (1.0 - 0.5 * sy) * By[k];
        bx[k] = sx * Bx[k];
        by[k] = -sy * By[k];
        c->A0[k] = (float)a0[k];
        c->Ax[k] = (float)ax[k];
        c->Ay[k] = (float)ay[k];
        c->B0[k] = (float)b0[k];
        c->Bx[k] = (float)bx[k];
        c->By[k] = (float)by[k];
    }
    // homogeneous list-grid coordinates: g_x w = hw (x + w), g_y w = hh (w - y)
    const double hw = 0.5 * v->desc.w, hh = 0.5 * v->desc.h;
    auto to_grid = [&](const double *q, double *g) {
        g[0] = hw * (q[0] + q[3]);
        g[1] = hh * (q[3] - q[1]);
        g[2] = q[3];
    };
    to_grid(a0, c->GA0);
    to_grid(ax, c->GAx);
    to_grid(ay, c->GAy);
    to_grid(b0, c->GB0);
    to_grid(bx, c->GBx);
    to_grid(by, c->GBy);
    c->a_affine = a_aff;
    c->b_affine = b_aff;
    c->frustum_clip = v->box_in_frustum ? 0 : 1;
    // V_N's rays start at V_O's eye when that eye's clip coordinates x, y, w
    // vanish: each ray then has one V_O NDC position and stays in one list
    {
        double bscale = 0.0;
        for (int k = 0; k < 4; ++k) bscale = fmax(bscale, fabs(b0[k]) + fabs(bx[k]) * W + fabs(by[k]) * H);
        c->single_list = (!a_aff && fabs(a0[0]) <= 1e-9 * bscale && fabs(a0[1]) <= 1e-9 * bscale &&
                          fabs(a0[3]) <= 1e-9 * bscale)
                             ? 1
                             : 0;
    }

    for (int k = 0; k < 3; ++k) {
        c->O0[k] = (float)O0[k];
        c->Ox[k] = (float)Ox[k];
        c->Oy[k] = (float)Oy[k];
        c->D0[k] = (float)D0[k];
        c->Dx[k] = (float)Dx[k];
        c->Dy[k] = (float)Dy[k];
        c->bmin[k] = (float)v->desc.bbox_min[k];
        c->bmax[k] = (float)v->desc.bbox_max[k];
    }
    c->t_lo = (float)t_lo;
    c->t_hi = (float)t_hi;
    c->inv_u = (float)(1.0 / v->desc.length_unit);
    c->W = W;
    c->H = H;
    // The pixel rectangle around the image of the box's eight corners under
    // V_N (their convex hull holds every pixel centre whose ray meets the
    // box), widened by a pixel; the whole image when a corner is not in front
    // of the camera.
    c->rx0 = 0;
    c->rx1 = W - 1;
    c->ry0 = 0;
    c->ry1 = H - 1;
    {
        double PV[16];
        mat4_mul(cam->proj, cam->view, PV);
        double xlo = INFINITY, xhi = -INFINITY, ylo = INFINITY, yhi = -INFINITY;
        bool front = true;
        for (int corner = 0; corner < 8 && front; ++corner) {
            const double p[4] = {(corner & 1) ? v->desc.bbox_max[0] : v->desc.bbox_min[0],
                                 (corner & 2) ? v->desc.bbox_max[1] : v->desc.bbox_min[1],
                                 (corner & 4) ? v->desc.bbox_max[2] : v->desc.bbox_min[2], 1.0};
            double q[4];
            mat4_apply(PV, p, q);
            if (!(q[3] > 1e-12)) {
                front = false;
                break;
            }
            const double px = (q[0] / q[3] + 1.0) * 0.5 * W - 0.5, py = (1.0 - q[1] / q[3]) * 0.5 * H - 0.5;
            xlo = fmin(xlo, px);
            xhi = fmax(xhi, px);
            ylo = fmin(ylo, py);
            yhi = fmax(yhi, py);
        }
        if (front && isfinite(xlo) && isfinite(xhi) && isfinite(ylo) && isfinite(yhi)) {
            c->rx0 = (int)fmax(floor(xlo) - 1.0, -1.0);
            c->rx1 = (int)fmin(ceil(xhi) + 1.0, (double)W);
            c->ry0 = (int)fmax(floor(ylo) - 1.0, -1.0);
            c->ry1 = (int)fmin(ceil(yhi) + 1.0, (double)H);
        }
    }
    // the render grid's tiles that meet the rectangle (clamped to the image)
    c->tiles_x = (W + 31) / 32;
    {
        const int x0 = max(c->rx0, 0), x1 = min(c->rx1, W - 1);
        const int y0 = max(c->ry0, 0), y1 = min(c->ry1, H - 1);
        if (x0 <= x1 && y0 <= y1) {
            c->tile_x0 = x0 / 32;
            c->tile_y0 = y0 / 8;
            c->tile_w = x1 / 32 - c->tile_x0 + 1;
            c->tile_h = y1 / 8 - c->tile_y0 + 1;
        } else {
            c->tile_x0 = c->tile_y0 = c->tile_w = c->tile_h = 0;
        }
    }
    c->sx = (float)(2.0 / W);
    c->sy = (float)(2.0 / H);
    c->d_r = d_r;
    c->cell_scale = (float)(v->desc.length_unit / (v->dz_cell * d_r));
    return VDI_OK;
}

}  // namespace vdi

using namespace vdi;

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------

VDI_API const char *vdi_status_str(vdi_status s) {
    switch (s) {
        case VDI_OK: return "VDI_OK";
        case VDI_ERR_INVALID_ARG: return "VDI_ERR_INVALID_ARG";
        case VDI_ERR_OOM: return "VDI_ERR_OOM";
        case VDI_ERR_CUDA: return "VDI_ERR_CUDA";
        case VDI_ERR_UNSORTED: return "VDI_ERR_UNSORTED";
        case VDI_ERR_TIMEOUT: return "VDI_ERR_TIMEOUT";
        case VDI_ERR_BUSY: return "VDI_ERR_BUSY";
        case VDI_ERR_UNSUPPORTED: return "VDI_ERR_UNSUPPORTED";
    }
    return "VDI_ERR_UNKNOWN";
}

VDI_API const char *vdi_last_error_message(void) { return g_err; }

VDI_API vdi_status vdi_ctx_create(int device, vdi_ctx **out) {
    if (!out) return fail(VDI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(VDI_ERR_INVALID_ARG, "device %d of %d", device, n);
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    vdi_ctx *c = new (std::nothrow) vdi_ctx();
    if (!c) return fail(VDI_ERR_OOM, "host allocation");
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if ((e = cudaStreamCreateWithFlags(&c->free_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaStreamCreate");
    }
    // VDIs and server images come from the stream-ordered allocator; keep freed
    // blocks in the pool instead of returning them to the driver at every sync
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return VDI_OK;
}

VDI_API void vdi_ctx_destroy(vdi_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    release_batch_cache(ctx);
    if (ctx->free_stream) {
        cudaStreamSynchronize(ctx->free_stream);
        cudaStreamDestroy(ctx->free_stream);
    }
    delete ctx;
}

VDI_API vdi_status vdi_layout_bytes(const vdi_desc *desc, vdi_layout *out) {
    if (!out) return fail(VDI_ERR_INVALID_ARG, "out is NULL");
    return check_desc(desc, out);
}

VDI_API vdi_status vdi_get_layout(const vdi_t *v, vdi_layout *out) {
    if (!v || !out) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    *out = v->layout;
    return VDI_OK;
}

#define CK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) {                      \
            st_ = cuda_fail(e_, #call);               \
            goto done;                                \
        }                                             \
    } while (0)

namespace vdi {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link against the driver library); null when the driver lacks it
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor maps of the staged one-list path over a VDI's arrays, all as 32-bit
// words: ranges (2 w) x h with 32 x 8-list boxes; depth slot pairs and colour
// records (4 w) x h x planes with boxes of 32 x 8 lists by the staged pairs
// (staged_pairs: FP16 colour) or twice as many slots (FP32 colour).  They
// need 16-byte row strides (w even) and 16-byte aligned arrays; false when a
// condition fails or the driver refuses.
static bool build_tile_maps(const DevVdi &d, TileMaps *m) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || (d.w & 1)) return false;
    const cuuint32_t np = (cuuint32_t)staged_pairs(d.nsp);
    if ((reinterpret_cast<uintptr_t>(d.depth) | reinterpret_cast<uintptr_t>(d.colour) |
         reinterpret_cast<uintptr_t>(d.range)) & 15)
        return false;
    const cuuint32_t es[3] = {1, 1, 1};
    const cuuint64_t w = (cuuint64_t)d.w, h = (cuuint64_t)d.h, plane = (cuuint64_t)d.nl * 16;
    {
        const cuuint64_t dim[2] = {2 * w, h}, stride[1] = {w * 8};
        const cuuint32_t box[2] = {64, 8};
        if (enc(&m->range, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<float2 *>(d.range), dim, stride, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    {
        const cuuint64_t dim[3] = {4 * w, h, (cuuint64_t)(d.nsp >> 1)}, stride[2] = {w * 16, plane};
        const cuuint32_t box[3] = {128, 8, np};
        if (enc(&m->depth, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<float4 *>(d.depth), dim, stride, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    {
        const bool f16 = d.fmt == 1;
        const cuuint64_t dim[3] = {4 * w, h, (cuuint64_t)(f16 ? (d.nsp >> 1) : d.nsp)}, stride[2] = {w * 16, plane};
        const cuuint32_t box[3] = {128, 8, f16 ? np : 2 * np};
        if (enc(&m->colour, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<void *>(d.colour), dim, stride, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

vdi_status alloc_vdi(vdi_ctx *ctx, const vdi_desc *desc, cudaStream_t stream, vdi_t **out) {
    vdi_layout L;
    vdi_status s = check_desc(desc, &L);
    if (s != VDI_OK) return s;
    vdi_t *v = new (std::nothrow) vdi_t();
    if (!v) return fail(VDI_ERR_OOM, "host allocation");
    v->ctx = ctx;
    v->desc = *desc;
    v->desc.grid_tile = desc->grid_tile ? desc->grid_tile : 8;
    v->desc.grid_nz = desc->grid_nz ? desc->grid_nz : 20;
    v->layout = L;
    mat4_mul(desc->orig.proj, desc->orig.view, v->M);
    const double dn = ndc_to_view_depth(desc->orig.proj, -1.0), df = ndc_to_view_depth(desc->orig.proj, 1.0);
    if (!(df > dn) || !isfinite(dn) || !isfinite(df)) {
        delete v;
        return fail(VDI_ERR_INVALID_ARG, "V_O near/far planes are degenerate");
    }
    v->dz_cell = (df - dn) / v->desc.grid_nz;
    // the V_O frustum clip of a render is redundant when the whole box lies
    // inside the frustum; the margin covers the FP32 rounding of the clip
    v->box_in_frustum = true;
    for (int corner = 0; corner < 8; ++corner) {
        const double p[4] = {(corner & 1) ? desc->bbox_max[0] : desc->bbox_min[0],
                             (corner & 2) ? desc->bbox_max[1] : desc->bbox_min[1],
                             (corner & 4) ? desc->bbox_max[2] : desc->bbox_min[2], 1.0};
        double q[4];
        mat4_apply(v->M, p, q);
        const double lim = q[3] * (1.0 - 1e-4);
        if (!(q[3] > 0.0) || !(fabs(q[0]) < lim) || !(fabs(q[1]) < lim) || !(fabs(q[2]) < lim))
            v->box_in_frustum = false;
    }
    DevVdi &d = v->dv;
    d.w = desc->w;
    d.h = desc->h;
    d.ns = desc->n_s;
    d.nsp = L.n_s_stored;
    d.fmt = desc->colour_fmt;
    d.nl = (long long)desc->w * desc->h;
    d.nl32 = (int)d.nl;
    d.T = v->desc.grid_tile;
    d.gw = L.grid_w;
    d.gh = L.grid_h;
    d.nz = L.grid_nz;
    grid_edges(desc->orig.proj, d.nz, d.edges);
    cudaError_t e;
    if ((e = cudaMallocAsync(&v->depth_mem, L.depth_bytes, stream)) != cudaSuccess ||
        (e = cudaMallocAsync(&v->colour_mem, L.colour_bytes, stream)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&v->grid_mem, L.grid_bytes, stream)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&v->range_mem, L.list_bytes, stream)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&v->status_mem, sizeof(uint32_t), stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(v->status_mem, 0, sizeof(uint32_t), stream)) != cudaSuccess) {
        vdi_status r = cuda_fail(e, "cudaMallocAsync(VDI)");
        if (v->depth_mem) cudaFreeAsync(v->depth_mem, stream);
        if (v->colour_mem) cudaFreeAsync(v->colour_mem, stream);
        if (v->grid_mem) cudaFreeAsync(v->grid_mem, stream);
        if (v->range_mem) cudaFreeAsync(v->range_mem, stream);
        if (v->status_mem) cudaFreeAsync(v->status_mem, stream);
        delete v;
        return r;
    }
    d.depth = reinterpret_cast<const float4 *>(v->depth_mem);
    d.colour = v->colour_mem;
    d.grid = v->grid_mem;
    d.range = v->range_mem;
    d.bw = div_up(desc->w, kB);
    d.bh = div_up(desc->h, kB);
    v->brange_mem = v->range_mem + d.nl;  // the block ranges follow the list ranges
    d.brange = v->brange_mem;
    v->maps_ok = build_tile_maps(d, &v->maps) ? 1 : 0;
    v->maps.status = v->status_mem;
    *out = v;
    return VDI_OK;
}

// Stream-ordered free on the context's free stream: the caller guarantees
// that no work still reads the VDI (vdi_destroy synchronises the device
// first; the server frees a VDI version only after its last batch retired).
void free_vdi(vdi_t *v) {
    if (!v) return;
    cudaSetDevice(v->ctx->device);
    cudaStream_t fs = v->ctx->free_stream;
    if (v->depth_mem) cudaFreeAsync(v->depth_mem, fs);
    if (v->colour_mem) cudaFreeAsync(v->colour_mem, fs);
    if (v->grid_mem) cudaFreeAsync(v->grid_mem, fs);
    if (v->range_mem) cudaFreeAsync(v->range_mem, fs);
    if (v->totals_mem) cudaFreeAsync(v->totals_mem, fs);
    if (v->status_mem) cudaFreeAsync(v->status_mem, fs);
    delete v;
}

}  // namespace vdi

VDI_API vdi_status vdi_create(vdi_ctx *ctx, const vdi_desc *desc, const float *rgba, const float *depth,
                              const int32_t *counts, int mem_kind, void *stream, vdi_t **out) {
    if (!ctx || !out || !rgba || !depth) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    if (mem_kind != VDI_MEM_HOST && mem_kind != VDI_MEM_DEVICE) return fail(VDI_ERR_INVALID_ARG, "mem_kind");
    *out = nullptr;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    vdi_t *v = nullptr;
    vdi_status st_ = alloc_vdi(ctx, desc, st, &v);
    if (st_ != VDI_OK) return st_;
    const size_t nl = (size_t)desc->w * desc->h, nslot = nl * desc->n_s;
    float *d_rgba = nullptr, *d_depth = nullptr;
    int32_t *d_counts = nullptr;
    unsigned *d_err = nullptr;
    unsigned h_err = 0;
    if (mem_kind == VDI_MEM_HOST) {
        CK(cudaMallocAsync((void **)&d_rgba, nslot * 16, st));
        CK(cudaMallocAsync((void **)&d_depth, nslot * 8, st));
        CK(cudaMemcpyAsync(d_rgba, rgba, nslot * 16, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_depth, depth, nslot * 8, cudaMemcpyHostToDevice, st));
    } else {
        d_rgba = const_cast<float *>(rgba);
        d_depth = const_cast<float *>(depth);
    }
    CK(cudaMallocAsync((void **)&d_counts, nl * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&d_err, sizeof(unsigned), st));
    CK(cudaMemsetAsync(d_err, 0, sizeof(unsigned), st));
    if (counts)
        CK(cudaMemcpyAsync(d_counts, counts, nl * sizeof(int32_t),
                           mem_kind == VDI_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    else
        CK(launch_count_leading(d_depth, desc->n_s, (long long)nl, d_counts, st));
    CK(launch_convert(desc->colour_fmt, d_rgba, d_depth, d_counts, desc->n_s, v->dv.nsp, (long long)nl,
                      reinterpret_cast<float4 *>(v->depth_mem), v->colour_mem, d_err, st));
    CK(launch_grid(v->dv, v->grid_mem, st));
    CK(launch_range(d_depth, d_counts, desc->n_s, (long long)nl, v->range_mem, st));
    CK(launch_block_range(v->dv, v->brange_mem, st));
    CK(cudaMemcpyAsync(&h_err, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_err & 1u)
        st_ = fail(VDI_ERR_UNSORTED, "supersegments not sorted/disjoint or depth not finite");
    else if (h_err & 2u)
        st_ = fail(VDI_ERR_INVALID_ARG, "colour outside 0 <= rgb <= alpha <= 1, or count outside 0..n_s");
done:
    if (mem_kind == VDI_MEM_HOST) {
        if (d_rgba) cudaFreeAsync(d_rgba, st);
        if (d_depth) cudaFreeAsync(d_depth, st);
    }
    if (d_counts) cudaFreeAsync(d_counts, st);
    if (d_err) cudaFreeAsync(d_err, st);
    if (st_ != VDI_OK) {
        cudaStreamSynchronize(st);
        free_vdi(v);
        return st_;
    }
    *out = v;
    return VDI_OK;
}

VDI_API vdi_status vdi_download(vdi_t *v, float *rgba, float *depth, int32_t *counts, uint32_t *grid,
                                void *stream) {
    if (!v) return fail(VDI_ERR_INVALID_ARG, "vdi is NULL");
    cudaSetDevice(v->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nl = (size_t)v->dv.nl, nslot = nl * v->dv.ns;
    vdi_status st_ = VDI_OK;
    float *d_rgba = nullptr, *d_depth = nullptr;
    int32_t *d_counts = nullptr;
    if (rgba) CK(cudaMallocAsync((void **)&d_rgba, nslot * 16, st));
    if (depth) CK(cudaMallocAsync((void **)&d_depth, nslot * 8, st));
    if (counts) CK(cudaMallocAsync((void **)&d_counts, nl * 4, st));
    if (rgba || depth || counts) CK(launch_download(v->dv, v->dv.ns, d_rgba, d_depth, d_counts, st));
    if (rgba) CK(cudaMemcpyAsync(rgba, d_rgba, nslot * 16, cudaMemcpyDeviceToHost, st));
    if (depth) CK(cudaMemcpyAsync(depth, d_depth, nslot * 8, cudaMemcpyDeviceToHost, st));
    if (counts) CK(cudaMemcpyAsync(counts, d_counts, nl * 4, cudaMemcpyDeviceToHost, st));
    if (grid) CK(cudaMemcpyAsync(grid, v->grid_mem, v->layout.grid_bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
done:
    if (d_rgba) cudaFreeAsync(d_rgba, st);
    if (d_depth) cudaFreeAsync(d_depth, st);
    if (d_counts) cudaFreeAsync(d_counts, st);
    if (st_ != VDI_OK) cudaStreamSynchronize(st);
    return st_;
}

VDI_API void vdi_destroy(vdi_t *v) {
    if (!v) return;
    cudaSetDevice(v->ctx->device);
    cudaDeviceSynchronize();  // work still reading the VDI on any stream completes first
    free_vdi(v);
}

namespace vdi {

// length in uint32 of the touch bitmap: depth, colour, grid padded to 16 bytes, list ranges
size_t touch_words(const vdi_t *v) {
    const size_t grid_words = ((size_t)v->dv.nz * v->dv.gh * v->dv.gw + 3) & ~(size_t)3;
    const size_t words = (v->layout.depth_bytes + v->layout.colour_bytes) / 4 + grid_words + v->layout.list_bytes / 4;  // list and block ranges
    return (words + 31) / 32;
}

vdi_status check_render_args(const vdi_t *v, int W, int H, int d_i, int d_r, const void *out, int out_fmt) {
    if (!v) return fail(VDI_ERR_INVALID_ARG, "vdi is NULL");
    if (!out) return fail(VDI_ERR_INVALID_ARG, "out_rgba is NULL");
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return fail(VDI_ERR_INVALID_ARG, "image %dx%d", W, H);
    if (d_i < 1 || d_i > 16 || d_r < 1 || d_r > 16) return fail(VDI_ERR_INVALID_ARG, "d_i=%d d_r=%d", d_i, d_r);
    if (out_fmt != VDI_F32 && out_fmt != VDI_F16) return fail(VDI_ERR_INVALID_ARG, "out_fmt=%d", out_fmt);
    return VDI_OK;
}

}  // namespace vdi

VDI_API vdi_status vdi_render_ex(vdi_t *v, const vdi_camera *view, int W, int H, int d_i, int d_r,
                                 void *out_rgba, int out_fmt, const vdi_render_opts *opts, void *stream) {
    vdi_status st_ = check_render_args(v, W, H, d_i, d_r, out_rgba, out_fmt);
    if (st_ != VDI_OK) return st_;
    vdi_render_opts o = {VDI_SEARCH_ALG2, 0, nullptr, nullptr, -1, 0, 0, 0};
    if (opts) o = *opts;
    if (o.search < 0 || o.search > 2) return fail(VDI_ERR_INVALID_ARG, "search=%d", o.search);
    if (o.warp_shape < -1 || o.warp_shape > 3) return fail(VDI_ERR_INVALID_ARG, "warp_shape=%d", o.warp_shape);
    if (o.record_stats && d_r != 1) return fail(VDI_ERR_UNSUPPORTED, "frame totals are counted on exact renders (d_r = 1)");
    cudaSetDevice(v->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int Wr = div_up(W, d_i), Hr = div_up(H, d_i);
    ViewConsts c;
    st_ = make_view_consts(v, view, Wr, Hr, d_r, &c);
    if (st_ != VDI_OK) return st_;
    const int ws = o.warp_shape >= 0 ? o.warp_shape : default_warp_shape(c);
    float4 *lo = nullptr;
    uint32_t *tmp_counters = nullptr;
    if (o.record_stats) {
        // per-ray counters (the caller's, or temporary ones) summed into the VDI's totals
        if (!v->totals_mem) CK(cudaMallocAsync((void **)&v->totals_mem, 3 * sizeof(unsigned long long), st));
        if (!o.ray_lists || !o.ray_segs) {
            CK(cudaMallocAsync((void **)&tmp_counters, 2 * (size_t)Wr * Hr * sizeof(uint32_t), st));
            if (!o.ray_lists) o.ray_lists = tmp_counters;
            if (!o.ray_segs) o.ray_segs = tmp_counters + (size_t)Wr * Hr;
        }
        CK(cudaMemsetAsync(v->totals_mem, 0, 3 * sizeof(unsigned long long), st));
    }
    if (d_i == 1) {
        CK(launch_render(c, v->dv, out_rgba, out_fmt, o.ray_lists, o.ray_segs, o.search, ws, !o.no_ert, o.ess != 0, o.blocks != 0, tile_maps(v), st));
    } else {
        CK(cudaMallocAsync((void **)&lo, (size_t)Wr * Hr * sizeof(float4), st));
        CK(launch_render(c, v->dv, lo, VDI_F32, o.ray_lists, o.ray_segs, o.search, ws, !o.no_ert, o.ess != 0, o.blocks != 0, tile_maps(v), st));
        CK(launch_upsample(lo, Wr, Hr, out_rgba, out_fmt, W, H, st));
    }
    if (o.record_stats) {
        CK(launch_count_totals(o.ray_lists, o.ray_segs, (long long)Wr * Hr, v->totals_mem, v->ctx->sm_count, st));
        v->frame_recorded = 1;
        v->frame_w = Wr;
        v->frame_h = Hr;
    }
done:
    if (lo) cudaFreeAsync(lo, st);
    if (tmp_counters) cudaFreeAsync(tmp_counters, st);
    return st_;
}

VDI_API vdi_status vdi_render_scaled(vdi_t *v, const vdi_camera *view, int W, int H, int Wr, int Hr, int d_r,
                                     void *out_rgba, int out_fmt, void *stream) {
    vdi_status st_ = check_render_args(v, W, H, 1, d_r, out_rgba, out_fmt);
    if (st_ != VDI_OK) return st_;
    if (Wr < 1 || Hr < 1 || Wr > W || Hr > H) return fail(VDI_ERR_INVALID_ARG, "rays %dx%d for image %dx%d", Wr, Hr, W, H);
    cudaSetDevice(v->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    ViewConsts c;
    st_ = make_view_consts(v, view, Wr, Hr, d_r, &c);
    if (st_ != VDI_OK) return st_;
    const int ws = default_warp_shape(c);
    float4 *lo = nullptr;
    if (Wr == W && Hr == H) {
        CK(launch_render(c, v->dv, out_rgba, out_fmt, nullptr, nullptr, VDI_SEARCH_ALG2, ws, true, false, false, tile_maps(v), st));
    } else {
        CK(cudaMallocAsync((void **)&lo, (size_t)Wr * Hr * sizeof(float4), st));
        CK(launch_render(c, v->dv, lo, VDI_F32, nullptr, nullptr, VDI_SEARCH_ALG2, ws, true, false, false, tile_maps(v), st));
        CK(launch_upsample(lo, Wr, Hr, out_rgba, out_fmt, W, H, st));
    }
done:
    if (lo) cudaFreeAsync(lo, st);
    return st_;
}

VDI_API vdi_status vdi_stats(vdi_t *v, vdi_stats_t *out, void *stream) {
    if (!v || !out) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    vdi_stats_t s{};
    s.layout = v->layout;
    s.w = v->desc.w;
    s.h = v->desc.h;
    s.n_s = v->desc.n_s;
    s.colour_fmt = v->desc.colour_fmt;
    s.grid_tile = v->desc.grid_tile;
    cudaSetDevice(v->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    {
        uint32_t flags = 0;
        cudaError_t e = cudaMemcpyAsync(&flags, v->status_mem, sizeof flags, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
        s.device_flags = flags;
    }
    if (v->frame_recorded && v->totals_mem) {
        unsigned long long t[3] = {0, 0, 0};
        cudaError_t e = cudaMemcpyAsync(t, v->totals_mem, sizeof t, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "reading frame totals");
        s.frame_recorded = 1;
        s.frame_w = v->frame_w;
        s.frame_h = v->frame_h;
        s.rays_hit = t[0];
        s.lists = t[1];
        s.pieces = t[2];
    }
    *out = s;
    return VDI_OK;
}

VDI_API vdi_status vdi_render(vdi_t *v, const vdi_camera *view, int W, int H, int d_i, int d_r, void *out_rgba,
                              int out_fmt, void *stream) {
    return vdi_render_ex(v, view, W, H, d_i, d_r, out_rgba, out_fmt, nullptr, stream);
}

VDI_API vdi_status vdi_search_first(vdi_t *v, int list, int search, const float *d_entry, const float *d_exit,
                                    const int32_t *seed, const int32_t *increasing, int32_t *result, int n,
                                    void *stream) {
    if (!v || !d_entry || !d_exit || !seed || !increasing || !result || n < 0)
        return fail(VDI_ERR_INVALID_ARG, "bad argument");
    if (list < 0 || list >= v->dv.nl) return fail(VDI_ERR_INVALID_ARG, "list %d out of range", list);
    if (search < 0 || search > 2) return fail(VDI_ERR_INVALID_ARG, "search=%d", search);
    if (n == 0) return VDI_OK;
    cudaSetDevice(v->ctx->device);
    vdi_status st_ = VDI_OK;
    CK(launch_search(v->dv, list, search, d_entry, d_exit, seed, increasing, result, n, (cudaStream_t)stream));
done:
    return st_;
}

VDI_API vdi_status vdi_touch_bitmap(vdi_t *v, const vdi_camera *view, int W, int H, uint32_t *bitmap, size_t words,
                                    void *stream) {
    vdi_status st_ = check_render_args(v, W, H, 1, 1, bitmap, VDI_F32);
    if (st_ != VDI_OK) return st_;
    const size_t need = touch_words(v);
    if (words < need) return fail(VDI_ERR_INVALID_ARG, "bitmap has %zu words, needs %zu", words, need);
    cudaSetDevice(v->ctx->device);
    ViewConsts c;
    st_ = make_view_consts(v, view, W, H, 1, &c);
    if (st_ != VDI_OK) return st_;
    CK(launch_touch(c, v->dv, bitmap, (cudaStream_t)stream));
done:
    return st_;
}
