// vdi_generate.cu -- VDI generation from a scalar volume (Section 3, Eq. 1
// with a fixed sensitivity gamma = tau or the ray-adaptive gamma of
// Algorithm 3), one thread per V_O pixel ray.
//
// Arithmetic uses explicit round-to-nearest FP32 intrinsics with no fused
// multiply-add, in a fixed order, so the integer outcome of generation (how
// many supersegments each list gets and where they start and end) is the
// reproducible result of IEEE FP32 operations.  The supersegment depths are
// written straight into the structure-of-arrays device layout; the colour is
// stored as (rgb / alpha, kappa) where kappa = -log2(segment transmittance)
// per length unit (the composite over the segment, Section 2.3).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/vdi.h"
#include "vdi_api_internal.h"
#include "vdi_internal.cuh"

namespace vdi {

constexpr long long kMaxSamples = 1 << 22;  // per ray; the host rejects steps that would need more

struct GenConsts {
    float E[3], D0[3], Dx[3], Dy[3];  // ray p(t) = E + t (D0 + x Dx + y Dy), t = V_O view depth
    float t_near, t_far, P22, P23;    // NDC z = P23 / t - P22
    float bmin[3], bmax[3], ext[3];
    float step, u, tau, adj_exp;
    int step_is_u;
    float kv[16], kc[16][4];
    int nk;
    int w, h, ns, nsp;
    long long nl;
    int nx, ny, nz, dtype;
    const void *data;
    int fmt;
    int adaptive;  // 1: per-ray gamma by Algorithm 3 (tau unused)
};

#define ADD __fadd_rn
#define SUB __fsub_rn
#define MUL __fmul_rn
#define DIV __fdiv_rn

__device__ __forceinline__ float lerp_rn(float a, float b, float t) { return ADD(a, MUL(t, SUB(b, a))); }

__device__ __forceinline__ float voxel(const GenConsts &g, int i, int j, int k) {
    const size_t o = ((size_t)k * g.ny + j) * g.nx + i;
    if (g.dtype == 0) return DIV((float)__ldg(reinterpret_cast<const uint8_t *>(g.data) + o), 255.f);
    if (g.dtype == 1) return DIV((float)__ldg(reinterpret_cast<const uint16_t *>(g.data) + o), 65535.f);
    return __ldg(reinterpret_cast<const float *>(g.data) + o);
}

__device__ __forceinline__ float trilinear(const GenConsts &g, const float p[3]) {
    const int n[3] = {g.nx, g.ny, g.nz};
    int i0[3], i1[3];
    float fr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float q = SUB(MUL(DIV(SUB(p[c], g.bmin[c]), g.ext[c]), (float)n[c]), 0.5f);
        const float fl = floorf(q);
        fr[c] = SUB(q, fl);
        const int i = (int)fl;
        i0[c] = min(max(i, 0), n[c] - 1);
        i1[c] = min(max(i + 1, 0), n[c] - 1);
    }
    const float c00 = lerp_rn(voxel(g, i0[0], i0[1], i0[2]), voxel(g, i1[0], i0[1], i0[2]), fr[0]);
    const float c10 = lerp_rn(voxel(g, i0[0], i1[1], i0[2]), voxel(g, i1[0], i1[1], i0[2]), fr[0]);
    const float c01 = lerp_rn(voxel(g, i0[0], i0[1], i1[2]), voxel(g, i1[0], i0[1], i1[2]), fr[0]);
    const float c11 = lerp_rn(voxel(g, i0[0], i1[1], i1[2]), voxel(g, i1[0], i1[1], i1[2]), fr[0]);
    return lerp_rn(lerp_rn(c00, c10, fr[1]), lerp_rn(c01, c11, fr[1]), fr[2]);
}

__device__ __forceinline__ void classify(const GenConsts &g, float v, float out[4]) {
    const int last = g.nk - 1;
    if (v <= g.kv[0]) {
#pragma unroll
        for (int c = 0; c < 4; ++c) out[c] = g.kc[0][c];
        return;
    }
    if (v >= g.kv[last]) {
#pragma unroll
        for (int c = 0; c < 4; ++c) out[c] = g.kc[last][c];
        return;
    }
    int i = 0;
    while (i < last - 1 && !(v < g.kv[i + 1])) ++i;
    const float s = DIV(SUB(v, g.kv[i]), SUB(g.kv[i + 1], g.kv[i]));
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] = lerp_rn(g.kc[i][c], g.kc[i + 1][c], s);
}

struct SegWriter {
    float pf, pb;      // pending even slot (depth)
    float4 pc;         // pending even slot (colour)
};

__device__ __forceinline__ unsigned h2bits(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned *>(&h);
}

__device__ __forceinline__ void write_pair(const GenConsts &g, float4 *depth, void *colour, long long li, int k,
                                           float f0, float b0, float4 c0, float f1, float b1, float4 c1) {
    depth[(size_t)k * g.nl + li] = make_float4(f0, b0, f1, b1);
    if (g.fmt == 0) {
        float4 *cp = reinterpret_cast<float4 *>(colour);
        cp[(size_t)(2 * k) * g.nl + li] = c0;
        cp[(size_t)(2 * k + 1) * g.nl + li] = c1;
    } else {
        uint4 q;
        q.x = h2bits(c0.x, c0.y);
        q.y = h2bits(c0.z, c0.w);
        q.z = h2bits(c1.x, c1.y);
        q.w = h2bits(c1.z, c1.w);
        reinterpret_cast<uint4 *>(colour)[(size_t)k * g.nl + li] = q;
    }
}

// The V_O pixel-centre ray of list (px, py), clipped to near/far and the box;
// K samples of view-depth step dt from t0.
struct GenRay {
    float dir[3];
    float len, t0, dt;
    long long K;
};

__device__ __forceinline__ GenRay gen_ray(const GenConsts &g, int px, int py) {
    GenRay r;
    const float x = SUB(DIV(MUL(2.f, ADD((float)px, 0.5f)), (float)g.w), 1.f);
    const float y = SUB(1.f, DIV(MUL(2.f, ADD((float)py, 0.5f)), (float)g.h));
#pragma unroll
    for (int c = 0; c < 3; ++c) r.dir[c] = ADD(ADD(g.D0[c], MUL(x, g.Dx[c])), MUL(y, g.Dy[c]));
    r.len = __fsqrt_rn(ADD(ADD(MUL(r.dir[0], r.dir[0]), MUL(r.dir[1], r.dir[1])), MUL(r.dir[2], r.dir[2])));
    float t0 = g.t_near, t1 = g.t_far;
    bool hit = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (r.dir[c] != 0.f) {
            float ta = DIV(SUB(g.bmin[c], g.E[c]), r.dir[c]), tb = DIV(SUB(g.bmax[c], g.E[c]), r.dir[c]);
            if (ta > tb) {
                const float s = ta;
                ta = tb;
                tb = s;
            }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        } else if (g.E[c] < g.bmin[c] || g.E[c] > g.bmax[c]) {
            hit = false;
        }
    }
    r.K = 0;
    r.t0 = t0;
    r.dt = 0.f;
    if (hit && t0 < t1) {
        const float L = MUL(SUB(t1, t0), r.len);
        const float kq = floorf(DIV(L, g.step));
        r.K = kq < (float)kMaxSamples ? (long long)kq : kMaxSamples;
        r.dt = DIV(g.step, r.len);
    }
    return r;
}

// One march along the ray with sensitivity tau (Eq. 1).  WRITE: supersegments
// go to the VDI, the N_S-th never closes, returns how many were written.
// !WRITE (the counting pass of Algorithm 3): no limit on the number, nothing
// written, and the count stops at ns + 1 ("more than N_S").
template <bool WRITE>
__device__ int gen_march(const GenConsts &g, const GenRay &r, float tau, float4 *__restrict__ depth,
                         void *__restrict__ colour, long long li, float &first_f, float &last_b) {
    const int limit = WRITE ? g.ns : g.ns + 2;  // supersegment number `limit` never closes
    int nseg = 0;
    SegWriter sw;
    sw.pf = sw.pb = INFINITY;
    sw.pc = make_float4(0.f, 0.f, 0.f, 0.f);
    bool open = false;
    float t_start = 0.f, t_end = 0.f, Tseg = 1.f, Tray = 1.f;
    float mean[3] = {0.f, 0.f, 0.f}, Cacc[3] = {0.f, 0.f, 0.f};
    int cnt = 0;
    const float tau2 = MUL(tau, tau);
    auto close = [&]() {
        if (WRITE) {
            const float f = SUB(DIV(g.P23, t_start), g.P22);
            const float b = SUB(DIV(g.P23, t_end), g.P22);
            const float aacc = 1.f - Tseg;
            const float Lu = (t_end - t_start) * r.len / g.u;  // world length in length units
            const float ia = aacc > 0.f ? 1.f / aacc : 0.f;
            const float kappa = (Lu > 0.f) ? -log2f(Tseg) / Lu : 0.f;
            const float4 col =
                make_float4(fminf(Cacc[0] * ia, 1.f), fminf(Cacc[1] * ia, 1.f), fminf(Cacc[2] * ia, 1.f), kappa);
            if (nseg == 0) first_f = f;
            last_b = b;
            if ((nseg & 1) == 0) {
                sw.pf = f;
                sw.pb = b;
                sw.pc = col;
            } else {
                write_pair(g, depth, colour, li, nseg >> 1, sw.pf, sw.pb, sw.pc, f, b, col);
            }
        }
        ++nseg;
        open = false;
    };
    for (long long k = 0; k < r.K; ++k) {
        const float fk = (float)k;
        const float ta = ADD(r.t0, MUL(fk, r.dt));
        const float tm = ADD(r.t0, MUL(ADD(fk, 0.5f), r.dt));
        const float tb = ADD(r.t0, MUL((float)(k + 1), r.dt));
        float p[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] = ADD(g.E[c], MUL(tm, r.dir[c]));
        float tf[4];
        classify(g, trilinear(g, p), tf);
        const float a = g.step_is_u ? tf[3] : 1.f - powf(1.f - tf[3], g.adj_exp);
        if (!(a > 0.f)) {
            if (open && nseg < limit - 1) {
                close();
                if (!WRITE && nseg > g.ns) return g.ns + 1;
            }
            continue;
        }
        const float xc[3] = {MUL(tf[0], a), MUL(tf[1], a), MUL(tf[2], a)};
        if (open && nseg < limit - 1) {
            const float d0 = SUB(mean[0], xc[0]), d1 = SUB(mean[1], xc[1]), d2 = SUB(mean[2], xc[2]);
            const float dist2 = ADD(ADD(MUL(d0, d0), MUL(d1, d1)), MUL(d2, d2));
            if (!(tau2 > dist2)) {
                close();
                if (!WRITE && nseg > g.ns) return g.ns + 1;
            }
        }
        if (!open) {
            open = true;
            t_start = ta;
            cnt = 0;
            Tseg = 1.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) mean[c] = Cacc[c] = 0.f;
        }
        ++cnt;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mean[c] = ADD(mean[c], DIV(SUB(xc[c], mean[c]), (float)cnt));
            Cacc[c] = ADD(Cacc[c], MUL(Tseg, xc[c]));
        }
        Tseg = MUL(Tseg, SUB(1.f, a));
        t_end = tb;
        Tray = MUL(Tray, SUB(1.f, a));
        if (Tray <= kErtT) break;
    }
    if (open) close();
    if (!WRITE) return nseg > g.ns ? g.ns + 1 : nseg;
    // pad the remaining slots
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    int j = nseg;
    if (j & 1) {
        write_pair(g, depth, colour, li, j >> 1, sw.pf, sw.pb, sw.pc, INFINITY, INFINITY, zero);
        ++j;
    }
    for (; j < g.nsp; j += 2)
        write_pair(g, depth, colour, li, j >> 1, INFINITY, INFINITY, zero, INFINITY, INFINITY, zero);
    return nseg;
}

// Ray-adaptive sensitivity (Section 3, Algorithm 3 of the supplement): a
// bisection for gamma in [0, sqrt(3)] (the largest L2 distance of two
// premultiplied RGB colours) until the ray gets between N_S - delta and N_S
// supersegments, delta = floor(0.15 N_S).  The search starts at 1e-5 and
// keeps it if that gives fewer than N_S; more than N_S raises the lower end,
// fewer than N_S - delta lowers the upper end; an interval narrower than
// 1e-6 (the supplement's value) ends the search with the upper end (the side
// that does not exceed N_S).  In [0, sqrt(3)] an FP32 ulp is at most 1.2e-7,
// so every interval still to be halved holds more than eight ulps and its
// midpoint lies strictly inside it.  FP32 with explicit rounding, like the
// march, so every ray's gamma is reproducible.
__device__ float adaptive_tau(const GenConsts &g, const GenRay &r) {
    const int delta = (15 * g.ns) / 100;
    float low = 0.f, high = (float)1.7320508075688772, gamma = (float)1e-5;
    const float eps = (float)1e-6;
    bool first = true, found = false;
    float ff = 0.f, lb = 0.f;
    while (!found) {
        const int n = gen_march<false>(g, r, gamma, nullptr, nullptr, 0, ff, lb);
        if (SUB(high, low) < eps) {
            found = true;
            gamma = high;
        } else if (n > g.ns) {
            low = gamma;
        } else if (n < g.ns - delta) {
            high = gamma;
        } else {
            found = true;
        }
        if (first) {
            first = false;
            if (n < g.ns) found = true;
        }
        if (!found) gamma = DIV(ADD(low, high), 2.f);
    }
    return gamma;
}

__global__ void __launch_bounds__(256) generate_kernel(const GenConsts g, float4 *__restrict__ depth,
                                                       void *__restrict__ colour, float2 *__restrict__ range,
                                                       float *__restrict__ tau_out) {
    const int px = blockIdx.x * 32 + (threadIdx.x & 31);
    const int py = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (px >= g.w || py >= g.h) return;
    const long long li = (long long)py * g.w + px;
    const GenRay r = gen_ray(g, px, py);
    const float tau = g.adaptive ? adaptive_tau(g, r) : g.tau;
    float first_f = INFINITY, last_b = -INFINITY;
    gen_march<true>(g, r, tau, depth, colour, li, first_f, last_b);
    range[li] = make_float2(first_f, last_b);
    if (tau_out) tau_out[li] = tau;
}

// Direct volume rendering (emission-absorption, front to back) of the volume
// from any perspective camera, at the generation's sampling rules: midpoints
// of world intervals of `step` from the box entry, trilinear interpolation,
// the transfer function, a' = 1 - (1 - alpha)^(step / u), early termination
// at transmittance 2^-12.  It is the ground truth the VDI renders are compared
// with (Section 6).  One thread per pixel; output premultiplied RGBA.
__global__ void __launch_bounds__(256) dvr_kernel(const GenConsts g, void *__restrict__ out, int out_fmt) {
    const int px = blockIdx.x * 32 + (threadIdx.x & 31);
    const int py = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (px >= g.w || py >= g.h) return;
    const GenRay r = gen_ray(g, px, py);
    float C[3] = {0.f, 0.f, 0.f}, T = 1.f;
    for (long long k = 0; k < r.K; ++k) {
        const float tm = ADD(r.t0, MUL(ADD((float)k, 0.5f), r.dt));
        float p[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] = ADD(g.E[c], MUL(tm, r.dir[c]));
        float tf[4];
        classify(g, trilinear(g, p), tf);
        const float a = g.step_is_u ? tf[3] : 1.f - powf(1.f - tf[3], g.adj_exp);
        if (!(a > 0.f)) continue;
        const float wgt = MUL(T, a);
#pragma unroll
        for (int c = 0; c < 3; ++c) C[c] = ADD(C[c], MUL(wgt, tf[c]));
        T = MUL(T, SUB(1.f, a));
        if (T <= kErtT) break;
    }
    const size_t idx = (size_t)py * g.w + px;
    if (out_fmt == 0) {
        reinterpret_cast<float4 *>(out)[idx] = make_float4(C[0], C[1], C[2], 1.f - T);
    } else {
        uint2 q;
        q.x = h2bits(C[0], C[1]);
        q.y = h2bits(C[2], 1.f - T);
        reinterpret_cast<uint2 *>(out)[idx] = q;
    }
}

cudaError_t launch_dvr(const GenConsts &g, void *out, int out_fmt, cudaStream_t st) {
    dim3 grid(div_up(g.w, 32), div_up(g.h, 8));
    dvr_kernel<<<grid, 256, 0, st>>>(g, out, out_fmt);
    return cudaGetLastError();
}

#undef ADD
#undef SUB
#undef MUL
#undef DIV

cudaError_t launch_grid(const DevVdi &v, uint32_t *grid, cudaStream_t st);

}  // namespace vdi

using namespace vdi;

#define VDI_API extern "C" __attribute__((visibility("default")))

static double pe(const double *m, int r, int c) { return m[c * 4 + r]; }

// Validation shared by generation and DVR: the volume, the transfer function,
// the sampling step and a perspective camera (the rays are parameterised by
// its view depth).
static vdi_status check_volume_tf_camera(const vdi_volume *vol, const vdi_tf *tf, const vdi_camera *cam, double step) {
    if (!vol->data || vol->nx < 1 || vol->ny < 1 || vol->nz < 1 || vol->dtype < 0 || vol->dtype > 2)
        return fail(VDI_ERR_INVALID_ARG, "bad volume");
    if (tf->n_knots < 2 || tf->n_knots > 16 || !tf->knots) return fail(VDI_ERR_INVALID_ARG, "n_knots in 2..16");
    for (int k = 0; k < tf->n_knots; ++k) {
        const float *kn = tf->knots + 5 * k;
        for (int c = 0; c < 5; ++c)
            if (!isfinite(kn[c])) return fail(VDI_ERR_INVALID_ARG, "non-finite knot");
        if (k > 0 && !(kn[0] > tf->knots[5 * (k - 1)])) return fail(VDI_ERR_INVALID_ARG, "knot values must increase");
        if (kn[4] < 0.f || kn[4] > 1.f) return fail(VDI_ERR_INVALID_ARG, "knot alpha outside [0,1]");
        for (int c = 1; c < 4; ++c)
            if (kn[c] < 0.f || kn[c] > 1.f) return fail(VDI_ERR_INVALID_ARG, "knot colour outside [0,1]");
    }
    if (!(step > 0.0)) return fail(VDI_ERR_INVALID_ARG, "step must be > 0");
    double diag = 0.0;
    for (int k = 0; k < 3; ++k) diag += (vol->bbox_max[k] - vol->bbox_min[k]) * (vol->bbox_max[k] - vol->bbox_min[k]);
    if (!(sqrt(diag) / step < (double)kMaxSamples))
        return fail(VDI_ERR_INVALID_ARG, "step too small: more than %lld samples per ray", kMaxSamples);
    const double *P = cam->proj;
    if (!(pe(P, 3, 0) == 0 && pe(P, 3, 1) == 0 && pe(P, 3, 2) == -1 && pe(P, 3, 3) == 0 && pe(P, 2, 0) == 0 &&
          pe(P, 2, 1) == 0 && pe(P, 0, 1) == 0 && pe(P, 1, 0) == 0 && pe(P, 0, 3) == 0 && pe(P, 1, 3) == 0))
        return fail(VDI_ERR_UNSUPPORTED, "generation and DVR need an OpenGL perspective frustum");
    return VDI_OK;
}

// Per-camera ray constants (host FP64, rounded to FP32 once).
static vdi_status make_gen_consts(const vdi_volume *vol, const vdi_tf *tf, const vdi_camera *cam, int w, int h,
                                  double step, double length_unit, GenConsts *g) {
    const double *P = cam->proj;
    double Vi[16];
    if (!mat4_inv(cam->view, Vi)) return fail(VDI_ERR_INVALID_ARG, "camera view is singular");
    *g = GenConsts{};
    const double dv0[3] = {pe(P, 0, 2) / pe(P, 0, 0), pe(P, 1, 2) / pe(P, 1, 1), -1.0};
    for (int r = 0; r < 3; ++r) {
        g->E[r] = (float)(pe(Vi, r, 3) / pe(Vi, 3, 3));
        double s0 = 0.0;
        for (int c = 0; c < 3; ++c) s0 += pe(Vi, r, c) * dv0[c];
        g->D0[r] = (float)s0;
        g->Dx[r] = (float)(pe(Vi, r, 0) * (1.0 / pe(P, 0, 0)));
        g->Dy[r] = (float)(pe(Vi, r, 1) * (1.0 / pe(P, 1, 1)));
        g->bmin[r] = (float)vol->bbox_min[r];
        g->bmax[r] = (float)vol->bbox_max[r];
        g->ext[r] = g->bmax[r] - g->bmin[r];  // one IEEE float subtraction (host code is built without contraction)
    }
    g->P22 = (float)pe(P, 2, 2);
    g->P23 = (float)pe(P, 2, 3);
    g->t_near = (float)(pe(P, 2, 3) / (pe(P, 2, 2) - 1.0));
    g->t_far = (float)(pe(P, 2, 3) / (pe(P, 2, 2) + 1.0));
    g->step = (float)step;
    g->u = (float)length_unit;
    g->step_is_u = g->step == g->u;
    g->adj_exp = g->step / g->u;
    g->nk = tf->n_knots;
    for (int k = 0; k < g->nk; ++k) {
        g->kv[k] = tf->knots[5 * k];
        for (int c = 0; c < 4; ++c) g->kc[k][c] = tf->knots[5 * k + 1 + c];
    }
    g->w = w;
    g->h = h;
    g->nx = vol->nx;
    g->ny = vol->ny;
    g->nz = vol->nz;
    g->dtype = vol->dtype;
    g->data = vol->data;
    return VDI_OK;
}

VDI_API vdi_status vdi_generate(vdi_ctx *ctx, const vdi_volume *vol, const vdi_tf *tf, const vdi_gen_params *prm,
                                void *stream, vdi_t **out) {
    if (!ctx || !vol || !tf || !prm || !out) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    vdi_status st_ = check_volume_tf_camera(vol, tf, &prm->orig, prm->step);
    if (st_ != VDI_OK) return st_;
    if (!(prm->tau >= 0.f) || !isfinite(prm->tau)) return fail(VDI_ERR_INVALID_ARG, "tau must be >= 0");
    vdi_desc d{};
    d.w = prm->w;
    d.h = prm->h;
    d.n_s = prm->n_s;
    d.orig = prm->orig;
    for (int k = 0; k < 3; ++k) {
        d.bbox_min[k] = vol->bbox_min[k];
        d.bbox_max[k] = vol->bbox_max[k];
    }
    d.length_unit = prm->length_unit;
    d.colour_fmt = prm->colour_fmt;
    d.grid_tile = prm->grid_tile;
    d.grid_nz = prm->grid_nz;
    GenConsts g;
    st_ = make_gen_consts(vol, tf, &prm->orig, d.w, d.h, prm->step, prm->length_unit, &g);
    if (st_ != VDI_OK) return st_;
    cudaSetDevice(ctx->device);
    vdi_t *v = nullptr;
    st_ = alloc_vdi(ctx, &d, (cudaStream_t)stream, &v);
    if (st_ != VDI_OK) return st_;
    g.tau = prm->tau;
    g.ns = d.n_s;
    g.nsp = v->dv.nsp;
    g.nl = v->dv.nl;
    g.fmt = d.colour_fmt;
    g.adaptive = prm->adaptive ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid(div_up(d.w, 32), div_up(d.h, 8));
    generate_kernel<<<grid, 256, 0, st>>>(g, reinterpret_cast<float4 *>(v->depth_mem), v->colour_mem, v->range_mem,
                                          prm->tau_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_grid(v->dv, v->grid_mem, st);
    if (e == cudaSuccess) e = launch_block_range(v->dv, v->brange_mem, st);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        free_vdi(v);
        return cuda_fail(e, "generate");
    }
    *out = v;
    return VDI_OK;
}

VDI_API vdi_status vdi_dvr(vdi_ctx *ctx, const vdi_volume *vol, const vdi_tf *tf, const vdi_camera *view, int W, int H,
                           double step, double length_unit, void *out_rgba, int out_fmt, void *stream) {
    if (!ctx || !vol || !tf || !view || !out_rgba) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    if (W < 1 || H < 1 || (long long)W * H > (1LL << 30)) return fail(VDI_ERR_INVALID_ARG, "image %dx%d", W, H);
    if (out_fmt != VDI_F32 && out_fmt != VDI_F16) return fail(VDI_ERR_INVALID_ARG, "out_fmt=%d", out_fmt);
    if (!(length_unit > 0.0)) return fail(VDI_ERR_INVALID_ARG, "length_unit must be > 0");
    vdi_status st_ = check_volume_tf_camera(vol, tf, view, step);
    if (st_ != VDI_OK) return st_;
    GenConsts g;
    st_ = make_gen_consts(vol, tf, view, W, H, step, length_unit, &g);
    if (st_ != VDI_OK) return st_;
    cudaSetDevice(ctx->device);
    cudaError_t e = launch_dvr(g, out_rgba, out_fmt, (cudaStream_t)stream);
    return e == cudaSuccess ? VDI_OK : cuda_fail(e, "dvr");
}
