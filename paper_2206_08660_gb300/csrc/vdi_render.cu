// vdi_render.cu -- new-view raycasting of a resident VDI (Section 4) and the
// subsampled previews (Section 4.4).
//
// One thread per pixel ray.  A block covers 32 x 8 pixels; its eight warps
// cover 32x1, 16x2 or 8x4 pixels each (the warp shape is a launch choice:
// lanes on neighbouring pixels walk neighbouring lists, so their 16-byte
// depth/colour loads coalesce).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "vdi_internal.cuh"

namespace vdi {

// A ray clipped to V_O's frustum and the volume box, as a straight segment in
// V_O NDC from P0 (s = 0) to P1 (s = 1).
struct Ray {
    float z0, dz;              // NDC z = z0 + s dz
    float gx0, gy0, dgx, dgy;  // list-grid coordinates (x right, y down), = g0 + s dg
    float w1, dw;              // D(s) = w1 + s (w0 - w1), clip w at the two ends mixed
    float lw;                  // world length / u of [sa, sb] = lw (sb - sa) / (D(sa) D(sb))
    float lu;                  // clipped world length / u
    float w0;
    float4 h0, h1;             // homogeneous clip coordinates of the two ends
};

__device__ __forceinline__ void clip_lin(float c0, float c1, float &t0, float &t1) {
    if (c1 > 0.f)
        t0 = fmaxf(t0, -c0 / c1);
    else if (c1 < 0.f)
        t1 = fminf(t1, -c0 / c1);
    else if (c0 < 0.f)
        t1 = -INFINITY;
}

// Ray setup (Section 4.1): FP64 only for the map of the pixel's ray into V_O
// clip space (a, b); everything after it is FP32.
__device__ __forceinline__ bool setup_ray(const ViewConsts &c, int px, int py, Ray &r) {
    const double x = fma((double)px + 0.5, c.sx, -1.0);
    const double y = fma(-((double)py + 0.5), c.sy, 1.0);
    float a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = c.a_affine ? (float)fma(y, c.Ay[k], fma(x, c.Ax[k], c.A0[k])) : (float)c.A0[k];
        b[k] = c.b_affine ? (float)fma(y, c.By[k], fma(x, c.Bx[k], c.B0[k])) : (float)c.B0[k];
    }
    const float xf = (float)x, yf = (float)y;
    float t0 = c.t_lo, t1 = c.t_hi;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        clip_lin(a[3] + a[k], b[3] + b[k], t0, t1);
        clip_lin(a[3] - a[k], b[3] - b[k], t0, t1);
    }
    float dl2 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float o = fmaf(yf, c.Oy[k], fmaf(xf, c.Ox[k], c.O0[k]));
        float d = fmaf(yf, c.Dy[k], fmaf(xf, c.Dx[k], c.D0[k]));
        clip_lin(o - c.bmin[k], d, t0, t1);
        clip_lin(c.bmax[k] - o, -d, t0, t1);
        dl2 = fmaf(d, d, dl2);
    }
    if (!(t0 < t1)) return false;
    float4 h0 = make_float4(fmaf(t0, b[0], a[0]), fmaf(t0, b[1], a[1]), fmaf(t0, b[2], a[2]),
                            fmaf(t0, b[3], a[3]));
    float4 h1 = make_float4(fmaf(t1, b[0], a[0]), fmaf(t1, b[1], a[1]), fmaf(t1, b[2], a[2]),
                            fmaf(t1, b[3], a[3]));
    if (!(h0.w > 0.f) || !(h1.w > 0.f)) return false;
    const float i0 = 1.f / h0.w, i1 = 1.f / h1.w;
    const float p0x = h0.x * i0, p0y = h0.y * i0, p0z = h0.z * i0;
    const float p1x = h1.x * i1, p1y = h1.y * i1, p1z = h1.z * i1;
    r.z0 = p0z;
    r.dz = p1z - p0z;
    r.h0 = h0;
    r.h1 = h1;
    r.w0 = h0.w;
    r.w1 = h1.w;
    r.dw = h0.w - h1.w;
    r.lu = sqrtf(dl2) * (t1 - t0) * c.inv_u;
    r.lw = r.lu * h0.w * h1.w;
    // grid coordinates are filled by the caller (needs the list resolution)
    r.gx0 = p0x;
    r.gy0 = p0y;
    r.dgx = p1x - p0x;
    r.dgy = p1y - p0y;
    return true;
}

struct Accum {
    float r, g, b, T;
};

__device__ __forceinline__ void add_piece(Accum &acc, float4 col, float len_u) {
    const float e = exp2f(-col.w * len_u);
    const float wgt = acc.T * (1.f - e);
    acc.r = fmaf(wgt, col.x, acc.r);
    acc.g = fmaf(wgt, col.y, acc.g);
    acc.b = fmaf(wgt, col.z, acc.b);
    acc.T *= e;
}

// ---------------------------------------------------------------------------
// Exact path: list walk (Amanatides-Woo in V_O NDC), Algorithm 2 per list,
// adjacency walk over the sorted supersegments, Eq. 2, front-to-back.
// ---------------------------------------------------------------------------
template <int FMT, int MODE, bool ERT, bool TOUCH = false>
__device__ __forceinline__ void march_exact(const DevVdi &v, Ray &r, Accum &acc, uint32_t &n_lists,
                                            uint32_t &n_segs, uint32_t *bm = nullptr) {
    const float hw = 0.5f * (float)v.w, hh = 0.5f * (float)v.h;
    const float gx0 = (r.gx0 + 1.f) * hw, gy0 = (1.f - r.gy0) * hh;
    const float dgx = r.dgx * hw, dgy = -r.dgy * hh;
    int ix = min(max((int)floorf(gx0), 0), v.w - 1);
    int iy = min(max((int)floorf(gy0), 0), v.h - 1);
    const int stx = dgx > 0.f ? 1 : -1, sty = dgy > 0.f ? 1 : -1;
    const float idgx = 1.f / dgx, idgy = 1.f / dgy;
    int bx = ix + (dgx > 0.f ? 1 : 0), by = iy + (dgy > 0.f ? 1 : 0);
    float sx = (dgx != 0.f) ? ((float)bx - gx0) * idgx : INFINITY;
    float sy = (dgy != 0.f) ? ((float)by - gy0) * idgy : INFINITY;
    const bool inc = r.dz >= 0.f;
    const float z0 = r.z0, dz = r.dz, idz = 1.f / r.dz;
    const float w1 = r.w1, dw = r.dw, lw = r.lw;
    int p = -1;
    float s_in = 0.f;
    const int maxit = v.w + v.h + 2;
    for (int it = 0; it < maxit; ++it) {
        const float s_out = fminf(fminf(sx, sy), 1.f);
        if (s_out > s_in) {
            const int li = iy * v.w + ix;
            const float d_in = fmaf(s_in, dz, z0), d_out = fmaf(s_out, dz, z0);
            PairCache pc;
            pc.k = -1;
            ColourCache<FMT> cc;
            cc.k = -1;
            ++n_lists;
            int last = -1, first;
            if (inc) {
                first = first_inc<MODE, TOUCH>(v, li, d_in, p, pc, bm);
                for (int j = first; j < v.nsp; ++j) {
                    float f, b;
                    get_fb(pc, v, li, j, f, b);
                    mark_depth<TOUCH>(v, bm, j, li, 0);
                    mark_depth<TOUCH>(v, bm, j, li, 1);
                    if (f > d_out) break;
                    const float sa = (f > d_in) ? fminf(fmaxf((f - z0) * idz, s_in), s_out) : s_in;
                    const float sb = (b < d_out) ? fminf(fmaxf((b - z0) * idz, s_in), s_out) : s_out;
                    last = j;
                    if (sb > sa) {
                        mark_colour<TOUCH>(v, bm, j, li);
                        const float4 col = get_colour<FMT>(cc, v, li, j);
                        const float da = fmaf(sa, dw, w1), db = fmaf(sb, dw, w1);
                        add_piece(acc, col, lw * (sb - sa) / (da * db));
                        ++n_segs;
                        if (ERT && acc.T <= kErtT) break;
                    }
                    if (b > d_out) break;
                }
            } else {
                first = first_dec<MODE, TOUCH>(v, li, d_in, p, pc, bm);
                for (int j = first; j >= 0; --j) {
                    float f, b;
                    get_fb(pc, v, li, j, f, b);
                    mark_depth<TOUCH>(v, bm, j, li, 0);
                    mark_depth<TOUCH>(v, bm, j, li, 1);
                    if (b < d_out) break;
                    const float sa = (b < d_in) ? fminf(fmaxf((b - z0) * idz, s_in), s_out) : s_in;
                    const float sb = (f > d_out) ? fminf(fmaxf((f - z0) * idz, s_in), s_out) : s_out;
                    last = j;
                    if (sb > sa) {
                        mark_colour<TOUCH>(v, bm, j, li);
                        const float4 col = get_colour<FMT>(cc, v, li, j);
                        const float da = fmaf(sa, dw, w1), db = fmaf(sb, dw, w1);
                        add_piece(acc, col, lw * (sb - sa) / (da * db));
                        ++n_segs;
                        if (ERT && acc.T <= kErtT) break;
                    }
                    if (f < d_out) break;
                }
            }
            p = (last >= 0) ? last : first;
            if (p < 0) p = 0;
            if (ERT && acc.T <= kErtT) break;
        }
        if (s_out >= 1.f) break;
        if (sx <= sy) {
            ix += stx;
            if ((unsigned)ix >= (unsigned)v.w) break;
            bx += stx;
            sx = ((float)bx - gx0) * idgx;
        } else {
            iy += sty;
            if ((unsigned)iy >= (unsigned)v.h) break;
            by += sty;
            sy = ((float)by - gy0) * idgy;
        }
        s_in = fmaxf(s_in, s_out);
    }
}

// ---------------------------------------------------------------------------
// Ray-subsampled preview (Section 4.4): walk the cells of the count grid; in a
// cell holding c supersegments over F lists, crossed over world length l_c,
// place n = ceil((c / F) (l_c / cell_depth) / D_R) samples at equal spacing,
// look each one up in its list (Algorithm 2 search, seeded by the previous
// sample) and composite with opacity corrected by the spacing.
// ---------------------------------------------------------------------------
template <int FMT, int MODE, bool ERT>
__device__ __forceinline__ void march_preview(const DevVdi &v, const ViewConsts &c, Ray &r,
                                              Accum &acc) {
    const float hw = 0.5f * (float)v.w, hh = 0.5f * (float)v.h;
    const float gx0 = (r.gx0 + 1.f) * hw, gy0 = (1.f - r.gy0) * hh;
    const float dgx = r.dgx * hw, dgy = -r.dgy * hh;
    const float fT = (float)v.T, iT = 1.f / fT;
    const float cx0 = gx0 * iT, cy0 = gy0 * iT, dcx = dgx * iT, dcy = dgy * iT;
    int cx = min(max((int)floorf(cx0), 0), v.gw - 1);
    int cy = min(max((int)floorf(cy0), 0), v.gh - 1);
    const int stx = dcx > 0.f ? 1 : -1, sty = dcy > 0.f ? 1 : -1;
    const float idcx = 1.f / dcx, idcy = 1.f / dcy;
    int bx = cx + (dcx > 0.f ? 1 : 0), by = cy + (dcy > 0.f ? 1 : 0);
    float sx = (dcx != 0.f) ? ((float)bx - cx0) * idcx : INFINITY;
    float sy = (dcy != 0.f) ? ((float)by - cy0) * idcy : INFINITY;
    const float z0 = r.z0, dz = r.dz, idz = 1.f / r.dz;
    const bool inc = dz >= 0.f;
    int cz = 0;
    while (cz + 1 < v.nz && z0 >= v.edges[cz + 1]) ++cz;
    int ez = inc ? cz + 1 : cz;  // index of the next slab edge met
    float sz = (dz != 0.f) ? (v.edges[ez] - z0) * idz : INFINITY;
    const float w0 = r.w0, w1 = r.w1, dw = r.dw;
    int p = -1, plist = -1;
    PairCache pc;
    pc.k = -1;
    ColourCache<FMT> cc;
    cc.k = -1;
    float s_in = 0.f;
    const int maxit = v.gw + v.gh + v.nz + 3;
    for (int it = 0; it < maxit; ++it) {
        const float s_out = fminf(fminf(fminf(sx, sy), sz), 1.f);
        if (s_out > s_in) {
            const uint32_t cnt = __ldg(v.grid + ((size_t)cz * v.gh + cy) * v.gw + cx);
            if (cnt) {
                const int fx = min(v.T, v.w - cx * v.T), fy = min(v.T, v.h - cy * v.T);
                const float ua = s_in * w0 / fmaf(s_in, dw, w1);
                const float ub = s_out * w0 / fmaf(s_out, dw, w1);
                const float lc = r.lu * (ub - ua);
                const float want = ((float)cnt / (float)(fx * fy)) * lc * c.cell_scale;
                // at least one sample per occupied cell; the cap only guards non-finite input
                const int n = (want < 65536.f) ? max(1, (int)ceilf(want)) : 65536;
                const float du = (ub - ua) / (float)n, spacing = lc / (float)n;
                for (int k = 0; k < n; ++k) {
                    const float uk = fmaf((float)k + 0.5f, du, ua);
                    const float hx = fmaf(uk, r.h1.x - r.h0.x, r.h0.x);
                    const float hy = fmaf(uk, r.h1.y - r.h0.y, r.h0.y);
                    const float hz = fmaf(uk, r.h1.z - r.h0.z, r.h0.z);
                    const float hwc = fmaf(uk, r.h1.w - r.h0.w, r.h0.w);
                    const float iw = 1.f / hwc;
                    const float nx = hx * iw, ny = hy * iw, nz = hz * iw;
                    const int jx = min(max((int)floorf((nx + 1.f) * hw), 0), v.w - 1);
                    const int jy = min(max((int)floorf((1.f - ny) * hh), 0), v.h - 1);
                    const int li = jy * v.w + jx;
                    if (li != plist) {
                        pc.k = -1;
                        cc.k = -1;
                        plist = li;
                    }
                    const int j = first_inc<MODE>(v, li, nz, p, pc);
                    p = min(j, v.nsp - 1);
                    if (j < v.nsp) {
                        float f, b;
                        get_fb(pc, v, li, j, f, b);
                        if (f <= nz) {
                            add_piece(acc, get_colour<FMT>(cc, v, li, j), spacing);
                            if (ERT && acc.T <= kErtT) return;
                        }
                    }
                }
            }
        }
        if (s_out >= 1.f) break;
        if (sx <= sy && sx <= sz) {
            cx += stx;
            if ((unsigned)cx >= (unsigned)v.gw) break;
            bx += stx;
            sx = ((float)bx - cx0) * idcx;
        } else if (sy <= sz) {
            cy += sty;
            if ((unsigned)cy >= (unsigned)v.gh) break;
            by += sty;
            sy = ((float)by - cy0) * idcy;
        } else {
            cz += inc ? 1 : -1;
            if ((unsigned)cz >= (unsigned)v.nz) break;
            ez += inc ? 1 : -1;
            sz = (v.edges[ez] - z0) * idz;
        }
        s_in = fmaxf(s_in, s_out);
    }
}

template <int WX>
__device__ __forceinline__ void tile_pixel(int &px, int &py) {
    constexpr int WY = 32 / WX, BWX = 32 / WX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    px = blockIdx.x * 32 + (warp % BWX) * WX + (lane % WX);
    py = blockIdx.y * 8 + (warp / BWX) * WY + (lane / WX);
}

__device__ __forceinline__ void store_px(void *out, int out_fmt, size_t idx, const Accum &acc) {
    const float a = 1.f - acc.T;
    if (out_fmt == 0) {
        reinterpret_cast<float4 *>(out)[idx] = make_float4(acc.r, acc.g, acc.b, a);
    } else {
        __half2 lo = __floats2half2_rn(acc.r, acc.g), hi = __floats2half2_rn(acc.b, a);
        uint2 u;
        u.x = *reinterpret_cast<unsigned *>(&lo);
        u.y = *reinterpret_cast<unsigned *>(&hi);
        reinterpret_cast<uint2 *>(out)[idx] = u;
    }
}

template <int FMT, int MODE, bool ERT, int WX, bool PREVIEW>
__global__ void __launch_bounds__(256) render_kernel(const ViewConsts c, const DevVdi v, void *out,
                                                     int out_fmt, uint32_t *ray_lists,
                                                     uint32_t *ray_segs) {
    int px, py;
    tile_pixel<WX>(px, py);
    if (px >= c.W || py >= c.H) return;
    Accum acc = {0.f, 0.f, 0.f, 1.f};
    uint32_t nl = 0, nsg = 0;
    Ray r;
    if (setup_ray(c, px, py, r)) {
        if (PREVIEW)
            march_preview<FMT, MODE, ERT>(v, c, r, acc);
        else
            march_exact<FMT, MODE, ERT>(v, r, acc, nl, nsg);
    }
    const size_t idx = (size_t)py * c.W + px;
    store_px(out, out_fmt, idx, acc);
    if (ray_lists) ray_lists[idx] = nl;
    if (ray_segs) ray_segs[idx] = nsg;
}

// Instrumented exact render: marks the VDI words the algorithm reads.
template <int FMT>
__global__ void __launch_bounds__(256) touch_kernel(const ViewConsts c, const DevVdi v, uint32_t *bm) {
    int px, py;
    tile_pixel<32>(px, py);
    if (px >= c.W || py >= c.H) return;
    Accum acc = {0.f, 0.f, 0.f, 1.f};
    uint32_t nl = 0, nsg = 0;
    Ray r;
    if (setup_ray(c, px, py, r)) march_exact<FMT, kSearchAlg2, true, true>(v, r, acc, nl, nsg, bm);
}

cudaError_t launch_touch(const ViewConsts &c, const DevVdi &v, uint32_t *bm, cudaStream_t st) {
    dim3 grid(div_up(c.W, 32), div_up(c.H, 8)), block(256);
    if (v.fmt == 0)
        touch_kernel<0><<<grid, block, 0, st>>>(c, v, bm);
    else
        touch_kernel<1><<<grid, block, 0, st>>>(c, v, bm);
    return cudaGetLastError();
}

// Bilinear upsampling of the D_I preview: half-pixel centres, clamp to edge.
__global__ void upsample_kernel(const float4 *__restrict__ lo, int w0, int h0, void *out, int out_fmt,
                                int W, int H) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y;
    if (X >= W || Y >= H) return;
    const float u = ((float)X + 0.5f) * ((float)w0 / (float)W) - 0.5f;
    const float vv = ((float)Y + 0.5f) * ((float)h0 / (float)H) - 0.5f;
    const int i0 = (int)floorf(u), j0 = (int)floorf(vv);
    const float fu = u - (float)i0, fv = vv - (float)j0;
    const int i1 = min(max(i0 + 1, 0), w0 - 1), j1 = min(max(j0 + 1, 0), h0 - 1);
    const int ic = min(max(i0, 0), w0 - 1), jc = min(max(j0, 0), h0 - 1);
    const float4 a = __ldg(lo + (size_t)jc * w0 + ic), b = __ldg(lo + (size_t)jc * w0 + i1);
    const float4 d = __ldg(lo + (size_t)j1 * w0 + ic), e = __ldg(lo + (size_t)j1 * w0 + i1);
    Accum acc;
    float4 top = make_float4(fmaf(fu, b.x - a.x, a.x), fmaf(fu, b.y - a.y, a.y), fmaf(fu, b.z - a.z, a.z),
                             fmaf(fu, b.w - a.w, a.w));
    float4 bot = make_float4(fmaf(fu, e.x - d.x, d.x), fmaf(fu, e.y - d.y, d.y), fmaf(fu, e.z - d.z, d.z),
                             fmaf(fu, e.w - d.w, d.w));
    acc.r = fmaf(fv, bot.x - top.x, top.x);
    acc.g = fmaf(fv, bot.y - top.y, top.y);
    acc.b = fmaf(fv, bot.z - top.z, top.z);
    acc.T = 1.f - fmaf(fv, bot.w - top.w, top.w);
    store_px(out, out_fmt, (size_t)Y * W + X, acc);
}

// First-supersegment search on one list for a batch of queries (diagnostic).
template <int MODE>
__global__ void search_kernel(const DevVdi v, int li, const float *d_entry, const float *d_exit,
                              const int32_t *seed, const int32_t *inc, int32_t *result, int n) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    PairCache pc;
    pc.k = -1;
    const float de = d_entry[q], dx = d_exit[q];
    int j;
    if (inc[q]) {
        j = first_inc<MODE>(v, li, de, seed[q], pc);
        if (j >= v.nsp || ld_front(v, j, li) > dx) j = -1;
    } else {
        j = first_dec<MODE>(v, li, de, seed[q], pc);
        if (j >= 0 && ld_back(v, j, li) < dx) j = -1;
    }
    result[q] = j;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <int FMT, int MODE, bool ERT, bool PREVIEW>
static cudaError_t launch_ws(const ViewConsts &c, const DevVdi &v, void *out, int out_fmt,
                             uint32_t *rl, uint32_t *rs, int warp_shape, cudaStream_t st) {
    dim3 grid(div_up(c.W, 32), div_up(c.H, 8)), block(256);
    switch (warp_shape) {
        case 1:
            render_kernel<FMT, MODE, ERT, 16, PREVIEW><<<grid, block, 0, st>>>(c, v, out, out_fmt, rl, rs);
            break;
        case 2:
            render_kernel<FMT, MODE, ERT, 8, PREVIEW><<<grid, block, 0, st>>>(c, v, out, out_fmt, rl, rs);
            break;
        default:
            render_kernel<FMT, MODE, ERT, 32, PREVIEW><<<grid, block, 0, st>>>(c, v, out, out_fmt, rl, rs);
            break;
    }
    return cudaGetLastError();
}

template <int FMT, int MODE>
static cudaError_t launch_m(const ViewConsts &c, const DevVdi &v, void *out, int out_fmt, uint32_t *rl,
                            uint32_t *rs, int warp_shape, bool ert, bool preview, cudaStream_t st) {
    if (preview)
        return ert ? launch_ws<FMT, MODE, true, true>(c, v, out, out_fmt, rl, rs, warp_shape, st)
                   : launch_ws<FMT, MODE, false, true>(c, v, out, out_fmt, rl, rs, warp_shape, st);
    return ert ? launch_ws<FMT, MODE, true, false>(c, v, out, out_fmt, rl, rs, warp_shape, st)
               : launch_ws<FMT, MODE, false, false>(c, v, out, out_fmt, rl, rs, warp_shape, st);
}

cudaError_t launch_render(const ViewConsts &c, const DevVdi &v, void *out, int out_fmt, uint32_t *rl,
                          uint32_t *rs, int search, int warp_shape, bool ert, cudaStream_t st) {
    const bool preview = c.d_r > 1;
    if (v.fmt == 0) {
        if (search == kSearchBinary)
            return launch_m<0, kSearchBinary>(c, v, out, out_fmt, rl, rs, warp_shape, ert, preview, st);
        if (search == kSearchLinear)
            return launch_m<0, kSearchLinear>(c, v, out, out_fmt, rl, rs, warp_shape, ert, preview, st);
        return launch_m<0, kSearchAlg2>(c, v, out, out_fmt, rl, rs, warp_shape, ert, preview, st);
    }
    if (search == kSearchBinary)
        return launch_m<1, kSearchBinary>(c, v, out, out_fmt, rl, rs, warp_shape, ert, preview, st);
    if (search == kSearchLinear)
        return launch_m<1, kSearchLinear>(c, v, out, out_fmt, rl, rs, warp_shape, ert, preview, st);
    return launch_m<1, kSearchAlg2>(c, v, out, out_fmt, rl, rs, warp_shape, ert, preview, st);
}

cudaError_t launch_upsample(const float4 *lo, int w0, int h0, void *out, int out_fmt, int W, int H,
                            cudaStream_t st) {
    dim3 block(32, 8), grid(div_up(W, 32), div_up(H, 8));
    upsample_kernel<<<grid, block, 0, st>>>(lo, w0, h0, out, out_fmt, W, H);
    return cudaGetLastError();
}

cudaError_t launch_search(const DevVdi &v, int li, int search, const float *de, const float *dx,
                          const int32_t *seed, const int32_t *inc, int32_t *res, int n, cudaStream_t st) {
    const int nb = div_up(n, 128);
    if (search == kSearchBinary)
        search_kernel<kSearchBinary><<<nb, 128, 0, st>>>(v, li, de, dx, seed, inc, res, n);
    else if (search == kSearchLinear)
        search_kernel<kSearchLinear><<<nb, 128, 0, st>>>(v, li, de, dx, seed, inc, res, n);
    else
        search_kernel<kSearchAlg2><<<nb, 128, 0, st>>>(v, li, de, dx, seed, inc, res, n);
    return cudaGetLastError();
}

}  // namespace vdi
