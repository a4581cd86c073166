// vdi_march.cuh -- per-ray device code of the render path (Section 4):
// ray setup in V_O clip space, the exact list walk with Algorithm 2 and Eq. 2,
// the ray-subsampled preview walk of Section 4.4, and pixel stores.  Shared
// by the single-view kernels (vdi_render.cu) and the batched persistent
// kernel (vdi_batch.cu).
#pragma once
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
    // list-grid position (x right, y down, in lists): g(s) = (ox + fx0, oy + fy0) + s (dgx, dgy);
    // the integer origin keeps the fraction, and every list crossing, at FP32 precision
    int ox, oy;
    float fx0, fy0, dgx, dgy;
    float w1, dw;              // D(s) = w1 + s (w0 - w1), clip w at the two ends mixed
    float lw;                  // world length / u of [sa, sb] = lw (sb - sa) / (D(sa) D(sb))
    float lu;                  // clipped world length / u
    float w0;
    float4 h0, h1;             // homogeneous clip coordinates of the two ends
};

__device__ __forceinline__ void clip_lin(float c0, float c1, float &t0, float &t1) {
    if (c1 > 0.f)
        t0 = fmaxf(t0, -c0 * rcp_fast(c1));
    else if (c1 < 0.f)
        t1 = fminf(t1, -c0 * rcp_fast(c1));
    else if (c0 < 0.f)
        t1 = -INFINITY;
}

// Ray setup (Section 4.1): the map of the pixel's ray into V_O clip space
// (a, b) as FP32 affine forms of the pixel indices; everything after it is
// FP32, except the exact start of rays that cross few lists (FP64, below).
constexpr float kPreciseSlope = 64.f;  // lists per ray below which list crossings need an FP64 start

// PRECISE_START: the FP64 start for rays that cross few lists (the exact list
// walk).  The ray-subsampled preview steps between grid cells eight lists
// apart and places samples in FP32 anyway, so it sets rays up in FP32 only.
template <bool PRECISE_START = true>
__device__ __forceinline__ bool setup_ray(const ViewConsts &c, int px, int py, int vw, int vh, Ray &r) {
    if (px < c.rx0 || px > c.rx1 || py < c.ry0 || py > c.ry1) return false;  // outside the box's image
    const float fpx = (float)px, fpy = (float)py;
    // pixel centre in V_N NDC (FP32 is enough for the world-space box clip)
    const float x = fmaf(fpx + 0.5f, c.sx, -1.f), y = fmaf(-(fpy + 0.5f), c.sy, 1.f);
    float t0 = c.t_lo, t1 = c.t_hi;
    // the volume box first (slabs, one reciprocal per axis): most rays that
    // miss the volume leave here
    float dl2 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float o = fmaf(y, c.Oy[k], fmaf(x, c.Ox[k], c.O0[k]));
        const float d = fmaf(y, c.Dy[k], fmaf(x, c.Dx[k], c.D0[k]));
        const float id = rcp_fast(d);
        float lo = (c.bmin[k] - o) * id, hi = (c.bmax[k] - o) * id;
        if (d == 0.f) {  // parallel to the slab: inside keeps the ray, outside rejects it
            hi = INFINITY;
            lo = (o < c.bmin[k] || o > c.bmax[k]) ? INFINITY : -INFINITY;
        }
        t0 = fmaxf(t0, fminf(lo, hi));
        t1 = fminf(t1, fmaxf(lo, hi));
        dl2 = fmaf(d, d, dl2);
    }
    if (!(t0 < t1)) return false;
    float a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = c.a_affine ? fmaf(fpx, c.Ax[k], fmaf(fpy, c.Ay[k], c.A0[k])) : c.A0[k];
        b[k] = c.b_affine ? fmaf(fpx, c.Bx[k], fmaf(fpy, c.By[k], c.B0[k])) : c.B0[k];
    }
    // V_O's frustum, -w <= x, y, z <= w; skipped when the host found the whole
    // box inside it (the clip could then never shorten the ray)
    if (c.frustum_clip) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            clip_lin(a[3] + a[k], b[3] + b[k], t0, t1);
            clip_lin(a[3] - a[k], b[3] - b[k], t0, t1);
        }
        if (!(t0 < t1)) return false;
    }
    float4 h0 = make_float4(fmaf(t0, b[0], a[0]), fmaf(t0, b[1], a[1]), fmaf(t0, b[2], a[2]),
                            fmaf(t0, b[3], a[3]));
    float4 h1 = make_float4(fmaf(t1, b[0], a[0]), fmaf(t1, b[1], a[1]), fmaf(t1, b[2], a[2]),
                            fmaf(t1, b[3], a[3]));
    if (!(h0.w > 0.f) || !(h1.w > 0.f)) return false;
    const float i0 = rcp_fast(h0.w), i1 = rcp_fast(h1.w);
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
    const float hw = 0.5f * (float)vw, hh = 0.5f * (float)vh;
    const float gx0 = (p0x + 1.f) * hw, gy0 = (1.f - p0y) * hh;
    const float gx1 = (p1x + 1.f) * hw, gy1 = (1.f - p1y) * hh;
    r.dgx = gx1 - gx0;
    r.dgy = gy1 - gy0;
    int ox = (int)floorf(gx0), oy = (int)floorf(gy0);
    float fx = gx0 - (float)ox, fy = gy0 - (float)oy;  // exact: the integer part is removed
    // A ray that drifts across few lists meets each list boundary at a grazing
    // angle: an FP32 start coordinate of magnitude w/2 (error ~ w 2^-25) would
    // move its crossings by that error / slope along the ray.  Such rays get
    // their start position relative to the integer origin in FP64.
    if (PRECISE_START && (((int)floorf(gx1) != ox && fabsf(r.dgx) < kPreciseSlope) ||
                          ((int)floorf(gy1) != oy && fabsf(r.dgy) < kPreciseSlope))) {
        // list-grid homogeneous coordinates G(t) = GA + t GB; the position
        // relative to the origin is (G_x - ox G_w) / G_w, whose numerator is
        // c + t d with c, d formed in FP64 before the cancellation
        const double dpx = (double)px, dpy = (double)py;
        double ga[3], gb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ga[k] = c.a_affine ? fma(dpx, c.GAx[k], fma(dpy, c.GAy[k], c.GA0[k])) : c.GA0[k];
            gb[k] = c.b_affine ? fma(dpx, c.GBx[k], fma(dpy, c.GBy[k], c.GB0[k])) : c.GB0[k];
        }
        const double dox = (double)ox, doy = (double)oy, td0 = (double)t0, td1 = (double)t1;
        const double cx = fma(-dox, ga[2], ga[0]), dx = fma(-dox, gb[2], gb[0]);
        const double cy = fma(-doy, ga[2], ga[1]), dy = fma(-doy, gb[2], gb[1]);
        fx = (float)fma(td0, dx, cx) * i0;
        fy = (float)fma(td0, dy, cy) * i0;
        r.dgx = (float)fma(td1, dx, cx) * i1 - fx;
        r.dgy = (float)fma(td1, dy, cy) * i1 - fy;
        if (fx < 0.f) {
            --ox;
            fx += 1.f;
        } else if (fx >= 1.f) {
            ++ox;
            fx -= 1.f;
        }
        if (fy < 0.f) {
            --oy;
            fy += 1.f;
        } else if (fy >= 1.f) {
            ++oy;
            fy -= 1.f;
        }
    }
    r.ox = ox;
    r.oy = oy;
    r.fx0 = fx;
    r.fy0 = fy;
    return true;
}

struct Accum {
    float r, g, b, T;
};

__device__ __forceinline__ void add_piece(Accum &acc, float4 col, float len_u) {
    const float e = exp2_fast(-col.w * len_u);
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
// Ray state shared by the list walks: NDC z = z0 + s dz, and the world length
// (in length units) of [sa, sb] is lw (sb - sa) / (D(sa) D(sb)) with
// D(s) = w1 + s dw (perspective-correct interpolation between the two ends).
struct Seg {
    float z0, dz, idz, w1, dw, lw;
};

// One list crossed by the ray over [s_in, s_out]: first supersegment by
// Algorithm 2 (seeded with p, the last index met in the previous list),
// adjacency walk, Eq. 2 per piece, front-to-back compositing.  Returns true
// once the ray is opaque (early termination).
// PRE: the caller has already loaded the list's range (rg_pre).  DIR: the
// sign of the ray's depth slope when the caller knows it (+1 / -1), 0 when it
// is decided at run time; the result is the same, the known sign saves work.
template <int FMT, int MODE, bool ERT, bool TOUCH, bool PRE = false, int DIR = 0>
__device__ __forceinline__ bool process_list(const DevVdi &v, const Seg &g, int li, float s_in, float s_out,
                                             int &p, Accum &acc, uint32_t &n_lists, uint32_t &n_segs,
                                             uint32_t *bm, bool &hot, float2 rg_pre = make_float2(0.f, 0.f)) {
    const float d_in = fmaf(s_in, g.dz, g.z0), d_out = fmaf(s_out, g.dz, g.z0);
    ++n_lists;
    PairCache pc;
    pc.k = -1;
    ColourCache<FMT> cc;
    cc.k = -1;
    {  // the ray crosses this list entirely before its first or after its last supersegment
        const float2 rg = PRE ? rg_pre : __ldg(v.range + li);
        if (MODE == kSearchAlg2 && p >= 0 && hot) {
            // the seed's depth and colour records, fetched together with the range
            // while the ray is in a run of lists it meets (hot: the previous
            // list passed its range test); a ray passing above or below the
            // data skips that speculative fetch
            pc.k = p >> 1;
            pc.d = ld_depth_pair(v, pc.k, li);
            fetch_colour_pair<FMT>(cc, v, li, pc.k);
        }
        if (TOUCH) {
            mark_word<TOUCH>(bm, range_word_base(v) + 2 * (size_t)li);
            mark_word<TOUCH>(bm, range_word_base(v) + 2 * (size_t)li + 1);
        }
        if (DIR > 0)
            hot = !(d_out < rg.x || d_in > rg.y);
        else if (DIR < 0)
            hot = !(d_in < rg.x || d_out > rg.y);
        else
            hot = !(fmaxf(d_in, d_out) < rg.x || fminf(d_in, d_out) > rg.y);
        if (!hot) return false;
    }
    int last = -1, first;
    if (DIR > 0 || (DIR == 0 && g.dz >= 0.f)) {
        first = first_inc<MODE, TOUCH>(v, li, d_in, p, pc, bm);
        for (int j = first; j < v.nsp; ++j) {
            float f, b;
            fetch_colour_pair<FMT>(cc, v, li, j >> 1);
            get_fb(pc, v, li, j, f, b);
            mark_depth<TOUCH>(v, bm, j, li, 0);
            mark_depth<TOUCH>(v, bm, j, li, 1);
            if (f > d_out) break;
            const float sa = (f > d_in) ? fminf(fmaxf((f - g.z0) * g.idz, s_in), s_out) : s_in;
            const float sb = (b < d_out) ? fminf(fmaxf((b - g.z0) * g.idz, s_in), s_out) : s_out;
            last = j;
            if (sb > sa) {
                mark_colour<TOUCH>(v, bm, j, li);
                const float4 col = get_colour<FMT>(cc, v, li, j);
                const float da = fmaf(sa, g.dw, g.w1), db = fmaf(sb, g.dw, g.w1);
                add_piece(acc, col, g.lw * (sb - sa) * rcp_fast(da * db));
                ++n_segs;
                if (ERT && acc.T <= kErtT) break;
            }
            if (b > d_out) break;
        }
    } else {
        first = first_dec<MODE, TOUCH>(v, li, d_in, p, pc, bm);
        for (int j = first; j >= 0; --j) {
            float f, b;
            fetch_colour_pair<FMT>(cc, v, li, j >> 1);
            get_fb(pc, v, li, j, f, b);
            mark_depth<TOUCH>(v, bm, j, li, 0);
            mark_depth<TOUCH>(v, bm, j, li, 1);
            if (b < d_out) break;
            const float sa = (b < d_in) ? fminf(fmaxf((b - g.z0) * g.idz, s_in), s_out) : s_in;
            const float sb = (f > d_out) ? fminf(fmaxf((f - g.z0) * g.idz, s_in), s_out) : s_out;
            last = j;
            if (sb > sa) {
                mark_colour<TOUCH>(v, bm, j, li);
                const float4 col = get_colour<FMT>(cc, v, li, j);
                const float da = fmaf(sa, g.dw, g.w1), db = fmaf(sb, g.dw, g.w1);
                add_piece(acc, col, g.lw * (sb - sa) * rcp_fast(da * db));
                ++n_segs;
                if (ERT && acc.T <= kErtT) break;
            }
            if (f < d_out) break;
        }
    }
    p = (last >= 0) ? last : first;
    if (p < 0) p = 0;
    return ERT && acc.T <= kErtT;
}

__device__ __forceinline__ Seg seg_of(const Ray &r) {
    Seg g;
    g.z0 = r.z0;
    g.dz = r.dz;
    g.idz = rcp_fast(r.dz);
    g.w1 = r.w1;
    g.dw = r.dw;
    g.lw = r.lw;
    return g;
}

// ---------------------------------------------------------------------------
// Exact path: every list the ray crosses (Amanatides-Woo in V_O NDC, Section
// 4.1) goes through process_list.  With BLOCKS, the walk first tests each
// kB x kB block of lists it enters: when the ray's depth range inside the
// block misses the block's [min front, max back] no list of the block can
// hold a supersegment the ray meets, and the walk jumps to where the ray
// leaves the block.  The image is the same; the skipped lists are not
// counted by the per-ray list counter, so counters use BLOCKS = false.
// ---------------------------------------------------------------------------
template <int FMT, int MODE, bool ERT, bool TOUCH = false, bool BLOCKS = false, int DIR = 0>
__device__ __forceinline__ void march_exact(const DevVdi &v, Ray &r, Accum &acc, uint32_t &n_lists,
                                            uint32_t &n_segs, uint32_t *bm = nullptr) {
    // list-grid position relative to the integer origin (ox, oy): boundary k is
    // crossed at s = ((k - ox) - f0) / dg, small exact integers minus a fraction
    const int ox = r.ox, oy = r.oy;
    const float gx0 = r.fx0, gy0 = r.fy0, dgx = r.dgx, dgy = r.dgy;
    int ix = min(max(ox, 0), v.w - 1);
    int iy = min(max(oy, 0), v.h - 1);
    const bool px_ = dgx > 0.f, py_ = dgy > 0.f;
    const int stx = px_ ? 1 : -1, sty = py_ ? 1 : -1;
    const float idgx = rcp_fast(dgx), idgy = rcp_fast(dgy);
    int bx = ix + (px_ ? 1 : 0), by = iy + (py_ ? 1 : 0);
    // crossing of the next boundary = (offset of the boundary from the origin) * idg - f0 * idg
    const float fsx = (float)stx, fsy = (float)sty, cx0 = -gx0 * idgx, cy0 = -gy0 * idgy;
    float fbx = (float)(bx - ox), fby = (float)(by - oy);
    float sx = (dgx != 0.f) ? fmaf(fbx, idgx, cx0) : INFINITY;
    float sy = (dgy != 0.f) ? fmaf(fby, idgy, cy0) : INFINITY;
    const Seg g = seg_of(r);
    // the first list has no previous list: a ray whose depth increases seeds
    // Algorithm 2 with the front-most supersegment (the one it most likely
    // meets first); a ray whose depth decreases runs the plain binary search
    int p = (g.dz >= 0.f) ? 0 : -1;
    bool hot = true;
    float s_in = 0.f;
    bool checked = !BLOCKS;
    const int maxit = v.w + v.h + 2 + (BLOCKS ? (v.bw + v.bh + 2) : 0);
    if (!BLOCKS) {
        // the walk with the next list's range requested one list ahead, so its
        // load overlaps the work on the current list
        int li = iy * v.w + ix;
        float2 rg = __ldg(v.range + li);
        for (int it = 0; it < maxit; ++it) {
            const float s_out = fminf(fminf(sx, sy), 1.f);
            const bool xs = sx <= sy;
            const int nix = xs ? ix + stx : ix, niy = xs ? iy : iy + sty;
            const bool nin = (unsigned)nix < (unsigned)v.w && (unsigned)niy < (unsigned)v.h;
            const int nli = nin ? niy * v.w + nix : li;
            float2 rg_next = rg;
            if (nin && s_out < 1.f) rg_next = __ldg(v.range + nli);  // not when the ray ends in this list
            if (s_out > s_in) {
                if (process_list<FMT, MODE, ERT, TOUCH, true, DIR>(v, g, li, s_in, s_out, p, acc, n_lists, n_segs,
                                                                   bm, hot, rg))
                    break;
            }
            if (s_out >= 1.f || !nin) break;
            if (xs) {
                fbx += fsx;
                sx = fmaf(fbx, idgx, cx0);
            } else {
                fby += fsy;
                sy = fmaf(fby, idgy, cy0);
            }
            ix = nix;
            iy = niy;
            li = nli;
            rg = rg_next;
            s_in = fmaxf(s_in, s_out);
        }
        return;
    }
    for (int it = 0; it < maxit; ++it) {
        if (BLOCKS && !checked) {
            const int cbx = ix / kB, cby = iy / kB;
            const int xb = (cbx + (px_ ? 1 : 0)) * kB, yb = (cby + (py_ ? 1 : 0)) * kB;  // exit faces, in lists
            const float sbx = (dgx != 0.f) ? fmaf((float)(xb - ox), idgx, cx0) : INFINITY;
            const float sby = (dgy != 0.f) ? fmaf((float)(yb - oy), idgy, cy0) : INFINITY;
            const float s_be = fminf(fminf(sbx, sby), 1.f);
            const float z_a = fmaf(s_in, g.dz, g.z0), z_b = fmaf(s_be, g.dz, g.z0);
            const float2 br = __ldg(v.brange + (size_t)cby * v.bw + cbx);
            if (TOUCH) {
                mark_word<TOUCH>(bm, brange_word_base(v) + 2 * ((size_t)cby * v.bw + cbx));
                mark_word<TOUCH>(bm, brange_word_base(v) + 2 * ((size_t)cby * v.bw + cbx) + 1);
            }
            checked = true;
            if (fmaxf(z_a, z_b) < br.x || fminf(z_a, z_b) > br.y) {
                // nothing in this block along the ray: continue from where it leaves the block
                if (s_be >= 1.f) break;
                if (sbx <= sby) {
                    ix = px_ ? xb : xb - 1;
                    if ((unsigned)ix >= (unsigned)v.w) break;
                    iy = min(max(oy + (int)floorf(fmaf(s_be, dgy, gy0)), cby * kB), min(cby * kB + kB, v.h) - 1);
                } else {
                    iy = py_ ? yb : yb - 1;
                    if ((unsigned)iy >= (unsigned)v.h) break;
                    ix = min(max(ox + (int)floorf(fmaf(s_be, dgx, gx0)), cbx * kB), min(cbx * kB + kB, v.w) - 1);
                }
                bx = ix + (px_ ? 1 : 0);
                by = iy + (py_ ? 1 : 0);
                fbx = (float)(bx - ox);
                fby = (float)(by - oy);
                sx = (dgx != 0.f) ? fmaf(fbx, idgx, cx0) : INFINITY;
                sy = (dgy != 0.f) ? fmaf(fby, idgy, cy0) : INFINITY;
                s_in = fmaxf(s_in, s_be);
                checked = false;
                continue;
            }
        }
        const float s_out = fminf(fminf(sx, sy), 1.f);
        if (s_out > s_in) {
            if (process_list<FMT, MODE, ERT, TOUCH>(v, g, iy * v.w + ix, s_in, s_out, p, acc, n_lists, n_segs, bm, hot))
                break;
        }
        if (s_out >= 1.f) break;
        if (sx <= sy) {
            ix += stx;
            if ((unsigned)ix >= (unsigned)v.w) break;
            fbx += fsx;
            sx = fmaf(fbx, idgx, cx0);
            if (BLOCKS && (ix & (kB - 1)) == (px_ ? 0 : kB - 1)) checked = false;  // entered a new block
        } else {
            iy += sty;
            if ((unsigned)iy >= (unsigned)v.h) break;
            fby += fsy;
            sy = fmaf(fby, idgy, cy0);
            if (BLOCKS && (iy & (kB - 1)) == (py_ ? 0 : kB - 1)) checked = false;
        }
        s_in = fmaxf(s_in, s_out);
    }
}

// ---------------------------------------------------------------------------
// Views from V_O's own eye (Section 4.1 at zero deviation): every ray projects
// to one point of V_O's image plane and stays in one list.  A ray that the
// list walk would treat as exactly one list over s in [0, 1] is composited
// here with the list's slot pairs (depth and colour records) requested PF at
// a time, instead of one dependent round trip per pair; its arithmetic is
// process_list's, so the image is the same.  Any other ray takes the list
// walk.
// ---------------------------------------------------------------------------
constexpr int kSinglePF = 2;  // slot pairs march_single requests at once

// The records a 32 x 8 tile of lists holds for the one-list path's first
// request, as TMA lays them out in shared memory: list ranges, the first
// kSinglePF depth slot pairs, their colour records (FP16 slot pairs, or FP32
// slots).  A VDI with fewer slot pairs stages all it has.
template <int FMT>
struct StagedTile {
    float2 range[8][32];
    float4 depth[kSinglePF][8][32];
    uint4 colour[(FMT == 1) ? kSinglePF : 2 * kSinglePF][8][32];
};

// slot pairs a VDI's staged tile holds, and the bytes its TMA requests bring
__host__ __device__ __forceinline__ int staged_pairs(int nsp) { return min(kSinglePF, nsp >> 1); }
template <int FMT>
__host__ __device__ __forceinline__ uint32_t staged_bytes(int nsp) {
    return (uint32_t)(8 * 32 * sizeof(float2) + (FMT == 1 ? 2 : 3) * staged_pairs(nsp) * 8 * 32 * sizeof(float4));
}

// STAGED: the list's range and first kSinglePF slot pairs come from the
// staged tile `st` (origin x0, y0) when it arrived (non-null) and holds the
// list, else from global memory; the arithmetic does not change.
template <int FMT, int MODE, bool ERT, bool STAGED = false>
__device__ __forceinline__ void march_single(const DevVdi &v, Ray &r, Accum &acc, uint32_t &n_lists,
                                             uint32_t &n_segs, const StagedTile<FMT> *st = nullptr, int x0 = 0,
                                             int y0 = 0) {
    constexpr int PF = kSinglePF;
    const int ox = r.ox, oy = r.oy;
    const float dgx = r.dgx, dgy = r.dgy;
    const int ix = min(max(ox, 0), v.w - 1), iy = min(max(oy, 0), v.h - 1);
    // the walk's first crossings, in the walk's own arithmetic
    const float idgx = rcp_fast(dgx), idgy = rcp_fast(dgy);
    const float cx0 = -r.fx0 * idgx, cy0 = -r.fy0 * idgy;
    const float fbx = (float)(ix + (dgx > 0.f ? 1 : 0) - ox), fby = (float)(iy + (dgy > 0.f ? 1 : 0) - oy);
    const float sx = (dgx != 0.f) ? fmaf(fbx, idgx, cx0) : INFINITY;
    const float sy = (dgy != 0.f) ? fmaf(fby, idgy, cy0) : INFINITY;
    if (!(fminf(sx, sy) >= 1.f) || !(r.dz >= 0.f)) {
        march_exact<FMT, MODE, ERT>(v, r, acc, n_lists, n_segs);
        return;
    }
    const Seg g = seg_of(r);
    const int li = iy * v.w + ix;
    const float d_in = fmaf(0.f, g.dz, g.z0), d_out = fmaf(1.f, g.dz, g.z0);
    ++n_lists;
    const int tlx = ix - x0, tly = iy - y0;
    const bool in_tile = STAGED && st != nullptr && (unsigned)tlx < 32u && (unsigned)tly < 8u;
    const int npairs = v.nsp >> 1;
    float2 rg;
    float4 dp[PF];
    uint4 cq[PF];
    if (in_tile) {  // slots past a short VDI's last pair are read but never used
        rg = st->range[tly][tlx];
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            dp[k] = st->depth[k][tly][tlx];
            if (FMT == 1) cq[k] = st->colour[k][tly][tlx];
        }
    } else {
        rg = __ldg(v.range + li);
#pragma unroll
        for (int k = 0; k < PF; ++k)
            if (k < npairs) {
                dp[k] = ld_depth_pair(v, k, li);
                if (FMT == 1) cq[k] = __ldg(reinterpret_cast<const uint4 *>(v.colour) + (k * v.nl32 + li));
            }
    }
    if (d_out < rg.x || d_in > rg.y) return;
    // slots in order; those with b < d_in lie before the first one met (b is
    // sorted).  The records come PF slot pairs at a time: the next PF pairs are
    // requested together once the current ones are used up.
    ColourCache<FMT> cc;
    cc.k = -1;
    bool done = false;
    for (int k0 = 0; k0 < npairs; k0 += PF) {
        if (k0 > 0) {
#pragma unroll
            for (int k = 0; k < PF; ++k)
                if (k0 + k < npairs) {
                    dp[k] = ld_depth_pair(v, k0 + k, li);
                    if (FMT == 1) cq[k] = __ldg(reinterpret_cast<const uint4 *>(v.colour) + ((k0 + k) * v.nl32 + li));
                }
        }
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            if (done || k0 + k >= npairs) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (done) break;
                const float f = h ? dp[k].z : dp[k].x, b = h ? dp[k].w : dp[k].y;
                if (b < d_in) continue;
                if (f > d_out) {
                    done = true;
                    break;
                }
                const float sa = (f > d_in) ? fminf(fmaxf((f - g.z0) * g.idz, 0.f), 1.f) : 0.f;
                const float sb = (b < d_out) ? fminf(fmaxf((b - g.z0) * g.idz, 0.f), 1.f) : 1.f;
                if (sb > sa) {
                    if (FMT == 1) {
                        cc.k = k0 + k;
                        cc.q = cq[k];
                    }
                    float4 col;
                    if (FMT == 0 && in_tile && k0 == 0) {
                        const uint4 q = st->colour[2 * k + h][tly][tlx];
                        col = make_float4(__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z),
                                          __uint_as_float(q.w));
                    } else {
                        col = get_colour<FMT>(cc, v, li, 2 * (k0 + k) + h);
                    }
                    const float da = fmaf(sa, g.dw, g.w1), db = fmaf(sb, g.dw, g.w1);
                    add_piece(acc, col, g.lw * (sb - sa) * rcp_fast(da * db));
                    ++n_segs;
                    if (ERT && acc.T <= kErtT) return;
                }
                if (b > d_out) done = true;
            }
        }
        if (done) return;
    }
}

// ---------------------------------------------------------------------------
// Exact path with empty-space skipping (Section 4.3): an outer walk over the
// cells of the count grid (T x T lists by slabs of equal V_O view depth)
// jumps over every cell whose count is 0 -- no supersegment overlaps it, so
// the ray can meet nothing there -- and runs the list walk of Section 4.1
// only inside occupied cells.  A list crossing several occupied cells is
// processed piecewise (pieces of one supersegment compose exactly, Eq. 2).
// Cell boundaries in x and y are computed with the list walk's own
// arithmetic, so both walks agree on where a cell ends.
// ---------------------------------------------------------------------------
template <int FMT, int MODE, bool ERT, bool TOUCH = false>
__device__ __forceinline__ void march_exact_ess(const DevVdi &v, Ray &r, Accum &acc, uint32_t &n_lists,
                                                uint32_t &n_segs, uint32_t *bm = nullptr) {
    const int ox = r.ox, oy = r.oy;
    const float gx0 = r.fx0, gy0 = r.fy0, dgx = r.dgx, dgy = r.dgy;
    const float idgx = rcp_fast(dgx), idgy = rcp_fast(dgy);
    const int stx = dgx > 0.f ? 1 : -1, sty = dgy > 0.f ? 1 : -1;
    const int T = v.T;
    const Seg g = seg_of(r);
    // cell walk
    int cx = min(max(ox, 0) / T, v.gw - 1);
    int cy = min(max(oy, 0) / T, v.gh - 1);
    int bcx = (cx + (dgx > 0.f ? 1 : 0)) * T, bcy = (cy + (dgy > 0.f ? 1 : 0)) * T;  // in lists
    float scx = (dgx != 0.f) ? ((float)(bcx - ox) - gx0) * idgx : INFINITY;
    float scy = (dgy != 0.f) ? ((float)(bcy - oy) - gy0) * idgy : INFINITY;
    const bool inc = g.dz >= 0.f;
    int cz = 0;
    while (cz + 1 < v.nz && g.z0 >= v.edges[cz + 1]) ++cz;
    int ez = inc ? cz + 1 : cz;
    float scz = (g.dz != 0.f) ? (v.edges[ez] - g.z0) * g.idz : INFINITY;
    float sc_in = 0.f, sc_out = 0.f;
    // list walk, (re)started lazily inside occupied cells
    int ix = 0, iy = 0, bx = 0, by = 0;
    float sx = 0.f, sy = 0.f, s_l_in = 0.f;
    bool lvalid = false, in_cell = false, fresh = true;
    bool hot = true;
    int p = -1;
    // One flat loop: every iteration is either one list step inside an occupied
    // cell or one cell step, so the lanes of a warp stay in step.
    const int maxit = 2 * (v.w + v.h) + v.gw + v.gh + v.nz + 8;
    for (int it = 0; it < maxit; ++it) {
        if (in_cell) {
            const float s_l_out = fminf(sx, sy);
            const float a = fmaxf(s_l_in, sc_in), b = fminf(s_l_out, sc_out);
            if (b > a &&
                process_list<FMT, MODE, ERT, TOUCH>(v, g, iy * v.w + ix, a, b, p, acc, n_lists, n_segs, bm, hot))
                return;
            if (s_l_out >= sc_out) {  // the list continues beyond this cell
                in_cell = false;
                continue;
            }
            if (sx <= sy) {
                ix += stx;
                if ((unsigned)ix >= (unsigned)v.w) return;
                bx += stx;
                sx = ((float)(bx - ox) - gx0) * idgx;
            } else {
                iy += sty;
                if ((unsigned)iy >= (unsigned)v.h) return;
                by += sty;
                sy = ((float)(by - oy) - gy0) * idgy;
            }
            s_l_in = s_l_out;
            continue;
        }
        if (!fresh) {  // advance to the next cell
            if (sc_out >= 1.f) return;
            if (scx <= scy && scx <= scz) {
                cx += stx;
                if ((unsigned)cx >= (unsigned)v.gw) return;
                bcx += stx * T;
                scx = ((float)(bcx - ox) - gx0) * idgx;
            } else if (scy <= scz) {
                cy += sty;
                if ((unsigned)cy >= (unsigned)v.gh) return;
                bcy += sty * T;
                scy = ((float)(bcy - oy) - gy0) * idgy;
            } else {
                cz += inc ? 1 : -1;
                if ((unsigned)cz >= (unsigned)v.nz) return;
                ez += inc ? 1 : -1;
                scz = (v.edges[ez] - g.z0) * g.idz;
            }
            sc_in = fmaxf(sc_in, sc_out);
        }
        fresh = false;
        sc_out = fminf(fminf(fminf(scx, scy), scz), 1.f);
        if (!(sc_out > sc_in)) continue;
        const size_t cell = ((size_t)cz * v.gh + cy) * v.gw + cx;
        mark_word<TOUCH>(bm, grid_word_base(v) + cell);
        if (__ldg(v.grid + cell) == 0u) {
            lvalid = false;
            continue;
        }
        if (!lvalid) {
            const float gx = fmaf(sc_in, dgx, gx0), gy = fmaf(sc_in, dgy, gy0);
            ix = min(max(ox + (int)floorf(gx), cx * T), min(cx * T + T, v.w) - 1);
            iy = min(max(oy + (int)floorf(gy), cy * T), min(cy * T + T, v.h) - 1);
            bx = ix + (dgx > 0.f ? 1 : 0);
            by = iy + (dgy > 0.f ? 1 : 0);
            sx = (dgx != 0.f) ? ((float)(bx - ox) - gx0) * idgx : INFINITY;
            sy = (dgy != 0.f) ? ((float)(by - oy) - gy0) * idgy : INFINITY;
            s_l_in = sc_in;
            lvalid = true;
        }
        in_cell = true;
    }
}

// Pixel of this thread inside a 32 x 8 tile whose warps cover WX x (32/WX)
// pixels each (lanes on neighbouring pixels walk neighbouring lists).
template <int WX>
__device__ __forceinline__ void tile_offset(int &dx, int &dy) {
    constexpr int WY = 32 / WX, BWX = 32 / WX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    dx = (warp % BWX) * WX + (lane % WX);
    dy = (warp / BWX) * WY + (lane / WX);
}

// The 32 x 8 tile of a linear block index: the tiles meeting the box's pixel
// rectangle come first (row by row), so the blocks that walk the VDI are
// dispatched together and fill the SMs; the tiles outside it (rays that miss
// the box: transparent pixels) follow in row order.
__device__ __forceinline__ void tile_of_block(const ViewConsts &c, int b, int &tx, int &ty) {
    const int nrect = c.tile_w * c.tile_h;
    if (b < nrect) {
        const int r = b / c.tile_w;
        ty = c.tile_y0 + r;
        tx = c.tile_x0 + (b - r * c.tile_w);
        return;
    }
    int k = b - nrect;
    const int above = c.tile_y0 * c.tiles_x;  // whole rows above the rectangle
    if (k < above) {
        ty = k / c.tiles_x;
        tx = k - ty * c.tiles_x;
        return;
    }
    k -= above;
    const int side = c.tiles_x - c.tile_w;  // tiles left and right of it in each of its rows
    if (k < c.tile_h * side) {
        const int r = k / side, q = k - r * side;
        ty = c.tile_y0 + r;
        tx = (q < c.tile_x0) ? q : q + c.tile_w;
        return;
    }
    k -= c.tile_h * side;  // whole rows below it
    const int r = k / c.tiles_x;
    ty = c.tile_y0 + c.tile_h + r;
    tx = k - r * c.tiles_x;
}

// Bilinear upsampling of a D_I preview (Section 4.4): output pixel (X, Y) of
// a W x H image from the w0 x h0 low-resolution one, half-pixel centres,
// clamp to edge.  The upsampling kernels give each thread kUpPixels output
// pixels 32 apart in x (stores stay coalesced; a thread has that many
// independent load chains).
constexpr int kUpPixels = 2;

__device__ __forceinline__ Accum upsample_px(const float4 *__restrict__ lo, int w0, int h0, int W, int H, int X,
                                             int Y) {
    const float u = ((float)X + 0.5f) * ((float)w0 / (float)W) - 0.5f;
    const float vv = ((float)Y + 0.5f) * ((float)h0 / (float)H) - 0.5f;
    const int i0 = (int)floorf(u), j0 = (int)floorf(vv);
    const float fu = u - (float)i0, fv = vv - (float)j0;
    const int i1 = min(max(i0 + 1, 0), w0 - 1), j1 = min(max(j0 + 1, 0), h0 - 1);
    const int ic = min(max(i0, 0), w0 - 1), jc = min(max(j0, 0), h0 - 1);
    const float4 a = __ldg(lo + (size_t)jc * w0 + ic), b = __ldg(lo + (size_t)jc * w0 + i1);
    const float4 d = __ldg(lo + (size_t)j1 * w0 + ic), e = __ldg(lo + (size_t)j1 * w0 + i1);
    const float4 top = make_float4(fmaf(fu, b.x - a.x, a.x), fmaf(fu, b.y - a.y, a.y), fmaf(fu, b.z - a.z, a.z),
                                   fmaf(fu, b.w - a.w, a.w));
    const float4 bot = make_float4(fmaf(fu, e.x - d.x, d.x), fmaf(fu, e.y - d.y, d.y), fmaf(fu, e.z - d.z, d.z),
                                   fmaf(fu, e.w - d.w, d.w));
    Accum acc;
    acc.r = fmaf(fv, bot.x - top.x, top.x);
    acc.g = fmaf(fv, bot.y - top.y, top.y);
    acc.b = fmaf(fv, bot.z - top.z, top.z);
    acc.T = 1.f - fmaf(fv, bot.w - top.w, top.w);
    return acc;
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

}  // namespace vdi
