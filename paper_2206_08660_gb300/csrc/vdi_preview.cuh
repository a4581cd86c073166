// vdi_preview.cuh -- the ray-subsampled preview of Section 4.4 with several
// lanes of a warp per ray.
//
// A preview ray's samples are independent of one another once their positions
// are known: each takes the supersegment that contains it, with opacity for
// the sample spacing (Eq. 2).  Compositing is associative, so a ray's grid
// cells can be composited in parallel and the partial results merged in
// order.  The ray walks the count grid in rounds of kRoundCells cells; in a
// round, each of the L lanes serving the ray composites kRoundCells / L
// consecutive cells into a partial result, and the lanes merge the partials
// with warp shuffles in a fixed balanced tree over the round's cells (so the
// image does not depend on L).  Early termination is checked once per round.
// Launches with few rays (a preview at a high D_I or D_R fills less than a
// wave of the GPU with one lane per ray) run with more lanes per ray, which
// cuts the chain of dependent loads each lane waits for.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "vdi_internal.cuh"
#include "vdi_march.cuh"

namespace vdi {

constexpr int kRoundCells = 8;    // grid cells per compositing round
constexpr int kPreviewProbe = 2;  // depth records a preview sample requests at once

// a in front of b
__device__ __forceinline__ Accum over(const Accum &a, const Accum &b) {
    Accum o;
    o.r = fmaf(a.T, b.r, a.r);
    o.g = fmaf(a.T, b.g, a.g);
    o.b = fmaf(a.T, b.b, a.b);
    o.T = a.T * b.T;
    return o;
}

// One grid cell of a ray: linear cell index, its footprint in lists, and the
// ray's NDC line parameter range inside it (sb <= sa: nothing to sample).
struct CellRec {
    int cell, lists;
    float sa, sb;
};

// The ray's walk over the cells of the count grid (T x T lists by slabs of
// equal V_O view depth): Amanatides-Woo with boundary crossings computed
// directly from integer offsets, as in the list walk.
struct CellWalk {
    int cx, cy, cz, bx, by, ez, stx, sty;
    float sx, sy, sz, s_in, idgx, idgy, idz;
    bool ended;
};

__device__ __forceinline__ void cell_walk_init(CellWalk &w, const DevVdi &v, const Ray &r, bool active) {
    const int T = v.T;
    w.cx = min(max(r.ox, 0) / T, v.gw - 1);
    w.cy = min(max(r.oy, 0) / T, v.gh - 1);
    w.stx = r.dgx > 0.f ? 1 : -1;
    w.sty = r.dgy > 0.f ? 1 : -1;
    w.idgx = rcp_fast(r.dgx);
    w.idgy = rcp_fast(r.dgy);
    w.bx = (w.cx + (r.dgx > 0.f ? 1 : 0)) * T;
    w.by = (w.cy + (r.dgy > 0.f ? 1 : 0)) * T;
    w.sx = (r.dgx != 0.f) ? ((float)(w.bx - r.ox) - r.fx0) * w.idgx : INFINITY;
    w.sy = (r.dgy != 0.f) ? ((float)(w.by - r.oy) - r.fy0) * w.idgy : INFINITY;
    w.idz = rcp_fast(r.dz);
    const bool inc = r.dz >= 0.f;
    w.cz = 0;
    while (w.cz + 1 < v.nz && r.z0 >= v.edges[w.cz + 1]) ++w.cz;
    w.ez = inc ? w.cz + 1 : w.cz;
    w.sz = (r.dz != 0.f) ? (v.edges[w.ez] - r.z0) * w.idz : INFINITY;
    w.s_in = 0.f;
    w.ended = !active;
}

// The current cell, then a step to the next one.
__device__ __forceinline__ CellRec cell_walk_next(CellWalk &w, const DevVdi &v, const Ray &r) {
    CellRec c;
    const float s_out = fminf(fminf(fminf(w.sx, w.sy), w.sz), 1.f);
    c.cell = (w.cz * v.gh + w.cy) * v.gw + w.cx;
    c.lists = min(v.T, v.w - w.cx * v.T) * min(v.T, v.h - w.cy * v.T);
    c.sa = w.s_in;
    c.sb = w.ended ? w.s_in : s_out;
    if (!w.ended) {
        if (s_out >= 1.f) {
            w.ended = true;
        } else if (w.sx <= w.sy && w.sx <= w.sz) {
            w.cx += w.stx;
            if ((unsigned)w.cx >= (unsigned)v.gw) w.ended = true;
            w.bx += w.stx * v.T;
            w.sx = ((float)(w.bx - r.ox) - r.fx0) * w.idgx;
        } else if (w.sy <= w.sz) {
            w.cy += w.sty;
            if ((unsigned)w.cy >= (unsigned)v.gh) w.ended = true;
            w.by += w.sty * v.T;
            w.sy = ((float)(w.by - r.oy) - r.fy0) * w.idgy;
        } else {
            const bool inc = r.dz >= 0.f;
            w.cz += inc ? 1 : -1;
            if ((unsigned)w.cz >= (unsigned)v.nz) w.ended = true;
            w.ez += inc ? 1 : -1;
            if (!w.ended) w.sz = (v.edges[w.ez] - r.z0) * w.idz;
        }
        w.s_in = fmaxf(w.s_in, s_out);
    }
    return c;
}

// The samples of one cell (Section 4.4): in a cell holding cnt supersegments
// over its lists, crossed over world length l_c, n = ceil((cnt / lists)
// (l_c / slab depth extent) / D_R) samples at the midpoints of n equal
// pieces; each finds the supersegment containing it with a probe of PW depth
// records at a time (the first slot whose back reaches the sample's depth:
// Algorithm 2's result) and is composited with opacity for the spacing.
template <int FMT, int PW>
__device__ __forceinline__ void preview_cell(const DevVdi &v, const ViewConsts &c, const Ray &r, const CellRec &rec,
                                             Accum &part) {
    if (!(rec.sb > rec.sa)) return;
    const uint32_t cnt = __ldg(v.grid + rec.cell);
    if (!cnt) return;
    const float hw = 0.5f * (float)v.w, hh = 0.5f * (float)v.h;
    const float s_in = rec.sa, s_out = rec.sb;
    const float ua = s_in * r.w0 * rcp_fast(fmaf(s_in, r.dw, r.w1));
    const float ub = s_out * r.w0 * rcp_fast(fmaf(s_out, r.dw, r.w1));
    const float lc = r.lu * (ub - ua);
    const float want = ((float)cnt / (float)rec.lists) * lc * c.cell_scale;
    // at least one sample per occupied cell; the cap only guards non-finite input
    const int n = (want < 65536.f) ? max(1, (int)ceilf(want)) : 65536;
    const float du = (ub - ua) / (float)n, spacing = lc / (float)n;
    const int npairs = v.nsp >> 1;
    for (int k = 0; k < n; ++k) {
        const float uk = fmaf((float)k + 0.5f, du, ua);
        const float hx = fmaf(uk, r.h1.x - r.h0.x, r.h0.x);
        const float hy = fmaf(uk, r.h1.y - r.h0.y, r.h0.y);
        const float hz = fmaf(uk, r.h1.z - r.h0.z, r.h0.z);
        const float hwc = fmaf(uk, r.h1.w - r.h0.w, r.h0.w);
        const float iw = rcp_fast(hwc);
        const float nx = hx * iw, ny = hy * iw, nz = hz * iw;
        const int jx = min(max((int)floorf((nx + 1.f) * hw), 0), v.w - 1);
        const int jy = min(max((int)floorf((1.f - ny) * hh), 0), v.h - 1);
        const int li = jy * v.w + jx;
        const float2 rg = __ldg(v.range + li);
        if (nz < rg.x || nz > rg.y) continue;  // outside every supersegment of the list
        int j = v.nsp;
        float fj = INFINITY;
        for (int k0 = 0; k0 < npairs && j == v.nsp; k0 += PW) {
            float4 d[PW];
#pragma unroll
            for (int i = 0; i < PW; ++i)
                if (k0 + i < npairs) d[i] = ld_depth_pair(v, k0 + i, li);
#pragma unroll
            for (int i = PW - 1; i >= 0; --i)
                if (k0 + i < npairs) {
                    if (d[i].w >= nz) {
                        j = 2 * (k0 + i) + 1;
                        fj = d[i].z;
                    }
                    if (d[i].y >= nz) {
                        j = 2 * (k0 + i);
                        fj = d[i].x;
                    }
                }
        }
        if (j < v.nsp && fj <= nz) {
            ColourCache<FMT> cc;
            cc.k = -1;
            add_piece(part, get_colour<FMT>(cc, v, li, j), spacing);
        }
    }
}

// The preview of one ray served by L lanes (L in {2, 4, 8}: the lanes
// threadIdx.x & ~(L - 1) .. + L - 1 of a warp; every lane of the warp must
// call this, lanes without a ray with active = false).  Returns the ray's
// composite in every lane of the group.
template <int FMT, int PW, int L>
__device__ __forceinline__ Accum march_preview_lanes(const DevVdi &v, const ViewConsts &c, const Ray &r,
                                                     bool active) {
    constexpr int G = kRoundCells / L;  // consecutive cells per lane and round
    static_assert(L >= 2 && L <= kRoundCells && G * L == kRoundCells, "lanes per ray");
    const unsigned full = 0xffffffffu;
    const int sub = threadIdx.x & (L - 1);
    CellWalk w;
    cell_walk_init(w, v, r, active);
    Accum acc = {0.f, 0.f, 0.f, 1.f};
    bool going = active;
    const int maxr = (v.gw + v.gh + v.nz + 3 + kRoundCells - 1) / kRoundCells + 1;
    for (int round = 0; round < maxr && __any_sync(full, going); ++round) {
        // every lane steps through the round's cells and keeps its own G
        CellRec rec[G];
#pragma unroll
        for (int i = 0; i < kRoundCells; ++i) {
            const CellRec cur = cell_walk_next(w, v, r);
            if (i / G == sub) rec[i % G] = cur;
        }
        Accum part[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            part[g] = {0.f, 0.f, 0.f, 1.f};
            if (going) preview_cell<FMT, PW>(v, c, r, rec[g], part[g]);
        }
        // the lane's cells, then the lanes, merged as one balanced tree over the round's cells
#pragma unroll
        for (int s = 1; s < G; s <<= 1)
#pragma unroll
            for (int g = 0; g + s < G; g += 2 * s) part[g] = over(part[g], part[g + s]);
        Accum x = part[0];
#pragma unroll
        for (int off = 1; off < L; off <<= 1) {
            Accum o;
            o.r = __shfl_down_sync(full, x.r, off, L);
            o.g = __shfl_down_sync(full, x.g, off, L);
            o.b = __shfl_down_sync(full, x.b, off, L);
            o.T = __shfl_down_sync(full, x.T, off, L);
            if ((sub & (2 * off - 1)) == 0) x = over(x, o);
        }
        Accum round_total;
        round_total.r = __shfl_sync(full, x.r, 0, L);
        round_total.g = __shfl_sync(full, x.g, 0, L);
        round_total.b = __shfl_sync(full, x.b, 0, L);
        round_total.T = __shfl_sync(full, x.T, 0, L);
        if (going) acc = over(acc, round_total);
        if (acc.T <= kErtT || w.ended) going = false;
    }
    return acc;
}

}  // namespace vdi
