// vdi_internal.cuh -- device-side data layout, per-view constants, loads and
// the first-supersegment searches shared by the render kernels.
//
// Device layout of a VDI (structure of arrays, slot-major so that lanes on
// neighbouring lists read neighbouring 16-byte records):
//   depth   float4 [nsp/2][nl]   (f_2k, b_2k, f_2k+1, b_2k+1)   FP32 V_O NDC z
//   colour  FP32: float4 [nsp][nl]   (r/a, g/a, b/a, kappa)
//           FP16: uint4  [nsp/2][nl] (two half4 (r/a, g/a, b/a, kappa) records)
//   grid    uint32 [nz][gh][gw]  supersegment counts per cell (Section 4.3)
//   range   float2 [nl]          (front of the first, back of the last supersegment)
//                                of each list, (+inf, -inf) when empty: a list the
//                                ray crosses entirely before or after it needs no search
//   brange  float2 [bh][bw]      the same for blocks of kB x kB lists (min front, max
//                                back): a ray whose depth range inside a block misses
//                                it skips the whole block
// nl = w*h lists, nsp = N_S rounded up to even; unused slots hold f = b = +inf
// and colour 0.  kappa = -log2(1 - alpha): Eq. 2's 1 - (1 - alpha)^l then is
// 1 - exp2(-kappa l), one exp2 per supersegment piece, and FP16 storage of
// kappa stays accurate for every l (storing alpha would lose 1 - alpha).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace vdi {

constexpr int kMaxNz = 64;
constexpr int kMaxNs = 64;
constexpr float kErtT = 1.0f / 4096.0f;  // stop once transmittance <= 2^-12
constexpr int kB = 4;                    // lists per side of a range block

enum { kSearchAlg2 = 0, kSearchBinary = 1, kSearchLinear = 2 };

struct DevVdi {
    int w, h, ns, nsp;
    int fmt;  // 0 = F32, 1 = F16
    long long nl;
    int nl32;  // nl as int: slot-plane offsets k * nl32 + li fit 32 bits (checked when the VDI is built)
    const float4 *depth;
    const void *colour;
    const uint32_t *grid;
    const float2 *range;
    const float2 *brange;
    int bw, bh;
    int T, gw, gh, nz;
    float edges[kMaxNz + 1];  // slab edges in V_O NDC z, edges[0] = -1, edges[nz] = 1
};

// Per-view constants built on the host in FP64 (vdi_api.cu, make_view_consts).
// A new-view ray through pixel NDC (x, y) is p(t) = O(x,y) + t D(x,y) in world
// space for t in [t_lo, t_hi] (V_N near plane to far plane).  Its image in
// V_O clip space is h(t) = a(x,y) + t b(x,y) with a = P_O V_O (O, 1) and
// b = P_O V_O (D, 0), both affine in (x, y); a is constant for a perspective
// V_N (O = eye), b is constant for an orthographic one.
struct ViewConsts {
    // a(px, py) = A0 + px Ax + py Ay for integer pixel indices (pixel centres
    // and the NDC scale folded in on the host), likewise b; FP32
    float A0[4], Ax[4], Ay[4];
    float B0[4], Bx[4], By[4];
    // the same affine forms in FP64, mapped to homogeneous list-grid
    // coordinates (hw (x + w), hh (w - y), w) of the VDI's w x h lists
    // (hw = w / 2, hh = h / 2): the exact start of rays that cross few lists
    double GA0[3], GAx[3], GAy[3];
    double GB0[3], GBx[3], GBy[3];
    int a_affine, b_affine;
    int frustum_clip;   // 0 when the volume box lies inside V_O's frustum
    int single_list;    // 1 when V_N's eye is V_O's eye: every ray stays in one list
    float O0[3], Ox[3], Oy[3];
    float D0[3], Dx[3], Dy[3];
    float t_lo, t_hi;
    float bmin[3], bmax[3];
    float inv_u;        // 1 / length_unit
    int W, H;           // rays rendered (after D_I)
    int rx0, rx1, ry0, ry1;  // pixel rectangle holding the box's image; rays outside it miss the box
    // 32 x 8 tiles of the render grid: tiles_x per row; the tiles meeting the
    // rectangle above span [tile_x0, tile_x0 + tile_w) x [tile_y0, tile_y0 + tile_h)
    // (tile_w = tile_h = 0 when it is empty)
    int tiles_x, tile_x0, tile_y0, tile_w, tile_h;
    float sx, sy;       // 2/W, 2/H
    int d_r;            // ray subsampling (1 = exact path)
    float cell_scale;   // length_unit / (slab view-depth extent * d_r)
};

// Bytes-touched instrumentation: one bit per 4-byte word of the depth array
// followed by the colour array.  The marks follow the algorithm's access rule
// (what a list visit and a supersegment piece need), not the width of the
// loads that serve it: the seed probe needs the two depths it compares, a
// binary-search probe one depth, a walked supersegment its front/back depth and
// its colour record.
template <bool TOUCH>
__device__ __forceinline__ void mark_word(uint32_t *bm, size_t w) {
    if (TOUCH) atomicOr(bm + (w >> 5), 1u << (w & 31));
}
template <bool TOUCH>
__device__ __forceinline__ void mark_depth(const DevVdi &v, uint32_t *bm, int j, int li, int which /*0 f, 1 b*/) {
    if (TOUCH) mark_word<TOUCH>(bm, ((size_t)(j >> 1) * v.nl + li) * 4 + 2 * (j & 1) + which);
}
// words of the touch bitmap: depth, then colour, then grid, then list ranges
__device__ __forceinline__ size_t grid_word_base(const DevVdi &v) {
    return (size_t)(v.nsp >> 1) * v.nl * 4 * ((v.fmt == 0) ? 3 : 2);
}
__device__ __forceinline__ size_t range_word_base(const DevVdi &v) {
    return grid_word_base(v) + (((size_t)v.nz * v.gh * v.gw + 3) & ~(size_t)3);
}
__device__ __forceinline__ size_t brange_word_base(const DevVdi &v) { return range_word_base(v) + 2 * (size_t)v.nl; }

template <bool TOUCH>
__device__ __forceinline__ void mark_colour(const DevVdi &v, uint32_t *bm, int j, int li) {
    if (TOUCH) {
        const size_t base = (size_t)(v.nsp >> 1) * v.nl * 4;
        if (v.fmt == 0) {
            for (int c = 0; c < 4; ++c) mark_word<TOUCH>(bm, base + ((size_t)j * v.nl + li) * 4 + c);
        } else {
            for (int c = 0; c < 2; ++c) mark_word<TOUCH>(bm, base + ((size_t)(j >> 1) * v.nl + li) * 4 + 2 * (j & 1) + c);
        }
    }
}

struct PairCache {
    int k;
    float4 d;
};

__device__ __forceinline__ float4 ld_depth_pair(const DevVdi &v, int k, int li) {
    return __ldg(v.depth + (k * v.nl32 + li));
}
__device__ __forceinline__ float ld_back(const DevVdi &v, int j, int li) {
    const float *p = reinterpret_cast<const float *>(v.depth + ((j >> 1) * v.nl32 + li));
    return __ldg(p + 2 * (j & 1) + 1);
}
__device__ __forceinline__ float ld_front(const DevVdi &v, int j, int li) {
    const float *p = reinterpret_cast<const float *>(v.depth + ((j >> 1) * v.nl32 + li));
    return __ldg(p + 2 * (j & 1));
}
__device__ __forceinline__ void get_fb(PairCache &pc, const DevVdi &v, int li, int j, float &f,
                                       float &b) {
    int k = j >> 1;
    if (k != pc.k) {
        pc.d = ld_depth_pair(v, k, li);
        pc.k = k;
    }
    f = (j & 1) ? pc.d.z : pc.d.x;
    b = (j & 1) ? pc.d.w : pc.d.y;
}

// colour of slot j: (r/a, g/a, b/a, kappa)
template <int FMT>
struct ColourCache {
    int k;
    uint4 q;
};

// FP16 colour: fetch the colour record of slot pair k (issued next to the
// pair's depth record, so that both loads are in flight together)
template <int FMT>
__device__ __forceinline__ void fetch_colour_pair(ColourCache<FMT> &cc, const DevVdi &v, int li, int k) {
    if (FMT == 1 && k != cc.k) {
        cc.q = __ldg(reinterpret_cast<const uint4 *>(v.colour) + (k * v.nl32 + li));
        cc.k = k;
    }
}

template <int FMT>
__device__ __forceinline__ float4 get_colour(ColourCache<FMT> &cc, const DevVdi &v, int li, int j) {
    if (FMT == 0) {
        return __ldg(reinterpret_cast<const float4 *>(v.colour) + (j * v.nl32 + li));
    } else {
        int k = j >> 1;
        if (k != cc.k) {
            cc.q = __ldg(reinterpret_cast<const uint4 *>(v.colour) + (k * v.nl32 + li));
            cc.k = k;
        }
        unsigned u0 = (j & 1) ? cc.q.z : cc.q.x;
        unsigned u1 = (j & 1) ? cc.q.w : cc.q.y;
        __half2 rg = *reinterpret_cast<__half2 *>(&u0);
        __half2 bk = *reinterpret_cast<__half2 *>(&u1);
        float2 a = __half22float2(rg), b = __half22float2(bk);
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

// ---------------------------------------------------------------------------
// First supersegment met by a ray entering a list (Section 4.2, Algorithm 2).
//
// Depth increasing along the ray: the answer is the smallest j with
// b_j >= d_entry (nsp if none).  Algorithm 2 seeds with p, the index of the
// last supersegment met in the previous list, reads b_{p-1} and b_p, counts
// how many of them lie at or beyond d_entry and then either keeps p or runs
// one binary search on the pruned range below or above p.  Here the seed is
// rounded up to odd, q = p | 1, so that b_{q-1} and b_q sit in one 16-byte
// depth record and the prefetch is a single load; the result is the same.
// Depth decreasing along the ray (the ray points back towards V_O): the mirror
// image, the largest j with f_j <= d_entry (-1 if none), seed q = p & ~1.
// ---------------------------------------------------------------------------
template <int MODE, bool TOUCH = false>
__device__ __forceinline__ int first_inc(const DevVdi &v, int li, float d, int p, PairCache &pc,
                                         uint32_t *bm = nullptr) {
    const int nsp = v.nsp;
    if (MODE == kSearchLinear) {
        int j = 0;
        for (; j < nsp; ++j) {
            float f, b;
            get_fb(pc, v, li, j, f, b);
            mark_depth<TOUCH>(v, bm, j, li, 1);
            if (b >= d) break;
        }
        return j;
    }
    int lo = 0, hi = nsp;  // answer in [lo, hi]; hi is either known to qualify or nsp
    if (MODE == kSearchAlg2 && p >= 0) {
        int q = p | 1;
        if (q >= nsp) q = nsp - 1;
        int k = q >> 1;
        if (pc.k != k) {
            pc.d = ld_depth_pair(v, k, li);
            pc.k = k;
        }
        mark_depth<TOUCH>(v, bm, q - 1, li, 1);
        mark_depth<TOUCH>(v, bm, q, li, 1);
        int interval = (pc.d.w >= d) + (pc.d.y >= d);
        if (interval == 1) {
            lo = hi = q;
        } else if (interval == 2) {
            lo = 0;
            hi = q - 1;
        } else {
            lo = q + 1;
            hi = nsp;
        }
    }
    while (lo < hi) {  // the single binary search of Algorithm 2 on [lo, hi)
        int mid = (lo + hi) >> 1;
        mark_depth<TOUCH>(v, bm, mid, li, 1);
        if (ld_back(v, mid, li) >= d)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

template <int MODE, bool TOUCH = false>
__device__ __forceinline__ int first_dec(const DevVdi &v, int li, float d, int p, PairCache &pc,
                                         uint32_t *bm = nullptr) {
    const int nsp = v.nsp;
    if (MODE == kSearchLinear) {
        int j = -1;
        for (; j + 1 < nsp; ++j) {
            float f, b;
            get_fb(pc, v, li, j + 1, f, b);
            mark_depth<TOUCH>(v, bm, j + 1, li, 0);
            if (!(f <= d)) break;
        }
        return j;
    }
    int lo = -1, hi = nsp - 1;  // answer in [lo, hi]; lo is either known to qualify or -1
    if (MODE == kSearchAlg2 && p >= 0) {
        int q = p & ~1;
        if (q >= nsp) q = nsp - 2;
        int k = q >> 1;
        if (pc.k != k) {
            pc.d = ld_depth_pair(v, k, li);
            pc.k = k;
        }
        mark_depth<TOUCH>(v, bm, q, li, 0);
        mark_depth<TOUCH>(v, bm, q + 1, li, 0);
        int interval = (pc.d.x <= d) + (pc.d.z <= d);
        if (interval == 1) {
            lo = hi = q;
        } else if (interval == 2) {
            lo = q + 1;
            hi = nsp - 1;
        } else {
            lo = -1;
            hi = q - 1;
        }
    }
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        mark_depth<TOUCH>(v, bm, mid, li, 0);
        if (ld_front(v, mid, li) <= d)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__host__ __device__ inline int div_up(int a, int b) { return (a + b - 1) / b; }

// PTX approximate reciprocal and base-2 exponential (documented relative
// errors of order 2^-23 and 2^-22): the render path needs no IEEE-rounded
// division, and Eq. 2's opacity 1 - 2^(-kappa l) tolerates a few ulp.
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float exp2_fast(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

}  // namespace vdi
