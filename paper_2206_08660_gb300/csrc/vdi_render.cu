// vdi_render.cu -- single-view kernels: new-view raycasting of a resident VDI
// (Section 4), the subsampled previews (Section 4.4), upsampling, the
// instrumented bytes-touched render and the search diagnostic.
//
// One thread per pixel ray.  A block covers a 32 x 8 tile that meets the
// volume box's pixel rectangle (those blocks are dispatched first); its eight
// warps cover 32x1, 16x2, 8x4 or 4x8 pixels each (the warp shape is a launch
// choice: lanes on neighbouring pixels walk neighbouring lists, so their
// 16-byte depth/colour loads coalesce).  The tiles outside the rectangle, whose
// rays all miss the box, are cleared by the last blocks, several tiles each.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "vdi_internal.cuh"
#include "vdi_march.cuh"
#include "vdi_preview.cuh"
#include "vdi_tma.cuh"

namespace vdi {

// PATH: 0 = exact walk over every list (the default), 1 = exact walk with
// empty-space skipping over the count grid, 3 = exact walk with range-block
// skipping, 5 = exact path for a view from V_O's eye (one list per ray).  The
// ray-subsampled previews (D_R > 1) have a kernel of their own below.
constexpr int kFillTiles = 8;  // tiles outside the box's pixel rectangle per block

// Fill block fb: kFillTiles tiles outside the box's pixel rectangle, whose
// rays all miss the box: transparent pixels (all-zero bytes in both output
// formats) and zero counters.  Where every tile row is a 16-byte multiple at
// a 16-byte boundary, the rows are bulk stores of a zeroed shared-memory row
// (one per thread of the first two warps); otherwise plain stores.  Every
// thread of the block must call this.
__device__ __forceinline__ void fill_tiles(const ViewConsts &c, void *out, int out_fmt, uint32_t *ray_lists,
                                           uint32_t *ray_segs, int fb) {
    const int nrect = c.tile_w * c.tile_h;
    const int ntiles = c.tiles_x * ((c.H + 7) >> 3);
    const int t0 = nrect + fb * kFillTiles, t1 = min(t0 + kFillTiles, ntiles);
    const bool bulk = ((reinterpret_cast<uintptr_t>(out) & 15) == 0) && (out_fmt == 0 || (c.W & 1) == 0) &&
                      !ray_lists && !ray_segs;
    if (bulk) {
        __shared__ alignas(128) uint4 zero_row[32];  // 32 pixels of FP32 RGBA
        if (threadIdx.x < 32) zero_row[threadIdx.x] = make_uint4(0u, 0u, 0u, 0u);
        fence_proxy_async_smem();
        __syncthreads();
        const int row = (int)threadIdx.x;  // tile t0 + row / 8, pixel row row % 8 of it
        if (row < (t1 - t0) * 8) {
            int tx, ty;
            tile_of_block(c, t0 + (row >> 3), tx, ty);
            const int py = ty * 8 + (row & 7), x0 = tx * 32;
            if (py < c.H && x0 < c.W) {
                const uint32_t bpp = out_fmt == 0 ? 16u : 8u;
                bulk_store_wait(reinterpret_cast<char *>(out) + ((size_t)py * c.W + x0) * bpp, zero_row,
                                (uint32_t)min(32, c.W - x0) * bpp);
            }
        }
        return;
    }
    const Accum miss = {0.f, 0.f, 0.f, 1.f};
    for (int t = t0; t < t1; ++t) {
        int tx, ty;
        tile_of_block(c, t, tx, ty);
        const int px = tx * 32 + (threadIdx.x & 31), py = ty * 8 + (threadIdx.x >> 5);
        if (px < c.W && py < c.H) {
            const size_t idx = (size_t)py * c.W + px;
            store_px(out, out_fmt, idx, miss);
            if (ray_lists) ray_lists[idx] = 0;
            if (ray_segs) ray_segs[idx] = 0;
        }
    }
}

// Resident blocks per SM the register allocation is held to: the one-list
// path for views from V_O's eye (PATH 5) waits on its records rather than on
// arithmetic and runs six (it requests slot pairs two at a time); the list
// walk four (64 registers); the walk with empty-space skipping three.
template <int PATH>
struct RenderOccupancy {
    static constexpr int blocks = PATH == 5 ? 6 : (PATH == 1 ? 3 : 4);
};

template <int FMT, int MODE, bool ERT, int WX, int PATH>
__global__ void __launch_bounds__(256, RenderOccupancy<PATH>::blocks) render_kernel(const ViewConsts c, const DevVdi v, void *out,
                                                     int out_fmt, uint32_t *ray_lists,
                                                     uint32_t *ray_segs) {
    const int nrect = c.tile_w * c.tile_h;
    if ((int)blockIdx.x >= nrect) {
        fill_tiles(c, out, out_fmt, ray_lists, ray_segs, (int)blockIdx.x - nrect);
        return;
    }
    int lx, ly, tx, ty;
    tile_offset<WX>(lx, ly);
    tile_of_block(c, blockIdx.x, tx, ty);
    const int px = tx * 32 + lx, py = ty * 8 + ly;
    if (px >= c.W || py >= c.H) return;
    Accum acc = {0.f, 0.f, 0.f, 1.f};
    uint32_t nl = 0, nsg = 0;
    Ray r;
    if (setup_ray(c, px, py, v.w, v.h, r)) {
        if (PATH == 1)
            march_exact_ess<FMT, MODE, ERT>(v, r, acc, nl, nsg);
        else if (PATH == 3)
            march_exact<FMT, MODE, ERT, false, true>(v, r, acc, nl, nsg);
        else if (PATH == 5)
            march_single<FMT, MODE, ERT>(v, r, acc, nl, nsg);
        else if (r.dz >= 0.f)  // two copies of the walk, one per depth direction
            march_exact<FMT, MODE, ERT, false, false, 1>(v, r, acc, nl, nsg);
        else
            march_exact<FMT, MODE, ERT, false, false, -1>(v, r, acc, nl, nsg);
    }
    const size_t idx = (size_t)py * c.W + px;
    store_px(out, out_fmt, idx, acc);
    if (ray_lists) ray_lists[idx] = nl;
    if (ray_segs) ray_segs[idx] = nsg;
}

// Exact path for a view from V_O's eye whose pixel (x, y) lands in list
// (x, y) (rendering from the original view): each 32 x 8 tile of rays reads
// one 32 x 8 tile of lists.  One thread requests that tile's list ranges and
// its first kSinglePF slot pairs (depth and colour) by TMA into shared memory
// as the block starts, so the copies overlap the ray setup; the rays then
// take their first records from there (march_single, STAGED) and request the
// later slot pairs from global memory.  The wait on the copies is bounded:
// when it runs out, the rays read global memory, the VDI's status word
// records it, and the block waits again before it exits.
template <int FMT, int MODE>
__global__ void __launch_bounds__(256, RenderOccupancy<5>::blocks)
    staged_single_kernel(const __grid_constant__ TileMaps tm, const ViewConsts c, const DevVdi v, void *out,
                         int out_fmt) {
    __shared__ alignas(128) StagedTile<FMT> st;
    __shared__ uint64_t bar;
    const int nrect = c.tile_w * c.tile_h;
    if ((int)blockIdx.x >= nrect) {
        fill_tiles(c, out, out_fmt, nullptr, nullptr, (int)blockIdx.x - nrect);
        return;
    }
    int tx, ty;
    tile_of_block(c, blockIdx.x, tx, ty);
    const int x0 = tx * 32, y0 = ty * 8;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, staged_bytes<FMT>(v.nsp));
        tma_load_2d(&st.range[0][0], &tm.range, 2 * x0, y0, &bar);
        tma_load_3d(&st.depth[0][0][0], &tm.depth, 4 * x0, y0, 0, &bar);
        tma_load_3d(&st.colour[0][0][0], &tm.colour, 4 * x0, y0, 0, &bar);
    }
    const int px = x0 + (int)(threadIdx.x & 31), py = y0 + (int)(threadIdx.x >> 5);
    const bool inside = px < c.W && py < c.H;
    Ray r;
    const bool hit = inside && setup_ray(c, px, py, v.w, v.h, r);
    const bool ready = mbar_wait(&bar, 0);
    if (!ready) atomicOr(tm.status, kStatusStageTimeout);
    Accum acc = {0.f, 0.f, 0.f, 1.f};
    uint32_t nl = 0, nsg = 0;
    if (hit) march_single<FMT, MODE, true, true>(v, r, acc, nl, nsg, ready ? &st : nullptr, x0, y0);
    if (inside) store_px(out, out_fmt, (size_t)py * c.W + px, acc);
    if (!ready) mbar_wait(&bar, 0);  // no copy into this block's shared memory may outlive it
}

// Ray-subsampled preview (Section 4.4) with L lanes per ray: the blocks of a
// 32 x 8 tile meeting the box's pixel rectangle (L blocks per tile, 256 / L
// rays each) come first, then the fill blocks of the tiles outside it.
template <int FMT, int L>
__global__ void __launch_bounds__(256, 4) preview_kernel(const ViewConsts c, const DevVdi v, void *out, int out_fmt) {
    constexpr int ROWS = 8 / L;  // tile rows per block
    const int nrect = c.tile_w * c.tile_h;
    if ((int)blockIdx.x >= nrect * L) {
        fill_tiles(c, out, out_fmt, nullptr, nullptr, (int)blockIdx.x - nrect * L);
        return;
    }
    const int tile = (int)blockIdx.x / L, unit = (int)blockIdx.x - tile * L;
    int tx, ty;
    tile_of_block(c, tile, tx, ty);
    const int g = (int)threadIdx.x / L;  // this lane's ray within the block
    const int px = tx * 32 + (g & 31), py = ty * 8 + unit * ROWS + (g >> 5);
    const bool inside = px < c.W && py < c.H;
    Ray r = {};
    const bool active = inside && setup_ray<false>(c, px, py, v.w, v.h, r);
    const Accum acc = march_preview_lanes<FMT, kPreviewProbe, L>(v, c, r, active);
    if (inside && (threadIdx.x & (L - 1)) == 0) store_px(out, out_fmt, (size_t)py * c.W + px, acc);
}

template <int FMT, int L>
static cudaError_t launch_preview_l(const ViewConsts &c, const DevVdi &v, void *out, int out_fmt, cudaStream_t st) {
    const int nrect = c.tile_w * c.tile_h, ntiles = div_up(c.W, 32) * div_up(c.H, 8);
    preview_kernel<FMT, L><<<nrect * L + div_up(ntiles - nrect, kFillTiles), 256, 0, st>>>(c, v, out, out_fmt);
    return cudaGetLastError();
}

// lanes per preview ray: more for launches with few rays, whose time is the
// longest ray's chain of dependent loads (the image is the same for any count)
template <int FMT>
static cudaError_t launch_preview(const ViewConsts &c, const DevVdi &v, void *out, int out_fmt, cudaStream_t st) {
    const long long rays = (long long)c.W * c.H;
    if (rays <= 300000) return launch_preview_l<FMT, 8>(c, v, out, out_fmt, st);
    if (rays <= 1200000) return launch_preview_l<FMT, 4>(c, v, out, out_fmt, st);
    return launch_preview_l<FMT, 2>(c, v, out, out_fmt, st);
}

// Instrumented exact render: marks the VDI words the algorithm reads.
template <int FMT>
__global__ void __launch_bounds__(256) touch_kernel(const ViewConsts c, const DevVdi v, uint32_t *bm) {
    int lx, ly;
    tile_offset<32>(lx, ly);
    const int px = blockIdx.x * 32 + lx, py = blockIdx.y * 8 + ly;
    if (px >= c.W || py >= c.H) return;
    Accum acc = {0.f, 0.f, 0.f, 1.f};
    uint32_t nl = 0, nsg = 0;
    Ray r;
    if (setup_ray(c, px, py, v.w, v.h, r)) march_exact<FMT, kSearchAlg2, true, true>(v, r, acc, nl, nsg, bm);
}

cudaError_t launch_touch(const ViewConsts &c, const DevVdi &v, uint32_t *bm, cudaStream_t st) {
    dim3 grid(div_up(c.W, 32), div_up(c.H, 8)), block(256);
    if (v.fmt == 0)
        touch_kernel<0><<<grid, block, 0, st>>>(c, v, bm);
    else
        touch_kernel<1><<<grid, block, 0, st>>>(c, v, bm);
    return cudaGetLastError();
}

// Bilinear upsampling of the D_I preview (upsample_px): a 32 x 8 block
// covers 32 kUpPixels x 8 output pixels.
__global__ void __launch_bounds__(256) upsample_kernel(const float4 *__restrict__ lo, int w0, int h0, void *out,
                                                        int out_fmt, int W, int H) {
    const int Y = blockIdx.y * blockDim.y + threadIdx.y;
    if (Y >= H) return;
    const int X0 = blockIdx.x * (32 * kUpPixels) + threadIdx.x;
    Accum acc[kUpPixels];
#pragma unroll
    for (int k = 0; k < kUpPixels; ++k)
        if (X0 + 32 * k < W) acc[k] = upsample_px(lo, w0, h0, W, H, X0 + 32 * k, Y);
#pragma unroll
    for (int k = 0; k < kUpPixels; ++k)
        if (X0 + 32 * k < W) store_px(out, out_fmt, (size_t)Y * W + X0 + 32 * k, acc[k]);
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

// Frame totals from per-ray counters: rays with at least one list, lists and
// pieces summed over the n rays (one atomic add per warp and total).
__global__ void count_totals_kernel(const uint32_t *__restrict__ lists, const uint32_t *__restrict__ segs, long long n,
                                    unsigned long long *totals) {
    unsigned long long hit = 0, nl = 0, ns = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t l = lists[i];
        hit += l > 0;
        nl += l;
        ns += segs[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        hit += __shfl_down_sync(0xffffffffu, hit, o);
        nl += __shfl_down_sync(0xffffffffu, nl, o);
        ns += __shfl_down_sync(0xffffffffu, ns, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(totals + 0, hit);
        atomicAdd(totals + 1, nl);
        atomicAdd(totals + 2, ns);
    }
}

cudaError_t launch_count_totals(const uint32_t *lists, const uint32_t *segs, long long n, unsigned long long *totals,
                                int sm_count, cudaStream_t st) {
    const int blocks = (int)std::min<long long>(div_up((int)std::min<long long>(n, 1LL << 30), 256), 4LL * sm_count);
    count_totals_kernel<<<std::max(blocks, 1), 256, 0, st>>>(lists, segs, n, totals);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

#define CK_RET(call)                      \
    do {                                  \
        cudaError_t e_ = (call);          \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

template <int FMT, int MODE, bool ERT, int PATH>
static cudaError_t launch_ws(const ViewConsts &c, const DevVdi &v, void *out, int out_fmt, uint32_t *rl,
                             uint32_t *rs, int warp_shape, cudaStream_t st) {
    // one block per 32 x 8 tile meeting the box's pixel rectangle, then one per
    // kFillTiles tiles outside it (tile_of_block's order)
    const int nrect = c.tile_w * c.tile_h, ntiles = div_up(c.W, 32) * div_up(c.H, 8);
    dim3 grid(nrect + div_up(ntiles - nrect, kFillTiles)), block(256);
    // the ablation searches are built with the default warp shape (4 x 8) only
    if (MODE == kSearchAlg2 && warp_shape == 0)
        render_kernel<FMT, MODE, ERT, 32, PATH><<<grid, block, 0, st>>>(c, v, out, out_fmt, rl, rs);
    else if (MODE == kSearchAlg2 && warp_shape == 1)
        render_kernel<FMT, MODE, ERT, 16, PATH><<<grid, block, 0, st>>>(c, v, out, out_fmt, rl, rs);
    else if (MODE == kSearchAlg2 && warp_shape == 2)
        render_kernel<FMT, MODE, ERT, 8, PATH><<<grid, block, 0, st>>>(c, v, out, out_fmt, rl, rs);
    else
        render_kernel<FMT, MODE, ERT, 4, PATH><<<grid, block, 0, st>>>(c, v, out, out_fmt, rl, rs);
    return cudaGetLastError();
}

// A view from V_O's eye renders the original image when pixel (x, y)'s ray
// lands in list (x, y): then a 32 x 8 tile of rays reads one 32 x 8 tile of
// lists, which the staged kernel loads by TMA.  The ray's list position is
// GB / GB_w (GA vanishes for such a view); a projective map that keeps the
// four corner pixel centres within a quarter list of their own list centres
// keeps every pixel in its list.  (Only the speed depends on this: a ray
// whose list lies outside its tile reads global memory.)
static bool stage_tiles(const ViewConsts &c, const DevVdi &v) {
    if (!c.single_list || c.d_r != 1 || c.W != v.w || c.H != v.h) return false;
    for (int corner = 0; corner < 4; ++corner) {
        const double px = (corner & 1) ? c.W - 1 : 0, py = (corner & 2) ? c.H - 1 : 0;
        double g[3];
        for (int k = 0; k < 3; ++k) g[k] = c.GB0[k] + px * c.GBx[k] + py * c.GBy[k];
        if (!(g[2] > 0.0) || !(fabs(g[0] / g[2] - (px + 0.5)) < 0.25) || !(fabs(g[1] / g[2] - (py + 0.5)) < 0.25))
            return false;
    }
    return true;
}

template <int FMT>
static cudaError_t launch_staged(const TileMaps &tm, const ViewConsts &c, const DevVdi &v, void *out, int out_fmt,
                                 cudaStream_t st) {
    const int nrect = c.tile_w * c.tile_h, ntiles = div_up(c.W, 32) * div_up(c.H, 8);
    staged_single_kernel<FMT, kSearchAlg2>
        <<<nrect + div_up(ntiles - nrect, kFillTiles), 256, 0, st>>>(tm, c, v, out, out_fmt);
    return cudaGetLastError();
}

template <int FMT, int MODE>
static cudaError_t launch_m(const ViewConsts &c, const DevVdi &v, void *out, int out_fmt, uint32_t *rl,
                            uint32_t *rs, int warp_shape, bool ert, bool ess, bool blocks, const TileMaps *tm,
                            cudaStream_t st) {
    if (c.d_r > 1) {
        // previews ignore the search mode and the warp shape (their samples use
        // a wide probe, several lanes serve a ray); their counters stay zero
        if (rl) CK_RET(cudaMemsetAsync(rl, 0, sizeof(uint32_t) * c.W * c.H, st));
        if (rs) CK_RET(cudaMemsetAsync(rs, 0, sizeof(uint32_t) * c.W * c.H, st));
        return launch_preview<FMT>(c, v, out, out_fmt, st);
    }
    // per-ray counters count whole lists, so they come from the walk over every list
    if (!ert) return launch_ws<FMT, MODE, false, 0>(c, v, out, out_fmt, rl, rs, warp_shape, st);
    if (rl || rs) return launch_ws<FMT, MODE, true, 0>(c, v, out, out_fmt, rl, rs, warp_shape, st);
    if (ess) return launch_ws<FMT, MODE, true, 1>(c, v, out, out_fmt, rl, rs, warp_shape, st);
    if (!blocks && c.single_list && MODE == kSearchAlg2) {
        // the staged kernel's warps cover 32 x 1 pixels (the default here); another
        // requested shape takes the unstaged one-list kernel with that shape
        if (tm && warp_shape == 0 && stage_tiles(c, v)) return launch_staged<FMT>(*tm, c, v, out, out_fmt, st);
        return launch_ws<FMT, MODE, true, 5>(c, v, out, out_fmt, rl, rs, warp_shape, st);
    }
    if (!blocks) return launch_ws<FMT, MODE, true, 0>(c, v, out, out_fmt, rl, rs, warp_shape, st);
    return launch_ws<FMT, MODE, true, 3>(c, v, out, out_fmt, rl, rs, warp_shape, st);
}

cudaError_t launch_render(const ViewConsts &c, const DevVdi &v, void *out, int out_fmt, uint32_t *rl, uint32_t *rs,
                          int search, int warp_shape, bool ert, bool ess, bool blocks, const TileMaps *tm,
                          cudaStream_t st) {
    if (v.fmt == 0) {
        if (search == kSearchBinary)
            return launch_m<0, kSearchBinary>(c, v, out, out_fmt, rl, rs, warp_shape, ert, ess, blocks, tm, st);
        if (search == kSearchLinear)
            return launch_m<0, kSearchLinear>(c, v, out, out_fmt, rl, rs, warp_shape, ert, ess, blocks, tm, st);
        return launch_m<0, kSearchAlg2>(c, v, out, out_fmt, rl, rs, warp_shape, ert, ess, blocks, tm, st);
    }
    if (search == kSearchBinary)
        return launch_m<1, kSearchBinary>(c, v, out, out_fmt, rl, rs, warp_shape, ert, ess, blocks, tm, st);
    if (search == kSearchLinear)
        return launch_m<1, kSearchLinear>(c, v, out, out_fmt, rl, rs, warp_shape, ert, ess, blocks, tm, st);
    return launch_m<1, kSearchAlg2>(c, v, out, out_fmt, rl, rs, warp_shape, ert, ess, blocks, tm, st);
}

cudaError_t launch_upsample(const float4 *lo, int w0, int h0, void *out, int out_fmt, int W, int H,
                            cudaStream_t st) {
    dim3 block(32, 8), grid(div_up(W, 32 * kUpPixels), div_up(H, 8));
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
