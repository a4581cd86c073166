// vdi_batch.cu -- many views of several resident VDIs in one persistent
// launch, optionally replayed from a CUDA graph, plus the batch autotuner.
//
// Exact requests are cut into 32 x 8 pixel tiles, ray-subsampled previews into
// 32 x 2 tiles; each kind forms one queue, drained by its own persistent grid
// (SM count x resident blocks per SM) pulling tiles from an atomic counter, so
// requests of different resolutions, previews and VDIs share the GPU without a
// launch per view.  Requests with image-space
// subsampling (D_I > 1) render into a low-resolution scratch image and a second
// batched kernel upsamples all of them.  The per-request view constants (ray
// setup, Section 4.1) travel as kernel parameters, so a captured graph is
// replayed with new views by updating its kernel nodes.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vdi.h"
#include "vdi_api_internal.h"
#include "vdi_internal.cuh"
#include "vdi_march.cuh"
#include "vdi_preview.cuh"

namespace vdi {

constexpr int kMaxBatchReq = VDI_BATCH_MAX_REQUESTS;
constexpr int kBatchLanes = 4;  // lanes per ray of a preview request
constexpr int kMaxBatchVdi = VDI_BATCH_MAX_VDIS;

struct BatchReq {
    ViewConsts c;
    void *out;       // final image, or the low-resolution scratch when fewer rays than pixels
    int out_fmt;
    int vdi;         // index into BatchParams::vdis
    int tiles_x;
    int tile_base;   // first tile of this request in the queue
};

// Two tile queues: exact requests (32 x 8 tiles, one lane per ray) and
// ray-subsampled previews (32 x (8 / kBatchLanes) tiles, kBatchLanes lanes per
// ray), each pulled by its own persistent kernel from its own counter.  A
// request's tile_base counts within its queue; ex_idx / pv_idx list the
// requests of each queue in queue order.
struct BatchParams {
    int n_req, total_tiles, total_ptiles, n_ex, n_pv;
    unsigned *counter, *pcounter;
    unsigned char ex_idx[kMaxBatchReq], pv_idx[kMaxBatchReq];
    DevVdi vdis[kMaxBatchVdi];
    BatchReq reqs[kMaxBatchReq];
};

// kernel parameters are limited to 32764 bytes
static_assert(sizeof(BatchParams) <= 32000, "batch parameters exceed the kernel parameter limit");

struct UpReq {
    const float4 *lo;
    void *out;
    int w0, h0, W, H, out_fmt, tiles_x, tile_base;
};

struct UpParams {
    int n, total_tiles;
    UpReq reqs[kMaxBatchReq];
};

// The request of queue tile t: the last request in idx (queue order) whose
// tile_base is at most t.
__device__ __forceinline__ int queue_request(const BatchParams &P, const unsigned char *idx, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.reqs[idx[mid]].tile_base <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return idx[lo];
}

// The next tile of a queue for the whole block (thread 0 takes it from the
// counter); returns the tile (>= total when the queue is drained) and its request.
__device__ __forceinline__ int next_tile(const BatchParams &P, unsigned *counter, const unsigned char *idx, int n,
                                         int total, int &req) {
    __shared__ int s_tile, s_req;
    if (threadIdx.x == 0) {
        const int t = (int)atomicAdd(counter, 1u);
        s_tile = t;
        s_req = (t < total) ? queue_request(P, idx, n, t) : 0;
    }
    __syncthreads();
    const int t = s_tile;
    req = s_req;
    __syncthreads();  // every thread has read s_tile / s_req before thread 0 writes them again
    return t;
}

// Exact requests: the list walk of vdi_render, one lane per ray.
template <int WX>
__global__ void __launch_bounds__(256, 4) batch_render_kernel(const BatchParams P) {
    for (;;) {
        int r;
        const int tile = next_tile(P, P.counter, P.ex_idx, P.n_ex, P.total_tiles, r);
        if (tile >= P.total_tiles) return;  // uniform: every thread read the same tile
        const BatchReq &q = P.reqs[r];
        const DevVdi &v = P.vdis[q.vdi];
        const int local = tile - q.tile_base;
        const int tx0 = (local % q.tiles_x) * 32, ty0 = (local / q.tiles_x) * 8;
        int lx, ly;
        tile_offset<WX>(lx, ly);
        const int px = tx0 + lx, py = ty0 + ly;
        if (px < q.c.W && py < q.c.H) {
            Accum acc = {0.f, 0.f, 0.f, 1.f};
            uint32_t nl = 0, nsg = 0;
            Ray ray;
            if (setup_ray(q.c, px, py, v.w, v.h, ray)) {
                if (v.fmt == 0)
                    march_exact<0, kSearchAlg2, true>(v, ray, acc, nl, nsg);
                else
                    march_exact<1, kSearchAlg2, true>(v, ray, acc, nl, nsg);
            }
            store_px(q.out, q.out_fmt, (size_t)py * q.c.W + px, acc);
        }
    }
}

// Ray-subsampled previews: kBatchLanes lanes per ray (the same image as the
// single-view kernels' lane counts).
__global__ void __launch_bounds__(256, 3) batch_preview_kernel(const BatchParams P) {
    constexpr int rows = 8 / kBatchLanes;
    const int g = (int)threadIdx.x / kBatchLanes;
    for (;;) {
        int r;
        const int tile = next_tile(P, P.pcounter, P.pv_idx, P.n_pv, P.total_ptiles, r);
        if (tile >= P.total_ptiles) return;
        const BatchReq &q = P.reqs[r];
        const DevVdi &v = P.vdis[q.vdi];
        const int local = tile - q.tile_base;
        const int px = (local % q.tiles_x) * 32 + (g & 31), py = (local / q.tiles_x) * rows + (g >> 5);
        const bool inside = px < q.c.W && py < q.c.H;
        Ray ray = {};
        const bool active = inside && setup_ray<false>(q.c, px, py, v.w, v.h, ray);
        const Accum acc = (v.fmt == 0) ? march_preview_lanes<0, kPreviewProbe, kBatchLanes>(v, q.c, ray, active)
                                       : march_preview_lanes<1, kPreviewProbe, kBatchLanes>(v, q.c, ray, active);
        if (inside && (threadIdx.x & (kBatchLanes - 1)) == 0) store_px(q.out, q.out_fmt, (size_t)py * q.c.W + px, acc);
    }
}

__global__ void __launch_bounds__(256) batch_upsample_kernel(const UpParams P) {
    const int tile = blockIdx.x;
    int lo = 0, hi = P.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.reqs[mid].tile_base <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    const UpReq &q = P.reqs[lo];
    const int local = tile - q.tile_base;
    const int X0 = (local % q.tiles_x) * (32 * kUpPixels) + (threadIdx.x & 31);
    const int Y = (local / q.tiles_x) * 8 + (threadIdx.x >> 5);
    if (Y >= q.H) return;
    Accum acc[kUpPixels];
#pragma unroll
    for (int k = 0; k < kUpPixels; ++k)
        if (X0 + 32 * k < q.W) acc[k] = upsample_px(q.lo, q.w0, q.h0, q.W, q.H, X0 + 32 * k, Y);
#pragma unroll
    for (int k = 0; k < kUpPixels; ++k)
        if (X0 + 32 * k < q.W) store_px(q.out, q.out_fmt, (size_t)Y * q.W + X0 + 32 * k, acc[k]);
}

static const void *render_fn(int ws) {
    if (ws == 0) return (const void *)batch_render_kernel<32>;
    if (ws == 1) return (const void *)batch_render_kernel<16>;
    if (ws == 2) return (const void *)batch_render_kernel<8>;
    return (const void *)batch_render_kernel<4>;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct BatchPlan {
    BatchParams *bp = nullptr;  // host copies (large structs live on the heap)
    UpParams *up = nullptr;
    size_t scratch_bytes = 0;             // counter + low-resolution images
    std::vector<size_t> lo_offset;        // per request, (size_t)-1 if it renders every pixel
    std::vector<void *> final_out;
    ~BatchPlan() {
        delete bp;
        delete up;
    }
};

static vdi_status plan_batch(vdi_ctx *ctx, const vdi_request *reqs, int n, BatchPlan &pl) {
    if (n < 1 || n > kMaxBatchReq) return fail(VDI_ERR_INVALID_ARG, "batch of %d requests (1..%d)", n, kMaxBatchReq);
    pl.bp = new BatchParams();
    pl.up = new UpParams();
    memset(pl.bp, 0, sizeof(BatchParams));
    memset(pl.up, 0, sizeof(UpParams));
    std::vector<const vdi_t *> vdis;
    size_t off = 256;  // the two queue counters live at offsets 0 and 4
    int tiles = 0, ptiles = 0, up_tiles = 0;
    pl.lo_offset.assign(n, (size_t)-1);
    pl.final_out.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        const vdi_request &r = reqs[i];
        vdi_status s = check_render_args(r.vdi, r.W, r.H, r.d_i, r.d_r, r.out, r.out_fmt);
        if (s != VDI_OK) {
            const std::string m = vdi_last_error_message();
            return fail(s, "request %d: %s", i, m.c_str());
        }
        if ((r.Wr != 0 || r.Hr != 0) && (r.Wr < 1 || r.Hr < 1 || r.Wr > r.W || r.Hr > r.H))
            return fail(VDI_ERR_INVALID_ARG, "request %d: rays %dx%d for image %dx%d", i, r.Wr, r.Hr, r.W, r.H);
        if (r.vdi->ctx != ctx) return fail(VDI_ERR_INVALID_ARG, "request %d: VDI of another context", i);

        int vi = -1;
        for (size_t k = 0; k < vdis.size(); ++k)
            if (vdis[k] == r.vdi) vi = (int)k;
        if (vi < 0) {
            if ((int)vdis.size() == kMaxBatchVdi)
                return fail(VDI_ERR_INVALID_ARG, "more than %d distinct VDIs in one batch", kMaxBatchVdi);
            vi = (int)vdis.size();
            vdis.push_back(r.vdi);
            pl.bp->vdis[vi] = r.vdi->dv;
        }
        int Wr, Hr;
        request_rays(r, Wr, Hr);
        BatchReq &q = pl.bp->reqs[i];
        s = make_view_consts(r.vdi, &r.view, Wr, Hr, r.d_r, &q.c);
        if (s != VDI_OK) {
            const std::string m = vdi_last_error_message();
            return fail(s, "request %d: %s", i, m.c_str());
        }
        q.vdi = vi;
        q.tiles_x = div_up(Wr, 32);
        if (r.d_r > 1) {  // preview queue: 32 x (8 / kBatchLanes) tiles
            q.tile_base = ptiles;
            ptiles += q.tiles_x * div_up(Hr, 8 / kBatchLanes);
            pl.bp->pv_idx[pl.bp->n_pv++] = (unsigned char)i;
        } else {  // exact queue: 32 x 8 tiles
            q.tile_base = tiles;
            tiles += q.tiles_x * div_up(Hr, 8);
            pl.bp->ex_idx[pl.bp->n_ex++] = (unsigned char)i;
        }
        pl.final_out[i] = r.out;
        if (Wr == r.W && Hr == r.H) {
            q.out = r.out;
            q.out_fmt = r.out_fmt;
        } else {
            pl.lo_offset[i] = off;
            off += ((size_t)Wr * Hr * sizeof(float4) + 255) & ~(size_t)255;
            q.out_fmt = VDI_F32;
            UpReq &u = pl.up->reqs[pl.up->n++];
            u.out = r.out;
            u.w0 = Wr;
            u.h0 = Hr;
            u.W = r.W;
            u.H = r.H;
            u.out_fmt = r.out_fmt;
            u.tiles_x = div_up(r.W, 32 * kUpPixels);
            u.tile_base = up_tiles;
            up_tiles += u.tiles_x * div_up(r.H, 8);
        }
    }
    pl.bp->n_req = n;
    pl.bp->total_tiles = tiles;
    pl.bp->total_ptiles = ptiles;
    pl.up->total_tiles = up_tiles;
    pl.scratch_bytes = off;
    return VDI_OK;
}

// point the plan at a scratch allocation
static void bind_scratch(BatchPlan &pl, char *scratch) {
    pl.bp->counter = reinterpret_cast<unsigned *>(scratch);
    pl.bp->pcounter = reinterpret_cast<unsigned *>(scratch) + 1;
    int k = 0;
    for (int i = 0; i < pl.bp->n_req; ++i)
        if (pl.lo_offset[i] != (size_t)-1) {
            pl.bp->reqs[i].out = scratch + pl.lo_offset[i];
            pl.up->reqs[k++].lo = reinterpret_cast<const float4 *>(scratch + pl.lo_offset[i]);
        }
}

// persistent grid of the exact kernel: resident blocks per SM (capped at bps
// when bps > 0) times the SM count, no more blocks than tiles
static int exact_grid(vdi_ctx *ctx, const BatchPlan &pl, int ws, int bps) {
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, render_fn(ws), 256, 0);
    if (bps > 0) occ = std::min(occ, bps);
    return std::min(std::max(1, occ) * ctx->sm_count, std::max(1, pl.bp->total_tiles));
}

static int preview_grid(vdi_ctx *ctx, const BatchPlan &pl) {
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)batch_preview_kernel, 256, 0);
    return std::min(std::max(1, occ) * ctx->sm_count, std::max(1, pl.bp->total_ptiles));
}

static cudaError_t enqueue_plain(vdi_ctx *ctx, BatchPlan &pl, int ws, int bps, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(pl.bp->counter, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    void *args[] = {pl.bp};
    if (pl.bp->n_ex) e = cudaLaunchKernel(render_fn(ws), dim3(exact_grid(ctx, pl, ws, bps)), dim3(256), args, 0, st);
    if (e != cudaSuccess) return e;
    if (pl.bp->n_pv)
        e = cudaLaunchKernel((const void *)batch_preview_kernel, dim3(preview_grid(ctx, pl)), dim3(256), args, 0, st);
    if (e != cudaSuccess || pl.up->n == 0) return e;
    void *uargs[] = {pl.up};
    return cudaLaunchKernel((const void *)batch_upsample_kernel, dim3(pl.up->total_tiles), dim3(256), uargs, 0, st);
}

// A cached executable graph for one batch shape: memset(counter) -> persistent
// render -> batched upsample, with its own scratch.
struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t render_node = nullptr, preview_node = nullptr, up_node = nullptr;
    void *scratch = nullptr;
    int grid = 0, pgrid = 0;
};

struct BatchCache {
    std::mutex mu;
    std::map<std::string, GraphEntry> graphs;
    std::map<std::string, vdi_batch_opts> tuned;
};

static BatchCache &cache_of(vdi_ctx *ctx) {
    static std::mutex mu;
    static std::map<vdi_ctx *, BatchCache *> m;
    std::lock_guard<std::mutex> g(mu);
    BatchCache *&c = m[ctx];
    if (!c) c = new BatchCache();
    return *c;
}

static std::string shape_key(const vdi_request *reqs, int n, const BatchPlan &pl, int ws, int bps, cudaStream_t st) {
    std::string k = std::to_string((unsigned long long)(uintptr_t)st) + "|" + std::to_string(ws) + "|" +
                    std::to_string(bps) + "|" + std::to_string(pl.scratch_bytes);
    for (int i = 0; i < n; ++i) {
        int Wr, Hr;
        request_rays(reqs[i], Wr, Hr);
        k += "|" + std::to_string(reqs[i].W) + "x" + std::to_string(reqs[i].H) + "/" + std::to_string(Wr) + "x" +
             std::to_string(Hr) + "/" + std::to_string(reqs[i].d_r);
    }
    return k;
}

// batch signature used by the autotuner: resolutions, previews and formats
static std::string tune_key(const vdi_request *reqs, int n) {
    std::vector<std::string> parts;
    for (int i = 0; i < n; ++i) {
        int Wr, Hr;
        request_rays(reqs[i], Wr, Hr);
        parts.push_back(std::to_string(reqs[i].W) + "x" + std::to_string(reqs[i].H) + "/" + std::to_string(Wr) + "x" +
                        std::to_string(Hr) + "/" + std::to_string(reqs[i].d_r) + "/" +
                        std::to_string(reqs[i].vdi->dv.nsp) + "/" + std::to_string(reqs[i].vdi->dv.fmt));
    }
    std::sort(parts.begin(), parts.end());
    std::string k;
    for (auto &p : parts) k += p + ";";
    return k;
}

static cudaKernelNodeParams kernel_node(const void *fn, int grid, void **args) {
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(fn);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    return kp;
}

// memset(counters) -> {persistent exact kernel, persistent preview kernel} ->
// batched upsample; a replay of the same shape only updates kernel parameters
static vdi_status enqueue_graph(vdi_ctx *ctx, const vdi_request *reqs, int n, BatchPlan &pl, int ws, int bps,
                                cudaStream_t st) {
    BatchCache &bc = cache_of(ctx);
    std::lock_guard<std::mutex> g(bc.mu);
    const std::string key = shape_key(reqs, n, pl, ws, bps, st);
    auto it = bc.graphs.find(key);
    cudaError_t e = cudaSuccess;
    void *args[] = {pl.bp};
    void *uargs[] = {pl.up};
    if (it == bc.graphs.end()) {
        GraphEntry ge;
        if ((e = cudaMalloc(&ge.scratch, pl.scratch_bytes)) != cudaSuccess) return cuda_fail(e, "graph scratch");
        bind_scratch(pl, (char *)ge.scratch);
        ge.grid = exact_grid(ctx, pl, ws, bps);
        ge.pgrid = preview_grid(ctx, pl);
        cudaGraphNode_t ms = nullptr;
        cudaMemsetParams mp{};
        mp.dst = ge.scratch;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 2;
        mp.height = 1;
        mp.pitch = 8;
        std::vector<cudaGraphNode_t> renders;
        e = cudaGraphCreate(&ge.graph, 0);
        if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&ms, ge.graph, nullptr, 0, &mp);
        if (e == cudaSuccess && pl.bp->n_ex) {
            const cudaKernelNodeParams kp = kernel_node(render_fn(ws), ge.grid, args);
            e = cudaGraphAddKernelNode(&ge.render_node, ge.graph, &ms, 1, &kp);
            renders.push_back(ge.render_node);
        }
        if (e == cudaSuccess && pl.bp->n_pv) {
            const cudaKernelNodeParams kp = kernel_node((const void *)batch_preview_kernel, ge.pgrid, args);
            e = cudaGraphAddKernelNode(&ge.preview_node, ge.graph, &ms, 1, &kp);
            renders.push_back(ge.preview_node);
        }
        if (e == cudaSuccess && pl.up->n) {
            const cudaKernelNodeParams kp = kernel_node((const void *)batch_upsample_kernel, pl.up->total_tiles, uargs);
            e = cudaGraphAddKernelNode(&ge.up_node, ge.graph, renders.data(), renders.size(), &kp);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge.exec, ge.graph, 0);
        if (e != cudaSuccess) {
            if (ge.graph) cudaGraphDestroy(ge.graph);
            cudaFree(ge.scratch);
            return cuda_fail(e, "graph build");
        }
        it = bc.graphs.emplace(key, ge).first;
    } else {
        GraphEntry &ge = it->second;
        bind_scratch(pl, (char *)ge.scratch);
        if (ge.render_node) {
            const cudaKernelNodeParams kp = kernel_node(render_fn(ws), ge.grid, args);
            e = cudaGraphExecKernelNodeSetParams(ge.exec, ge.render_node, &kp);
        }
        if (e == cudaSuccess && ge.preview_node) {
            const cudaKernelNodeParams kp = kernel_node((const void *)batch_preview_kernel, ge.pgrid, args);
            e = cudaGraphExecKernelNodeSetParams(ge.exec, ge.preview_node, &kp);
        }
        if (e == cudaSuccess && ge.up_node) {
            const cudaKernelNodeParams kp = kernel_node((const void *)batch_upsample_kernel, pl.up->total_tiles, uargs);
            e = cudaGraphExecKernelNodeSetParams(ge.exec, ge.up_node, &kp);
        }
        if (e != cudaSuccess) return cuda_fail(e, "graph update");
    }
    if ((e = cudaGraphLaunch(it->second.exec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
    return VDI_OK;
}

vdi_status render_batch(vdi_ctx *ctx, const vdi_request *reqs, int n, const vdi_batch_opts *opts, cudaStream_t st) {
    BatchPlan pl;
    vdi_status s = plan_batch(ctx, reqs, n, pl);
    if (s != VDI_OK) return s;
    vdi_batch_opts o = {-1, 0, 1};
    if (opts) o = *opts;
    if (o.warp_shape < 0) {
        BatchCache &bc = cache_of(ctx);
        std::lock_guard<std::mutex> g(bc.mu);
        auto it = bc.tuned.find(tune_key(reqs, n));
        if (it != bc.tuned.end()) {
            o.warp_shape = it->second.warp_shape;
            if (o.blocks_per_sm == 0) o.blocks_per_sm = it->second.blocks_per_sm;
        } else {
            o.warp_shape = 3;  // 4 x 8 pixels per warp, the single-view default
        }
    }
    if (o.warp_shape > 3) return fail(VDI_ERR_INVALID_ARG, "warp_shape=%d", o.warp_shape);
    if (o.blocks_per_sm < 0) return fail(VDI_ERR_INVALID_ARG, "blocks_per_sm=%d", o.blocks_per_sm);
    if (o.use_graph) return enqueue_graph(ctx, reqs, n, pl, o.warp_shape, o.blocks_per_sm, st);
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, pl.scratch_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch scratch");
    bind_scratch(pl, (char *)scratch);
    e = enqueue_plain(ctx, pl, o.warp_shape, o.blocks_per_sm, st);
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return VDI_OK;
}

void release_batch_cache(vdi_ctx *ctx) {
    BatchCache &bc = cache_of(ctx);
    std::lock_guard<std::mutex> g(bc.mu);
    for (auto &kv : bc.graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
        cudaFree(kv.second.scratch);
    }
    bc.graphs.clear();
}

}  // namespace vdi

using namespace vdi;

#define VDI_API extern "C" __attribute__((visibility("default")))

VDI_API vdi_status vdi_render_batch(vdi_ctx *ctx, const vdi_request *reqs, int n, const vdi_batch_opts *opts,
                                    void *stream) {
    if (!ctx || !reqs) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(ctx->device);
    return render_batch(ctx, reqs, n, opts, (cudaStream_t)stream);
}

// Time every launch configuration on this batch (renders into the requests'
// outputs) and remember the fastest for batches with the same signature.
VDI_API vdi_status vdi_autotune_batch(vdi_ctx *ctx, const vdi_request *reqs, int n, void *stream,
                                      vdi_batch_opts *best, float *best_ms) {
    if (!ctx || !reqs) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    vdi_batch_opts winner = {0, 0, 0};
    float wms = INFINITY;
    vdi_status s = VDI_OK;
    for (int ws = 0; ws <= 3 && s == VDI_OK; ++ws) {
        int occ_max = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_max, render_fn(ws), 256, 0);
        for (int bps = 1; bps <= std::max(1, occ_max) && s == VDI_OK; ++bps) {
            vdi_batch_opts o = {ws, bps, 0};
            s = render_batch(ctx, reqs, n, &o, st);  // warm-up
            if (s != VDI_OK) break;
            float tot = 0.f;
            const int reps = 3;
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && s == VDI_OK; ++r) s = render_batch(ctx, reqs, n, &o, st);
            cudaEventRecord(e1, st);
            cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) {
                s = cuda_fail(ce, "autotune");
                break;
            }
            cudaEventElapsedTime(&tot, e0, e1);
            if (tot / reps < wms) {
                wms = tot / reps;
                winner = o;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != VDI_OK) return s;
    winner.use_graph = 1;
    {
        BatchCache &bc = cache_of(ctx);
        std::lock_guard<std::mutex> g(bc.mu);
        bc.tuned[tune_key(reqs, n)] = winner;
    }
    if (best) *best = winner;
    if (best_ms) *best_ms = wms;
    return VDI_OK;
}
