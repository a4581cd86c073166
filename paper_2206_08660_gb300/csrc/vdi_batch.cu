// vdi_batch.cu -- many views of several resident VDIs in one persistent
// launch, optionally replayed from a CUDA graph, plus the batch autotuner.
//
// Every request is cut into 32 x 8 pixel tiles; all tiles of all requests form
// one queue.  A persistent grid (SM count x resident blocks per SM) pulls tiles
// from an atomic counter, so requests of different resolutions, previews and
// VDIs share the GPU without a launch per view.  Requests with image-space
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

struct BatchParams {
    int n_req, total_tiles;
    unsigned *counter;
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

// PREVIEW: the batch holds ray-subsampled previews (d_r > 1); without them the
// kernel carries only the exact walk, which needs fewer registers, so more
// blocks fit on an SM.
template <int WX, bool PREVIEW>
__global__ void __launch_bounds__(256, PREVIEW ? 3 : 4) batch_render_kernel(const BatchParams P) {
    __shared__ int s_tile, s_req;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = (int)atomicAdd(P.counter, 1u);
            int r = 0;
            if (t < P.total_tiles) {
                int lo = 0, hi = P.n_req - 1;  // last request with tile_base <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (P.reqs[mid].tile_base <= t)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                r = lo;
            }
            s_tile = t;
            s_req = r;
        }
        __syncthreads();
        const int tile = s_tile, r = s_req;
        if (tile >= P.total_tiles) return;  // uniform: every thread read the same s_tile
        const BatchReq &q = P.reqs[r];
        const DevVdi &v = P.vdis[q.vdi];
        const int local = tile - q.tile_base;
        const int tx0 = (local % q.tiles_x) * 32, ty0 = (local / q.tiles_x) * 8;
        if (PREVIEW && q.c.d_r > 1) {
            // a preview tile in kBatchLanes passes of 256 / kBatchLanes rays with
            // kBatchLanes lanes per ray (the same image as any lane count)
            const int g = (int)threadIdx.x / kBatchLanes;
            for (int unit = 0; unit < kBatchLanes; ++unit) {
                const int px = tx0 + (g & 31), py = ty0 + unit * (8 / kBatchLanes) + (g >> 5);
                const bool inside = px < q.c.W && py < q.c.H;
                Ray ray = {};
                const bool active = inside && setup_ray(q.c, px, py, v.w, v.h, ray);
                const Accum acc = (v.fmt == 0) ? march_preview_lanes<0, kPreviewProbe, kBatchLanes>(v, q.c, ray, active)
                                               : march_preview_lanes<1, kPreviewProbe, kBatchLanes>(v, q.c, ray, active);
                if (inside && (threadIdx.x & (kBatchLanes - 1)) == 0)
                    store_px(q.out, q.out_fmt, (size_t)py * q.c.W + px, acc);
            }
        } else {
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
        __syncthreads();  // every thread has read s_tile / s_req before thread 0 writes them again
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
    const int X = (local % q.tiles_x) * 32 + (threadIdx.x & 31);
    const int Y = (local / q.tiles_x) * 8 + (threadIdx.x >> 5);
    if (X >= q.W || Y >= q.H) return;
    const float u = ((float)X + 0.5f) * ((float)q.w0 / (float)q.W) - 0.5f;
    const float vv = ((float)Y + 0.5f) * ((float)q.h0 / (float)q.H) - 0.5f;
    const int i0 = (int)floorf(u), j0 = (int)floorf(vv);
    const float fu = u - (float)i0, fv = vv - (float)j0;
    const int i1 = min(max(i0 + 1, 0), q.w0 - 1), j1 = min(max(j0 + 1, 0), q.h0 - 1);
    const int ic = min(max(i0, 0), q.w0 - 1), jc = min(max(j0, 0), q.h0 - 1);
    const float4 a = __ldg(q.lo + (size_t)jc * q.w0 + ic), b = __ldg(q.lo + (size_t)jc * q.w0 + i1);
    const float4 d = __ldg(q.lo + (size_t)j1 * q.w0 + ic), e = __ldg(q.lo + (size_t)j1 * q.w0 + i1);
    const float4 top = make_float4(fmaf(fu, b.x - a.x, a.x), fmaf(fu, b.y - a.y, a.y), fmaf(fu, b.z - a.z, a.z),
                                   fmaf(fu, b.w - a.w, a.w));
    const float4 bot = make_float4(fmaf(fu, e.x - d.x, d.x), fmaf(fu, e.y - d.y, d.y), fmaf(fu, e.z - d.z, d.z),
                                   fmaf(fu, e.w - d.w, d.w));
    Accum acc;
    acc.r = fmaf(fv, bot.x - top.x, top.x);
    acc.g = fmaf(fv, bot.y - top.y, top.y);
    acc.b = fmaf(fv, bot.z - top.z, top.z);
    acc.T = 1.f - fmaf(fv, bot.w - top.w, top.w);
    store_px(q.out, q.out_fmt, (size_t)Y * q.W + X, acc);
}

template <bool PREVIEW>
static const void *render_fn_p(int ws) {
    if (ws == 0) return (const void *)batch_render_kernel<32, PREVIEW>;
    if (ws == 1) return (const void *)batch_render_kernel<16, PREVIEW>;
    if (ws == 2) return (const void *)batch_render_kernel<8, PREVIEW>;
    return (const void *)batch_render_kernel<4, PREVIEW>;
}

static const void *render_fn(int ws, bool preview) {
    return preview ? render_fn_p<true>(ws) : render_fn_p<false>(ws);
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
    bool preview = false;                 // some request has d_r > 1
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
    size_t off = 256;  // the counter lives at offset 0
    int tiles = 0, up_tiles = 0;
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
        if (r.d_r > 1) pl.preview = true;
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
        q.tile_base = tiles;
        tiles += q.tiles_x * div_up(Hr, 8);
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
            u.tiles_x = div_up(r.W, 32);
            u.tile_base = up_tiles;
            up_tiles += u.tiles_x * div_up(r.H, 8);
        }
    }
    pl.bp->n_req = n;
    pl.bp->total_tiles = tiles;
    pl.up->total_tiles = up_tiles;
    pl.scratch_bytes = off;
    return VDI_OK;
}

// point the plan at a scratch allocation
static void bind_scratch(BatchPlan &pl, char *scratch) {
    pl.bp->counter = reinterpret_cast<unsigned *>(scratch);
    int k = 0;
    for (int i = 0; i < pl.bp->n_req; ++i)
        if (pl.lo_offset[i] != (size_t)-1) {
            pl.bp->reqs[i].out = scratch + pl.lo_offset[i];
            pl.up->reqs[k++].lo = reinterpret_cast<const float4 *>(scratch + pl.lo_offset[i]);
        }
}

static int persistent_blocks(vdi_ctx *ctx, int ws, int bps, bool preview) {
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, render_fn(ws, preview), 256, 0);
    if (bps > 0) occ = std::min(occ, bps);
    return std::max(1, occ) * ctx->sm_count;
}

static cudaError_t enqueue_plain(vdi_ctx *ctx, BatchPlan &pl, int ws, int bps, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(pl.bp->counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int grid = std::min(persistent_blocks(ctx, ws, bps, pl.preview), std::max(1, pl.bp->total_tiles));
    void *args[] = {pl.bp};
    e = cudaLaunchKernel(render_fn(ws, pl.preview), dim3(grid), dim3(256), args, 0, st);
    if (e != cudaSuccess || pl.up->n == 0) return e;
    void *uargs[] = {pl.up};
    return cudaLaunchKernel((const void *)batch_upsample_kernel, dim3(pl.up->total_tiles), dim3(256), uargs, 0, st);
}

// A cached executable graph for one batch shape: memset(counter) -> persistent
// render -> batched upsample, with its own scratch.
struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t render_node = nullptr, up_node = nullptr;
    void *scratch = nullptr;
    int grid = 0;
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

static vdi_status enqueue_graph(vdi_ctx *ctx, const vdi_request *reqs, int n, BatchPlan &pl, int ws, int bps,
                                cudaStream_t st) {
    BatchCache &bc = cache_of(ctx);
    std::lock_guard<std::mutex> g(bc.mu);
    const std::string key = shape_key(reqs, n, pl, ws, bps, st);
    auto it = bc.graphs.find(key);
    cudaError_t e = cudaSuccess;
    if (it == bc.graphs.end()) {
        GraphEntry ge;
        if ((e = cudaMalloc(&ge.scratch, pl.scratch_bytes)) != cudaSuccess) return cuda_fail(e, "graph scratch");
        bind_scratch(pl, (char *)ge.scratch);
        ge.grid = std::min(persistent_blocks(ctx, ws, bps, pl.preview), std::max(1, pl.bp->total_tiles));
        cudaGraphNode_t ms = nullptr;
        cudaMemsetParams mp{};
        mp.dst = ge.scratch;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 1;
        mp.height = 1;
        mp.pitch = 4;
        void *args[] = {pl.bp};
        cudaKernelNodeParams kp{};
        kp.func = (void *)render_fn(ws, pl.preview);
        kp.gridDim = dim3(ge.grid);
        kp.blockDim = dim3(256);
        kp.kernelParams = args;
        if ((e = cudaGraphCreate(&ge.graph, 0)) != cudaSuccess ||
            (e = cudaGraphAddMemsetNode(&ms, ge.graph, nullptr, 0, &mp)) != cudaSuccess ||
            (e = cudaGraphAddKernelNode(&ge.render_node, ge.graph, &ms, 1, &kp)) != cudaSuccess) {
            cudaFree(ge.scratch);
            return cuda_fail(e, "graph build");
        }
        if (pl.up->n) {
            void *uargs[] = {pl.up};
            cudaKernelNodeParams up{};
            up.func = (void *)batch_upsample_kernel;
            up.gridDim = dim3(pl.up->total_tiles);
            up.blockDim = dim3(256);
            up.kernelParams = uargs;
            if ((e = cudaGraphAddKernelNode(&ge.up_node, ge.graph, &ge.render_node, 1, &up)) != cudaSuccess) {
                cudaGraphDestroy(ge.graph);
                cudaFree(ge.scratch);
                return cuda_fail(e, "graph build");
            }
        }
        if ((e = cudaGraphInstantiate(&ge.exec, ge.graph, 0)) != cudaSuccess) {
            cudaGraphDestroy(ge.graph);
            cudaFree(ge.scratch);
            return cuda_fail(e, "graph instantiate");
        }
        it = bc.graphs.emplace(key, ge).first;
    } else {
        GraphEntry &ge = it->second;
        bind_scratch(pl, (char *)ge.scratch);
        void *args[] = {pl.bp};
        cudaKernelNodeParams kp{};
        kp.func = (void *)render_fn(ws, pl.preview);
        kp.gridDim = dim3(ge.grid);
        kp.blockDim = dim3(256);
        kp.kernelParams = args;
        if ((e = cudaGraphExecKernelNodeSetParams(ge.exec, ge.render_node, &kp)) != cudaSuccess)
            return cuda_fail(e, "graph update");
        if (pl.up->n) {
            void *uargs[] = {pl.up};
            cudaKernelNodeParams up{};
            up.func = (void *)batch_upsample_kernel;
            up.gridDim = dim3(pl.up->total_tiles);
            up.blockDim = dim3(256);
            up.kernelParams = uargs;
            if ((e = cudaGraphExecKernelNodeSetParams(ge.exec, ge.up_node, &up)) != cudaSuccess)
                return cuda_fail(e, "graph update");
        }
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
    bool preview = false;
    for (int i = 0; i < n; ++i) preview = preview || reqs[i].d_r > 1;
    vdi_status s = VDI_OK;
    for (int ws = 0; ws <= 3 && s == VDI_OK; ++ws) {
        int occ_max = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_max, render_fn(ws, preview), 256, 0);
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
