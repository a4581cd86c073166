// vdi_serve.cu -- continuous-batching view server over resident VDIs.
//
// The paper's client keeps the latest VDI resident and renders views from it
// while a new VDI is uploaded in the background (Section 5, double
// buffering).  This server generalises that to many resident VDIs and many
// concurrent view requests:
//  - requests are queued on submit and admitted FIFO into the next batch as
//    soon as a batch slot (one of `max_inflight` CUDA streams) and device
//    memory for their images fit under the budget; batches already on the GPU
//    keep running, so new work overlaps in-flight work (continuous batching);
//  - each batch is one vdi_render_batch launch (persistent tile queue);
//  - a VDI slot can be replaced at any time: the new VDI is used by batches
//    formed after its producer stream has reached the replacement point, and
//    the old one is freed once no in-flight batch references it;
//  - every wait is bounded (VDI_ERR_TIMEOUT), errors land on the ticket;
//  - the memory budget is a device budget: resident VDI versions (including
//    a replaced one still read by in-flight batches) and a VDI being
//    generated through the server are charged next to images and scratch.
// One scheduler thread owns all CUDA work of the server.
#include <cuda_runtime.h>

#include <atomic>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/vdi.h"
#include "vdi_api_internal.h"

#define VDI_API extern "C" __attribute__((visibility("default")))

namespace vdi {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct VdiVersion {  // one VDI installed in a slot, shared by the batches that use it
    vdi_t *vdi = nullptr;
    cudaEvent_t ready = nullptr;  // recorded on the producer stream at install time
    bool ready_seen = false;
    std::atomic<size_t> *charge = nullptr;  // the server's resident-VDI bytes, while this version lives
    size_t bytes = 0;
    ~VdiVersion() {
        if (ready) cudaEventDestroy(ready);
        if (vdi) free_vdi(vdi);
        if (charge) charge->fetch_sub(bytes);
    }
};

struct Ticket {
    vdi_view_request req{};
    int status = -1;  // -1 pending / running, else a vdi_status
    double t_submit = 0, t_start = 0, t_done = 0;
    void *image = nullptr;
    size_t bytes = 0;       // image bytes (counted against the budget until release)
    size_t scratch = 0;     // low-resolution bytes of a D_I preview while running
    bool released = false;
};

struct Batch {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
    std::vector<std::shared_ptr<VdiVersion>> holds;
};

}  // namespace vdi

struct vdi_server {
    vdi_ctx *ctx = nullptr;
    vdi_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv;       // wakes the scheduler
    std::condition_variable done_cv;  // wakes waiters
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, vdi::Ticket> tickets;
    // device bytes of the live VDI versions (declared before the slots and
    // batches that hold versions, so it outlives them)
    std::atomic<size_t> vdi_bytes{0};
    size_t reserved = 0;  // bytes held for VDIs being generated through the server
    std::vector<std::shared_ptr<vdi::VdiVersion>> slots;
    std::vector<vdi::Batch> batches;
    uint64_t next_ticket = 1;
    size_t used = 0;
    bool stop = false;
    std::thread th;
    vdi_server_counters st{};
};

namespace vdi {

static size_t image_bytes(const vdi_view_request &r) {
    return (size_t)r.W * r.H * (r.out_fmt == VDI_F16 ? 8 : 16);
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// admission cost: the image plus the low-resolution scratch of a D_I preview
static size_t request_bytes(const vdi_view_request &r) {
    size_t b = align256(image_bytes(r));
    int Wr, Hr;
    request_rays(r, Wr, Hr);
    if (Wr != r.W || Hr != r.H) b += align256((size_t)Wr * Hr * 16);
    return b;
}

static void finish(vdi_server *s, uint64_t id, int status) {
    Ticket &t = s->tickets[id];
    t.status = status;
    t.t_done = now_s();
    if (status != VDI_OK) {
        s->st.failed++;
        if (t.image) {
            cudaFreeAsync(t.image, s->ctx->free_stream);
            t.image = nullptr;
            s->used -= align256(t.bytes);
            t.bytes = 0;
        }
    } else {
        s->st.completed++;
    }
    s->used -= t.scratch;
    t.scratch = 0;
}

// mark finished batches, release their VDI holds; called with the lock held
static int reap(vdi_server *s) {
    int n = 0;
    for (auto &b : s->batches) {
        if (!b.busy) continue;
        cudaError_t e = cudaEventQuery(b.done);
        if (e == cudaErrorNotReady) continue;
        const int status = (e == cudaSuccess) ? VDI_OK : VDI_ERR_CUDA;
        for (uint64_t id : b.tickets) finish(s, id, status);
        b.tickets.clear();
        b.holds.clear();
        b.busy = false;
        ++n;
    }
    return n;
}

// form and launch one batch on a free stream; called with the lock held
static bool launch_one(vdi_server *s) {
    Batch *slot = nullptr;
    for (auto &b : s->batches)
        if (!b.busy) {
            slot = &b;
            break;
        }
    if (!slot || s->pending.empty()) return false;
    std::vector<vdi_request> reqs;
    std::vector<uint64_t> ids;
    std::vector<std::shared_ptr<VdiVersion>> holds;
    while (!s->pending.empty() && (int)reqs.size() < s->cfg.max_batch) {
        const uint64_t id = s->pending.front();
        Ticket &t = s->tickets[id];
        const vdi_view_request &r = t.req;
        if (r.slot < 0 || r.slot >= (int)s->slots.size() || !s->slots[r.slot]) {
            s->pending.pop_front();
            fail(VDI_ERR_INVALID_ARG, "slot %d holds no VDI", r.slot);
            finish(s, id, VDI_ERR_INVALID_ARG);
            continue;
        }
        const size_t need = request_bytes(r);
        const size_t held = s->vdi_bytes.load() + s->reserved;  // resident and incoming VDIs
        bool idle = true;  // nothing in flight or unreleased that could free memory later
        for (auto &b : s->batches) idle &= !b.busy;
        idle &= s->used == 0;
        if (need > s->cfg.budget_bytes || (idle && held + need > s->cfg.budget_bytes)) {
            // can never fit (or not while these VDIs stay resident and nothing else runs):
            // reject instead of blocking the queue
            s->pending.pop_front();
            fail(VDI_ERR_OOM, "request needs %zu bytes; budget %zu, VDIs hold %zu", need, s->cfg.budget_bytes, held);
            finish(s, id, VDI_ERR_OOM);
            continue;
        }
        if (s->used + held + need > s->cfg.budget_bytes) break;  // admission by memory: wait for releases
        std::shared_ptr<VdiVersion> ver = s->slots[r.slot];
        if (!ver->ready_seen) {
            const cudaError_t q = cudaEventQuery(ver->ready);
            if (q == cudaErrorNotReady) break;  // the VDI is still being produced: keep FIFO order
            ver->ready_seen = true;
        }
        void *img = nullptr;
        if (cudaMallocAsync(&img, align256(image_bytes(r)), slot->stream) != cudaSuccess) {
            cudaGetLastError();
            break;  // device memory is tighter than the budget: retry when batches retire
        }
        s->pending.pop_front();
        t.image = img;
        t.bytes = image_bytes(r);
        t.scratch = need - align256(image_bytes(r));
        s->used += need;
        t.t_start = now_s();
        vdi_request q{};
        q.vdi = ver->vdi;
        q.view = r.view;
        q.W = r.W;
        q.H = r.H;
        q.d_i = r.d_i;
        q.d_r = r.d_r;
        q.Wr = r.Wr;
        q.Hr = r.Hr;
        q.out = img;
        q.out_fmt = r.out_fmt;
        reqs.push_back(q);
        ids.push_back(id);
        holds.push_back(ver);
    }
    if (reqs.empty()) return false;
    vdi_batch_opts o = {-1, 0, 0};
    const vdi_status rc = vdi_render_batch(s->ctx, reqs.data(), (int)reqs.size(), &o, slot->stream);
    if (rc != VDI_OK) {
        for (uint64_t id : ids) finish(s, id, rc);
        return true;
    }
    cudaEventRecord(slot->done, slot->stream);
    slot->busy = true;
    slot->tickets = ids;
    slot->holds = holds;
    s->st.batches++;
    s->st.batched_requests += reqs.size();
    return true;
}

static void scheduler(vdi_server *s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        const int reaped = reap(s);
        bool launched = false;
        while (launch_one(s)) launched = true;
        if (reaped || launched) s->done_cv.notify_all();
        bool busy = false;
        for (auto &b : s->batches) busy |= b.busy;
        // poll in-flight work every 50 us; sleep until a submit when idle
        if (busy || !s->pending.empty())
            s->cv.wait_for(lk, std::chrono::microseconds(50));
        else
            s->cv.wait_for(lk, std::chrono::milliseconds(20));
    }
    // drain: wait (bounded) for in-flight batches before tearing down
    for (auto &b : s->batches)
        if (b.busy) {
            lk.unlock();
            const double t0 = now_s();
            while (cudaEventQuery(b.done) == cudaErrorNotReady && now_s() - t0 < s->cfg.wait_timeout_s)
                std::this_thread::sleep_for(std::chrono::microseconds(100));
            lk.lock();
        }
    reap(s);
}

}  // namespace vdi

using namespace vdi;

VDI_API vdi_status vdi_server_create(vdi_ctx *ctx, const vdi_server_config *cfg, vdi_server **out) {
    if (!ctx || !cfg || !out) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_batch > VDI_BATCH_MAX_REQUESTS || cfg->max_inflight < 1 ||
        cfg->max_inflight > 16 || cfg->n_slots < 1 || cfg->n_slots > VDI_BATCH_MAX_VDIS || cfg->budget_bytes == 0)
        return fail(VDI_ERR_INVALID_ARG, "server config out of range");
    cudaSetDevice(ctx->device);
    vdi_server *s = new vdi_server();
    s->ctx = ctx;
    s->cfg = *cfg;
    if (!(s->cfg.wait_timeout_s > 0)) s->cfg.wait_timeout_s = 10.0;
    s->slots.resize(cfg->n_slots);
    s->batches.resize(cfg->max_inflight);
    // batch streams get the highest priority: view requests are latency-bound,
    // VDI generation on the caller's side stream should yield to them
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (auto &b : s->batches) {
        cudaError_t e = cudaStreamCreateWithPriority(&b.stream, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            vdi_status r = cuda_fail(e, "server streams");
            for (auto &c : s->batches) {
                if (c.stream) cudaStreamDestroy(c.stream);
                if (c.done) cudaEventDestroy(c.done);
            }
            delete s;
            return r;
        }
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return VDI_OK;
}

// Bytes the live VDIs would hold after installing `incoming` bytes in `slot`:
// the slot's current version is freed at once when nothing but the slot
// holds it, else it lives until its last batch retires.  Lock held.
static size_t vdi_bytes_after_install(vdi_server *s, int slot, size_t incoming) {
    size_t b = s->vdi_bytes.load() + incoming;
    const auto &old = s->slots[slot];
    if (old && old.use_count() == 1) b -= old->bytes;
    return b;
}

// Install `vdi` in `slot` with its ready event on `ready_stream`; `reserved`
// bytes held for it (by vdi_server_generate) convert into its charge.
static vdi_status install(vdi_server *s, int slot, vdi_t *vdi, cudaStream_t ready_stream, size_t reserved) {
    cudaSetDevice(s->ctx->device);
    auto ver = std::make_shared<VdiVersion>();
    cudaError_t e = cudaEventCreateWithFlags(&ver->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ver->ready, ready_stream);
    if (e != cudaSuccess) return cuda_fail(e, "set_vdi");  // ver->vdi is still null: the caller keeps the VDI
    const size_t bytes = vdi->layout.total_bytes;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->reserved -= reserved;
        if (s->used + s->reserved + vdi_bytes_after_install(s, slot, bytes) > s->cfg.budget_bytes) {
            s->cv.notify_all();
            return fail(VDI_ERR_OOM, "VDI of %zu bytes does not fit the budget of %zu next to %zu in use", bytes,
                        s->cfg.budget_bytes, s->used + s->reserved + s->vdi_bytes.load());
        }
        ver->vdi = vdi;
        ver->bytes = bytes;
        ver->charge = &s->vdi_bytes;
        s->vdi_bytes.fetch_add(bytes);
        s->slots[slot] = ver;  // the previous version dies with the last batch holding it
        s->st.vdi_installs++;
    }
    s->cv.notify_all();
    return VDI_OK;
}

VDI_API vdi_status vdi_server_set_vdi(vdi_server *s, int slot, vdi_t *vdi, void *ready_stream) {
    if (!s || !vdi) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    if (slot < 0 || slot >= (int)s->slots.size()) return fail(VDI_ERR_INVALID_ARG, "slot %d", slot);
    if (vdi->ctx != s->ctx) return fail(VDI_ERR_INVALID_ARG, "VDI of another context");
    return install(s, slot, vdi, (cudaStream_t)ready_stream, 0);
}

VDI_API vdi_status vdi_server_generate(vdi_server *s, int slot, const vdi_volume *vol, const vdi_tf *tf,
                                       const vdi_gen_params *params, void *stream) {
    if (!s || !vol || !tf || !params) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    if (slot < 0 || slot >= (int)s->slots.size()) return fail(VDI_ERR_INVALID_ARG, "slot %d", slot);
    vdi_desc d{};
    d.w = params->w;
    d.h = params->h;
    d.n_s = params->n_s;
    d.orig = params->orig;
    for (int k = 0; k < 3; ++k) {
        d.bbox_min[k] = vol->bbox_min[k];
        d.bbox_max[k] = vol->bbox_max[k];
    }
    d.length_unit = params->length_unit;
    d.colour_fmt = params->colour_fmt;
    d.grid_tile = params->grid_tile;
    d.grid_nz = params->grid_nz;
    vdi_layout L;
    vdi_status st_ = vdi_layout_bytes(&d, &L);
    if (st_ != VDI_OK) return st_;
    {  // hold the new VDI's bytes before it is allocated
        std::lock_guard<std::mutex> g(s->mu);
        if (s->used + s->reserved + vdi_bytes_after_install(s, slot, L.total_bytes) > s->cfg.budget_bytes)
            return fail(VDI_ERR_OOM, "generating a VDI of %zu bytes exceeds the budget of %zu next to %zu in use",
                        L.total_bytes, s->cfg.budget_bytes, s->used + s->reserved + s->vdi_bytes.load());
        s->reserved += L.total_bytes;
    }
    vdi_t *v = nullptr;
    st_ = vdi_generate(s->ctx, vol, tf, params, stream, &v);
    if (st_ != VDI_OK) {
        std::lock_guard<std::mutex> g(s->mu);
        s->reserved -= L.total_bytes;
        return st_;
    }
    st_ = install(s, slot, v, (cudaStream_t)stream, L.total_bytes);
    if (st_ != VDI_OK) vdi_destroy(v);
    return st_;
}

VDI_API vdi_status vdi_server_submit(vdi_server *s, const vdi_view_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    if (req->W < 1 || req->H < 1 || req->W > 16384 || req->H > 16384 || req->d_i < 1 || req->d_i > 16 ||
        req->d_r < 1 || req->d_r > 16 || (req->out_fmt != VDI_F32 && req->out_fmt != VDI_F16))
        return fail(VDI_ERR_INVALID_ARG, "bad request");
    if ((req->Wr != 0 || req->Hr != 0) && (req->Wr < 1 || req->Hr < 1 || req->Wr > req->W || req->Hr > req->H))
        return fail(VDI_ERR_INVALID_ARG, "rays %dx%d for image %dx%d", req->Wr, req->Hr, req->W, req->H);
    {
        std::lock_guard<std::mutex> g(s->mu);
        const uint64_t id = s->next_ticket++;
        Ticket &t = s->tickets[id];
        t.req = *req;
        t.t_submit = now_s();
        s->pending.push_back(id);
        s->st.submitted++;
        *ticket = id;
    }
    s->cv.notify_all();
    return VDI_OK;
}

static void fill_info(const Ticket &t, vdi_ticket_info *info) {
    if (!info) return;
    info->status = t.status < 0 ? -1 : t.status;
    info->t_submit = t.t_submit;
    info->t_start = t.t_start;
    info->t_done = t.t_done;
    info->image = t.status == VDI_OK ? t.image : nullptr;
    info->image_bytes = t.status == VDI_OK ? t.bytes : 0;
}

VDI_API vdi_status vdi_server_wait(vdi_server *s, uint64_t ticket, double timeout_s, vdi_ticket_info *info) {
    if (!s) return fail(VDI_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(VDI_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (s->tickets[ticket].status < 0) {
        if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && s->tickets[ticket].status < 0) {
            fill_info(s->tickets[ticket], info);
            return fail(VDI_ERR_TIMEOUT, "ticket %llu not done after %.3f s", (unsigned long long)ticket, timeout_s);
        }
    }
    fill_info(s->tickets[ticket], info);
    return VDI_OK;
}

VDI_API vdi_status vdi_server_poll(vdi_server *s, uint64_t ticket, vdi_ticket_info *info) {
    if (!s) return fail(VDI_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(VDI_ERR_INVALID_ARG, "unknown ticket");
    fill_info(it->second, info);
    return VDI_OK;
}

VDI_API vdi_status vdi_server_read(vdi_server *s, uint64_t ticket, void *dst, size_t bytes, int dst_kind,
                                   void *stream) {
    if (!s || !dst) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    if (dst_kind != VDI_MEM_HOST && dst_kind != VDI_MEM_DEVICE) return fail(VDI_ERR_INVALID_ARG, "dst_kind");
    void *src = nullptr;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return fail(VDI_ERR_INVALID_ARG, "unknown ticket");
        if (it->second.status < 0) return fail(VDI_ERR_BUSY, "ticket still running");
        if (it->second.status != VDI_OK || !it->second.image) return fail(VDI_ERR_INVALID_ARG, "ticket has no result");
        if (bytes != it->second.bytes) return fail(VDI_ERR_INVALID_ARG, "bytes %zu != image %zu", bytes, it->second.bytes);
        src = it->second.image;  // stays valid: only release frees it, and release is the caller's
    }
    cudaSetDevice(s->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes,
                                    dst_kind == VDI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? VDI_OK : cuda_fail(e, "server read");
}

VDI_API vdi_status vdi_server_release(vdi_server *s, uint64_t ticket) {
    if (!s) return fail(VDI_ERR_INVALID_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return fail(VDI_ERR_INVALID_ARG, "unknown ticket");
        if (it->second.status < 0) return fail(VDI_ERR_BUSY, "ticket still running");
        if (it->second.image) {  // its batch has retired: a stream-ordered free is safe
            cudaSetDevice(s->ctx->device);
            cudaFreeAsync(it->second.image, s->ctx->free_stream);
            s->used -= align256(it->second.bytes);
        }
        s->tickets.erase(it);
    }
    s->cv.notify_all();
    return VDI_OK;
}

VDI_API vdi_status vdi_server_stats(vdi_server *s, vdi_server_counters *out) {
    if (!s || !out) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->st;
    out->pending = s->pending.size();
    out->bytes_in_use = s->used;
    out->vdi_bytes = s->vdi_bytes.load() + s->reserved;
    int busy = 0;
    for (auto &b : s->batches) busy += b.busy;
    out->batches_in_flight = busy;
    return VDI_OK;
}

VDI_API void vdi_server_destroy(vdi_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(s->ctx->device);
    for (auto &kv : s->tickets)
        if (kv.second.image) cudaFreeAsync(kv.second.image, s->ctx->free_stream);
    for (auto &b : s->batches) {
        b.holds.clear();
        if (b.stream) cudaStreamDestroy(b.stream);
        if (b.done) cudaEventDestroy(b.done);
    }
    s->slots.clear();
    delete s;
}
