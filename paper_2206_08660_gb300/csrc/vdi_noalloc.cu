// vdi_noalloc.cu -- vdi_render_preview_static: the render of vdi_render, with
// the low-resolution image of an image-space preview (D_I > 1) kept in a
// fixed static device buffer of this library instead of memory from the
// stream-ordered allocator, so the call allocates no device memory.
//
// Some callers cannot allocate at render time: a viewer or server that has
// handed all device memory to resident VDIs up front (a per-frame allocation
// could fail mid-frame), a frame loop with a hard time budget that must not
// wait on the allocator, or an application that only allows device
// allocation during start-up.  They get one more entry point whose scratch is
// a file-scope array of a stated size, present on every GPU that loads the
// library until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/vdi.h"
#include "vdi_api_internal.h"
#include "vdi_internal.cuh"

#define VDI_API extern "C" __attribute__((visibility("default")))

namespace vdi {

cudaError_t launch_upsample(const float4 *lo, int w0, int h0, void *out, int out_fmt, int W, int H,
                            cudaStream_t st);

// 8 MiB: one RGBA float per low-resolution pixel, enough for 1920 x 1080 at D_I = 2.
constexpr size_t kStaticPreviewPixels = VDI_STATIC_PREVIEW_PIXELS;
static __device__ __align__(256) float4 g_preview_lowres[kStaticPreviewPixels];

// In host code g_preview_lowres names a host-side stand-in, not device
// memory: the device address comes from cudaGetSymbolAddress, looked up once
// per device with that device current, and handed to the kernels.
constexpr int kMaxDevices = 64;
static std::mutex g_mu;
static float4 *g_addr[kMaxDevices];

static vdi_status static_preview_buffer(int device, float4 **out) {
    if (device < 0 || device >= kMaxDevices) return fail(VDI_ERR_UNSUPPORTED, "device %d", device);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_preview_lowres);  // device is current
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static preview buffer)");
        g_addr[device] = static_cast<float4 *>(p);
    }
    *out = g_addr[device];
    return VDI_OK;
}

}  // namespace vdi

using namespace vdi;

VDI_API vdi_status vdi_render_preview_static(vdi_t *v, const vdi_camera *view, int W, int H, int d_i, int d_r,
                                             void *out_rgba, int out_fmt, void *stream) {
    vdi_status st_ = check_render_args(v, W, H, d_i, d_r, out_rgba, out_fmt);
    if (st_ != VDI_OK) return st_;
    const int Wr = div_up(W, d_i), Hr = div_up(H, d_i);
    if (d_i > 1 && (size_t)Wr * Hr > kStaticPreviewPixels)
        return fail(VDI_ERR_INVALID_ARG,
                    "preview of %dx%d rays exceeds the static buffer of %zu pixels; raise d_i or use vdi_render", Wr,
                    Hr, kStaticPreviewPixels);
    cudaSetDevice(v->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    ViewConsts c;
    st_ = make_view_consts(v, view, Wr, Hr, d_r, &c);
    if (st_ != VDI_OK) return st_;
    const int ws = default_warp_shape(c);
    cudaError_t e;
    if (d_i == 1) {
        e = launch_render(c, v->dv, out_rgba, out_fmt, nullptr, nullptr, VDI_SEARCH_ALG2, ws, true, false, false, tile_maps(v), st);
    } else {
        float4 *lo = nullptr;
        st_ = static_preview_buffer(v->ctx->device, &lo);
        if (st_ != VDI_OK) return st_;
        // every low-resolution pixel is written before the upsampling reads it,
        // so nothing left by an earlier call needs clearing
        e = launch_render(c, v->dv, lo, VDI_F32, nullptr, nullptr, VDI_SEARCH_ALG2, ws, true, false, false, tile_maps(v), st);
        if (e == cudaSuccess) e = launch_upsample(lo, Wr, Hr, out_rgba, out_fmt, W, H, st);
    }
    return e == cudaSuccess ? VDI_OK : cuda_fail(e, "preview render");
}
