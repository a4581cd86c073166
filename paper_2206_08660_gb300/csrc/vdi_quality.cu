// vdi_quality.cu -- image quality of a render against a reference image, the
// measures of the paper's evaluation (Section 6 and its supplement): SSIM
// (Wang, Bovik, Sheikh and Simoncelli, 2004) and PSNR.
//
// Both run over the R, G and B channels of premultiplied RGBA images (the
// images over a black background), data range 1:
//  * SSIM: for every 7 x 7 window that lies inside the image, with window
//    means mu, sample variances s^2 (divided by 49 - 1) and sample covariance
//    s_ab, SSIM = (2 mu_a mu_b + C1)(2 s_ab + C2) / ((mu_a^2 + mu_b^2 + C1)
//    (s_a^2 + s_b^2 + C2)), C1 = 0.01^2, C2 = 0.03^2; the result is the mean
//    over the windows and the three channels.
//  * PSNR = 10 log10(1 / MSE), MSE over every pixel and the three channels.
// One thread per window centre; a block stages its 38 x 14 pixel footprint of
// both images in shared memory.  Per-block sums are reduced in a fixed order,
// so the result is deterministic.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/vdi.h"
#include "vdi_api_internal.h"
#include "vdi_internal.cuh"

#define VDI_API extern "C" __attribute__((visibility("default")))

namespace vdi {

constexpr int kWin = 7, kHalf = 3;
constexpr int kTx = 32, kTy = 8;                         // window centres per block
constexpr int kSx = kTx + 2 * kHalf, kSy = kTy + 2 * kHalf;  // staged footprint

__device__ __forceinline__ float3 load_rgb(const void *img, int fmt, size_t i) {
    if (fmt == 0) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(img) + i);
        return make_float3(v.x, v.y, v.z);
    }
    const uint2 q = __ldg(reinterpret_cast<const uint2 *>(img) + i);
    const __half2 rg = *reinterpret_cast<const __half2 *>(&q.x), ba = *reinterpret_cast<const __half2 *>(&q.y);
    const float2 a = __half22float2(rg), b = __half22float2(ba);
    return make_float3(a.x, a.y, b.x);
}

__device__ __forceinline__ float ssim_window(const float (*A)[kSx], const float (*B)[kSx], int lx, int ly) {
    float sa = 0.f, sb = 0.f;
    for (int j = 0; j < kWin; ++j)
        for (int i = 0; i < kWin; ++i) {
            sa += A[ly + j][lx + i];
            sb += B[ly + j][lx + i];
        }
    const float n = (float)(kWin * kWin);
    const float ma = sa / n, mb = sb / n;
    float vaa = 0.f, vbb = 0.f, vab = 0.f;  // two-pass: deviations from the window means
    for (int j = 0; j < kWin; ++j)
        for (int i = 0; i < kWin; ++i) {
            const float da = A[ly + j][lx + i] - ma, db = B[ly + j][lx + i] - mb;
            vaa = fmaf(da, da, vaa);
            vbb = fmaf(db, db, vbb);
            vab = fmaf(da, db, vab);
        }
    vaa /= n - 1.f;
    vbb /= n - 1.f;
    vab /= n - 1.f;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    return ((2.f * ma * mb + C1) * (2.f * vab + C2)) / ((ma * ma + mb * mb + C1) * (vaa + vbb + C2));
}

// partial[block] = (sum of SSIM over the block's windows and channels, sum of squared errors)
__global__ void __launch_bounds__(kTx * kTy) quality_kernel(const void *__restrict__ a, const void *__restrict__ b,
                                                            int fmt, int W, int H, double2 *__restrict__ partial) {
    __shared__ float A[3][kSy][kSx], B[3][kSy][kSx];
    __shared__ double red_s[kTx * kTy / 32], red_e[kTx * kTy / 32];
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * kTx, y0 = blockIdx.y * kTy;  // first window centre is (x0 + 3, y0 + 3)
    for (int k = t; k < kSx * kSy; k += blockDim.x) {
        const int sx = k % kSx, sy = k / kSx;
        const int X = x0 + sx, Y = y0 + sy;
        float3 va = make_float3(0.f, 0.f, 0.f), vb = va;
        if (X < W && Y < H) {
            va = load_rgb(a, fmt, (size_t)Y * W + X);
            vb = load_rgb(b, fmt, (size_t)Y * W + X);
        }
        A[0][sy][sx] = va.x;
        A[1][sy][sx] = va.y;
        A[2][sy][sx] = va.z;
        B[0][sy][sx] = vb.x;
        B[1][sy][sx] = vb.y;
        B[2][sy][sx] = vb.z;
    }
    __syncthreads();
    const int lx = t % kTx, ly = t / kTx;
    double s_sum = 0.0, e_sum = 0.0;
    // window centred at (x0 + lx + 3, y0 + ly + 3): inside the image when its corner fits
    if (x0 + lx + kWin <= W && y0 + ly + kWin <= H)
        for (int c = 0; c < 3; ++c) s_sum += (double)ssim_window(A[c], B[c], lx, ly);
    // squared error: each pixel once, by the thread of its position in the block's tile
    {
        const int X = x0 + lx, Y = y0 + ly;
        if (X < W && Y < H)
            for (int c = 0; c < 3; ++c) {
                const double d = (double)A[c][ly][lx] - (double)B[c][ly][lx];
                e_sum += d * d;
            }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s_sum += __shfl_down_sync(0xffffffffu, s_sum, o);
        e_sum += __shfl_down_sync(0xffffffffu, e_sum, o);
    }
    if ((t & 31) == 0) {
        red_s[t >> 5] = s_sum;
        red_e[t >> 5] = e_sum;
    }
    __syncthreads();
    if (t == 0) {
        double s = 0.0, e = 0.0;
        for (int w = 0; w < kTx * kTy / 32; ++w) {
            s += red_s[w];
            e += red_e[w];
        }
        partial[blockIdx.y * gridDim.x + blockIdx.x] = make_double2(s, e);
    }
}

// one block: sums the per-block partials in a fixed order
__global__ void quality_reduce_kernel(const double2 *__restrict__ partial, int n, double2 *__restrict__ total) {
    __shared__ double rs[256], re[256];
    double s = 0.0, e = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        s += partial[i].x;
        e += partial[i].y;
    }
    rs[threadIdx.x] = s;
    re[threadIdx.x] = e;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            rs[threadIdx.x] += rs[threadIdx.x + o];
            re[threadIdx.x] += re[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = make_double2(rs[0], re[0]);
}

}  // namespace vdi

using namespace vdi;

VDI_API vdi_status vdi_image_quality(const void *a, const void *b, int W, int H, int fmt, double *ssim,
                                     double *psnr, void *stream) {
    if (!a || !b || !ssim || !psnr) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    if (W < kWin || H < kWin || (long long)W * H > (1LL << 30))
        return fail(VDI_ERR_INVALID_ARG, "image %dx%d: at least 7 x 7 pixels", W, H);
    if (fmt != VDI_F32 && fmt != VDI_F16) return fail(VDI_ERR_INVALID_ARG, "fmt=%d", fmt);
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 grid(div_up(W, kTx), div_up(H, kTy));
    const int nb = (int)(grid.x * grid.y);
    double2 *d = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d, sizeof(double2) * (size_t)(nb + 1), st);
    if (e != cudaSuccess) return cuda_fail(e, "quality scratch");
    quality_kernel<<<grid, kTx * kTy, 0, st>>>(a, b, fmt, W, H, d + 1);
    e = cudaGetLastError();
    double2 h = make_double2(0.0, 0.0);
    if (e == cudaSuccess) {
        quality_reduce_kernel<<<1, 256, 0, st>>>(d + 1, nb, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "image quality");
    const double windows = 3.0 * (double)(W - kWin + 1) * (double)(H - kWin + 1);
    const double mse = h.y / (3.0 * (double)W * (double)H);
    *ssim = h.x / windows;
    *psnr = mse > 0.0 ? 10.0 * log10(1.0 / mse) : INFINITY;
    return VDI_OK;
}
