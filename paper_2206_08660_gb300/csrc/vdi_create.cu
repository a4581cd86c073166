// vdi_create.cu -- building the device-resident VDI: validation, conversion
// from the array-of-structures input (Section 5: colour RGBA32F + front/back
// depth per slot) into the structure-of-arrays device layout, the
// supersegment-count grid (Section 4.3) and the reverse conversion.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "vdi_internal.cuh"

namespace vdi {

enum { kErrUnsorted = 1, kErrInvalid = 2 };

// Per list: number of leading slots with a finite front depth.
__global__ void count_leading_kernel(const float *__restrict__ depth, int ns, long long nl,
                                     int32_t *__restrict__ counts) {
    const long long li = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nl) return;
    int n = 0;
    while (n < ns && isfinite(depth[((size_t)li * ns + n) * 2])) ++n;
    counts[li] = n;
}

__device__ __forceinline__ unsigned pack_half2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned *>(&h);
}

// One thread per (list, slot pair): validate, convert, pad.
template <int FMT>
__global__ void convert_kernel(const float *__restrict__ rgba, const float *__restrict__ depth,
                               const int32_t *__restrict__ counts, int ns, int nsp, long long nl,
                               float4 *__restrict__ dpair, void *__restrict__ colour,
                               unsigned *__restrict__ err) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = nsp >> 1;
    if (tid >= nl * npairs) return;
    const int k = (int)(tid / nl);
    const long long li = tid - (long long)k * nl;  // list-fastest: coalesced stores
    const int n = counts[li];
    unsigned e = 0;
    if (n < 0 || n > ns) e |= kErrInvalid;
    float fb[4];
    float4 col[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int j = 2 * k + s;
        if (j < n && j < ns) {
            const size_t o = (size_t)li * ns + j;
            const float f = depth[o * 2], b = depth[o * 2 + 1];
            if (!isfinite(f) || !isfinite(b) || !(f <= b)) e |= kErrUnsorted;
            if (j > 0 && !(depth[(o - 1) * 2 + 1] <= f)) e |= kErrUnsorted;
            const float4 c = *reinterpret_cast<const float4 *>(rgba + o * 4);
            if (!(c.w >= 0.f && c.w <= 1.f) || !(c.x >= 0.f && c.x <= c.w) || !(c.y >= 0.f && c.y <= c.w) ||
                !(c.z >= 0.f && c.z <= c.w))
                e |= kErrInvalid;
            fb[2 * s] = f;
            fb[2 * s + 1] = b;
            const float ia = c.w > 0.f ? 1.f / c.w : 0.f;
            // kappa = -log2(1 - alpha); alpha = 1 gives +inf (fully opaque for any l > 0)
            const float kappa = -log1pf(-c.w) * 1.4426950408889634f;
            col[s] = make_float4(fminf(c.x * ia, 1.f), fminf(c.y * ia, 1.f), fminf(c.z * ia, 1.f), kappa);
        } else {
            fb[2 * s] = INFINITY;
            fb[2 * s + 1] = INFINITY;
            col[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    dpair[(size_t)k * nl + li] = make_float4(fb[0], fb[1], fb[2], fb[3]);
    if (FMT == 0) {
        float4 *c = reinterpret_cast<float4 *>(colour);
        c[(size_t)(2 * k) * nl + li] = col[0];
        c[(size_t)(2 * k + 1) * nl + li] = col[1];
    } else {
        uint4 q;
        q.x = pack_half2(col[0].x, col[0].y);
        q.y = pack_half2(col[0].z, col[0].w);
        q.z = pack_half2(col[1].x, col[1].y);
        q.w = pack_half2(col[1].z, col[1].w);
        reinterpret_cast<uint4 *>(colour)[(size_t)k * nl + li] = q;
    }
    if (e) atomicOr(err, e);
}

// Supersegment-count grid: one block per T x T column of lists; per-slab
// counts accumulate in shared memory and are written once (deterministic,
// no global atomics).  A supersegment [f, b] counts in slab k when
// f < edge[k+1] and b > edge[k]; a zero-length one (f == b) counts in the
// slab with edge[k] <= f < edge[k+1].
__global__ void grid_kernel(const DevVdi v, uint32_t *__restrict__ grid) {
    __shared__ unsigned cnt[kMaxNz];
    __shared__ float edges[kMaxNz + 1];
    const int cx = blockIdx.x, cy = blockIdx.y;
    for (int k = threadIdx.x; k < v.nz; k += blockDim.x) cnt[k] = 0;
    for (int k = threadIdx.x; k <= v.nz; k += blockDim.x) edges[k] = v.edges[k];
    __syncthreads();
    const int x0 = cx * v.T, y0 = cy * v.T;
    const int fx = min(v.T, v.w - x0), fy = min(v.T, v.h - y0);
    const int npairs = v.nsp >> 1;
    const int items = fx * fy * npairs;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int k = it / (fx * fy);
        const int r = it - k * fx * fy;
        const int li = (y0 + r / fx) * v.w + (x0 + r % fx);
        const float4 d = v.depth[(size_t)k * v.nl + li];
        const float fs[2] = {d.x, d.z}, bs[2] = {d.y, d.w};
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float f = fs[s], b = bs[s];
            if (!isfinite(f)) continue;
            for (int z = 0; z < v.nz; ++z) {
                const bool hit = (f == b) ? (edges[z] <= f && f < edges[z + 1]) : (f < edges[z + 1] && b > edges[z]);
                if (hit) atomicAdd(&cnt[z], 1u);
            }
        }
    }
    __syncthreads();
    for (int z = threadIdx.x; z < v.nz; z += blockDim.x)
        grid[((size_t)z * v.gh + cy) * v.gw + cx] = cnt[z];
}

// Per list: front of the first and back of the last valid supersegment.
__global__ void range_kernel(const float *__restrict__ depth, const int32_t *__restrict__ counts, int ns,
                             long long nl, float2 *__restrict__ range) {
    const long long li = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nl) return;
    const int n = min(max(counts[li], 0), ns);
    range[li] = n ? make_float2(depth[(size_t)li * ns * 2], depth[((size_t)li * ns + n - 1) * 2 + 1])
                  : make_float2(INFINITY, -INFINITY);
}

// Per block of kB x kB lists: the smallest first front and the largest last back.
__global__ void block_range_kernel(const DevVdi v, float2 *__restrict__ brange) {
    const int bxi = blockIdx.x * blockDim.x + threadIdx.x, byi = blockIdx.y;
    if (bxi >= v.bw) return;
    float lo = INFINITY, hi = -INFINITY;
    for (int y = byi * kB; y < min(byi * kB + kB, v.h); ++y)
        for (int x = bxi * kB; x < min(bxi * kB + kB, v.w); ++x) {
            const float2 r = v.range[(size_t)y * v.w + x];
            lo = fminf(lo, r.x);
            hi = fmaxf(hi, r.y);
        }
    brange[(size_t)byi * v.bw + bxi] = make_float2(lo, hi);
}

cudaError_t launch_block_range(const DevVdi &v, float2 *brange, cudaStream_t st) {
    block_range_kernel<<<dim3(div_up(v.bw, 128), v.bh), 128, 0, st>>>(v, brange);
    return cudaGetLastError();
}

// Device layout -> array-of-structures (premultiplied rgba, alpha per unit).
template <int FMT>
__global__ void download_kernel(const DevVdi v, int ns, float *__restrict__ rgba, float *__restrict__ depth,
                                int32_t *__restrict__ counts) {
    const long long li = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= v.nl) return;
    int n = 0;
    ColourCache<FMT> cc;
    cc.k = -1;
    for (int j = 0; j < ns; ++j) {
        const float f = ld_front(v, j, (int)li), b = ld_back(v, j, (int)li);
        const size_t o = (size_t)li * ns + j;
        if (depth) {
            depth[o * 2] = f;
            depth[o * 2 + 1] = b;
        }
        if (isfinite(f)) ++n;
        if (rgba) {
            float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
            if (isfinite(f)) {
                const float4 c = get_colour<FMT>(cc, v, (int)li, j);
                const float a = -expm1f(-c.w * 0.69314718055994531f);
                out = make_float4(c.x * a, c.y * a, c.z * a, a);
            }
            *reinterpret_cast<float4 *>(rgba + o * 4) = out;
        }
    }
    if (counts) counts[li] = n;
}

cudaError_t launch_count_leading(const float *depth, int ns, long long nl, int32_t *counts, cudaStream_t st) {
    count_leading_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(depth, ns, nl, counts);
    return cudaGetLastError();
}

cudaError_t launch_convert(int fmt, const float *rgba, const float *depth, const int32_t *counts, int ns,
                           int nsp, long long nl, float4 *dpair, void *colour, unsigned *err, cudaStream_t st) {
    const long long items = nl * (nsp / 2);
    const unsigned nb = (unsigned)((items + 255) / 256);
    if (fmt == 0)
        convert_kernel<0><<<nb, 256, 0, st>>>(rgba, depth, counts, ns, nsp, nl, dpair, colour, err);
    else
        convert_kernel<1><<<nb, 256, 0, st>>>(rgba, depth, counts, ns, nsp, nl, dpair, colour, err);
    return cudaGetLastError();
}

cudaError_t launch_grid(const DevVdi &v, uint32_t *grid, cudaStream_t st) {
    dim3 g(v.gw, v.gh);
    grid_kernel<<<g, 256, 0, st>>>(v, grid);
    return cudaGetLastError();
}

cudaError_t launch_range(const float *depth, const int32_t *counts, int ns, long long nl, float2 *range,
                         cudaStream_t st) {
    range_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(depth, counts, ns, nl, range);
    return cudaGetLastError();
}

cudaError_t launch_download(const DevVdi &v, int ns, float *rgba, float *depth, int32_t *counts,
                            cudaStream_t st) {
    const unsigned nb = (unsigned)((v.nl + 255) / 256);
    if (v.fmt == 0)
        download_kernel<0><<<nb, 256, 0, st>>>(v, ns, rgba, depth, counts);
    else
        download_kernel<1><<<nb, 256, 0, st>>>(v, ns, rgba, depth, counts);
    return cudaGetLastError();
}

}  // namespace vdi
