// vdi_api_internal.h -- host-side object definitions shared by the ABI
// translation units (contexts, VDI handles, helpers).
#pragma once
#include <cuda_runtime.h>

#include "../../include/vdi.h"
#include "vdi_internal.cuh"
#include "vdi_tma.cuh"

struct vdi_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t free_stream = nullptr;  // stream-ordered frees of VDI memory
};

struct vdi_t {
    vdi_ctx *ctx = nullptr;
    vdi_desc desc{};
    vdi_layout layout{};
    vdi::DevVdi dv{};
    double M[16]{};       // P_O * V_O
    double dz_cell = 0.0; // V_O view-depth extent of one grid slab
    bool box_in_frustum = false;  // all eight box corners strictly inside V_O's clip volume
    void *depth_mem = nullptr;
    void *colour_mem = nullptr;
    uint32_t *grid_mem = nullptr;
    float2 *range_mem = nullptr;
    float2 *brange_mem = nullptr;
    // frame totals of the last counted render (vdi_stats): rays hit, lists, pieces
    unsigned long long *totals_mem = nullptr;
    int frame_recorded = 0, frame_w = 0, frame_h = 0;
    uint32_t *status_mem = nullptr;  // device status word (TileMaps::status)
    // TMA tensor maps over the depth, colour and range arrays (the staged
    // one-list path); maps_ok = 0 when the layout does not allow them
    vdi::TileMaps maps{};
    int maps_ok = 0;
};

namespace vdi {

vdi_status fail(vdi_status s, const char *fmt, ...);
vdi_status cuda_fail(cudaError_t e, const char *what);
vdi_status check_desc(const vdi_desc *d, vdi_layout *L);
vdi_status make_view_consts(const vdi_t *v, const vdi_camera *cam, int W, int H, int d_r, ViewConsts *c);
vdi_status alloc_vdi(vdi_ctx *ctx, const vdi_desc *desc, cudaStream_t stream, vdi_t **out);
void free_vdi(vdi_t *v);
void mat4_mul(const double *A, const double *B, double *C);
bool mat4_inv(const double *m, double *out);
double ndc_to_view_depth(const double *P, double Z);
void grid_edges(const double *P, int nz, float *edges);
size_t touch_words(const vdi_t *v);
vdi_status check_render_args(const vdi_t *v, int W, int H, int d_i, int d_r, const void *out, int out_fmt);
void release_batch_cache(vdi_ctx *ctx);
cudaError_t launch_render(const ViewConsts &c, const DevVdi &v, void *out, int out_fmt, uint32_t *rl, uint32_t *rs,
                          int search, int warp_shape, bool ert, bool ess, bool blocks, const TileMaps *tm,
                          cudaStream_t st);
// the VDI's tensor maps for launch_render, or null when it has none
inline const TileMaps *tile_maps(const vdi_t *v) { return v->maps_ok ? &v->maps : nullptr; }
cudaError_t launch_block_range(const DevVdi &v, float2 *brange, cudaStream_t st);

// warp shape used when the caller does not choose one: 4 x 8 pixels per warp
// (lanes whose rays cross neighbouring lists together), except for exact
// renders from V_O's eye, where each lane reads one list and 32 x 1 pixels
// per warp read 32 neighbouring lists' records at once
inline int default_warp_shape(const vdi::ViewConsts &c) { return (c.single_list && c.d_r == 1) ? 0 : 3; }

// rays a request renders: explicit (Wr, Hr) when given, else ceil(W / d_i) x ceil(H / d_i)
template <class R>
inline void request_rays(const R &r, int &Wr, int &Hr) {
    if (r.Wr > 0 && r.Hr > 0) {
        Wr = r.Wr;
        Hr = r.Hr;
    } else {
        Wr = (r.W + r.d_i - 1) / r.d_i;
        Hr = (r.H + r.d_i - 1) / r.d_i;
    }
}

}  // namespace vdi
