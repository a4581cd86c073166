/*
 * vdi.h -- C ABI of the GB300 (sm_103a) Volumetric Depth Image renderer.
 *
 * Method: "Efficient Raycasting of Volumetric Depth Images for Remote
 * Visualization of Large Volumes at High Frame Rates" (arXiv 2206.08660).
 *
 * A VDI (Section 2.3) stores, for every pixel of an original view V_O, a
 * depth-sorted list of up to N_S supersegments, each with a front and back
 * depth and a classified colour/opacity.  The library renders a resident VDI
 * from a new view V_N by raycasting in V_O's NDC space (Section 4.1), finds
 * supersegments with the carried-index search of Algorithm 2 (Section 4.2),
 * corrects opacity by intersection length (Eq. 2) and composites front to
 * back; it also renders the subsampled previews of Section 4.4 and generates
 * VDIs from volumes (Section 3, Eq. 1, fixed sensitivity).
 *
 * Conventions used by every entry point
 *  - Matrices are OpenGL column-major double[16]; clip = proj * view * x_world;
 *    NDC = clip.xyz / clip.w in [-1,1]^3 (Fig. 3).
 *  - Supersegment depth is V_O NDC z (OpenGL, -1 = near plane).  V_O's
 *    near/far planes should bracket the volume tightly so FP32 depth keeps
 *    its resolution.
 *  - Colour is premultiplied RGBA; alpha is the opacity accumulated over one
 *    `length_unit` of world length, so a ray piece of world length l inside a
 *    supersegment contributes opacity 1 - (1 - alpha)^(l / length_unit)
 *    (Eq. 2) with colour rgb / alpha.
 *  - Image pixel (px, py) of a W x H image has NDC centre
 *    (2 (px + 1/2) / W - 1, 1 - 2 (py + 1/2) / H): row 0 is the top row;
 *    VDI list i = iy * w + ix uses the same convention.
 *  - Output images are premultiplied RGBA, row-major [H][W][4], background
 *    transparent black; VDI_F32 = float, VDI_F16 = IEEE half.
 *  - All device work is ordered on the caller's CUDA stream (`stream` is a
 *    cudaStream_t; NULL = legacy default stream).  A call returns after
 *    enqueueing unless stated otherwise.  Argument errors are reported
 *    synchronously; CUDA faults surface as VDI_ERR_CUDA from the call that
 *    observes them.
 *  - Every entry point returns vdi_status; no C++ exception crosses the ABI.
 *  - Objects (vdi_ctx, vdi_t) are owned by the library and released with
 *    their destroy call; caller-provided buffers stay owned by the caller.
 */
#ifndef VDI_H
#define VDI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VDI_OK = 0,
    VDI_ERR_INVALID_ARG = 1, /* bad pointer, size, enum or camera */
    VDI_ERR_OOM = 2,         /* device allocation failed or budget exceeded */
    VDI_ERR_CUDA = 3,        /* a CUDA call failed; see vdi_last_error_message() */
    VDI_ERR_UNSORTED = 4,    /* supersegments not sorted/disjoint, or non-finite depth */
    VDI_ERR_TIMEOUT = 5,     /* a bounded wait ran out */
    VDI_ERR_BUSY = 6,        /* object still referenced by in-flight work */
    VDI_ERR_UNSUPPORTED = 7  /* valid request outside what this build implements */
} vdi_status;

enum { VDI_F32 = 0, VDI_F16 = 1 };            /* colour / output formats */
enum { VDI_MEM_HOST = 0, VDI_MEM_DEVICE = 1 }; /* where an input buffer lives */
enum {                                          /* first-supersegment search (Section 4.2, Fig. 4) */
    VDI_SEARCH_ALG2 = 0,   /* carried index + pruned binary search (Algorithm 2), default */
    VDI_SEARCH_BINARY = 1, /* binary search seeded at the middle of the list */
    VDI_SEARCH_LINEAR = 2  /* linear search from the first slot */
};

typedef struct vdi_ctx vdi_ctx; /* one per device */
typedef struct vdi_t vdi_t;     /* a device-resident VDI */

typedef struct {
    double view[16]; /* world -> eye, column-major */
    double proj[16]; /* eye -> clip, column-major; perspective or orthographic */
} vdi_camera;

typedef struct {
    int w, h;                 /* lists (= V_O viewport pixels) */
    int n_s;                  /* supersegments per list, 1..64 (N_S) */
    vdi_camera orig;          /* V_O */
    double bbox_min[3];       /* volume box in world space; rays are clipped to it */
    double bbox_max[3];
    double length_unit;       /* world length over which the stored alpha is defined (> 0) */
    int colour_fmt;           /* device colour storage: VDI_F32 or VDI_F16 (depth is always FP32) */
    int grid_tile;            /* supersegment-count grid: lists per cell side, 0 -> 8 */
    int grid_nz;              /* grid slabs of equal V_O view depth, 1..64, 0 -> 20 */
} vdi_desc;

typedef struct {
    size_t depth_bytes;  /* front/back FP32 depths on the device */
    size_t colour_bytes; /* colour + opacity on the device */
    size_t grid_bytes;   /* uint32 supersegment counts */
    size_t list_bytes;   /* per list, then per block of 4 x 4 lists: front of the first and back of the last
                            supersegment (float2 each) */
    size_t total_bytes;  /* everything the VDI holds on the device */
    size_t paper_bytes;  /* size in the paper's RGBA32F + 2 x R32F layout: 24 B per slot (Section 5) */
    int grid_w, grid_h, grid_nz;
    int n_s_stored;      /* slots per list as stored (N_S rounded up to even) */
} vdi_layout;

typedef struct {
    int search;          /* VDI_SEARCH_*; default VDI_SEARCH_ALG2 (the exact path; D_R previews read
                            a list's depth records several pairs at a time whatever the mode) */
    int no_ert;          /* 1: keep compositing past full opacity (for exact counters) */
    uint32_t *ray_lists; /* nullable device [H'][W']: lists traversed with positive length per ray */
    uint32_t *ray_segs;  /* nullable device [H'][W']: supersegment pieces of positive length per ray */
    int warp_shape;      /* -1: default (32x1 for exact renders from V_O's eye, else 4x8); 0: 32x1, 1: 16x2, 2: 8x4, 3: 4x8 pixels per warp.
                            A view from V_O's eye at V_O's own pixel grid with 32x1 warps loads each
                            32x8 tile's list ranges and first slot pairs into shared memory by TMA;
                            the image does not depend on the shape. */
    int ess;             /* 1: empty-space skipping over the count grid (Section 4.3): occupied cells
                            only.  Off by default (measured slower on the benchmark workloads); the
                            image is the same up to where early termination lands; per-ray
                            counters always come from the walk over every list. */
    int blocks;          /* 1: skip 4 x 4 blocks of lists whose merged depth range the ray misses.
                            Off by default (measured slower on the benchmark workloads); the image
                            is bit-identical either way. */
    int record_stats;    /* 1: count this frame's rays, lists and supersegment pieces into the
                            VDI's totals, read back by vdi_stats (exact renders only, d_r = 1; the
                            rays walk every list as with ray_lists; temporary per-ray counters
                            come from the stream-ordered allocator when ray_lists / ray_segs are
                            NULL) */
} vdi_render_opts;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device` (made current by every call that
 * uses the context).  *out owned by the caller; release with vdi_ctx_destroy. */
vdi_status vdi_ctx_create(int device, vdi_ctx **out);
void vdi_ctx_destroy(vdi_ctx *ctx);

/* Text of a status code (static storage). */
const char *vdi_status_str(vdi_status s);
/* Message of the last error raised on this host thread (thread-local storage). */
const char *vdi_last_error_message(void);

/* ---- layout ------------------------------------------------------------ */

/* Device bytes a VDI with this descriptor occupies.  Host only, no GPU
 * needed.  Section 5: the paper's VDI is an RGBA32F colour texture plus an
 * R32F depth texture holding front and back (24 B per slot); Section 6.3
 * quotes 422 MiB / 950 MiB at 1280x720 / 1920x1080 with N_S = 20 and a
 * 2.5 MiB empty-space grid at 1920x1080.  Device layout here is
 * structure-of-arrays: slot pairs of FP32 (front, back) depths [N_S/2][h*w]
 * as 16-byte records, and per slot (rgb / alpha, -log2(1 - alpha)) in FP32
 * ([N_S][h*w], 16 B) or FP16 ([N_S/2][h*w], two slots per 16 B). */
vdi_status vdi_layout_bytes(const vdi_desc *desc, vdi_layout *out);

/* ---- create / download / destroy --------------------------------------- */

/* Build a device-resident VDI from supersegment buffers (Section 2.3).
 *  rgba   [h][w][n_s][4] float, premultiplied, alpha per length_unit, 0 <= rgb <= alpha <= 1
 *  depth  [h][w][n_s][2] float, V_O NDC z (front, back)
 *  counts [h][w] int32 supersegments per list (0..n_s), or NULL: the leading
 *         slots whose front depth is finite are used
 * Valid slots must satisfy f <= b, b_j <= f_{j+1}, finite depths; slots beyond
 * the count are ignored.  `mem_kind` says whether the three buffers are host
 * or device memory; they are copied and may be freed when the call returns
 * (it synchronises `stream` to report VDI_ERR_UNSORTED / VDI_ERR_INVALID_ARG).
 * Also builds the supersegment-count grid of Section 4.3 (grid_tile x
 * grid_tile lists by grid_nz slabs of equal V_O view depth; a supersegment
 * counts in every slab its [f, b] overlaps).  *out released with vdi_destroy. */
vdi_status vdi_create(vdi_ctx *ctx, const vdi_desc *desc, const float *rgba, const float *depth,
                      const int32_t *counts, int mem_kind, void *stream, vdi_t **out);

/* Copy a VDI back to HOST buffers in the vdi_create layout (any may be NULL).
 * Depths, counts and the grid are exact; colour is reconverted from the
 * device form (FP32: within a few ulp; FP16: half precision).  Unused slots
 * come back as depth +inf and colour 0.  grid: [grid_nz][grid_h][grid_w]
 * uint32.  Synchronises `stream`. */
vdi_status vdi_download(vdi_t *vdi, float *rgba, float *depth, int32_t *counts, uint32_t *grid,
                        void *stream);

/* Layout of an existing VDI. */
vdi_status vdi_get_layout(const vdi_t *vdi, vdi_layout *out);

/* What a resident VDI holds and what its last counted frame did.  Sizes:
 * Section 5 stores a VDI as an RGBA32F colour texture plus an R32F texture
 * holding front and back depth (24 B per slot: 950 MiB at 1920 x 1080,
 * N_S = 20, Section 6.3), and a count grid of 2.5 MiB at 1920 x 1080
 * (Section 4.3); `layout` gives this library's bytes per array and the
 * paper-layout size.  Frame totals: the last vdi_render_ex call with
 * record_stats = 1 on this VDI, summed over its rays (Section 4.1: the lists
 * a ray passes through; Section 4.2 / Eq. 2: the supersegment pieces it
 * composites; with early termination unless no_ert).  Reading the totals
 * synchronises `stream` (the stream that render was ordered on).  Before any
 * counted frame, frame_recorded is 0 and the totals are 0.  device_flags:
 * bits the render kernels set on the device for this VDI, read on every call
 * (VDI_FLAG_STAGE_TIMEOUT: a bounded wait for a TMA-staged tile of list
 * records ran out; those rays read global memory instead, so the image is
 * unaffected, and the flag means the copies were far slower than expected). */
#define VDI_FLAG_STAGE_TIMEOUT 1u
typedef struct {
    vdi_layout layout;      /* device bytes by array, grid dims, slots stored per list */
    int w, h, n_s;          /* lists and supersegments per list */
    int colour_fmt;         /* VDI_F32 or VDI_F16 */
    int grid_tile;          /* lists per grid cell side */
    int frame_recorded;     /* 1 when the totals below describe a counted frame */
    int frame_w, frame_h;   /* rays of that frame (after d_i) */
    uint64_t rays_hit;      /* rays that passed through at least one list with positive length */
    uint64_t lists;         /* lists passed through with positive length, summed over the rays */
    uint64_t pieces;        /* supersegment pieces of positive length composited, summed over the rays */
    uint32_t device_flags;  /* VDI_FLAG_* bits set by kernels on this VDI since it was created */
} vdi_stats_t;
vdi_status vdi_stats(vdi_t *vdi, vdi_stats_t *out, void *stream);

/* Free the VDI's device memory.  Stream-ordered on the stream it was created
 * on; the caller must not destroy a VDI that other streams still render. */
void vdi_destroy(vdi_t *vdi);

/* ---- render --------------------------------------------------------------
 * Render `vdi` from the new view `view` into the caller's DEVICE buffer
 * out_rgba ([H][W][4] of out_fmt).
 *  d_i = 1, d_r = 1: the full method of Section 4: per pixel ray clipped to
 *    V_O's frustum and the box (Section 4.1, Fig. 2), walked list by list
 *    through V_O's NDC grid (Amanatides-Woo), first supersegment per list by
 *    Algorithm 2 with the index carried from the previous list, adjacency
 *    walk, opacity corrected by world intersection length (Eq. 2),
 *    front-to-back compositing with early termination at alpha >= 1 - 2^-12.
 *  d_r = k > 1: ray-subsampled preview (Section 4.4): per grid cell crossed,
 *    ceil((count / lists_in_cell) * (l_cell / cell_depth) / k) samples at equal
 *    world spacing; each takes the colour of the supersegment containing it,
 *    opacity corrected by the spacing.
 *  d_i = k > 1: image-space preview (Section 4.4): ceil(W/k) x ceil(H/k) rays,
 *    bilinearly upsampled to W x H (half-pixel centres, clamp to edge).
 *  W, H in 1..16384; d_i, d_r in 1..16.  Temporary device memory for d_i > 1
 *  comes from the stream-ordered allocator. */
vdi_status vdi_render(vdi_t *vdi, const vdi_camera *view, int W, int H, int d_i, int d_r,
                      void *out_rgba, int out_fmt, void *stream);

/* vdi_render with options (NULL opts = defaults).  Counters are written for
 * the rendered (pre-upsampling) resolution. */
vdi_status vdi_render_ex(vdi_t *vdi, const vdi_camera *view, int W, int H, int d_i, int d_r,
                         void *out_rgba, int out_fmt, const vdi_render_opts *opts, void *stream);

/* vdi_render with any image-space scale (the paper's fractional D_I, Section
 * 4.4): Wr x Hr rays (1 <= Wr <= W, 1 <= Hr <= H) over the same image plane,
 * bilinearly upsampled to the W x H output (half-pixel centres, clamp to
 * edge); Wr = ceil(W / d_i), Hr = ceil(H / d_i) gives exactly vdi_render's
 * d_i preview.  The low-resolution image comes from the stream-ordered
 * allocator.  Errors as vdi_render. */
vdi_status vdi_render_scaled(vdi_t *vdi, const vdi_camera *view, int W, int H, int Wr, int Hr, int d_r,
                             void *out_rgba, int out_fmt, void *stream);

/* ---- preview-rate controller (Section 4.4) ---------------------------------
 * A proportional-integral controller that picks the image-space scale s (the
 * paper's D_I: fraction of the display resolution rendered per axis) so that
 * frames keep a target frame time; the caller keeps D_R.  The paper names the
 * controller type only; the law here runs on logarithms (frame time grows
 * about with s^2): e = ln(target / measured), I += ki e (skipped while s sits
 * at a bound and e pushes it further out), ln s = clamp(ln scale_start + kp e
 * + I, ln scale_min, ln scale_max).  The next frame is rendered at
 * round(s W) x round(s H) rays, halves rounding up (vdi_render_scaled).  Host-only
 * state; no GPU work.  vdi_pi_update takes the measured time of the frame
 * rendered at the current scale and returns the scale and ray counts of the
 * next one. */
typedef struct {
    double target_ms;                 /* target frame time (> 0) */
    double kp, ki;                    /* gains (>= 0); 0.1 and 0.3 are the defaults of the binding */
    double scale_min, scale_max;      /* 0 < scale_min <= scale_max <= 1 */
    double scale_start;               /* first frame's scale, inside the bounds */
    int W, H;                         /* display resolution */
} vdi_pi_config;
typedef struct vdi_pi vdi_pi;
vdi_status vdi_pi_create(const vdi_pi_config *cfg, vdi_pi **out);
vdi_status vdi_pi_current(const vdi_pi *pi, double *scale, int *Wr, int *Hr);
vdi_status vdi_pi_update(vdi_pi *pi, double frame_ms, double *scale, int *Wr, int *Hr);
void vdi_pi_destroy(vdi_pi *pi);

/* ---- batched multi-view rendering ---------------------------------------
 * Render up to VDI_BATCH_MAX_REQUESTS views of up to VDI_BATCH_MAX_VDIS
 * resident VDIs (of any resolutions, formats, previews) in one batched
 * launch: exact requests are cut into 32x8-pixel tiles and previews (d_r > 1)
 * into 32x2-pixel tiles served with four lanes per ray; each kind forms a queue
 * that a persistent grid of (SM count x resident blocks per SM) blocks drains.
 * Each request renders exactly as vdi_render would (the same per-pixel
 * arithmetic, so results do not depend on what else is in the batch).
 * With use_graph the launch sequence is replayed from a CUDA graph cached per
 * batch shape (resolutions, previews, launch configuration, stream); a replay
 * only updates the graph's kernel parameters.  The graph path keeps its
 * scratch (tile counter, low-resolution images for D_I > 1) with the cached
 * graph: batches of one shape on one stream run one after another; the plain
 * path takes scratch from the stream-ordered allocator.  A cached graph lives
 * until vdi_ctx_destroy.  warp_shape = -1 uses the configuration stored by
 * vdi_autotune_batch for batches with the same signature (resolutions,
 * previews, N_S, colour formats), else 4x8. */
enum { VDI_BATCH_MAX_REQUESTS = 64, VDI_BATCH_MAX_VDIS = 8 };

typedef struct {
    vdi_t *vdi;          /* resident VDI (of this context) */
    vdi_camera view;     /* V_N */
    int W, H, d_i, d_r;  /* as in vdi_render */
    void *out;           /* DEVICE [H][W][4] of out_fmt */
    int out_fmt;
    int Wr, Hr;          /* rays rendered, as in vdi_render_scaled (1..W, 1..H; d_i is then ignored);
                            0, 0: ceil(W / d_i) x ceil(H / d_i) */
} vdi_request;

typedef struct {
    int warp_shape;      /* -1 autotuned/default (4x8), 0: 32x1, 1: 16x2, 2: 8x4, 3: 4x8 pixels per warp */
    int blocks_per_sm;   /* resident blocks per SM of the persistent grid, 0 = occupancy limit */
    int use_graph;       /* 1: replay a cached CUDA graph for this batch shape */
} vdi_batch_opts;

vdi_status vdi_render_batch(vdi_ctx *ctx, const vdi_request *reqs, int n, const vdi_batch_opts *opts, void *stream);

/* Autotuner: time every (warp shape, blocks per SM) on this batch -- it
 * renders into the requests' outputs -- remember the fastest for batches of
 * the same signature in this context and return it (with use_graph = 1) and
 * its time per batch in milliseconds.  Synchronises `stream`. */
vdi_status vdi_autotune_batch(vdi_ctx *ctx, const vdi_request *reqs, int n, void *stream, vdi_batch_opts *best,
                              float *best_ms);

/* ---- serving ---------------------------------------------------------------
 * A continuous-batching view server over resident VDIs.  The paper's client
 * renders views from the resident VDI while the next one is uploaded in the
 * background (Section 5, double buffering); here up to n_slots VDIs stay
 * resident and any number of clients submit view requests:
 *  - vdi_server_submit queues a request and returns a ticket at once;
 *  - a scheduler thread admits queued requests FIFO into the next batch as
 *    soon as one of `max_inflight` batch streams is free and their image
 *    memory (plus low-resolution scratch for D_I > 1) fits under
 *    `budget_bytes` next to everything not yet released and the resident
 *    VDIs; a request that can never fit fails with VDI_ERR_OOM; batches run
 *    while new requests are admitted behind them (continuous batching, work
 *    overlaps on the device);
 *  - each batch is one vdi_render_batch launch: every result equals the same
 *    view rendered alone by vdi_render;
 *  - vdi_server_set_vdi installs or replaces a slot's VDI at any time (the
 *    server takes ownership).  Batches formed after the work enqueued on
 *    `ready_stream` (e.g. the side stream of a vdi_generate) has completed use
 *    the new VDI; the old one is freed when the last batch using it retires;
 *  - the budget is a device budget: every live VDI version (layout
 *    total_bytes; a replaced one until its last batch retires) counts against
 *    it next to images and scratch.  vdi_server_set_vdi returns VDI_ERR_OOM
 *    (the caller keeps the VDI) when the VDI does not fit;
 *    vdi_server_generate charges the new VDI's bytes before generating it
 *    (vdi_generate on `stream`, then an install ready on that stream) and
 *    returns VDI_ERR_OOM without generating when they do not fit;
 *  - results stay in server-owned DEVICE memory until vdi_server_release;
 *  - waits are bounded: vdi_server_wait returns VDI_ERR_TIMEOUT;
 *  - batches run on streams of the highest priority, so work the caller
 *    enqueues on default-priority streams (e.g. generation) yields to them.
 * Times are seconds of a host monotonic clock. */
typedef struct vdi_server vdi_server;

typedef struct {
    size_t budget_bytes;   /* device memory for resident VDIs, unreleased results and preview scratch */
    int max_batch;         /* requests per launch, 1..VDI_BATCH_MAX_REQUESTS */
    int max_inflight;      /* batches on the device at once (streams), 1..16 */
    int n_slots;           /* resident VDI slots, 1..VDI_BATCH_MAX_VDIS */
    double wait_timeout_s; /* bound on internal waits at shutdown (0 -> 10 s) */
} vdi_server_config;

typedef struct {
    int slot;              /* resident VDI slot */
    vdi_camera view;
    int W, H, d_i, d_r, out_fmt;
    int Wr, Hr;            /* rays rendered (as in vdi_request); 0, 0: from d_i.  A client that
                              keeps a frame rate with the preview controller (vdi_pi_*) passes
                              the ray counts vdi_pi_update returned */
} vdi_view_request;

typedef struct {
    int status;            /* -1 while queued or running, else a vdi_status */
    double t_submit, t_start, t_done;
    void *image;           /* DEVICE [H][W][4] of out_fmt when status == VDI_OK */
    size_t image_bytes;
} vdi_ticket_info;

typedef struct {
    uint64_t submitted, completed, failed, batches, batched_requests, vdi_installs;
    uint64_t pending, batches_in_flight;
    size_t bytes_in_use;   /* unreleased images and preview scratch */
    size_t vdi_bytes;      /* live VDI versions and VDIs being generated through the server */
} vdi_server_counters;

vdi_status vdi_server_create(vdi_ctx *ctx, const vdi_server_config *cfg, vdi_server **out);
vdi_status vdi_server_set_vdi(vdi_server *s, int slot, vdi_t *vdi, void *ready_stream);
/* vdi_server_generate (after vdi_generate below): generation into a slot, its
 * bytes charged to the budget first. */
vdi_status vdi_server_submit(vdi_server *s, const vdi_view_request *req, uint64_t *ticket);
vdi_status vdi_server_wait(vdi_server *s, uint64_t ticket, double timeout_s, vdi_ticket_info *info);
vdi_status vdi_server_poll(vdi_server *s, uint64_t ticket, vdi_ticket_info *info);
/* Copy a finished ticket's image into the caller's buffer (`dst_kind` is
 * VDI_MEM_HOST or VDI_MEM_DEVICE; `bytes` must equal the image size), ordered
 * on `stream` and synchronised before returning. */
vdi_status vdi_server_read(vdi_server *s, uint64_t ticket, void *dst, size_t bytes, int dst_kind, void *stream);
/* Free a finished ticket's result (VDI_ERR_BUSY while it is still running). */
vdi_status vdi_server_release(vdi_server *s, uint64_t ticket);
vdi_status vdi_server_stats(vdi_server *s, vdi_server_counters *out);
/* Stops admitting, waits (bounded) for batches in flight, frees everything
 * including the installed VDIs. */
void vdi_server_destroy(vdi_server *s);

/* ---- generation ----------------------------------------------------------
 * Build a VDI from a scalar volume (Section 3) with the homogeneity
 * criterion of Eq. 1 at a fixed sensitivity gamma = tau: along each V_O
 * pixel-centre ray (clipped to V_O's near/far planes and the volume box),
 * samples at the midpoints of consecutive intervals of world length `step`
 * are classified by the transfer function, given opacity
 * a' = 1 - (1 - alpha_tf)^(step / length_unit), and merged into the current
 * supersegment while tau > || mean premultiplied colour of the supersegment
 * - premultiplied colour of the sample ||_2; otherwise a new supersegment
 * starts.  A fully transparent sample closes the current supersegment; the
 * n_s-th supersegment absorbs everything that follows.  Rays stop once their
 * opacity reaches 1 - 2^-12.  Each supersegment stores the exact composite of
 * its samples, so rendering at V_O reproduces the samples' compositing.
 * FP32 arithmetic is IEEE round-to-nearest without fused operations, in a
 * fixed order (supersegment counts and depths are reproducible bit for bit).
 * Also builds the count grid.  Returns after enqueueing on `stream`. */
enum { VDI_VOL_U8 = 0, VDI_VOL_U16 = 1, VDI_VOL_F32 = 2 };

typedef struct {
    int nx, ny, nz;      /* voxels; element (i, j, k) at data[(k * ny + j) * nx + i] */
    int dtype;           /* VDI_VOL_*; u8 / 255, u16 / 65535 and f32 values are the scalar */
    const void *data;    /* DEVICE pointer, owned by the caller, read until the work completes */
    double bbox_min[3];  /* world box the volume fills; voxel centres at (index + 1/2) / n of it, */
    double bbox_max[3];  /* trilinear interpolation with clamp to edge */
} vdi_volume;

typedef struct {
    int n_knots;         /* 2..16 */
    const float *knots;  /* HOST [n_knots][5]: value, r, g, b, alpha (opacity per length_unit);
                            values strictly increasing; piecewise linear, constant beyond the ends */
} vdi_tf;

typedef struct {
    int w, h, n_s;       /* lists and supersegments per list (1..64) */
    vdi_camera orig;     /* V_O: an OpenGL perspective frustum */
    float tau;           /* gamma of Eq. 1 (>= 0) */
    double step;         /* world sampling step (> 0) */
    double length_unit;  /* world length the stored and transfer-function alphas refer to */
    int colour_fmt;      /* VDI_F32 or VDI_F16 */
    int grid_tile, grid_nz; /* count grid (0 -> 8, 20) */
    int adaptive;        /* 0: gamma = tau for every ray; 1: each ray finds its own gamma by the
                            bisection of Section 3 (Algorithm 3 of the supplement): in [0, sqrt(3)],
                            from 1e-5, until it gets N_S - floor(0.15 N_S) .. N_S supersegments or
                            the interval is narrower than 1e-4; tau is then ignored */
    float *tau_out;      /* DEVICE [h][w] or NULL: the gamma each list used */
} vdi_gen_params;

vdi_status vdi_generate(vdi_ctx *ctx, const vdi_volume *vol, const vdi_tf *tf, const vdi_gen_params *params,
                        void *stream, vdi_t **out);

/* Serving (above): generate a VDI on `stream` (vdi_generate of the server's
 * context) and install it in `slot` once that stream reaches the end of the
 * generation, with its device bytes (vdi_layout_bytes of the parameters)
 * charged to the server's budget before anything is allocated.  VDI_ERR_OOM
 * when they do not fit next to the resident VDIs and unreleased results;
 * other errors as vdi_generate.  Returns after enqueueing. */
vdi_status vdi_server_generate(vdi_server *s, int slot, const vdi_volume *vol, const vdi_tf *tf,
                               const vdi_gen_params *params, void *stream);

/* ---- ground truth and image quality (Section 6) ----------------------------
 * vdi_dvr: direct volume rendering of the volume from `view` (an OpenGL
 * perspective frustum; the ray of pixel (px, py) runs through its centre from
 * the near to the far plane, clipped to the box), with the sampling rules of
 * vdi_generate: samples at the midpoints of world intervals of `step` from the
 * box entry, trilinear interpolation, the transfer function, opacity
 * 1 - (1 - alpha)^(step / length_unit), front-to-back emission-absorption
 * compositing, early termination at transmittance 2^-12.  out_rgba: DEVICE
 * W x H premultiplied RGBA of out_fmt (row 0 on top), caller-owned.
 * Stream-ordered; argument errors are returned synchronously.
 *
 * vdi_image_quality: SSIM and PSNR of image `a` against reference `b`, the
 * measures of the paper's evaluation (SSIM of Wang et al. 2004).  a, b: DEVICE
 * W x H RGBA images of fmt (W, H >= 7); both measures use the R, G, B channels
 * with data range 1.  SSIM: 7 x 7 windows fully inside the image, window
 * means, sample variances and covariance (divided by 48), C1 = 0.01^2,
 * C2 = 0.03^2, mean over windows and channels.  PSNR = 10 log10(1 / MSE) over
 * all pixels and channels (+inf for identical images).  Results are written to
 * the host doubles; the call synchronises `stream`. */
vdi_status vdi_dvr(vdi_ctx *ctx, const vdi_volume *vol, const vdi_tf *tf, const vdi_camera *view, int W, int H,
                   double step, double length_unit, void *out_rgba, int out_fmt, void *stream);
vdi_status vdi_image_quality(const void *a, const void *b, int W, int H, int fmt, double *ssim, double *psnr,
                             void *stream);

/* ---- render without device allocation -------------------------------------
 * The paper has no counterpart to this entry point.  It renders exactly what
 * vdi_render renders, but the low-resolution image of an image-space preview
 * (d_i > 1) lives in a fixed buffer of this library -- a static device array
 * of VDI_STATIC_PREVIEW_PIXELS RGBA floats (8 MiB; enough for 1920 x 1080 at
 * d_i = 2), held on every GPU that loads the library until the process exits
 * -- so the call performs no device allocation.  It is for callers that
 * cannot allocate while rendering: an application that has given all device
 * memory to resident VDIs (a per-frame allocation could fail), a frame loop
 * that must not wait on an allocator, or a program that allocates only at
 * start-up.
 *  - ceil(W/d_i) * ceil(H/d_i) above VDI_STATIC_PREVIEW_PIXELS (with d_i > 1)
 *    returns VDI_ERR_INVALID_ARG; d_i = 1 needs no buffer.
 *  - The first call with d_i > 1 on a device looks up the buffer's device
 *    address (cudaGetSymbolAddress with that device current); make that first
 *    call before any stream capture.
 *  - Every call shares the buffer, which keeps the last call's contents (a
 *    call writes every pixel it reads, so nothing needs clearing): calls that
 *    overlap on the GPU -- on different streams or from different threads --
 *    race on it.  Order them on one stream or synchronise between them. */
#define VDI_STATIC_PREVIEW_PIXELS 524288
vdi_status vdi_render_preview_static(vdi_t *vdi, const vdi_camera *view, int W, int H, int d_i, int d_r,
                                     void *out_rgba, int out_fmt, void *stream);

/* ---- diagnostics --------------------------------------------------------
 * Run the device first-supersegment search on a batch of queries against
 * list `list` of `vdi` (Algorithm 2 and the ablation searches).  Device
 * buffers of length n: d_entry, d_exit (float), seed (int32, -1 = none),
 * increasing (int32 0/1); result (int32): index of the first supersegment
 * met, or -1.  Exposed so the index contract can be tested bit-exactly. */
vdi_status vdi_search_first(vdi_t *vdi, int list, int search, const float *d_entry,
                            const float *d_exit, const int32_t *seed, const int32_t *increasing,
                            int32_t *result, int n, void *stream);

/* Mark, in a caller-provided zeroed DEVICE bitmap, every 4-byte word of the
 * VDI's depth and colour arrays that an exact render (d_i = d_r = 1,
 * Algorithm 2) of `view` at W x H reads under the method's access rule
 * (Section 4.2: per list passed through, its depth range (front of the
 * first, back of the last supersegment); the two depths of Algorithm 2's seed
 * probe, one depth per binary-search probe, front/back depth of each
 * supersegment walked, the colour record of each supersegment piece
 * composited).  Bit (w mod 32) of word w / 32 stands for the 4-byte word w of
 * the VDI's device arrays laid end to end (vdi_layout_bytes): the depth array
 * ([n_s_stored / 2][h*w] records of (f_2k, b_2k, f_2k+1, b_2k+1)), the colour
 * array (FP32: [n_s_stored][h*w] records of 4 words; FP16: [n_s_stored / 2][h*w]
 * records holding two slots of 2 words), the count grid
 * (grid_nz * grid_h * grid_w words, padded to a multiple of 4) and the list
 * ranges ([h*w] pairs (front, back)).  `words` is the bitmap length in uint32
 * and must be at least ceil((depth_bytes + colour_bytes + 4 * grid words
 * + list_bytes) / 128).  The popcount times 4 is the number of unique VDI
 * bytes one frame needs (the roofline numerator). */
vdi_status vdi_touch_bitmap(vdi_t *vdi, const vdi_camera *view, int W, int H, uint32_t *bitmap, size_t words,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VDI_H */
