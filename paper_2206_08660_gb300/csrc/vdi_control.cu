// vdi_control.cu -- the preview-rate controller of the remote-visualisation
// application (Section 4.4): a proportional-integral (PI) controller that
// modulates the image-space sampling D_I so that VDI frames keep a target
// frame time chosen by the user, while the user also picks the ray sampling
// D_R.  The paper names the controller type but not its law.  Frame time
// grows about with the number of rays, i.e. with s^2 for image-space scale s,
// so the loop runs on logarithms, where that plant has a constant gain:
//
//   e_k = ln(T* / T_k)                          frame-time error of frame k
//   I_k = I_{k-1} + K_i e_k                     unless s is pinned at a bound
//                                               and e_k pushes it further out
//   ln s_{k+1} = clamp(ln s_0 + K_p e_k + I_k, ln s_min, ln s_max)
//
// with T* the target, T_k the measured time of frame k, s the paper's D_I
// (the fraction of the display resolution rendered per axis) and s_0 the
// starting scale.  For a plant T = a s^2 the error then shrinks by the roots
// of z^2 - (1 - 2 K_p - 2 K_i) z - 2 K_p (0.56 and -0.36 for the default
// gains K_p = 0.1, K_i = 0.3).  The next frame is rendered at
// round(s W) x round(s H) rays (halves round up) and bilinearly upsampled to
// W x H (vdi_render_scaled).  Host code only.
#include <math.h>
#include <stdlib.h>

#include <new>

#include "../../include/vdi.h"
#include "vdi_api_internal.h"

#define VDI_API extern "C" __attribute__((visibility("default")))

struct vdi_pi {
    vdi_pi_config cfg;
    double integ;
    double scale;
    long long frames;
};

static int render_size(double scale, int n) {
    const long long r = llround(scale * (double)n);
    return (int)(r < 1 ? 1 : (r > n ? n : r));
}

VDI_API vdi_status vdi_pi_create(const vdi_pi_config *cfg, vdi_pi **out) {
    using vdi::fail;
    if (!cfg || !out) return fail(VDI_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (!(cfg->target_ms > 0.0) || !isfinite(cfg->target_ms)) return fail(VDI_ERR_INVALID_ARG, "target_ms must be > 0");
    if (!(cfg->scale_min > 0.0) || !(cfg->scale_min <= cfg->scale_max) || !(cfg->scale_max <= 1.0))
        return fail(VDI_ERR_INVALID_ARG, "need 0 < scale_min <= scale_max <= 1");
    if (!(cfg->scale_start >= cfg->scale_min && cfg->scale_start <= cfg->scale_max))
        return fail(VDI_ERR_INVALID_ARG, "scale_start outside [scale_min, scale_max]");
    if (!(cfg->kp >= 0.0) || !(cfg->ki >= 0.0) || !isfinite(cfg->kp) || !isfinite(cfg->ki))
        return fail(VDI_ERR_INVALID_ARG, "gains must be finite and >= 0");
    if (cfg->W < 1 || cfg->H < 1) return fail(VDI_ERR_INVALID_ARG, "display %dx%d", cfg->W, cfg->H);
    vdi_pi *p = new (std::nothrow) vdi_pi();
    if (!p) return fail(VDI_ERR_OOM, "host allocation");
    p->cfg = *cfg;
    p->integ = 0.0;
    p->scale = cfg->scale_start;
    p->frames = 0;
    *out = p;
    return VDI_OK;
}

VDI_API vdi_status vdi_pi_current(const vdi_pi *p, double *scale, int *Wr, int *Hr) {
    if (!p || !scale || !Wr || !Hr) return vdi::fail(VDI_ERR_INVALID_ARG, "NULL argument");
    *scale = p->scale;
    *Wr = render_size(p->scale, p->cfg.W);
    *Hr = render_size(p->scale, p->cfg.H);
    return VDI_OK;
}

VDI_API vdi_status vdi_pi_update(vdi_pi *p, double frame_ms, double *scale, int *Wr, int *Hr) {
    if (!p || !scale || !Wr || !Hr) return vdi::fail(VDI_ERR_INVALID_ARG, "NULL argument");
    if (!(frame_ms >= 0.0) || !isfinite(frame_ms)) return vdi::fail(VDI_ERR_INVALID_ARG, "frame_ms=%g", frame_ms);
    const vdi_pi_config &c = p->cfg;
    const double e = log(c.target_ms / (frame_ms > 1e-9 ? frame_ms : 1e-9));
    const bool pinned_high = p->scale >= c.scale_max && e > 0.0;
    const bool pinned_low = p->scale <= c.scale_min && e < 0.0;
    if (!pinned_high && !pinned_low) p->integ += c.ki * e;  // conditional integration (no wind-up)
    double s = exp(log(c.scale_start) + c.kp * e + p->integ);
    s = s < c.scale_min ? c.scale_min : (s > c.scale_max ? c.scale_max : s);
    p->scale = s;
    ++p->frames;
    return vdi_pi_current(p, scale, Wr, Hr);
}

VDI_API void vdi_pi_destroy(vdi_pi *p) { delete p; }
