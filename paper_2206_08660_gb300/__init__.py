"""Python binding of the GB300 VDI renderer (C ABI in ``include/vdi.h``).

Argument marshalling only: every step of the render, create and generate
paths runs in the CUDA library ``_build/libvdi.so``.  There is no CPU
fallback; if the library is missing or cannot be loaded every call raises.

Functions keep the C names (``vdi_create``, ``vdi_render``, ...).  Device
buffers are passed as torch CUDA tensors (or raw integer device pointers),
host buffers as numpy arrays; streams default to torch's current stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "VDI_F32", "VDI_F16", "VDI_MEM_HOST", "VDI_MEM_DEVICE", "VDI_SEARCH_ALG2", "VDI_SEARCH_BINARY", "VDI_FLAG_STAGE_TIMEOUT",
    "VDI_SEARCH_LINEAR", "VdiError", "VdiCamera", "VdiDesc", "VdiLayout", "VdiRenderOpts", "load",
    "vdi_ctx_create", "vdi_ctx_destroy", "vdi_layout_bytes", "vdi_create", "vdi_download", "vdi_get_layout", "vdi_stats",
    "vdi_destroy", "vdi_render", "vdi_render_ex", "vdi_render_preview_static", "VDI_STATIC_PREVIEW_PIXELS", "vdi_search_first", "vdi_generate", "vdi_touch_bitmap", "vdi_render_batch", "vdi_autotune_batch", "request",
    "vdi_server_create", "vdi_server_set_vdi", "vdi_server_generate", "vdi_server_submit", "vdi_server_wait", "vdi_server_poll",
    "vdi_server_release", "vdi_server_read", "vdi_server_stats", "vdi_server_destroy", "VdiViewRequest", "VdiTicketInfo",
    "VdiRequest", "VdiBatchOpts", "camera", "desc",
]

VDI_F32, VDI_F16 = 0, 1
VDI_STATIC_PREVIEW_PIXELS = 524288
VDI_MEM_HOST, VDI_MEM_DEVICE = 0, 1
VDI_SEARCH_ALG2, VDI_SEARCH_BINARY, VDI_SEARCH_LINEAR = 0, 1, 2
VDI_FLAG_STAGE_TIMEOUT = 1
STATUS = ["VDI_OK", "VDI_ERR_INVALID_ARG", "VDI_ERR_OOM", "VDI_ERR_CUDA", "VDI_ERR_UNSORTED",
          "VDI_ERR_TIMEOUT", "VDI_ERR_BUSY", "VDI_ERR_UNSUPPORTED"]


class VdiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {msg}")


class VdiCamera(C.Structure):
    _fields_ = [("view", C.c_double * 16), ("proj", C.c_double * 16)]


class VdiDesc(C.Structure):
    _fields_ = [("w", C.c_int), ("h", C.c_int), ("n_s", C.c_int), ("orig", VdiCamera),
                ("bbox_min", C.c_double * 3), ("bbox_max", C.c_double * 3), ("length_unit", C.c_double),
                ("colour_fmt", C.c_int), ("grid_tile", C.c_int), ("grid_nz", C.c_int)]


class VdiLayout(C.Structure):
    _fields_ = [("depth_bytes", C.c_size_t), ("colour_bytes", C.c_size_t), ("grid_bytes", C.c_size_t),
                ("list_bytes", C.c_size_t), ("total_bytes", C.c_size_t), ("paper_bytes", C.c_size_t), ("grid_w", C.c_int),
                ("grid_h", C.c_int), ("grid_nz", C.c_int), ("n_s_stored", C.c_int)]


class VdiStats(C.Structure):
    _fields_ = [("layout", VdiLayout), ("w", C.c_int), ("h", C.c_int), ("n_s", C.c_int), ("colour_fmt", C.c_int),
                ("grid_tile", C.c_int), ("frame_recorded", C.c_int), ("frame_w", C.c_int), ("frame_h", C.c_int),
                ("rays_hit", C.c_uint64), ("lists", C.c_uint64), ("pieces", C.c_uint64),
                ("device_flags", C.c_uint32)]


class VdiVolume(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dtype", C.c_int), ("data", C.c_void_p),
                ("bbox_min", C.c_double * 3), ("bbox_max", C.c_double * 3)]


class VdiTf(C.Structure):
    _fields_ = [("n_knots", C.c_int), ("knots", C.c_void_p)]


class VdiGenParams(C.Structure):
    _fields_ = [("w", C.c_int), ("h", C.c_int), ("n_s", C.c_int), ("orig", VdiCamera), ("tau", C.c_float),
                ("step", C.c_double), ("length_unit", C.c_double), ("colour_fmt", C.c_int),
                ("grid_tile", C.c_int), ("grid_nz", C.c_int), ("adaptive", C.c_int), ("tau_out", C.c_void_p)]


class VdiRequest(C.Structure):
    _fields_ = [("vdi", C.c_void_p), ("view", VdiCamera), ("W", C.c_int), ("H", C.c_int), ("d_i", C.c_int),
                ("d_r", C.c_int), ("out", C.c_void_p), ("out_fmt", C.c_int), ("Wr", C.c_int), ("Hr", C.c_int)]


class VdiBatchOpts(C.Structure):
    _fields_ = [("warp_shape", C.c_int), ("blocks_per_sm", C.c_int), ("use_graph", C.c_int)]


class VdiServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("max_batch", C.c_int), ("max_inflight", C.c_int),
                ("n_slots", C.c_int), ("wait_timeout_s", C.c_double)]


class VdiViewRequest(C.Structure):
    _fields_ = [("slot", C.c_int), ("view", VdiCamera), ("W", C.c_int), ("H", C.c_int), ("d_i", C.c_int),
                ("d_r", C.c_int), ("out_fmt", C.c_int), ("Wr", C.c_int), ("Hr", C.c_int)]


class VdiTicketInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("image", C.c_void_p), ("image_bytes", C.c_size_t)]


class VdiServerCounters(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("batches", C.c_uint64), ("batched_requests", C.c_uint64), ("vdi_installs", C.c_uint64),
                ("pending", C.c_uint64), ("batches_in_flight", C.c_uint64), ("bytes_in_use", C.c_size_t),
                ("vdi_bytes", C.c_size_t)]


class VdiRenderOpts(C.Structure):
    _fields_ = [("search", C.c_int), ("no_ert", C.c_int), ("ray_lists", C.c_void_p),
                ("ray_segs", C.c_void_p), ("warp_shape", C.c_int), ("ess", C.c_int), ("blocks", C.c_int),
                ("record_stats", C.c_int)]


_lib = None
P = C.c_void_p


def _sig(L, name, args, res=C.c_int):
    f = getattr(L, name)
    f.argtypes = args
    f.restype = res
    return f


def load(build_if_needed: bool = True):
    """Load libvdi.so (building it first when sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_needed and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = C.CDLL(path)
    _sig(L, "vdi_status_str", [C.c_int], C.c_char_p)
    _sig(L, "vdi_last_error_message", [], C.c_char_p)
    _sig(L, "vdi_ctx_create", [C.c_int, C.POINTER(P)])
    _sig(L, "vdi_ctx_destroy", [P], None)
    _sig(L, "vdi_layout_bytes", [P, P])
    _sig(L, "vdi_create", [P, P, P, P, P, C.c_int, P, C.POINTER(P)])
    _sig(L, "vdi_download", [P, P, P, P, P, P])
    _sig(L, "vdi_get_layout", [P, P])
    _sig(L, "vdi_stats", [P, P, P])
    _sig(L, "vdi_destroy", [P], None)
    _sig(L, "vdi_render", [P, P, C.c_int, C.c_int, C.c_int, C.c_int, P, C.c_int, P])
    _sig(L, "vdi_render_ex", [P, P, C.c_int, C.c_int, C.c_int, C.c_int, P, C.c_int, P, P])
    _sig(L, "vdi_search_first", [P, C.c_int, C.c_int, P, P, P, P, P, C.c_int, P])
    _sig(L, "vdi_generate", [P, P, P, P, P, C.POINTER(P)])
    _sig(L, "vdi_dvr", [P, P, P, P, C.c_int, C.c_int, C.c_double, C.c_double, P, C.c_int, P])
    _sig(L, "vdi_render_scaled", [P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, C.c_int, P])
    _sig(L, "vdi_pi_create", [P, C.POINTER(P)])
    _sig(L, "vdi_pi_current", [P, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int)])
    _sig(L, "vdi_pi_update", [P, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int)])
    _sig(L, "vdi_pi_destroy", [P], None)
    _sig(L, "vdi_image_quality", [P, P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), P])
    _sig(L, "vdi_touch_bitmap", [P, P, C.c_int, C.c_int, P, C.c_size_t, P])
    _sig(L, "vdi_render_batch", [P, P, C.c_int, P, P])
    _sig(L, "vdi_autotune_batch", [P, P, C.c_int, P, P, P])
    _sig(L, "vdi_server_create", [P, P, C.POINTER(P)])
    _sig(L, "vdi_server_set_vdi", [P, C.c_int, P, P])
    _sig(L, "vdi_server_generate", [P, C.c_int, P, P, P, P])
    _sig(L, "vdi_server_submit", [P, P, C.POINTER(C.c_uint64)])
    _sig(L, "vdi_server_wait", [P, C.c_uint64, C.c_double, P])
    _sig(L, "vdi_server_poll", [P, C.c_uint64, P])
    _sig(L, "vdi_server_release", [P, C.c_uint64])
    _sig(L, "vdi_server_read", [P, C.c_uint64, P, C.c_size_t, C.c_int, P])
    _sig(L, "vdi_render_preview_static", [P, P, C.c_int, C.c_int, C.c_int, C.c_int, P, C.c_int, P])
    _sig(L, "vdi_server_stats", [P, P])
    _sig(L, "vdi_server_destroy", [P], None)
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise VdiError(rc, load().vdi_last_error_message().decode(errors="replace"))


def _dptr(x):
    """Device pointer of a torch CUDA tensor (or an int pointer / None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(type(x))


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _mat(m):
    m = np.asarray(m, np.float64)
    if m.shape == (4, 4):
        m = np.ascontiguousarray(m.T).reshape(16)
    return (C.c_double * 16)(*m.tolist())


def camera(view, proj) -> VdiCamera:
    """VdiCamera from (4,4) row-major matrices or column-major [16] arrays."""
    c = VdiCamera()
    c.view, c.proj = _mat(view), _mat(proj)
    return c


def desc(w, h, n_s, view_o, proj_o, bbox_min, bbox_max, length_unit, colour_fmt=VDI_F32, grid_tile=0,
         grid_nz=0) -> VdiDesc:
    d = VdiDesc()
    d.w, d.h, d.n_s = int(w), int(h), int(n_s)
    d.orig = camera(view_o, proj_o)
    d.bbox_min = (C.c_double * 3)(*map(float, bbox_min))
    d.bbox_max = (C.c_double * 3)(*map(float, bbox_max))
    d.length_unit = float(length_unit)
    d.colour_fmt, d.grid_tile, d.grid_nz = int(colour_fmt), int(grid_tile), int(grid_nz)
    return d


def vdi_ctx_create(device: int = 0):
    out = P()
    _check(load().vdi_ctx_create(int(device), C.byref(out)))
    return out


def vdi_ctx_destroy(ctx):
    load().vdi_ctx_destroy(ctx)


def vdi_layout_bytes(d: VdiDesc) -> VdiLayout:
    out = VdiLayout()
    _check(load().vdi_layout_bytes(C.byref(d), C.byref(out)))
    return out


def vdi_create(ctx, d: VdiDesc, rgba, depth, counts=None, stream=None):
    """rgba/depth/counts: numpy (host) or torch CUDA tensors (device)."""
    if isinstance(rgba, np.ndarray):
        rgba = np.ascontiguousarray(rgba, np.float32)
        depth = np.ascontiguousarray(depth, np.float32)
        if counts is not None:
            counts = np.ascontiguousarray(counts, np.int32)
        ptrs = [rgba.ctypes.data, depth.ctypes.data, None if counts is None else counts.ctypes.data]
        kind = VDI_MEM_HOST
    else:
        ptrs = [_dptr(rgba), _dptr(depth), _dptr(counts)]
        kind = VDI_MEM_DEVICE
    out = P()
    _check(load().vdi_create(ctx, C.byref(d), ptrs[0], ptrs[1], ptrs[2], kind, _stream(stream), C.byref(out)))
    return out


def vdi_stats(vdi, stream=None) -> VdiStats:
    """Bytes by array, grid shape and the last counted frame's totals (synchronises ``stream``)."""
    out = VdiStats()
    _check(load().vdi_stats(vdi, C.byref(out), _stream(stream)))
    return out


def vdi_get_layout(vdi) -> VdiLayout:
    out = VdiLayout()
    _check(load().vdi_get_layout(vdi, C.byref(out)))
    return out


def vdi_download(vdi, w, h, n_s, stream=None):
    """Returns host (rgba[h,w,n_s,4], depth[h,w,n_s,2], counts[h,w], grid[nz,gh,gw])."""
    L = vdi_get_layout(vdi)
    rgba = np.zeros((h, w, n_s, 4), np.float32)
    depth = np.zeros((h, w, n_s, 2), np.float32)
    counts = np.zeros((h, w), np.int32)
    grid = np.zeros((L.grid_nz, L.grid_h, L.grid_w), np.uint32)
    _check(load().vdi_download(vdi, rgba.ctypes.data, depth.ctypes.data, counts.ctypes.data, grid.ctypes.data,
                               _stream(stream)))
    return rgba, depth, counts, grid


def vdi_destroy(vdi):
    load().vdi_destroy(vdi)


def vdi_render(vdi, cam: VdiCamera, W, H, d_i, d_r, out, out_fmt=VDI_F32, stream=None):
    _check(load().vdi_render(vdi, C.byref(cam), int(W), int(H), int(d_i), int(d_r), _dptr(out), int(out_fmt),
                             _stream(stream)))


def vdi_render_preview_static(vdi, cam: VdiCamera, W, H, d_i, d_r, out, out_fmt=VDI_F32, stream=None):
    """vdi_render without device allocation (low-resolution preview image in a static library buffer)."""
    _check(load().vdi_render_preview_static(vdi, C.byref(cam), int(W), int(H), int(d_i), int(d_r), _dptr(out),
                                            int(out_fmt), _stream(stream)))


def vdi_render_ex(vdi, cam: VdiCamera, W, H, d_i, d_r, out, out_fmt=VDI_F32, search=VDI_SEARCH_ALG2,
                  no_ert=False, ray_lists=None, ray_segs=None, warp_shape=-1, ess=False, blocks=False,
                  record_stats=False, stream=None):
    o = VdiRenderOpts()
    o.search, o.no_ert, o.warp_shape, o.ess = int(search), int(bool(no_ert)), int(warp_shape), int(bool(ess))
    o.blocks, o.record_stats = int(bool(blocks)), int(bool(record_stats))
    o.ray_lists, o.ray_segs = _dptr(ray_lists), _dptr(ray_segs)
    _check(load().vdi_render_ex(vdi, C.byref(cam), int(W), int(H), int(d_i), int(d_r), _dptr(out),
                                int(out_fmt), C.byref(o), _stream(stream)))


def vdi_search_first(vdi, list_index, search, d_entry, d_exit, seed, increasing, result, stream=None):
    n = int(d_entry.numel())
    _check(load().vdi_search_first(vdi, int(list_index), int(search), _dptr(d_entry), _dptr(d_exit), _dptr(seed),
                                   _dptr(increasing), _dptr(result), n, _stream(stream)))


_VOL_DTYPE = {"uint8": 0, "uint16": 1, "float32": 2}


def vdi_generate(ctx, volume, bbox_min, bbox_max, knots, cam_o: VdiCamera, w, h, n_s, tau, step, length_unit,
                 colour_fmt=VDI_F32, grid_tile=0, grid_nz=0, stream=None, adaptive=False, tau_out=None):
    """volume: torch CUDA tensor [nz, ny, nx] of uint8/uint16/float32; knots: (n, 5) array.
    adaptive: per-ray gamma (Algorithm 3) instead of tau; tau_out: optional float32 CUDA
    tensor [h, w] that receives each list's gamma."""
    vol = VdiVolume()
    vol.nz, vol.ny, vol.nx = (int(x) for x in volume.shape)
    vol.dtype = _VOL_DTYPE[str(volume.dtype).replace("torch.", "")]
    vol.data = _dptr(volume)
    vol.bbox_min = (C.c_double * 3)(*map(float, bbox_min))
    vol.bbox_max = (C.c_double * 3)(*map(float, bbox_max))
    kn = np.ascontiguousarray(knots, np.float32)
    tf = VdiTf()
    tf.n_knots, tf.knots = len(kn), kn.ctypes.data
    p = VdiGenParams()
    p.w, p.h, p.n_s, p.orig = int(w), int(h), int(n_s), cam_o
    p.tau, p.step, p.length_unit = float(tau), float(step), float(length_unit)
    p.colour_fmt, p.grid_tile, p.grid_nz = int(colour_fmt), int(grid_tile), int(grid_nz)
    p.adaptive = 1 if adaptive else 0
    if tau_out is not None:
        assert str(tau_out.dtype) == "torch.float32" and tau_out.numel() >= int(w) * int(h)
        p.tau_out = _dptr(tau_out)
    out = P()
    _check(load().vdi_generate(ctx, C.byref(vol), C.byref(tf), C.byref(p), _stream(stream), C.byref(out)))
    return out


def _volume_tf(volume, bbox_min, bbox_max, knots):
    vol = VdiVolume()
    vol.nz, vol.ny, vol.nx = (int(x) for x in volume.shape)
    vol.dtype = _VOL_DTYPE[str(volume.dtype).replace("torch.", "")]
    vol.data = _dptr(volume)
    vol.bbox_min = (C.c_double * 3)(*map(float, bbox_min))
    vol.bbox_max = (C.c_double * 3)(*map(float, bbox_max))
    kn = np.ascontiguousarray(knots, np.float32)
    tf = VdiTf()
    tf.n_knots, tf.knots = len(kn), kn.ctypes.data
    return vol, tf, kn


def vdi_dvr(ctx, volume, bbox_min, bbox_max, knots, view: VdiCamera, W, H, step, length_unit, out,
            out_fmt=VDI_F32, stream=None):
    """Direct volume rendering (ground truth) into ``out`` (CUDA tensor [H, W, 4] of out_fmt)."""
    vol, tf, kn = _volume_tf(volume, bbox_min, bbox_max, knots)
    _check(load().vdi_dvr(ctx, C.byref(vol), C.byref(tf), C.byref(view), int(W), int(H), float(step),
                          float(length_unit), _dptr(out), int(out_fmt), _stream(stream)))
    del kn


def vdi_image_quality(a, b, fmt=VDI_F32, stream=None):
    """(SSIM, PSNR) of image ``a`` against reference ``b`` (CUDA tensors [H, W, 4] of fmt)."""
    H, W = int(a.shape[0]), int(a.shape[1])
    assert tuple(b.shape[:2]) == (H, W)
    ssim, psnr = C.c_double(), C.c_double()
    _check(load().vdi_image_quality(_dptr(a), _dptr(b), W, H, int(fmt), C.byref(ssim), C.byref(psnr),
                                    _stream(stream)))
    return ssim.value, psnr.value


def vdi_render_scaled(vdi, view: VdiCamera, W, H, Wr, Hr, d_r, out, out_fmt=VDI_F32, stream=None):
    """Render Wr x Hr rays and upsample bilinearly into ``out`` (CUDA tensor [H, W, 4])."""
    _check(load().vdi_render_scaled(vdi, C.byref(view), int(W), int(H), int(Wr), int(Hr), int(d_r), _dptr(out),
                                    int(out_fmt), _stream(stream)))


class VdiPiConfig(C.Structure):
    _fields_ = [("target_ms", C.c_double), ("kp", C.c_double), ("ki", C.c_double), ("scale_min", C.c_double),
                ("scale_max", C.c_double), ("scale_start", C.c_double), ("W", C.c_int), ("H", C.c_int)]


class PiController:
    """The preview-rate PI controller (vdi_pi_*): ``update(frame_ms)`` returns
    (scale, Wr, Hr) for the next frame."""

    def __init__(self, target_ms, W, H, kp=0.1, ki=0.3, scale_min=0.1, scale_max=1.0, scale_start=1.0):
        cfg = VdiPiConfig(float(target_ms), float(kp), float(ki), float(scale_min), float(scale_max),
                          float(scale_start), int(W), int(H))
        self._p = P()
        _check(load().vdi_pi_create(C.byref(cfg), C.byref(self._p)))

    def current(self):
        s, w, h = C.c_double(), C.c_int(), C.c_int()
        _check(load().vdi_pi_current(self._p, C.byref(s), C.byref(w), C.byref(h)))
        return s.value, w.value, h.value

    def update(self, frame_ms):
        s, w, h = C.c_double(), C.c_int(), C.c_int()
        _check(load().vdi_pi_update(self._p, float(frame_ms), C.byref(s), C.byref(w), C.byref(h)))
        return s.value, w.value, h.value

    def __del__(self):
        if getattr(self, "_p", None):
            load().vdi_pi_destroy(self._p)
            self._p = None


def vdi_touch_bitmap(vdi, cam: VdiCamera, W, H, bitmap, stream=None):
    """bitmap: zeroed int32 CUDA tensor of at least the length touched_bytes() allocates (see vdi.h)."""
    _check(load().vdi_touch_bitmap(vdi, C.byref(cam), int(W), int(H), _dptr(bitmap), int(bitmap.numel()),
                                   _stream(stream)))


def touched_bytes(vdi, cam: VdiCamera, W, H, stream=None) -> int:
    """Unique VDI bytes an exact render of this view reads (popcount of the touch bitmap x 4)."""
    import torch

    L = vdi_get_layout(vdi)
    grid_words = (L.grid_w * L.grid_h * L.grid_nz + 3) // 4 * 4
    words = ((L.depth_bytes + L.colour_bytes) // 4 + grid_words + L.list_bytes // 4 + 31) // 32
    bm = torch.zeros(words, dtype=torch.int32, device="cuda")
    vdi_touch_bitmap(vdi, cam, W, H, bm, stream)
    torch.cuda.synchronize()
    b = bm.cpu().numpy().view(np.uint8)
    return int(np.unpackbits(b).sum()) * 4


def request(vdi, cam: VdiCamera, W, H, d_i, d_r, out, out_fmt=VDI_F32, Wr=0, Hr=0) -> VdiRequest:
    r = VdiRequest()
    r.vdi, r.view, r.W, r.H, r.d_i, r.d_r = vdi, cam, int(W), int(H), int(d_i), int(d_r)
    r.out, r.out_fmt = _dptr(out), int(out_fmt)
    r.Wr, r.Hr = int(Wr), int(Hr)
    return r


def _req_array(reqs):
    arr = (VdiRequest * len(reqs))()
    for i, r in enumerate(reqs):
        arr[i] = r
    return arr


def vdi_render_batch(ctx, reqs, warp_shape=-1, blocks_per_sm=0, use_graph=True, stream=None):
    o = VdiBatchOpts()
    o.warp_shape, o.blocks_per_sm, o.use_graph = int(warp_shape), int(blocks_per_sm), int(bool(use_graph))
    arr = _req_array(reqs)
    _check(load().vdi_render_batch(ctx, arr, len(reqs), C.byref(o), _stream(stream)))


def vdi_autotune_batch(ctx, reqs, stream=None):
    """Returns (VdiBatchOpts of the fastest configuration, milliseconds per batch)."""
    best = VdiBatchOpts()
    ms = C.c_float()
    arr = _req_array(reqs)
    _check(load().vdi_autotune_batch(ctx, arr, len(reqs), _stream(stream), C.byref(best), C.byref(ms)))
    return best, ms.value


def vdi_server_create(ctx, budget_bytes, max_batch=32, max_inflight=2, n_slots=8, wait_timeout_s=10.0):
    c = VdiServerConfig()
    c.budget_bytes, c.max_batch, c.max_inflight = int(budget_bytes), int(max_batch), int(max_inflight)
    c.n_slots, c.wait_timeout_s = int(n_slots), float(wait_timeout_s)
    out = P()
    _check(load().vdi_server_create(ctx, C.byref(c), C.byref(out)))
    return out


def vdi_server_set_vdi(server, slot, vdi, ready_stream=None):
    """Install or replace the VDI of a slot; the server takes ownership of `vdi`
    (on VDI_ERR_OOM the caller keeps it)."""
    _check(load().vdi_server_set_vdi(server, int(slot), vdi, _stream(ready_stream)))


def vdi_server_generate(server, slot, volume, bbox_min, bbox_max, knots, cam_o: VdiCamera, w, h, n_s, tau, step,
                        length_unit, colour_fmt=VDI_F32, grid_tile=0, grid_nz=0, stream=None, adaptive=False):
    """vdi_generate into a slot of the server, its bytes charged to the budget first."""
    vol, tf, kn = _volume_tf(volume, bbox_min, bbox_max, knots)
    p = VdiGenParams()
    p.w, p.h, p.n_s, p.orig = int(w), int(h), int(n_s), cam_o
    p.tau, p.step, p.length_unit = float(tau), float(step), float(length_unit)
    p.colour_fmt, p.grid_tile, p.grid_nz = int(colour_fmt), int(grid_tile), int(grid_nz)
    p.adaptive = 1 if adaptive else 0
    _check(load().vdi_server_generate(server, int(slot), C.byref(vol), C.byref(tf), C.byref(p), _stream(stream)))
    del kn


def view_request(slot, cam: VdiCamera, W, H, d_i=1, d_r=1, out_fmt=VDI_F16, Wr=0, Hr=0) -> VdiViewRequest:
    r = VdiViewRequest()
    r.slot, r.view, r.W, r.H, r.d_i, r.d_r, r.out_fmt = int(slot), cam, int(W), int(H), int(d_i), int(d_r), \
        int(out_fmt)
    r.Wr, r.Hr = int(Wr), int(Hr)
    return r


def vdi_server_submit(server, req: VdiViewRequest) -> int:
    t = C.c_uint64()
    _check(load().vdi_server_submit(server, C.byref(req), C.byref(t)))
    return t.value


def vdi_server_wait(server, ticket, timeout_s=10.0) -> VdiTicketInfo:
    info = VdiTicketInfo()
    _check(load().vdi_server_wait(server, C.c_uint64(ticket), float(timeout_s), C.byref(info)))
    return info


def vdi_server_poll(server, ticket) -> VdiTicketInfo:
    info = VdiTicketInfo()
    _check(load().vdi_server_poll(server, C.c_uint64(ticket), C.byref(info)))
    return info


def vdi_server_read(server, ticket, dst, stream=None):
    """Copy a finished result into `dst` (numpy array -> host copy, CUDA tensor -> device copy)."""
    if isinstance(dst, np.ndarray):
        ptr, kind, n = dst.ctypes.data, VDI_MEM_HOST, dst.nbytes
    else:
        ptr, kind, n = _dptr(dst), VDI_MEM_DEVICE, dst.numel() * dst.element_size()
    _check(load().vdi_server_read(server, C.c_uint64(ticket), ptr, n, kind, _stream(stream)))


def vdi_server_release(server, ticket):
    _check(load().vdi_server_release(server, C.c_uint64(ticket)))


def vdi_server_stats(server) -> VdiServerCounters:
    st = VdiServerCounters()
    _check(load().vdi_server_stats(server, C.byref(st)))
    return st


def vdi_server_destroy(server):
    load().vdi_server_destroy(server)
