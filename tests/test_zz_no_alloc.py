"""vdi_render_preview_static: the same render as vdi_render without any device
allocation, for callers that cannot allocate while rendering (all device
memory already handed to resident VDIs, a frame loop that must not wait on
an allocator, programs that allocate only at start-up).  Its low-resolution
preview image lives in a fixed static buffer of the library.

Collected last on purpose: run alone in a fresh process or after every other
test, two calls in a row must each equal vdi_render of the same view bit for
bit, and a call must not raise the high-water mark of the device's
stream-ordered memory pool (where vdi_render takes its preview scratch)."""
import ctypes

import numpy as np
import pytest

import vdi_synth as S
from helpers import random_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    import paper_2206_08660_gb300 as V

    V.load()
    ctx = V.vdi_ctx_create(0)
    case = random_case(96, 54, 6, seed=12, fill=0.8)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 1), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    yield V, case, vdi
    V.vdi_destroy(vdi)
    V.vdi_ctx_destroy(ctx)


def render(V, fn, vdi, cam, W, H, d_i, d_r):
    out = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    fn(vdi, V.camera(cam.view, cam.proj), W, H, d_i, d_r, out, V.VDI_F32)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_two_calls_in_a_row_match_vdi_render(setup):
    V, case, vdi = setup
    calls = [(25.0, 1920, 1080, 2, 1), (-40.0, 1280, 720, 2, 2)]  # the first fills the whole buffer's capacity
    for az, W, H, d_i, d_r in calls:
        cam = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=az, el_deg=20.0)
        got = render(V, V.vdi_render_preview_static, vdi, cam, W, H, d_i, d_r)
        ref = render(V, V.vdi_render, vdi, cam, W, H, d_i, d_r)
        assert ref[..., 3].max() > 0.2
        assert np.array_equal(got, ref), f"static preview {W}x{H} d_i={d_i} d_r={d_r}"


class _Pool:
    """High-water mark of the device's current stream-ordered memory pool, read
    through the CUDA runtime the library itself links (libcudart.so.13)."""

    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8  # cudaMemPoolAttr

    def __init__(self, device=0):
        self.rt = ctypes.CDLL("libcudart.so.13")
        self.pool = ctypes.c_void_p()
        assert self.rt.cudaDeviceGetMemPool(ctypes.byref(self.pool), device) == 0

    def attr(self, a):
        v = ctypes.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, a, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)  # the high-water mark can only be reset (to the current use)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0
        return self.attr(self.USED_MEM_HIGH)


def test_no_device_allocation(setup):
    """The static-buffer preview leaves the pool's high-water mark where it was;
    vdi_render of the same preview raises it by its scratch image."""
    V, case, vdi = setup
    W, H, d_i, d_r = 1280, 720, 2, 1
    cam = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=15.0, el_deg=20.0)
    out = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    args = (vdi, V.camera(cam.view, cam.proj), W, H, d_i, d_r, out, V.VDI_F32)
    V.vdi_render_preview_static(*args)  # first call on the device: the buffer's address is looked up
    torch.cuda.synchronize()
    pool = _Pool(0)
    base = pool.reset_high()
    V.vdi_render_preview_static(*args)
    torch.cuda.synchronize()
    assert pool.attr(pool.USED_MEM_HIGH) == base
    base = pool.reset_high()
    V.vdi_render(*args)
    torch.cuda.synchronize()
    scratch = (-(-W // d_i)) * (-(-H // d_i)) * 16
    assert pool.attr(pool.USED_MEM_HIGH) >= base + scratch


def test_oversized_preview_is_rejected(setup):
    V, case, vdi = setup
    cam = S.orbit_camera(case.bmin, case.bmax, 1.0)
    out = torch.zeros((2048, 2048, 4), dtype=torch.float16, device="cuda")
    with pytest.raises(V.VdiError) as e:  # 1024 x 1024 low-resolution pixels > 524288
        V.vdi_render_preview_static(vdi, V.camera(cam.view, cam.proj), 2048, 2048, 2, 1, out, V.VDI_F16)
    assert e.value.status == 1
