"""vdi_render_preview_static: the same render as vdi_render without any device
allocation, for callers that cannot allocate while rendering (all device
memory already handed to resident VDIs, a frame loop that must not wait on
an allocator, programs that allocate only at start-up).  Its low-resolution
preview image lives in a fixed static buffer of the library.

Collected last on purpose: run alone in a fresh process or after every other
test, two calls in a row must each match vdi_render of the same view."""
import numpy as np
import pytest

import vdi_synth as S
from helpers import check_tolerance, random_case

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
        check_tolerance(got, ref, 0, what=f"static preview {W}x{H} d_i={d_i} d_r={d_r}")


def test_oversized_preview_is_rejected(setup):
    V, case, vdi = setup
    cam = S.orbit_camera(case.bmin, case.bmax, 1.0)
    out = torch.zeros((2048, 2048, 4), dtype=torch.float16, device="cuda")
    with pytest.raises(V.VdiError) as e:  # 1024 x 1024 low-resolution pixels > 524288
        V.vdi_render_preview_static(vdi, V.camera(cam.view, cam.proj), 2048, 2048, 2, 1, out, V.VDI_F16)
    assert e.value.status == 1
