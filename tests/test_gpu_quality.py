"""GPU ground truth and image quality (Section 6), through the C ABI.

* vdi_dvr against the oracle's FP64 DVR from new perspective views (rays whose
  sample count sits at a rounding boundary excluded), FP32 and FP16 output.
* vdi_image_quality (SSIM, PSNR) against the oracle's definitions on random
  images of ragged sizes and on real renders.
* The quality study in small: a VDI render from a new view is close to DVR
  from that view (the paper's Fig. 9 measure).
"""
import numpy as np
import pytest

import vdi_synth as S
from helpers import check_tolerance, check_with_alternatives

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    import paper_2206_08660_gb300 as V

    V.load()
    return V


@pytest.fixture(scope="module")
def ctx(V):
    c = V.vdi_ctx_create(0)
    yield c
    V.vdi_ctx_destroy(c)


@pytest.mark.parametrize("name", ["blobs", "noise"])
@pytest.mark.parametrize("fmt", [0, 1])
def test_dvr_matches_oracle(V, ctx, orc, name, fmt):
    vol = S.blobs_volume(48, seed=1) if name == "blobs" else S.value_noise_volume(40, seed=2, dtype=np.uint16)
    bmin, bmax = S.bbox_for_dims(vol.shape)
    kn = S.tf_knots("dense" if name == "blobs" else "sparse")
    u = 1.0 / max(vol.shape)
    vd = torch.from_numpy(vol).cuda()
    for az, step in ((0.0, u), (25.0, 0.7 * u), (160.0, u)):
        W, H = 70, 45  # ragged tiles
        cam = S.orbit_camera(bmin, bmax, W / H, az_deg=az, el_deg=20.0)
        out = torch.zeros((H, W, 4), dtype=torch.float32 if fmt == 0 else torch.float16, device="cuda")
        V.vdi_dvr(ctx, vd, bmin, bmax, kn, V.camera(cam.view, cam.proj), W, H, step, u, out, fmt)
        torch.cuda.synchronize()
        ref, fl = orc.dvr(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, W, H, step, u, with_flags=True)
        assert ref[:, 3].max() > 0.3
        # rays whose sample count sits at a rounding boundary: the GPU decides in FP32,
        # as the oracle's FP32 DVR does
        ref32 = orc.dvr(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, W, H, step, u, fp32=True)
        check_with_alternatives(out.float().cpu().numpy(), ref, fmt, fl, ref32[fl != 0][None],
                                what=f"dvr {name} {az}")


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("W,H", [(7, 7), (101, 37), (64, 64), (333, 190)])
def test_quality_measures_match_oracle(V, fmt, W, H):
    from oracle import quality as Q

    rng = np.random.default_rng(W * 1000 + H)
    a = rng.uniform(0, 1, (H, W, 4)).astype(np.float32)
    b = np.clip(a + rng.normal(0, 0.05, a.shape), 0, 1).astype(np.float32)
    dt = torch.float32 if fmt == 0 else torch.float16
    ta, tb = torch.from_numpy(a).to(dt).cuda(), torch.from_numpy(b).to(dt).cuda()
    ssim, psnr = V.vdi_image_quality(ta, tb, fmt)
    # the oracle on the values the GPU read (FP16 storage rounds them)
    ha, hb = ta.float().cpu().numpy(), tb.float().cpu().numpy()
    assert abs(ssim - Q.ssim(ha, hb)) < 2e-6
    assert abs(psnr - Q.psnr(ha, hb)) < 1e-6
    s2, p2 = V.vdi_image_quality(ta, ta, fmt)
    assert abs(s2 - 1.0) < 1e-6 and p2 == float("inf")


def test_vdi_render_close_to_dvr_from_new_views(V, ctx, orc):
    """The tiny workload: a 128 x 128, N_S = 8 VDI from 64^3 blobs rendered
    from views 0..30 degrees away scores close to DVR from the same views,
    and the score falls as the view moves away from V_O (Fig. 9)."""
    from oracle import quality as Q

    vol = S.blobs_volume(64, seed=0)
    bmin, bmax = S.bbox_for_dims(vol.shape)
    u = 1.0 / 64
    kn = S.tf_knots("dense")
    cam_o = S.orbit_camera(bmin, bmax, 1.0, el_deg=15.0)
    vd = torch.from_numpy(vol).cuda()
    vdi = V.vdi_generate(ctx, vd, bmin, bmax, kn, V.camera(cam_o.view, cam_o.proj), 128, 128, 8, 0.02, u, u, 0)
    try:
        scores = []
        for az in (0.0, 10.0, 30.0):
            cam = S.orbit_camera(bmin, bmax, 1.0, az_deg=az, el_deg=15.0)
            img = torch.zeros((128, 128, 4), device="cuda")
            ref = torch.zeros((128, 128, 4), device="cuda")
            V.vdi_render(vdi, V.camera(cam.view, cam.proj), 128, 128, 1, 1, img)
            V.vdi_dvr(ctx, vd, bmin, bmax, kn, V.camera(cam.view, cam.proj), 128, 128, u, u, ref)
            torch.cuda.synchronize()
            ssim, psnr = V.vdi_image_quality(img, ref)
            assert abs(ssim - Q.ssim(img.cpu().numpy(), ref.cpu().numpy())) < 2e-6
            scores.append((ssim, psnr))
        assert scores[0][0] > 0.99 and scores[0][1] > 40  # at V_O the VDI reproduces DVR
        assert scores[2][0] > 0.8 and scores[2][0] < scores[0][0]
    finally:
        V.vdi_destroy(vdi)
