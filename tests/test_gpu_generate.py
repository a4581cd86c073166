"""GPU vdi_generate (Section 3, Eq. 1) against the oracle, through the C ABI.

* Supersegment counts and FP32 depths are bit-identical to the oracle's FP32
  generation (same IEEE operations, no contraction); colour within FP32 /
  FP16 storage tolerance.
* Check a': the GPU-generated VDI rendered by the GPU at V_O reproduces the
  oracle's FP64 DVR at the same samples (rays whose sample count sits at a
  rounding boundary are excluded).
* End to end on the tiny workload (64^3 Gaussian blobs, 128x128 VDI, N_S = 8,
  tau = 0.02, new view 10 degrees away): GPU generate + render against oracle
  generate + exact render.
* Ray-adaptive gamma (Algorithm 3): per-list gamma, counts and depths
  bit-identical to the oracle's FP32 generation.
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


VOLUMES = {
    "blobs_f32": lambda: S.blobs_volume(64, seed=0),
    "noise_u16": lambda: S.value_noise_volume(48, octaves=4, seed=3, dtype=np.uint16),
    "layer_u8": lambda: S.mixing_layer_volume(64, modes=8, seed=1, dtype=np.uint8),
}
TF = {"blobs_f32": "dense", "noise_u16": "sparse", "layer_u8": "interface"}


def gen_both(V, ctx, orc, name, w, h, ns, tau, fmt, step_scale=1.0, el=15.0, az=0.0):
    vol = VOLUMES[name]()
    bmin, bmax = S.bbox_for_dims(vol.shape)
    u = 1.0 / max(vol.shape)
    step = u * step_scale
    cam = S.orbit_camera(bmin, bmax, w / h, el_deg=el, az_deg=az)
    kn = S.tf_knots(TF[name])
    vdi = V.vdi_generate(ctx, torch.from_numpy(vol).cuda(), bmin, bmax, kn, V.camera(cam.view, cam.proj), w, h, ns,
                         tau, step, u, fmt)
    ref = orc.generate(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, w, h, ns, tau, step, u, fp32=True)
    return vol, bmin, bmax, u, step, cam, kn, vdi, ref


@pytest.mark.parametrize("name", list(VOLUMES))
@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("tau,ns", [(0.02, 8), (0.0, 5), (0.005, 20)])
def test_counts_and_depths_bit_exact(V, ctx, orc, name, fmt, tau, ns):
    w, h = 72, 40
    vol, bmin, bmax, u, step, cam, kn, vdi, (rgba, depth, counts) = gen_both(V, ctx, orc, name, w, h, ns, tau, fmt)
    try:
        g_rgba, g_depth, g_counts, g_grid = V.vdi_download(vdi, w, h, ns)
        assert counts.sum() > w * h // 4
        assert np.array_equal(g_counts, counts)
        valid = np.arange(ns)[None, None, :] < counts[:, :, None]
        assert np.array_equal(g_depth[valid].view(np.uint32), depth[valid].view(np.uint32))
        tol = 2e-5 if fmt == 0 else 3e-3
        assert np.abs(g_rgba[valid] - rgba[valid]).max() < tol
        sc = orc.Scene(S.VdiArrays(w, h, ns, rgba, depth, counts), cam.view, cam.proj, bmin, bmax, u)
        assert np.array_equal(g_grid, orc.grid_counts(sc, 8, 20))
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("name", list(VOLUMES))
@pytest.mark.parametrize("fmt", [0, 1])
def test_render_at_original_view_equals_dvr(V, ctx, orc, name, fmt):
    """Check a': independent of the segmentation, rendering at V_O reproduces DVR."""
    w, h, ns = 96, 64, 6
    vol, bmin, bmax, u, step, cam, kn, vdi, _ = gen_both(V, ctx, orc, name, w, h, ns, 0.01, fmt)
    try:
        out = torch.zeros((h, w, 4), device="cuda")
        V.vdi_render(vdi, V.camera(cam.view, cam.proj), w, h, 1, 1, out)
        torch.cuda.synchronize()
        dvr, fl = orc.dvr(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, w, h, step, u, with_flags=True)
        assert dvr[:, 3].max() > 0.3
        # a ray whose sample count floor(L / step) sits at a rounding boundary has two
        # valid values; the VDI took the FP32 decision, which the oracle's FP32 DVR repeats
        dvr32 = orc.dvr(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, w, h, step, u, fp32=True)
        check_with_alternatives(out.cpu().numpy(), dvr, fmt, fl, dvr32[fl != 0][None], what=f"a' {name}")
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("fmt", [0, 1])
def test_tiny_workload_end_to_end(V, ctx, orc, fmt):
    """64^3 blobs, VDI 128x128, N_S = 8, tau = 0.02, view rotated 10 degrees."""
    w = h = 128
    vol, bmin, bmax, u, step, cam, kn, vdi, (rgba, depth, counts) = gen_both(V, ctx, orc, "blobs_f32", w, h, 8, 0.02,
                                                                             fmt)
    try:
        sc = orc.Scene(S.VdiArrays(w, h, 8, rgba, depth, counts), cam.view, cam.proj, bmin, bmax, u)
        for az in (10.0, -10.0, 35.0):
            cn = S.orbit_camera(bmin, bmax, 1.0, az_deg=az, el_deg=15.0)
            ref = orc.render_exact(sc, cn.view, cn.proj, w, h)[0]
            out = torch.zeros((h, w, 4), device="cuda")
            V.vdi_render(vdi, V.camera(cn.view, cn.proj), w, h, 1, 1, out)
            torch.cuda.synchronize()
            assert ref[:, 3].max() > 0.5
            check_tolerance(out.cpu().numpy(), ref, fmt, what=f"tiny az={az}")
    finally:
        V.vdi_destroy(vdi)


def test_generate_rejects_bad_input(V, ctx):
    vol = torch.zeros((4, 4, 4), device="cuda")
    cam = S.orbit_camera(np.zeros(3), np.ones(3), 1.0)
    kn = S.tf_knots("dense")
    with pytest.raises(V.VdiError):
        V.vdi_generate(ctx, vol, (0, 0, 0), (1, 1, 1), kn[::-1].copy(), V.camera(cam.view, cam.proj), 8, 8, 4, 0.01,
                       0.25, 0.25)
    ortho = S.orbit_camera(np.zeros(3), np.ones(3), 1.0, ortho=True)
    with pytest.raises(V.VdiError) as e:
        V.vdi_generate(ctx, vol, (0, 0, 0), (1, 1, 1), kn, V.camera(ortho.view, ortho.proj), 8, 8, 4, 0.01, 0.25, 0.25)
    assert e.value.status == 7


@pytest.mark.parametrize("name", list(VOLUMES))
@pytest.mark.parametrize("ns", [6, 20])
def test_adaptive_gamma_bit_exact(V, ctx, orc, name, ns):
    """Ray-adaptive gamma (Algorithm 3): every list's gamma, supersegment
    count and FP32 depth equal the oracle's FP32 generation bit for bit, and
    the VDI still renders to DVR at V_O (check a')."""
    w, h, fmt = 64, 40, 1
    vol = VOLUMES[name]()
    bmin, bmax = S.bbox_for_dims(vol.shape)
    u = 1.0 / max(vol.shape)
    cam = S.orbit_camera(bmin, bmax, w / h, el_deg=15.0)
    kn = S.tf_knots(TF[name])
    taus = torch.zeros((h, w), dtype=torch.float32, device="cuda")
    vdi = V.vdi_generate(ctx, torch.from_numpy(vol).cuda(), bmin, bmax, kn, V.camera(cam.view, cam.proj), w, h, ns,
                         0.0, u, u, fmt, adaptive=True, tau_out=taus)
    rgba, depth, counts, r_taus = orc.generate(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, w, h, ns, 0.0, u,
                                               u, fp32=True, adaptive=True, with_tau=True)
    try:
        torch.cuda.synchronize()
        assert np.array_equal(taus.cpu().numpy().view(np.uint32), r_taus.view(np.uint32))
        assert len(np.unique(r_taus)) > 5  # many lists searched
        _, g_depth, g_counts, _ = V.vdi_download(vdi, w, h, ns)
        assert np.array_equal(g_counts, counts) and counts.max() <= ns
        valid = np.arange(ns)[None, None, :] < counts[:, :, None]
        assert np.array_equal(g_depth[valid].view(np.uint32), depth[valid].view(np.uint32))
        out = torch.zeros((h, w, 4), device="cuda")
        V.vdi_render(vdi, V.camera(cam.view, cam.proj), w, h, 1, 1, out)
        torch.cuda.synchronize()
        dvr, fl = orc.dvr(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, w, h, u, u, with_flags=True)
        dvr32 = orc.dvr(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, w, h, u, u, fp32=True)
        check_with_alternatives(out.cpu().numpy(), dvr, fmt, fl, dvr32[fl != 0][None], what=f"adaptive a' {name}")
    finally:
        V.vdi_destroy(vdi)
