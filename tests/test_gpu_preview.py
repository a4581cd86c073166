"""GPU parity of the subsampled previews (Section 4.4) against the FP64 oracle.

D_R: samples per grid cell proportional to the cell's supersegment count and
the ray's length in it, thinned by D_R.  Every ray is compared: a ray the
oracle flags (a sample within rounding distance of a list or supersegment
boundary, or a sample count at a rounding boundary) may match any of the
oracle's limits with those tie decisions flipped.
D_I: fewer rays, then bilinear upsampling; the low-resolution image (checked
ray by ray as above) is upsampled by the oracle and compared everywhere.
"""
import numpy as np
import pytest

import vdi_synth as S
from helpers import (check_tolerance, check_with_alternatives, closest_alternative, preview_alternatives,
                     random_case)

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


def render(V, vdi, cam, W, H, d_i, d_r):
    out = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    V.vdi_render(vdi, V.camera(cam.view, cam.proj), W, H, d_i, d_r, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(-1, 4)


T, NZ = 8, 10


@pytest.fixture(scope="module")
def scene(V, ctx, orc):
    case = random_case(64, 48, 6, seed=21, u=0.15, alpha_range=(0.05, 0.6))
    vdi = {fmt: V.vdi_create(ctx, case.gpu_desc(V, fmt, T, NZ), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
           for fmt in (0, 1)}
    sc = case.oracle_scene(orc)
    yield case, sc, vdi, orc.grid_counts(sc, T, NZ)
    for v in vdi.values():
        V.vdi_destroy(v)


def lowres_reference(V, orc, sc, grid, vdi, cn, Wr, Hr, d_r, fmt=0):
    """The oracle's low-resolution image, with each flagged ray set to its limit
    nearest the GPU's (all limits checked against the GPU within tolerance)."""
    if d_r == 1:
        return orc.render_exact(sc, cn.view, cn.proj, Wr, Hr)[0]
    lo, fl = orc.render_preview(sc, cn.view, cn.proj, Wr, Hr, d_r, T, NZ, grid=grid)
    idx = np.nonzero(fl)[0]
    if len(idx):
        alts = preview_alternatives(orc, sc, cn, Wr, Hr, d_r, T, NZ, grid, idx)
        got_lo = render(V, vdi, cn, Wr, Hr, 1, d_r)
        check_with_alternatives(got_lo, lo, fmt, fl, alts, what=f"low-res {Wr}x{Hr} D_R={d_r}")
        lo = lo.copy()
        lo[idx] = closest_alternative(got_lo[idx], alts)
    return lo


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("d_r", [2, 4])
@pytest.mark.parametrize("az,el", [(20.0, 10.0), (-45.0, 30.0), (160.0, 0.0)])
def test_ray_subsampled_preview(V, orc, scene, fmt, d_r, az, el):
    case, sc, vdi, grid = scene
    W, H = 75, 53
    cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=az, el_deg=el, zoom=1.1)
    ref, fl = orc.render_preview(sc, cn.view, cn.proj, W, H, d_r, T, NZ, grid=grid)
    got = render(V, vdi[fmt], cn, W, H, 1, d_r)
    assert ref[:, 3].max() > 0.2
    alts = preview_alternatives(orc, sc, cn, W, H, d_r, T, NZ, grid, np.nonzero(fl)[0])
    frac, _ = check_with_alternatives(got, ref, fmt, fl, alts, what=f"D_R={d_r} view {az},{el}")
    assert frac < 0.2


@pytest.mark.parametrize("d_i,d_r", [(2, 1), (3, 1), (2, 2), (4, 4)])
def test_image_space_preview(V, orc, scene, d_i, d_r):
    case, sc, vdi, grid = scene
    W, H = 90, 61
    Wr, Hr = -(-W // d_i), -(-H // d_i)
    cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=30, el_deg=20)
    ref = orc.upsample(lowres_reference(V, orc, sc, grid, vdi[0], cn, Wr, Hr, d_r), Wr, Hr, W, H)
    got = render(V, vdi[0], cn, W, H, d_i, d_r)
    check_tolerance(got, ref, 0, what=f"D_I={d_i} D_R={d_r}")


@pytest.mark.parametrize("Wr,Hr,d_r", [(45, 31, 1), (37, 61, 1), (90, 61, 1), (52, 35, 2)])
def test_fractional_image_scale(V, orc, scene, Wr, Hr, d_r):
    """vdi_render_scaled: any ray count per axis (the paper's fractional D_I),
    upsampled to the display; against the oracle's render at Wr x Hr and its
    bilinear upsampling."""
    case, sc, vdi, grid = scene
    W, H = 90, 61
    cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=30, el_deg=20)
    ref = orc.upsample(lowres_reference(V, orc, sc, grid, vdi[0], cn, Wr, Hr, d_r), Wr, Hr, W, H)
    out = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    V.vdi_render_scaled(vdi[0], V.camera(cn.view, cn.proj), W, H, Wr, Hr, d_r, out)
    torch.cuda.synchronize()
    check_tolerance(out.cpu().numpy().reshape(-1, 4), ref, 0, what=f"{Wr}x{Hr} D_R={d_r}")


def test_scaled_render_equals_integer_preview(V, scene):
    case, sc, vdi, grid = scene
    W, H = 90, 61
    cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=-20, el_deg=10)
    for d_i in (1, 2, 3):
        a = render(V, vdi[1], cn, W, H, d_i, 1)
        out = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
        V.vdi_render_scaled(vdi[1], V.camera(cn.view, cn.proj), W, H, -(-W // d_i), -(-H // d_i), 1, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().reshape(-1, 4), a)
