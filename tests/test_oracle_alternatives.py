"""The oracle's other limits of a flagged ray (used by the GPU parity tests to
check flagged rays instead of dropping them).

* The D_R preview with no tie decision flipped is the plain preview, bit for
  bit; flipping decisions changes only rays that met a tie.
* The exact render through explicit NDC points at the pixel centres is the
  plain render; a ray that runs along a list boundary has two limits, one on
  each side, and the pixel centre moved by a thousandth of a pixel reaches
  both.
"""
import numpy as np

import vdi_synth as S
from helpers import NUDGE, pixel_ndc, random_case


def test_preview_alt_plain_equals_preview_and_flips_only_tied_rays(orc):
    case = random_case(64, 48, 6, seed=21, u=0.15, alpha_range=(0.05, 0.6))
    sc = case.oracle_scene(orc)
    T, nz, W, H = 8, 10, 75, 53
    grid = orc.grid_counts(sc, T, nz)
    cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=20.0, el_deg=10.0, zoom=1.1)
    for d_r in (2, 4):
        ref, fl = orc.render_preview(sc, cn.view, cn.proj, W, H, d_r, T, nz, grid=grid)
        pix = np.arange(W * H, dtype=np.int32)
        plain, nt = orc.render_preview_alt(sc, cn.view, cn.proj, W, H, d_r, T, nz, grid, pix, 0)
        assert np.array_equal(plain, ref)
        assert np.all(nt[fl == 0] == 0) and np.all(nt <= 64)
        flipped, nt2 = orc.render_preview_alt(sc, cn.view, cn.proj, W, H, d_r, T, nz, grid, pix, 0xFFFFFFFF)
        assert np.array_equal(flipped[nt == 0], ref[nt == 0])
        moved = np.abs(flipped - ref).max(axis=1) > 1e-9
        assert moved.any() and np.all(nt[moved] > 0)


def test_exact_ndc_equals_render_and_boundary_rays_have_two_limits(orc):
    bmin, bmax = np.zeros(3), np.ones(3)
    vdi = S.random_vdi(37, 23, 5, seed=11, alpha_range=(0.05, 0.8))
    cam_o = S.orbit_camera(bmin, bmax, 37 / 23, az_deg=0.0, el_deg=15.0, zoom=1.8)
    sc = orc.Scene(vdi, cam_o.view, cam_o.proj, bmin, bmax, 0.15)
    W, H = 70, 45
    cn = S.orbit_camera(bmin, bmax, W / H, az_deg=0.0, el_deg=15.0)  # V_O's direction: rays along list edges
    ref, nl, ns, fl = orc.render_exact(sc, cn.view, cn.proj, W, H)
    x, y = pixel_ndc(np.arange(W * H), W, H)
    again, nl2, ns2, fl2 = orc.render_exact_ndc(sc, cn.view, cn.proj, np.stack([x, y], 1))
    assert np.array_equal(again, ref) and np.array_equal(nl2, nl) and np.array_equal(fl2, fl)
    idx = np.nonzero(fl)[0]
    assert len(idx) > 0
    sides = []
    for dx in (1, -1):
        for dy in (1, -1):
            xy = np.stack([x[idx] + dx * NUDGE * 2 / W, y[idx] + dy * NUDGE * 2 / H], 1)
            sides.append(orc.render_exact_ndc(sc, cn.view, cn.proj, xy)[0])
    sides = np.stack(sides)
    spread = (sides.max(axis=0) - sides.min(axis=0)).max(axis=1)
    assert (spread > 1e-3).any()  # both sides of a list boundary, visibly different
    # away from boundaries the nudge moves the result continuously and only a little
    unflagged = np.nonzero(fl == 0)[0][:200]
    xy = np.stack([x[unflagged] + NUDGE * 2 / W, y[unflagged] + NUDGE * 2 / H], 1)
    assert np.abs(orc.render_exact_ndc(sc, cn.view, cn.proj, xy)[0] - ref[unflagged]).max() < 1e-3
