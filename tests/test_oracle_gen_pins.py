"""Pins of the oracle's VDI generation (Section 3, Eq. 1) and DVR.

* Check a': a VDI stores the exact composite of its supersegments' samples,
  so compositing each list directly at V_O (a routine that shares no code
  with generation) must reproduce DVR at the same samples, whatever the
  sensitivity tau and the budget N_S (including N_S = 1, where one
  supersegment absorbs everything).
* Closed forms on a constant volume, computed here from numpy's matrix
  inverse and a slab test: one supersegment per list spanning floor(L/step)
  samples with opacity 1 - (1 - a)^(K step / u); with tau = 0 every sample
  starts a new supersegment until the budget is used.
"""
import numpy as np
import pytest

import vdi_synth as S


def pixel_rays(cam, w, h):
    inv = np.linalg.inv(cam.proj @ cam.view)
    px, py = np.meshgrid(np.arange(w), np.arange(h))
    x = 2 * (px.ravel() + 0.5) / w - 1
    y = 1 - 2 * (py.ravel() + 0.5) / h
    out = []
    for xi, yi in zip(x, y):
        a = inv @ np.array([xi, yi, -1.0, 1.0])
        b = inv @ np.array([xi, yi, 1.0, 1.0])
        out.append((a[:3] / a[3], b[:3] / b[3]))
    return out


def chord(pn, pf, bmin, bmax):
    d = pf - pn
    t0, t1 = 0.0, 1.0
    for k in range(3):
        if d[k] != 0:
            ta, tb = sorted([(bmin[k] - pn[k]) / d[k], (bmax[k] - pn[k]) / d[k]])
            t0, t1 = max(t0, ta), min(t1, tb)
        elif not (bmin[k] <= pn[k] <= bmax[k]):
            return None
    return (t0, t1, np.linalg.norm(d)) if t0 < t1 else None


@pytest.mark.parametrize("tau", [0.0, 0.005, 0.02, 0.1, 10.0])
@pytest.mark.parametrize("ns", [1, 3, 8])
def test_direct_render_of_generated_vdi_equals_dvr(orc, tau, ns):
    vol = S.blobs_volume(32, seed=2)
    bmin, bmax = S.bbox_for_dims(vol.shape)
    cam = S.orbit_camera(bmin, bmax, 1.0, el_deg=25, az_deg=15)
    V = orc.Volume(vol, bmin, bmax)
    kn = S.tf_knots("dense")
    u = 1 / 32
    for step in (u, 0.7 * u):
        rgba, depth, counts = orc.generate(V, kn, cam.view, cam.proj, 40, 40, ns, tau, step, u)
        assert counts.max() <= ns
        sc = orc.Scene(S.VdiArrays(40, 40, ns, rgba, depth, counts), cam.view, cam.proj, bmin, bmax, u)
        direct = orc.render_direct(sc)
        dvr = orc.dvr(V, kn, cam.view, cam.proj, 40, 40, step, u)
        assert dvr[:, 3].max() > 0.5
        assert np.abs(direct - dvr).max() < 2e-6, (tau, ns, step)


def test_noise_u16_generation_invariants_and_direct_equals_dvr(orc):
    vol = S.value_noise_volume(48, octaves=4, seed=3, dtype=np.uint16)
    bmin, bmax = S.bbox_for_dims(vol.shape)
    cam = S.orbit_camera(bmin, bmax, 1.5, el_deg=10)
    V = orc.Volume(vol, bmin, bmax)
    kn = S.tf_knots("sparse")
    u = 1 / 48
    rgba, depth, counts = orc.generate(V, kn, cam.view, cam.proj, 60, 40, 6, 0.01, u, u)
    valid = np.arange(6)[None, None, :] < counts[:, :, None]
    f, b = depth[..., 0], depth[..., 1]
    assert np.all(f[valid] <= b[valid])
    nxt = valid[:, :, 1:]
    assert np.all(b[:, :, :-1][nxt] <= f[:, :, 1:][nxt])
    assert np.all(np.abs(f[valid]) <= 1) and np.all(np.abs(b[valid]) <= 1)
    assert np.all(rgba[valid][:, :3] <= rgba[valid][:, 3:4])
    assert counts.mean() > 1.0
    sc = orc.Scene(S.VdiArrays(60, 40, 6, rgba, depth, counts), cam.view, cam.proj, bmin, bmax, u)
    assert np.abs(orc.render_direct(sc) - orc.dvr(V, kn, cam.view, cam.proj, 60, 40, u, u)).max() < 2e-6


@pytest.mark.parametrize("tau,ns", [(0.05, 4), (0.0, 4), (0.0, 64)])
def test_constant_volume_closed_form(orc, tau, ns):
    n = 16
    vol = np.full((n, n, n), 0.45, np.float32)
    bmin, bmax = np.zeros(3), np.ones(3)
    cam = S.orbit_camera(bmin, bmax, 1.0, el_deg=20, az_deg=30)
    kn = S.tf_knots("dense")
    # the transfer function at 0.45, by linear interpolation between knots 1 and 2
    s = (0.45 - kn[1, 0]) / (kn[2, 0] - kn[1, 0])
    c = kn[1, 1:].astype(np.float64) + s * (kn[2, 1:] - kn[1, 1:])
    u, step, w, h = 1 / n, 1 / n, 12, 12
    V = orc.Volume(vol, bmin, bmax)
    rgba, depth, counts = orc.generate(V, kn, cam.view, cam.proj, w, h, ns, tau, step, u)
    dvr = orc.dvr(V, kn, cam.view, cam.proj, w, h, step, u)
    M = cam.proj @ cam.view
    hits = 0
    for i, (pn, pf) in enumerate(pixel_rays(cam, w, h)):
        iy, ix = divmod(i, w)
        ch = chord(pn, pf, bmin, bmax)
        if ch is None:
            assert counts[iy, ix] == 0
            continue
        t0, t1, dl = ch
        K = int(np.floor((t1 - t0) * dl / step + 1e-9))
        # stop once transmittance falls to 2^-12
        Kert = int(np.ceil(np.log(2.0 ** -12) / np.log(1 - c[3]) - 1e-9))
        Keff = min(K, Kert)
        if Keff == 0:
            continue
        hits += 1
        a = 1 - (1 - c[3]) ** Keff
        assert np.abs(dvr[i] - np.append(c[:3] * a, a)).max() < 1e-5
        expect_n = 1 if tau > 0 else min(Keff, ns)
        assert counts[iy, ix] == expect_n
        if tau > 0:
            p_in = pn + t0 * (pf - pn)
            p_out = p_in + (pf - pn) / dl * Keff * step
            z = [(M @ np.append(p, 1))[2] / (M @ np.append(p, 1))[3] for p in (p_in, p_out)]
            assert abs(depth[iy, ix, 0, 0] - z[0]) < 2e-5 and abs(depth[iy, ix, 0, 1] - z[1]) < 2e-5
            assert abs(rgba[iy, ix, 0, 3] - c[3]) < 1e-5  # per-unit opacity of a homogeneous segment
    assert hits > 50


def test_transparent_volume_gives_empty_vdi(orc):
    vol = np.zeros((8, 8, 8), np.float32)
    bmin, bmax = np.zeros(3), np.ones(3)
    cam = S.orbit_camera(bmin, bmax, 1.0)
    V = orc.Volume(vol, bmin, bmax)
    rgba, depth, counts = orc.generate(V, S.tf_knots("sparse"), cam.view, cam.proj, 10, 10, 4, 0.01, 1 / 8, 1 / 8)
    assert counts.sum() == 0 and np.all(np.isinf(depth)) and np.all(rgba == 0)


def test_linear_ramp_is_interpolated_exactly(orc):
    """Trilinear interpolation of a ramp sampled at voxel centres (i + 1/2) / n
    reproduces the ramp; with alpha = value / 2 the DVR of one ray is the
    product over its sample x-coordinates (closed form, computed here)."""
    n = 32
    g = ((np.arange(n) + 0.5) / n).astype(np.float32)
    vol = np.broadcast_to(g[None, None, :], (n, n, n)).copy()
    bmin, bmax = np.zeros(3), np.ones(3)
    kn = np.array([[0, 1, 1, 1, 0], [1, 1, 1, 1, 0.5]], np.float32)
    cam = S.orbit_camera(bmin, bmax, 1.0, el_deg=0.0, az_deg=90.0)  # looks along -x
    u = step = 1 / n
    w = h = 8
    dvr = orc.dvr(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, w, h, step, u)
    checked = 0
    for i, (pn, pf) in enumerate(pixel_rays(cam, w, h)):
        ch = chord(pn, pf, bmin, bmax)
        if ch is None:
            continue
        t0, t1, dl = ch
        K = int(np.floor((t1 - t0) * dl / step))
        d = (pf - pn) / dl
        T = 1.0
        for k in range(K):
            p = pn + t0 * (pf - pn) + (k + 0.5) * step * d
            x = min(max(p[0], 0.5 / n), 1 - 0.5 / n)  # the ramp is flat beyond the outer centres
            T *= 1 - 0.5 * x
            if T <= 2.0 ** -12:
                break
        assert abs(dvr[i, 3] - (1 - T)) < 1e-6
        checked += 1
    assert checked > 20


def test_transparent_gap_closes_supersegment(orc):
    """Two opaque slabs separated by empty space: with a huge tau each
    non-transparent run is one supersegment, so rays through both get two."""
    n = 40
    vol = np.zeros((n, n, n), np.float32)
    vol[:, :, 8:16] = 0.8
    vol[:, :, 24:32] = 0.8
    bmin, bmax = np.zeros(3), np.ones(3)
    kn = np.array([[0, 0, 0, 0, 0], [1, 1, 0.5, 0.2, 0.02]], np.float32)
    cam = S.orbit_camera(bmin, bmax, 1.0, el_deg=0.0, az_deg=90.0)
    _, _, counts = orc.generate(orc.Volume(vol, bmin, bmax), kn, cam.view, cam.proj, 9, 9, 6, 10.0, 1 / n, 1 / n)
    assert counts[4, 4] == 2 and counts[2:7, 2:7].min() == 2


def test_near_plane_inside_the_box_clips_generation(orc):
    n = 16
    vol = np.full((n, n, n), 0.45, np.float32)
    bmin, bmax = np.zeros(3), np.ones(3)
    eye = np.array([0.5, 0.5, 2.0])
    view = S.look_at(eye, np.array([0.5, 0.5, 0.5]))
    proj = S.perspective(np.radians(30.0), 1.0, 1.3, 3.0)  # near plane at z = 0.7, inside the box
    cam = S.Camera(view, proj, eye)
    kn = S.tf_knots("dense")
    w = h = 6
    rgba, depth, counts = orc.generate(orc.Volume(vol, bmin, bmax), kn, view, proj, w, h, 4, 0.05, 1 / n, 1 / n)
    M = proj @ view
    for i, (pn, pf) in enumerate(pixel_rays(cam, w, h)):
        iy, ix = divmod(i, w)
        ch = chord(pn, pf, bmin, bmax)
        assert ch is not None and ch[0] == 0.0  # the ray starts on the near plane, inside the box
        assert counts[iy, ix] == 1 and abs(depth[iy, ix, 0, 0] - (-1.0)) < 1e-5


# ---------------------------------------------------------------------------
# Ray-adaptive sensitivity (Section 3, Algorithm 3 of the supplement)
# ---------------------------------------------------------------------------
GAMMA0 = np.float32(1e-5)


def test_adaptive_gamma_on_a_constant_volume_keeps_the_start_value(orc):
    """Every sample of a constant volume is identical, so gamma = 1e-5 already
    gives one supersegment (< N_S): each ray keeps gamma = 1e-5 and the VDI is
    the fixed-gamma one (the closed form of test_constant_volume_closed_form)."""
    n = 16
    vol = np.full((n, n, n), 0.45, np.float32)
    bmin, bmax = np.zeros(3), np.ones(3)
    cam = S.orbit_camera(bmin, bmax, 1.0, el_deg=20, az_deg=30)
    kn = S.tf_knots("dense")
    V = orc.Volume(vol, bmin, bmax)
    for fp32 in (False, True):
        rgba, depth, counts, taus = orc.generate(V, kn, cam.view, cam.proj, 12, 12, 4, 0.3, 1 / n, 1 / n, fp32=fp32,
                                                 adaptive=True, with_tau=True)
        fixed = orc.generate(V, kn, cam.view, cam.proj, 12, 12, 4, float(GAMMA0), 1 / n, 1 / n, fp32=fp32)
        assert np.all(taus == GAMMA0)
        assert counts.max() == 1 and counts.sum() > 50
        for a, b in zip((rgba, depth, counts), fixed):
            assert np.array_equal(a, b)


def _band_check(orc, V, kn, cam, w, h, ns, u, rgba, depth, counts, taus):
    """Classify every list's gamma with the writing path of fixed-gamma
    generation at budget N_S + 1, which yields min(n(gamma), N_S + 1)."""
    delta = (15 * ns) // 100
    n_at = np.zeros((h, w), np.int64)
    for t in np.unique(taus):
        sel = taus == t
        _, _, c = orc.generate(V, kn, cam.view, cam.proj, w, h, ns + 1, float(t), u, u, fp32=True)
        n_at[sel] = c[sel]
    first = taus == GAMMA0
    band = (n_at >= ns - delta) & (n_at <= ns)
    converged = ~first & ~band
    # gamma = 1e-5 is kept only when it already gives at most N_S (fewer than
    # N_S, or inside the band)
    assert np.all(n_at[first] <= ns)
    # the generated VDI is the fixed-gamma VDI of each list's gamma
    assert np.all(counts <= ns)
    assert np.all(counts[band] == n_at[band])
    # lists that ended by the interval width took the upper end, a gamma that
    # gave fewer than N_S - delta
    assert np.all(n_at[converged] < ns - delta)
    searched = ~first
    return searched.mean(), band[searched].mean(), converged[searched].mean()


@pytest.mark.parametrize("ns", [6, 12])
def test_adaptive_gamma_lands_in_the_budget_band(orc, ns):
    vol = S.value_noise_volume(32, octaves=4, seed=5, dtype=np.uint16)
    bmin, bmax = S.bbox_for_dims(vol.shape)
    cam = S.orbit_camera(bmin, bmax, 1.0, el_deg=15, az_deg=20)
    V = orc.Volume(vol, bmin, bmax)
    kn = S.tf_knots("dense")
    u = 1 / 32
    w = h = 20
    rgba, depth, counts, taus = orc.generate(V, kn, cam.view, cam.proj, w, h, ns, 0.0, u, u, fp32=True,
                                             adaptive=True, with_tau=True)
    f_searched, f_band, f_conv = _band_check(orc, V, kn, cam, w, h, ns, u, rgba, depth, counts, taus)
    # of the lists that had to search, most end inside the band
    assert f_searched > 0.2 and f_band > 0.75 and f_conv < 0.25, (f_searched, f_band, f_conv)
    # the budget is used: adaptive lists carry more supersegments than a coarse fixed gamma
    assert counts[taus != GAMMA0].mean() >= ns - (15 * ns) // 100 - 1


def test_adaptive_vdi_still_renders_to_dvr_at_the_original_view(orc):
    """Check a' holds for any per-ray gamma: every supersegment stores the exact
    composite of its samples."""
    vol = S.blobs_volume(32, seed=4)
    bmin, bmax = S.bbox_for_dims(vol.shape)
    cam = S.orbit_camera(bmin, bmax, 1.0, el_deg=25, az_deg=40)
    V = orc.Volume(vol, bmin, bmax)
    kn = S.tf_knots("dense")
    u = 1 / 32
    for fp32 in (False, True):
        rgba, depth, counts, taus = orc.generate(V, kn, cam.view, cam.proj, 32, 32, 5, 0.0, u, u, fp32=fp32,
                                                 adaptive=True, with_tau=True)
        assert counts.max() <= 5 and len(np.unique(taus)) > 10
        sc = orc.Scene(S.VdiArrays(32, 32, 5, rgba, depth, counts), cam.view, cam.proj, bmin, bmax, u)
        dvr = orc.dvr(V, kn, cam.view, cam.proj, 32, 32, u, u)
        assert dvr[:, 3].max() > 0.5
        assert np.abs(orc.render_direct(sc) - dvr).max() < 2e-6


def test_eq1_threshold_is_the_l2_distance_of_premultiplied_colours(orc):
    """Two constant slabs, red then blue, with the same opacity: the
    premultiplied colours of their samples are a'(1, 0, 0) and a'(0, 0, 1),
    L2 distance D = sqrt(2) a', and samples near the interface lie between
    them.  A sensitivity above D merges everything into one supersegment per
    ray; one well below D must split at the interface."""
    n = 32
    vol = np.zeros((n, n, n), np.float32)
    vol[:, :, : n // 2] = 0.25
    vol[:, :, n // 2:] = 0.75
    bmin, bmax = np.zeros(3), np.ones(3)
    a = 0.05
    kn = np.array([[0.25, 1, 0, 0, a], [0.75, 0, 0, 1, a]], np.float32)
    cam = S.orbit_camera(bmin, bmax, 1.0, el_deg=0.0, az_deg=90.0)  # looks along -x, across the interface
    V = orc.Volume(vol, bmin, bmax)
    D = np.sqrt(2.0) * a  # step = u: a' = a
    _, _, c_hi = orc.generate(V, kn, cam.view, cam.proj, 9, 9, 8, 1.1 * D, 1 / n, 1 / n)
    _, _, c_lo = orc.generate(V, kn, cam.view, cam.proj, 9, 9, 8, 0.4 * D, 1 / n, 1 / n)
    hit = c_hi > 0
    assert hit.sum() >= 25
    assert np.all(c_hi[hit] == 1)
    assert np.all(c_lo[hit] >= 2)
