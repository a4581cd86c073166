"""Pins of the FP64 CPU oracle against closed forms, invariants and brute force.

None of these compares the oracle with itself: every expected value comes from
an independent derivation written here with numpy (camera-basis rays,
Cyrus-Beck clipping against world planes, Beer-Lambert attenuation) or from a
library primitive (numpy.searchsorted), or from a different oracle routine
that does not share the traversal (direct per-list compositing at V_O,
midpoint sampling).
"""
import math

import numpy as np
import pytest

import vdi_synth as S

BMIN, BMAX = np.zeros(3), np.ones(3)


# ---------------------------------------------------------------- helpers


def cam_rays(cam, W, H, fovy, aspect):
    """Pixel-centre rays of a perspective camera from its basis (no matrix inverse).

    Returns origin (3,), directions (H*W, 3) with unit view-space depth, i.e.
    p(s) = eye + s * dir sits at view depth s.
    """
    px, py = np.meshgrid(np.arange(W), np.arange(H))
    x = 2 * (px.ravel() + 0.5) / W - 1
    y = 1 - 2 * (py.ravel() + 0.5) / H
    th = math.tan(fovy / 2)
    R = cam.view[:3, :3]  # rows: right, up, -forward
    dv = np.stack([x * th * aspect, y * th, -np.ones_like(x)], 1)
    return cam.eye, dv @ R


def fovy_of(cam):
    return 2 * math.atan(1.0 / cam.proj[1, 1])


def near_far(cam):
    P = cam.proj
    n = P[2, 3] / (P[2, 2] - 1)
    f = P[2, 3] / (P[2, 2] + 1)
    return n, f


def view_depth(cam, Z):
    P = cam.proj
    return -(P[2, 3] - Z * P[3, 3]) / (Z * P[3, 2] - P[2, 2])


def clip_interval(o, d, planes, s0, s1):
    """Cyrus-Beck: keep s in [s0,s1] where n.(o + s d) + c >= 0 for every (n, c)."""
    for n, c in planes:
        num = n @ o + c
        den = n @ d
        if abs(den) < 1e-300:
            if num < 0:
                return s0, s0
            continue
        t = -num / den
        if den > 0:
            s0 = max(s0, t)
        else:
            s1 = min(s1, t)
    return s0, s1


def box_planes(bmin, bmax):
    out = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1
        out.append((e, -bmin[k]))
        out.append((-e, bmax[k]))
    return out


def clip_planes(M, rows):
    """World half-spaces (row_a - X row_w) . (p, 1) >= 0 from clip-space rows of M = P V."""
    out = []
    for (r, X, sign) in rows:
        v = sign * (M[r] - X * M[3])
        out.append((v[:3], v[3]))
    return out


def frustum_planes(M):
    return clip_planes(M, [(0, -1, 1), (0, 1, -1), (1, -1, 1), (1, 1, -1), (2, -1, 1), (2, 1, -1)])


def scene(orc, vdi, cam, u):
    return orc.Scene(vdi, cam.view, cam.proj, BMIN, BMAX, u)


# ---------------------------------------------------------------- (a) V_O render == direct compositing


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_at_original_view_equals_direct(orc, seed):
    w, h, ns = 12, 9, 4
    vdi = S.random_vdi(w, h, ns, seed=seed, alpha_range=(0.02, 0.6))
    co = S.orbit_camera(BMIN, BMAX, w / h, az_deg=10 * seed, el_deg=15)
    sc = scene(orc, vdi, co, 0.1)
    direct = orc.render_direct(sc)
    exact, nl, nsg, fl = orc.render_exact(sc, co.view, co.proj, w, h)
    assert np.abs(direct - exact).max() < 1e-12
    # at V_O every ray stays in its own list
    assert nl.max() <= 1
    assert direct[:, 3].max() > 0.05


# ---------------------------------------------------------------- (b) Beer-Lambert slab


@pytest.mark.parametrize("az,el", [(25.0, 15.0), (-40.0, 5.0), (60.0, 30.0)])
def test_slab_matches_beer_lambert(orc, az, el):
    w, h = 40, 30
    co = S.orbit_camera(BMIN, BMAX, w / h, el_deg=10)
    n, f = near_far(co)
    d_f, d_b = n + 0.35 * (f - n), n + 0.55 * (f - n)
    zf = np.float32(S.ndc_z_of_view_depth(co.proj, d_f))
    zb = np.float32(S.ndc_z_of_view_depth(co.proj, d_b))
    chat, alpha, u = np.array([0.8, 0.5, 0.2]), 0.3, 0.05
    vdi = S.slab_vdi(w, h, 2, zf, zb, chat=chat, alpha=alpha)
    sc = scene(orc, vdi, co, u)
    W, H = 48, 36
    cn = S.orbit_camera(BMIN, BMAX, W / H, az_deg=az, el_deg=el, zoom=1.2)
    got, _, _, _ = orc.render_exact(sc, cn.view, cn.proj, W, H)

    # closed form: chord between the two planes of constant V_O view depth
    a32 = np.float32(alpha)
    chat_eff = (chat.astype(np.float32) * a32).astype(np.float32).astype(np.float64) / float(a32)
    fo = -co.view[2, :3]  # V_O forward
    dfz, dbz = view_depth(co, float(zf)), view_depth(co, float(zb))
    eye, dirs = cam_rays(cn, W, H, fovy_of(cn), W / H)
    nN, fN = near_far(cn)
    M = co.proj @ co.view
    ok = 0
    for q in range(W * H):
        d = dirs[q]
        base = fo @ (eye - co.eye)
        rate = fo @ d
        s_a, s_b = sorted([(dfz - base) / rate, (dbz - base) / rate])
        # chord must be inside V_N's depth range, the V_O frustum and the box, with margin
        inside = nN < s_a and s_b < fN
        for s in (s_a, s_b):
            p = eye + s * d
            hc = M @ np.append(p, 1.0)
            ndc = hc[:3] / hc[3]
            inside &= bool(np.all(np.abs(ndc[:2]) < 0.99) and np.all(p > 0.01) and np.all(p < 0.99))
        if not inside:
            continue
        ok += 1
        chord = (s_b - s_a) * np.linalg.norm(d)
        a = 1 - (1 - float(a32)) ** (chord / u)
        expect = np.append(chat_eff * a, a)
        assert np.abs(got[q] - expect).max() < 1e-9, (q, got[q], expect)
    assert ok > 50


# ---------------------------------------------------------------- (c) single supersegment: Cyrus-Beck hexahedron


@pytest.mark.parametrize("az", [15.0, 35.0, -70.0])
def test_single_supersegment_matches_hexahedron(orc, az):
    w, h = 6, 5
    co = S.orbit_camera(BMIN, BMAX, w / h, el_deg=10)
    n, f = near_far(co)
    ix, iy = 3, 2
    zf = np.float32(S.ndc_z_of_view_depth(co.proj, n + 0.3 * (f - n)))
    zb = np.float32(S.ndc_z_of_view_depth(co.proj, n + 0.7 * (f - n)))
    chat, alpha, u = np.array([0.3, 0.9, 0.6], np.float32), np.float32(0.6), 0.04
    vdi = S.single_vdi(w, h, 3, ix, iy, zf, zb, chat=chat, alpha=alpha)
    sc = scene(orc, vdi, co, u)
    W, H = 64, 48
    cn = S.orbit_camera(BMIN, BMAX, W / H, az_deg=az, el_deg=25, zoom=1.5)
    got, _, nsg, _ = orc.render_exact(sc, cn.view, cn.proj, W, H)

    M = co.proj @ co.view
    X0, X1 = -1 + 2 * ix / w, -1 + 2 * (ix + 1) / w
    Y0, Y1 = 1 - 2 * (iy + 1) / h, 1 - 2 * iy / h
    planes = clip_planes(M, [(0, X0, 1), (0, X1, -1), (1, Y0, 1), (1, Y1, -1),
                             (2, float(zf), 1), (2, float(zb), -1)])
    planes += box_planes(BMIN, BMAX) + frustum_planes(M)
    eye, dirs = cam_rays(cn, W, H, fovy_of(cn), W / H)
    nN, fN = near_far(cn)
    hits = 0
    for q in range(W * H):
        s0, s1 = clip_interval(eye, dirs[q], planes, nN, fN)
        l = max(0.0, s1 - s0) * np.linalg.norm(dirs[q])
        a = 1 - (1 - float(alpha)) ** (l / u)
        expect = np.append((chat * alpha).astype(np.float32).astype(np.float64) / float(alpha) * a, a)
        assert np.abs(got[q] - expect).max() < 1e-9, (q, got[q], expect)
        hits += l > 0
        assert nsg[q] == (1 if l > 1e-9 else nsg[q])
    assert hits > 20


# ---------------------------------------------------------------- (d) brute-force sampling converges to the exact render


def test_sampled_converges_to_exact(orc):
    w, h, ns = 8, 6, 4
    vdi = S.random_vdi(w, h, ns, seed=5, alpha_range=(0.05, 0.5), zero_len_p=0.0)
    co = S.orbit_camera(BMIN, BMAX, w / h, el_deg=15)
    sc = scene(orc, vdi, co, 0.2)
    cn = S.orbit_camera(BMIN, BMAX, 1.0, az_deg=30, el_deg=5)
    W = H = 24
    ex, _, _, _ = orc.render_exact(sc, cn.view, cn.proj, W, H)
    errs = []
    for hw in (4e-3, 2e-3, 1e-3, 5e-4):
        s = orc.render_sampled(sc, cn.view, cn.proj, W, H, hw)
        errs.append(np.abs(s - ex).mean())
    # first order in the step: each halving roughly halves the mean error
    for a, b in zip(errs, errs[1:]):
        assert 1.4 < a / b < 3.0, errs
    assert errs[-1] < 2e-3


# ---------------------------------------------------------------- special cases and invariants


def test_empty_vdi_and_missing_view_give_zero(orc):
    w, h = 8, 8
    vdi = S.random_vdi(w, h, 4, seed=0, fill=0.0)
    co = S.orbit_camera(BMIN, BMAX, 1.0)
    sc = scene(orc, vdi, co, 0.1)
    out, nl, nsg, _ = orc.render_exact(sc, co.view, co.proj, 16, 16)
    assert np.all(out == 0) and np.all(nsg == 0)
    full = S.random_vdi(w, h, 4, seed=3)
    sc2 = scene(orc, full, co, 0.1)
    away = S.Camera(S.look_at(co.eye, 2 * co.eye - 0.5), co.proj, co.eye)  # looks away
    out2, nl2, _, _ = orc.render_exact(sc2, away.view, away.proj, 16, 16)
    assert np.all(out2 == 0) and np.all(nl2 == 0)


def test_invariants_and_alpha_monotonicity(orc):
    w, h = 10, 10
    vdi = S.random_vdi(w, h, 4, seed=9)
    co = S.orbit_camera(BMIN, BMAX, 1.0, el_deg=10)
    cn = S.orbit_camera(BMIN, BMAX, 1.0, az_deg=40, el_deg=-10)
    sc = scene(orc, vdi, co, 0.1)
    out, _, _, _ = orc.render_exact(sc, cn.view, cn.proj, 20, 20)
    rgb, a = out[:, :3], out[:, 3]
    assert np.all(out >= -1e-15) and np.all(a <= 1 + 1e-15)
    assert np.all(rgb <= a[:, None] + 1e-12)
    weaker = S.VdiArrays(w, h, 4, vdi.rgba * np.float32(0.5), vdi.depth, vdi.counts)
    out2, _, _, _ = orc.render_exact(scene(orc, weaker, co, 0.1), cn.view, cn.proj, 20, 20)
    assert np.all(out2[:, 3] <= a + 1e-12)
    assert (out2[:, 3] < a - 1e-6).sum() > 10


def test_counts_null_means_leading_finite_slots(orc):
    vdi = S.random_vdi(9, 7, 5, seed=4)
    co = S.orbit_camera(BMIN, BMAX, 9 / 7)
    cn = S.orbit_camera(BMIN, BMAX, 1.0, az_deg=20)
    a = orc.render_exact(orc.Scene(vdi, co.view, co.proj, BMIN, BMAX, 0.1), cn.view, cn.proj, 16, 16)[0]
    b = orc.render_exact(orc.Scene(vdi, co.view, co.proj, BMIN, BMAX, 0.1, use_counts=False),
                         cn.view, cn.proj, 16, 16)[0]
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- first-supersegment contract (Algorithm 2)


def test_first_index_contract_matches_searchsorted(orc):
    rng = np.random.default_rng(0)
    for _ in range(3000):
        n = int(rng.integers(1, 9))
        pts = np.sort(rng.uniform(-1, 1, 2 * n)).astype(np.float32)
        f, b = pts[0::2].copy(), pts[1::2].copy()
        if rng.random() < 0.3:  # ties and zero-length pieces
            k = int(rng.integers(0, n))
            b[k] = f[k]
        d0, d1 = np.sort(rng.uniform(-1.1, 1.1, 2)).astype(np.float32)
        if rng.random() < 0.2:
            d0 = b[int(rng.integers(0, n))]
        j = int(np.searchsorted(b, d0, side="left"))
        exp_inc = j if (j < n and f[j] <= d1) else -1
        assert orc.first_index(f, b, d0, d1, True) == exp_inc
        k = int(np.searchsorted(f, d1, side="right")) - 1
        exp_dec = k if (k >= 0 and b[k] >= d0) else -1
        assert orc.first_index(f, b, d1, d0, False) == exp_dec


# ---------------------------------------------------------------- grid of supersegment counts (Section 4.3)


def test_grid_edges_are_uniform_in_view_depth(orc):
    co = S.orbit_camera(BMIN, BMAX, 16 / 9)
    vdi = S.random_vdi(16, 9, 2, seed=0, fill=0)
    e = orc.grid_edges(scene(orc, vdi, co, 0.1), 20).astype(np.float64)
    d = view_depth(co, e)
    n, f = near_far(co)
    assert abs(d[0] - n) < 1e-4 * n and abs(d[-1] - f) < 1e-4 * f
    assert np.abs(np.diff(d) - (f - n) / 20).max() < 1e-5 * (f - n)


def test_grid_counts_of_slab_on_cell_edges(orc):
    w, h, T, nz = 32, 24, 8, 10
    co = S.orbit_camera(BMIN, BMAX, w / h)
    e = orc.grid_edges(scene(orc, S.random_vdi(w, h, 2, fill=0), co, 0.1), nz)
    vdi = S.slab_vdi(w, h, 2, e[3], e[6])  # covers slabs 3, 4, 5 exactly
    g = orc.grid_counts(scene(orc, vdi, co, 0.1), T, nz)
    assert g.shape == (nz, h // T, w // T)
    expect = np.zeros(nz)
    expect[3:6] = T * T
    assert np.array_equal(g.reshape(nz, -1), np.repeat(expect[:, None], g[0].size, 1))
    # a zero-length piece on an edge belongs to the slab above the edge
    vdi0 = S.slab_vdi(w, h, 2, e[4], e[4])
    g0 = orc.grid_counts(scene(orc, vdi0, co, 0.1), T, nz)
    assert g0.sum() == w * h and np.all(g0[4] == T * T)


# ---------------------------------------------------------------- D_I / D_R previews (Section 4.4)


def test_upsample_is_exact_on_affine_images(orc):
    w0, h0, W, H = 7, 5, 28, 20
    yy, xx = np.meshgrid((np.arange(h0) + 0.5) / h0, (np.arange(w0) + 0.5) / w0, indexing="ij")
    lo = np.stack([0.3 + 0.2 * xx - 0.1 * yy, 0.5 * xx, 0.7 * yy, np.full_like(xx, 0.25)], -1)
    hi = orc.upsample(lo.reshape(-1, 4), w0, h0, W, H).reshape(H, W, 4)
    Y, X = np.meshgrid((np.arange(H) + 0.5) / H, (np.arange(W) + 0.5) / W, indexing="ij")
    expect = np.stack([0.3 + 0.2 * X - 0.1 * Y, 0.5 * X, 0.7 * Y, np.full_like(X, 0.25)], -1)
    # inside the band of low-res pixel centres bilinear interpolation of an affine image is exact
    m = (X >= 0.5 / w0) & (X <= 1 - 0.5 / w0) & (Y >= 0.5 / h0) & (Y <= 1 - 0.5 / h0)
    assert np.abs(hi - expect)[m].max() < 1e-14
    c = orc.upsample(np.full((h0 * w0, 4), 0.625), w0, h0, W, H)
    assert np.all(c == 0.625)


@pytest.mark.parametrize("d_r", [2, 4])
def test_ray_subsampled_preview_exact_on_slab_with_faces_on_edges(orc, d_r):
    w, h, T, nz = 32, 24, 8, 10
    co = S.orbit_camera(BMIN, BMAX, w / h, el_deg=5)
    e = orc.grid_edges(scene(orc, S.random_vdi(w, h, 2, fill=0), co, 0.1), nz)
    vdi = S.slab_vdi(w, h, 2, e[2], e[7], alpha=0.2)
    sc = scene(orc, vdi, co, 0.05)
    cn = S.orbit_camera(BMIN, BMAX, 1.0, az_deg=20, el_deg=10, zoom=1.3)
    ex, _, _, _ = orc.render_exact(sc, cn.view, cn.proj, 32, 32)
    pv, fl = orc.render_preview(sc, cn.view, cn.proj, 32, 32, d_r, T, nz)
    # every occupied cell lies inside the slab, so equal spacing composes to the exact length
    assert np.abs(pv - ex).max() < 1e-9
    assert ex[:, 3].max() > 0.1


# ---------------------------------------------------------------- D_R sample count (Section 4.4): an image that depends on n


def _stack_in_slab(w, h, ns, co, e, k0, d_r_pattern=None):
    """Every list holds supersegments inside grid slab k0 only (view-depth
    fractions of the slab): S1 = [0.02, 0.60]; lists with even ix also hold
    three thin ones, [0.70, 0.72], [0.80, 0.82], [0.90, 0.92].  Returns the VDI
    and, per list parity, the supersegments' view-depth ranges and (chat, alpha)."""
    dk, dk1 = view_depth(co, float(e[k0])), view_depth(co, float(e[k0 + 1]))
    fr = [(0.02, 0.60), (0.70, 0.72), (0.80, 0.82), (0.90, 0.92)]
    cols = [((0.9, 0.3, 0.1), 0.35), ((0.1, 0.8, 0.2), 0.5), ((0.2, 0.2, 0.9), 0.4), ((0.7, 0.7, 0.1), 0.6)]
    v = S.VdiArrays(w, h, ns, np.zeros((h, w, ns, 4), np.float32), np.full((h, w, ns, 2), np.inf, np.float32),
                    np.zeros((h, w), np.int32))
    segs = {}
    for parity, m in ((0, 4), (1, 1)):
        rows = []
        for j in range(m):
            zf = np.float32(S.ndc_z_of_view_depth(co.proj, dk + fr[j][0] * (dk1 - dk)))
            zb = np.float32(S.ndc_z_of_view_depth(co.proj, dk + fr[j][1] * (dk1 - dk)))
            chat, a = np.asarray(cols[j][0], np.float32), np.float32(cols[j][1])
            c32 = (chat * a).astype(np.float32)
            v.depth[:, parity::2, j] = (zf, zb)
            v.rgba[:, parity::2, j, :3] = c32
            v.rgba[:, parity::2, j, 3] = a
            # the field the VDI defines: chat = C / alpha of the stored FP32 values
            rows.append((view_depth(co, float(zf)), view_depth(co, float(zb)),
                         c32.astype(np.float64) / float(a), float(a)))
        v.counts[:, parity::2] = m
        segs[parity] = rows
    return v, segs, (dk, dk1)


@pytest.mark.parametrize("d_r", [1, 2])
def test_ray_subsampled_preview_sample_count(orc, d_r):
    """Rendered from V_O's own camera at the VDI's resolution, every ray runs down
    its list's centre and crosses only slabs of the count grid.  The one occupied
    slab holds c supersegments over the cell's F lists; the preview places
    n = ceil((c / F) (l_c / slab depth extent) / D_R) samples at the midpoints of n
    equal pieces of the ray's chord through the slab, and each takes the colour
    of the supersegment containing it with opacity for the spacing l_c / n.
    Expected values come from camera-basis rays, Cyrus-Beck box clipping and the
    closed-form view depth of the stored faces; the supersegments are thinner
    than the slab, so the image depends on n (planted floor-for-ceil, x D_R, and
    T instead of the cell's list count each fail here)."""
    w, h, T, nz, k0, u = 43, 30, 8, 10, 5, 0.03  # ragged last cell column (3 lists) and row (6 lists)
    co = S.orbit_camera(BMIN, BMAX, w / h, el_deg=15, zoom=2.6)  # the box fills the view, ragged cells included
    e = orc.grid_edges(scene(orc, S.random_vdi(w, h, 2, fill=0), co, u), nz)
    vdi, segs, (dk, dk1) = _stack_in_slab(w, h, 4, co, e, k0)
    sc = scene(orc, vdi, co, u)
    got, fl = orc.render_preview(sc, co.view, co.proj, w, h, d_r, T, nz)

    nN, fN = near_far(co)
    dz_cell = (fN - nN) / nz
    eye, dirs = cam_rays(co, w, h, fovy_of(co), w / h)
    checked, ns_seen = 0, {}
    for q in range(w * h):
        ix, iy = q % w, q // w
        s0, s1 = clip_interval(eye, dirs[q], box_planes(BMIN, BMAX), nN, fN)
        sa, sb = max(s0, dk), min(s1, dk1)  # view depth along these rays
        if not sb > sa:
            assert np.all(got[q] == 0)
            checked += 1
            continue
        L = np.linalg.norm(dirs[q])
        lc = (sb - sa) * L
        cx, cy = ix // T, iy // T
        xs, ys = range(cx * T, min(cx * T + T, w)), range(cy * T, min(cy * T + T, h))
        c = sum(len(segs[x % 2]) for x in xs) * len(ys)
        want = (c / (len(xs) * len(ys))) * (lc / dz_cell) / d_r
        if abs(want - round(want)) < 1e-7 * want:
            continue  # a count at a rounding boundary
        n = max(1, math.ceil(want))
        acc = np.zeros(4)
        tie = False
        for i in range(n):
            s = sa + (i + 0.5) * (sb - sa) / n
            for (vf, vb, chat, a) in segs[ix % 2]:
                if min(abs(s - vf), abs(s - vb)) < 1e-9:
                    tie = True
                if vf <= s <= vb:
                    at = 1 - (1 - a) ** ((lc / n) / u)
                    acc[:3] += (1 - acc[3]) * chat * at
                    acc[3] += (1 - acc[3]) * at
                    break
        if tie:
            continue
        assert np.abs(got[q] - acc).max() < 1e-9, (q, n, got[q], acc)
        checked += 1
        ns_seen[n] = ns_seen.get(n, 0) + 1
    assert checked > 0.95 * w * h
    assert got.reshape(h, w, 4)[:, -1, 3].min() > 0 and got.reshape(h, w, 4)[-1, :, 3].min() > 0
    assert len(ns_seen) >= 2 and sum(ns_seen.values()) > 200, ns_seen  # the image depends on n across the view
    assert got[:, 3].max() > 0.3


# ---------------------------------------------------------------- per-ray counters: lists crossed, pieces inside supersegments


def pixel_rays(cam, W, H):
    """Pixel-centre rays of a perspective or orthographic camera from its basis:
    origins (n, 3) and directions (n, 3) with unit view-space depth, so
    o + s d sits at view depth s (no matrix inverse)."""
    px, py = np.meshgrid(np.arange(W), np.arange(H))
    x = 2 * (px.ravel() + 0.5) / W - 1
    y = 1 - 2 * (py.ravel() + 0.5) / H
    R = cam.view[:3, :3]  # rows: right, up, -forward
    P = cam.proj
    if P[3, 3] == 1.0:  # orthographic: parallel rays from points of the view plane
        o = cam.eye + (x / P[0, 0])[:, None] * R[0] + (y / P[1, 1])[:, None] * R[1]
        d = np.repeat(-R[2][None, :], len(x), 0)
        return o, d
    th = 1.0 / P[1, 1]
    dv = np.stack([x * th * (P[1, 1] / P[0, 0]), y * th, -np.ones_like(x)], 1)
    return np.repeat(cam.eye[None, :], len(x), 0), dv @ R


def lines_between(a, b, n):
    """Interior grid lines k (1 <= k <= n - 1) strictly between grid coordinates a and b."""
    lo, hi = min(a, b), max(a, b)
    return [k for k in range(max(1, math.floor(lo) + 1), min(n - 1, math.ceil(hi) - 1) + 1) if lo < k < hi]


@pytest.mark.parametrize("az,el,zoom,ortho", [(20.0, 10.0, 1.3, False), (-50.0, 30.0, 1.0, False),
                                             (35.0, 15.0, 1.2, True), (125.0, -10.0, 1.4, False)])
def test_ray_counters_match_lines_crossed(orc, az, el, zoom, ortho):
    """A new-view ray is a straight segment in V_O's NDC, so the lists it passes
    through with positive length number one more than the interior list-grid
    lines between the NDC images of its clipped ends (Fig. 3), empty lists
    included.  With a slab in every non-empty list, the pieces inside
    supersegments are the lists crossed by the part of the ray between the two
    slab planes.  Clip ends come from Cyrus-Beck against the box, V_O's frustum
    planes and V_N's near/far range; rays with a tie (an end or a crossing
    within 1e-9 list widths of a grid line) are skipped."""
    w, h = 23, 17
    co = S.orbit_camera(BMIN, BMAX, w / h, el_deg=10, zoom=2.0)  # V_O's frustum cuts the box
    n0, f0 = near_far(co)
    zf = np.float32(S.ndc_z_of_view_depth(co.proj, n0 + 0.4 * (f0 - n0)))
    zb = np.float32(S.ndc_z_of_view_depth(co.proj, n0 + 0.55 * (f0 - n0)))
    vdi = S.slab_vdi(w, h, 2, zf, zb, alpha=0.2)
    empty = (np.add.outer(np.arange(h), np.arange(w)) % 3) == 0  # every third diagonal of lists is empty
    vdi.depth[empty] = np.inf
    vdi.rgba[empty] = 0
    vdi.counts[empty] = 0
    sc = scene(orc, vdi, co, 0.1)
    W, H = 40, 30
    cn = S.orbit_camera(BMIN, BMAX, W / H, az_deg=az, el_deg=el, zoom=zoom, ortho=ortho)
    _, nl, nsg, _ = orc.render_exact(sc, cn.view, cn.proj, W, H)

    M = co.proj @ co.view
    planes = box_planes(BMIN, BMAX) + frustum_planes(M)
    origins, dirs = pixel_rays(cn, W, H)
    nN, fN = near_far(cn) if not ortho else ((cn.proj[2, 3] + 1) / cn.proj[2, 2], (cn.proj[2, 3] - 1) / cn.proj[2, 2])
    fo, vd_f, vd_b = -co.view[2, :3], view_depth(co, float(zf)), view_depth(co, float(zb))

    def grid_of(p):
        hc = M @ np.append(p, 1.0)
        return (hc[0] / hc[3] + 1) * 0.5 * w, (1 - hc[1] / hc[3]) * 0.5 * h

    def crossed(o, d, s0, s1):
        """(lists crossed, tie) for the segment s in [s0, s1] of the ray."""
        (ax, ay), (bx, by) = grid_of(o + s0 * d), grid_of(o + s1 * d)
        # an end on an interior grid line (ends on the frustum's sides, grid 0 or w, are no tie)
        tie = any(abs(g - round(g)) < 1e-9 and 0 < round(g) < n
                  for g, n in ((ax, w), (ay, h), (bx, w), (by, h)))
        kx, ky = lines_between(ax, bx, w), lines_between(ay, by, h)
        for k in kx:  # a corner: an x line met where y is also on a line
            lam = (k - ax) / (bx - ax)
            tie |= abs((ay + lam * (by - ay)) - round(ay + lam * (by - ay))) < 1e-9
        return 1 + len(kx) + len(ky), tie

    checked = crossings = 0
    for q in range(W * H):
        o, d = origins[q], dirs[q]
        s0, s1 = clip_interval(o, d, planes, nN, fN)
        if not s1 > s0 + 1e-12:
            assert nl[q] == 0 and nsg[q] == 0
            checked += 1
            continue
        want_l, tie = crossed(o, d, s0, s1)
        # part of the ray between the slab's planes of constant V_O view depth
        base, rate = fo @ (o - co.eye), fo @ d
        ta, tb = sorted([(vd_f - base) / rate, (vd_b - base) / rate])
        ca, cb = max(s0, ta), min(s1, tb)
        if cb > ca + 1e-12:
            # pieces inside the slab: lists crossed by [ca, cb] that are not empty
            (ax, ay), (bx, by) = grid_of(o + ca * d), grid_of(o + cb * d)
            want_s, tie2 = crossed(o, d, ca, cb)
            tie |= tie2
            # walk the crossed lists in order to drop the empty ones
            ts = [0.0, 1.0] + [(k - ax) / (bx - ax) for k in lines_between(ax, bx, w)] + \
                 [(k - ay) / (by - ay) for k in lines_between(ay, by, h)]
            ts = sorted(ts)
            want_s = 0
            for t0, t1 in zip(ts, ts[1:]):
                if t1 - t0 < 1e-12:
                    continue
                # the grid point at the middle of the NDC sub-segment (NDC is affine in the
                # sub-segment's own parameter, which is what the crossings above measure)
                gx, gy = ax + 0.5 * (t0 + t1) * (bx - ax), ay + 0.5 * (t0 + t1) * (by - ay)
                ix, iy = min(int(gx), w - 1), min(int(gy), h - 1)
                want_s += 0 if empty[iy, ix] else 1
        else:
            want_s = 0
        if tie:
            continue
        assert nl[q] == want_l, (q, nl[q], want_l)
        assert nsg[q] == want_s, (q, nsg[q], want_s)
        checked += 1
        crossings += want_l - 1
    assert checked > 0.97 * W * H and crossings > 200
