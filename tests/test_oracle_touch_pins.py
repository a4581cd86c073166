"""Pins of the oracle's replay of the exact render's access rule (the bytes a
frame touches: the roofline numerator).

* Per ray, the lists whose depth range it reads are the lists it passes
  through with positive length, and the supersegments whose colour it reads
  are its pieces inside supersegments: the replay's counts equal the exact
  render's per-ray counters (themselves pinned against lines crossed in V_O
  NDC) while early termination cannot trigger.
* At V_O every ray stays in its own list with depth increasing, so the
  supersegments it walks (front and back read) are the run from Algorithm 2's
  answer min{j : b_j >= d_entry} (numpy.searchsorted) up to and including the
  first one that reaches past d_exit, with d_entry, d_exit the NDC depths of
  the ray's box-clipped ends from camera-basis rays.  Search probes read backs
  only: at most the two seed depths and ceil(log2(N_S + 1)) probes per list.
* A supersegment opaque enough to end every ray inside it is the last colour
  any ray reads.
"""
import math

import numpy as np
import pytest

import vdi_synth as S
from helpers import random_case
from test_oracle_pins import box_planes, cam_rays, clip_interval, fovy_of, near_far


@pytest.mark.parametrize("az,el,ortho", [(25.0, 10.0, False), (-60.0, 25.0, False), (150.0, -15.0, False),
                                         (30.0, 15.0, True)])
def test_touch_counts_equal_ray_counters(orc, az, el, ortho):
    case = random_case(19, 13, 5, seed=7, u=0.5, alpha_range=(0.005, 0.02), zero_len_p=0.3)  # too faint to end a ray
    sc = case.oracle_scene(orc)
    W, H = 21, 17
    cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=az, el_deg=el, zoom=1.2, ortho=ortho)
    ref, nl, nsg, fl = orc.render_exact(sc, cn.view, cn.proj, W, H)
    assert ref[:, 3].max() < 0.9
    checked = 0
    for q in range(W * H):
        if fl[q]:
            continue
        d, c, r, tf = orc.touch_exact(sc, cn.view, cn.proj, W, H, pix=[q])
        assert tf[0] == 0
        assert r.sum() == nl[q], (q, r.sum(), nl[q])
        assert c.sum() == nsg[q], (q, c.sum(), nsg[q])
        assert np.all(d[c][:, 0] & d[c][:, 1])  # a composited supersegment had both faces read
        checked += nl[q] > 0
    assert checked > 50


def test_touch_at_original_view_walks_from_the_first_index(orc):
    w, h, ns = 14, 10, 7  # odd N_S: one padding slot
    case = random_case(w, h, ns, seed=12, u=0.5, alpha_range=(0.005, 0.02), fill=0.9, zero_len_p=0.0)
    sc = case.oracle_scene(orc)
    co = case.cam_o
    d, c, r, fl = orc.touch_exact(sc, co.view, co.proj, w, h)
    nsp = ns + 1
    eye, dirs = cam_rays(co, w, h, fovy_of(co), w / h)
    nN, fN = near_far(co)
    P = co.proj
    ndc_z = lambda depth: (P[2, 2] * -depth + P[2, 3]) / (P[3, 2] * -depth + P[3, 3])
    budget = 2 + math.ceil(math.log2(nsp + 1))
    checked = 0
    for q in range(w * h):
        s0, s1 = clip_interval(eye, dirs[q], box_planes(case.bmin, case.bmax), nN, fN)
        if not s1 > s0:
            assert not r[q] and not d[q].any()
            continue
        assert r[q]
        n = int(case.vdi.counts.reshape(-1)[q])
        f = np.full(nsp, np.inf)
        b = np.full(nsp, np.inf)
        f[:n] = case.vdi.depth.reshape(-1, ns, 2)[q, :n, 0]
        b[:n] = case.vdi.depth.reshape(-1, ns, 2)[q, :n, 1]
        d_in, d_out = ndc_z(s0), ndc_z(s1)
        if n and np.min(np.abs(np.concatenate([f[:n], b[:n]])[:, None] - [d_in, d_out])) < 1e-6:
            continue  # a face at the ray's end: a tie
        if n == 0 or d_out < f[0] or d_in > b[n - 1]:
            assert not d[q].any() and not c[q].any()  # the depth range alone rules the list out
            continue
        first = int(np.searchsorted(b, d_in, side="left"))
        walked = []
        for j in range(first, nsp):
            walked.append(j)
            if f[j] > d_out or b[j] > d_out:
                break
        assert list(np.nonzero(d[q, :, 0])[0]) == walked, (q, np.nonzero(d[q, :, 0])[0], walked)
        back_only = d[q, :, 1] & ~d[q, :, 0]
        assert back_only.sum() <= budget
        expect_c = [j for j in walked if min(b[j], d_out) > max(f[j], d_in)]
        assert list(np.nonzero(c[q])[0]) == expect_c
        checked += 1
    assert checked > 40


def test_touch_stops_at_an_opaque_supersegment(orc):
    w, h = 16, 12
    co = S.orbit_camera(np.zeros(3), np.ones(3), w / h, el_deg=10)
    n0, f0 = near_far(co)
    vdi = S.random_vdi(w, h, 4, seed=2, alpha_range=(0.05, 0.1), fill=1.0, zero_len_p=0.0)
    # every list's first supersegment becomes an opaque slab-like block in front of the rest
    zf = np.float32(S.ndc_z_of_view_depth(co.proj, n0 + 0.05 * (f0 - n0)))
    zb = np.float32(S.ndc_z_of_view_depth(co.proj, n0 + 0.5 * (f0 - n0)))
    vdi.depth[:, :, 0] = (zf, zb)
    vdi.depth[:, :, 1:, :] = np.maximum(vdi.depth[:, :, 1:, :], np.float32(zb + 1e-3))
    vdi.depth[:, :, 1:, :] = np.sort(vdi.depth[:, :, 1:, :].reshape(h, w, -1), axis=2).reshape(h, w, 3, 2)
    vdi.rgba[:, :, 0] = (0.9, 0.5, 0.1, 0.9)
    sc = orc.Scene(vdi, co.view, co.proj, np.zeros(3), np.ones(3), 0.01)
    W, H = 24, 18  # V_O's direction at another resolution: a ray meets the block before anything else
    ref = orc.render_exact(sc, co.view, co.proj, W, H)[0]
    stopped = 0
    for q in range(W * H):
        d, c, r, fl = orc.touch_exact(sc, co.view, co.proj, W, H, pix=[q])
        if fl[0] or not c[:, 0].any():
            continue
        # once the opaque block ends the ray, nothing behind it is read
        assert not c[:, 1:].any() and ref[q, 3] >= 1 - 2 ** -12
        stopped += 1
    assert stopped > 50
