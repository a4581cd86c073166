"""Shared test helpers: tolerance checks and scene set-up for GPU-vs-oracle parity.

Tolerances (per-channel maximum absolute error against the FP64 oracle):
FP32 colour <= 1e-3 on 99.9% of pixels and <= 4e-3 everywhere; FP16 colour
storage <= 4e-3 / <= 8e-3 (against the oracle on the unquantised FP32 VDI).
"""
import numpy as np

import vdi_synth as S

TOL = {0: (1e-3, 4e-3), 1: (4e-3, 8e-3)}  # colour format -> (99.9% bound, max bound)


def check_tolerance(got, ref, fmt, mask=None, what=""):
    got = np.asarray(got, np.float64).reshape(-1, 4)
    ref = np.asarray(ref, np.float64).reshape(-1, 4)
    err = np.abs(got - ref).max(axis=1)
    if mask is not None:
        err = err[np.asarray(mask, bool).reshape(-1)]
    p999, pmax = TOL[fmt]
    q = float(np.quantile(err, 0.999)) if err.size else 0.0
    m = float(err.max()) if err.size else 0.0
    assert q <= p999 and m <= pmax, f"{what}: 99.9% err {q:.3g} (<= {p999}), max err {m:.3g} (<= {pmax})"
    return q, m


class Case:
    """One VDI (ABI arrays) with its original camera, box and length unit."""

    def __init__(self, vdi, cam_o, bmin, bmax, u):
        self.vdi, self.cam_o, self.bmin, self.bmax, self.u = vdi, cam_o, np.asarray(bmin), np.asarray(bmax), u

    def oracle_scene(self, orc):
        return orc.Scene(self.vdi, self.cam_o.view, self.cam_o.proj, self.bmin, self.bmax, self.u)

    def gpu_desc(self, V, fmt, T=0, nz=0):
        return V.desc(self.vdi.w, self.vdi.h, self.vdi.ns, self.cam_o.view, self.cam_o.proj, self.bmin, self.bmax,
                      self.u, fmt, T, nz)


def random_case(w, h, ns, seed, u=0.1, el=15.0, **kw):
    bmin, bmax = np.zeros(3), np.ones(3)
    vdi = S.random_vdi(w, h, ns, seed=seed, **kw)
    cam = S.orbit_camera(bmin, bmax, w / h, az_deg=0.0, el_deg=el)
    return Case(vdi, cam, bmin, bmax, u)


# ---------------------------------------------------------------------------
# rays the oracle flags: every valid limit is accepted
#
# The oracle flags a ray whose result turns on a decision within rounding
# distance of a tie (a list boundary, a supersegment face, a D_R sample count
# at an integer).  The GPU takes those decisions in FP32, so either side is a
# correct answer.  Flagged rays are therefore checked, not dropped: the GPU
# value must lie within the tolerance of the plain oracle value or of one of
# the oracle's other limits -- for the exact render the rays through the pixel
# centre moved by NUDGE pixel widths in eight directions (rays the GPU's
# rounding can stand for), for the D_R preview the same ray with its tie
# decisions flipped.
# ---------------------------------------------------------------------------

NUDGE = 1e-3  # pixel widths


def pixel_ndc(idx, W, H):
    idx = np.asarray(idx)
    px, py = idx % W, idx // W
    return 2 * (px + 0.5) / W - 1, 1 - 2 * (py + 0.5) / H


def exact_alternatives(orc, sc, cam, W, H, idx):
    """[8, len(idx), 4] oracle values, and [8, len(idx)] list / supersegment
    counters, of the rays through the pixel centres of ``idx`` moved by NUDGE
    pixel widths in eight directions."""
    x, y = pixel_ndc(idx, W, H)
    vals, nls, nss = [], [], []
    for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (1, -1), (-1, 1), (-1, -1)):
        xy = np.stack([x + dx * NUDGE * 2.0 / W, y + dy * NUDGE * 2.0 / H], 1)
        o, nl, ns, _ = orc.render_exact_ndc(sc, cam.view, cam.proj, xy)
        vals.append(o)
        nls.append(nl)
        nss.append(ns)
    return np.stack(vals), np.stack(nls), np.stack(nss)


def preview_alternatives(orc, sc, cam, W, H, d_r, T, nz, grid, idx):
    """[k, len(idx), 4] oracle D_R preview values of the pixels ``idx`` with their
    near-tie decisions flipped: none, all, each one alone, and every combination
    of the first five."""
    idx = np.asarray(idx, np.int32)
    base, nt = orc.render_preview_alt(sc, cam.view, cam.proj, W, H, d_r, T, nz, grid, idx, 0)
    k = int(nt.max()) if len(idx) else 0
    masks = {0xFFFFFFFF} | {1 << b for b in range(min(k, 32))} | set(range(1, 1 << min(k, 5)))
    vals = [base] + [orc.render_preview_alt(sc, cam.view, cam.proj, W, H, d_r, T, nz, grid, idx, m)[0]
                     for m in sorted(masks)]
    return np.stack(vals)


def check_with_alternatives(got, ref, fmt, flags, alts, what=""):
    """check_tolerance over every pixel: a flagged pixel's error is the smallest
    over the plain oracle value and its alternatives (``alts``: [k, n_flagged, 4]
    for the pixels where ``flags`` is set, in index order).  Returns the flagged
    fraction and how many flagged pixels needed an alternative."""
    got = np.asarray(got, np.float64).reshape(-1, 4)
    ref = np.asarray(ref, np.float64).reshape(-1, 4)
    err = np.abs(got - ref).max(axis=1)
    flagged = np.nonzero(np.asarray(flags).reshape(-1))[0]
    used = 0
    if len(flagged):
        e_alt = np.abs(np.asarray(alts) - got[flagged][None]).max(axis=2).min(axis=0)
        used = int(np.sum(e_alt < err[flagged] - 1e-12))
        err[flagged] = np.minimum(err[flagged], e_alt)
    p999, pmax = TOL[fmt]
    q = float(np.quantile(err, 0.999)) if err.size else 0.0
    m = float(err.max()) if err.size else 0.0
    frac = len(flagged) / max(1, err.size)
    print(f"{what}: flagged {frac:.4f} of {err.size} rays, {used} matched another limit; "
          f"99.9% err {q:.3g}, max err {m:.3g}")
    assert q <= p999 and m <= pmax, f"{what}: 99.9% err {q:.3g} (<= {p999}), max err {m:.3g} (<= {pmax})"
    return frac, used


def closest_alternative(got_idx, alts):
    """Per flagged pixel, the oracle alternative nearest to the GPU value ([n, 4])."""
    alts = np.asarray(alts)
    e = np.abs(alts - np.asarray(got_idx, np.float64)[None]).max(axis=2)
    return alts[np.argmin(e, axis=0), np.arange(alts.shape[1])]


def check_exact(orc, sc, cam, W, H, got, fmt, ref=None, fl=None, what=""):
    """Exact render of W x H against the oracle, flagged rays against their nudged limits."""
    if ref is None:
        ref, _, _, fl = orc.render_exact(sc, cam.view, cam.proj, W, H)
    idx = np.nonzero(fl)[0]
    alts = exact_alternatives(orc, sc, cam, W, H, idx)[0] if len(idx) else np.zeros((1, 0, 4))
    return check_with_alternatives(got, ref, fmt, fl, alts, what=what)
