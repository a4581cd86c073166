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
