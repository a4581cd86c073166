"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle harness.

This module only *creates inputs*: cameras (OpenGL view/projection matrices),
scalar volumes, transfer-function knots and small VDIs in the ABI's array-of-
structures format.  It holds none of the rendering or generation arithmetic of
the method (no ray setup, no list traversal, no compositing), so the CUDA path
and the CPU oracle can both consume its outputs without sharing method code.

Conventions
-----------
* Matrices are float64 numpy (4, 4) arrays in the usual row-major math layout;
  ``colmajor(M)`` flattens one into the column-major ``double[16]`` that the C
  interfaces take (OpenGL convention, clip = P * V * x_world).
* World space is y-up.  A volume array ``vol[k, j, i]`` (z, y, x; x fastest)
  fills the box ``[0, n/nmax]^3``; one voxel is ``1/nmax`` world units, which
  is also the default opacity length unit ``u``.
* The workloads stand in for the paper's datasets (Engine, Kingsnake,
  Rayleigh-Taylor, Richtmyer-Meshkov; Section 2, Table 1), which are not
  available: Gaussian blobs, multi-octave value noise and a perturbed tanh
  mixing layer.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------


def colmajor(m: np.ndarray) -> np.ndarray:
    """(4,4) row-major math matrix -> contiguous column-major float64[16]."""
    return np.ascontiguousarray(np.asarray(m, dtype=np.float64).T).reshape(16)


def look_at(eye, center, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    center = np.asarray(center, np.float64)
    up = np.asarray(up, np.float64)
    f = center - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[0, 3], m[1, 3], m[2, 3] = -s @ eye, -u @ eye, f @ eye
    return m


def perspective(fovy_rad: float, aspect: float, near: float, far: float) -> np.ndarray:
    f = 1.0 / math.tan(fovy_rad / 2.0)
    m = np.zeros((4, 4))
    m[0, 0] = f / aspect
    m[1, 1] = f
    m[2, 2] = (far + near) / (near - far)
    m[2, 3] = 2.0 * far * near / (near - far)
    m[3, 2] = -1.0
    return m


def orthographic(half_w: float, half_h: float, near: float, far: float) -> np.ndarray:
    m = np.eye(4)
    m[0, 0] = 1.0 / half_w
    m[1, 1] = 1.0 / half_h
    m[2, 2] = -2.0 / (far - near)
    m[2, 3] = -(far + near) / (far - near)
    return m


@dataclass
class Camera:
    view: np.ndarray  # (4,4)
    proj: np.ndarray  # (4,4)
    eye: np.ndarray

    @property
    def view_cm(self):
        return colmajor(self.view)

    @property
    def proj_cm(self):
        return colmajor(self.proj)


def bbox_for_dims(dims_zyx) -> tuple[np.ndarray, np.ndarray]:
    nz, ny, nx = dims_zyx
    nmax = float(max(dims_zyx))
    return np.zeros(3), np.array([nx / nmax, ny / nmax, nz / nmax])


def orbit_camera(bmin, bmax, aspect, az_deg=0.0, el_deg=20.0, zoom=1.0,
                 dist_factor=3.0, ortho=False) -> Camera:
    """Camera facing the box centre from distance ``dist_factor * r``.

    ``r`` is the bounding-sphere radius.  The vertical field of view is fitted
    to the sphere (divided by ``zoom``) and near/far bracket the sphere tightly
    (``D - r``, ``D + r``), which keeps FP32 NDC depth well resolved.  The
    evaluation camera path of the paper (Section 6) rotates about the dataset
    centre while facing it; ``az_deg`` is that rotation about the vertical
    axis.
    """
    bmin = np.asarray(bmin, np.float64)
    bmax = np.asarray(bmax, np.float64)
    c = 0.5 * (bmin + bmax)
    r = 0.5 * np.linalg.norm(bmax - bmin)
    d = dist_factor * r
    az, el = math.radians(az_deg), math.radians(el_deg)
    eye = c + d * np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)])
    view = look_at(eye, c)
    near, far = d - r, d + r
    if ortho:
        hh = r / zoom
        proj = orthographic(hh * aspect, hh, near, far)
    else:
        half = math.asin(r / d)
        fovy = 2.0 * math.atan(math.tan(half) / zoom)
        proj = perspective(fovy, aspect, near, far)
    return Camera(view, proj, eye)


# --------------------------------------------------------------------------
# volumes
# --------------------------------------------------------------------------


def blobs_volume(n=64, n_blobs=6, seed=0) -> np.ndarray:
    """Sum of Gaussian blobs, centres U[0.2,0.8]^3, sigma U[0.05,0.15], clamped to [0,1]."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(n_blobs, 3))
    sig = rng.uniform(0.05, 0.15, size=n_blobs)
    g = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    v = np.zeros((n, n, n))
    for (cx, cy, cz), s in zip(centres, sig):
        v += np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2 * s * s))
    return np.clip(v, 0.0, 1.0).astype(np.float32)


def _smooth_upsample_axis(a: np.ndarray, axis: int, n: int, freq: int) -> np.ndarray:
    """Resample lattice values (freq+1 points) to n voxel centres, smoothstep weights."""
    pos = (np.arange(n) + 0.5) / n * freq
    i0 = np.minimum(np.floor(pos).astype(np.int64), freq - 1)
    t = (pos - i0).astype(np.float32)
    t = t * t * (3.0 - 2.0 * t)
    shape = [1] * a.ndim
    shape[axis] = n
    t = t.reshape(shape)
    lo = np.take(a, i0, axis=axis)
    hi = np.take(a, i0 + 1, axis=axis)
    return lo + (hi - lo) * t


def value_noise_volume(n=256, octaves=5, base_freq=4, seed=0, dtype=np.uint16) -> np.ndarray:
    """Multi-octave value noise: seeded lattice values, smoothstep trilinear, amplitude 2^-k."""
    rng = np.random.default_rng(seed)
    acc = np.zeros((n, n, n), np.float32)
    amp_sum = 0.0
    for k in range(octaves):
        f = base_freq << k
        lat = rng.random((f + 1, f + 1, f + 1), dtype=np.float32)
        v = _smooth_upsample_axis(lat, 2, n, f)
        v = _smooth_upsample_axis(v, 1, n, f)
        v = _smooth_upsample_axis(v, 0, n, f)
        amp = 0.5 ** k
        acc += np.float32(amp) * v
        amp_sum += amp
    acc /= np.float32(amp_sum)
    lo, hi = float(acc.min()), float(acc.max())
    acc = (acc - lo) / max(hi - lo, 1e-12)
    if dtype == np.float32:
        return acc.astype(np.float32)
    top = np.iinfo(dtype).max
    return np.clip(np.rint(acc * top), 0, top).astype(dtype)


def mixing_layer_volume(n=1024, modes=64, amp_max=0.05, width=0.01, seed=0,
                        dtype=np.uint8) -> np.ndarray:
    """Perturbed tanh interface at mid-height (world y), Rayleigh-Taylor-like.

    rho = 1/2 + 1/2 tanh((y - 1/2 - sum_m a_m sin(2 pi (k_m . (x, z)) + phi_m)) / width),
    with a_m ~ U[0, amp_max], integer k_m in [1, 8]^2, phi_m ~ U[0, 2 pi).
    """
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, amp_max, size=modes)
    kx = rng.integers(1, 9, size=modes)
    kz = rng.integers(1, 9, size=modes)
    ph = rng.uniform(0.0, 2 * np.pi, size=modes)
    g = ((np.arange(n) + 0.5) / n).astype(np.float64)
    h = np.zeros((n, n))  # [z, x]
    zz, xx = np.meshgrid(g, g, indexing="ij")
    for m in range(modes):
        h += a[m] * np.sin(2 * np.pi * (kx[m] * xx + kz[m] * zz) + ph[m])
    h = (0.5 + h).astype(np.float32)  # interface height per (z, x)
    top = np.iinfo(dtype).max if dtype != np.float32 else 1.0
    out = np.empty((n, n, n), dtype=dtype)
    gy = g.astype(np.float32)
    inv_w = np.float32(1.0 / width)
    for k in range(n):  # one z slice at a time keeps memory bounded
        arg = (gy[:, None] - h[k][None, :]) * inv_w  # [y, x]
        rho = 0.5 + 0.5 * np.tanh(arg)
        if dtype == np.float32:
            out[k] = rho
        else:
            out[k] = np.rint(rho * top).astype(dtype)
    return out


# --------------------------------------------------------------------------
# transfer functions (4-knot piecewise-linear RGBA)
# --------------------------------------------------------------------------


def tf_knots(kind: str = "dense") -> np.ndarray:
    """(4, 5) float32 knots: value, r, g, b, a (a = opacity per length unit, capped at 0.5)."""
    if kind == "dense":
        k = [[0.00, 0.10, 0.20, 0.80, 0.00],
             [0.30, 0.20, 0.60, 0.90, 0.05],
             [0.60, 0.95, 0.60, 0.20, 0.35],
             [1.00, 0.90, 0.20, 0.10, 0.50]]
    elif kind == "sparse":
        k = [[0.00, 0.00, 0.00, 0.00, 0.00],
             [0.45, 0.30, 0.50, 0.90, 0.00],
             [0.60, 0.95, 0.70, 0.30, 0.25],
             [1.00, 1.00, 0.30, 0.20, 0.50]]
    elif kind == "interface":
        # mixing layer: transparent light fluid, thin opaque-ish sheet, hazy heavy fluid
        k = [[0.00, 0.20, 0.40, 0.90, 0.00],
             [0.30, 0.30, 0.70, 0.90, 0.20],
             [0.60, 1.00, 0.55, 0.15, 0.45],
             [1.00, 0.25, 0.35, 0.80, 0.03]]
    else:
        raise ValueError(kind)
    return np.asarray(k, np.float32)


# --------------------------------------------------------------------------
# small VDIs in the ABI layout (rgba[h][w][ns][4] premultiplied, depth[h][w][ns][2])
# --------------------------------------------------------------------------


@dataclass
class VdiArrays:
    w: int
    h: int
    ns: int
    rgba: np.ndarray   # float32 [h, w, ns, 4], premultiplied, alpha per length unit
    depth: np.ndarray  # float32 [h, w, ns, 2], V_O NDC z (front, back)
    counts: np.ndarray  # int32 [h, w]


def _empty_vdi(w, h, ns) -> VdiArrays:
    rgba = np.zeros((h, w, ns, 4), np.float32)
    depth = np.full((h, w, ns, 2), np.inf, np.float32)
    return VdiArrays(w, h, ns, rgba, depth, np.zeros((h, w), np.int32))


def random_vdi(w, h, ns, seed=0, z_lo=-0.95, z_hi=0.95, fill=0.8, touch_p=0.2,
               zero_len_p=0.05, alpha_range=(0.05, 0.9)) -> VdiArrays:
    """Random sorted supersegment lists with gaps, touching neighbours and zero-length pieces."""
    rng = np.random.default_rng(seed)
    v = _empty_vdi(w, h, ns)
    for iy in range(h):
        for ix in range(w):
            if rng.random() > fill:
                continue
            n = int(rng.integers(1, ns + 1))
            pts = np.sort(rng.uniform(z_lo, z_hi, size=2 * n)).astype(np.float32)
            f = pts[0::2].copy()
            b = pts[1::2].copy()
            for j in range(n - 1):
                if rng.random() < touch_p:
                    b[j] = f[j + 1]
            for j in range(n):
                if rng.random() < zero_len_p:
                    b[j] = f[j]
            a = rng.uniform(*alpha_range, size=n).astype(np.float32)
            chat = rng.random((n, 3)).astype(np.float32)
            v.depth[iy, ix, :n, 0] = f
            v.depth[iy, ix, :n, 1] = b
            v.rgba[iy, ix, :n, :3] = (chat * a[:, None]).astype(np.float32)
            v.rgba[iy, ix, :n, 3] = a
            v.counts[iy, ix] = n
    return v


def slab_vdi(w, h, ns, z_front, z_back, chat=(0.8, 0.5, 0.2), alpha=0.3) -> VdiArrays:
    """Every list holds one supersegment [z_front, z_back]: a slab of constant V_O view depth."""
    v = _empty_vdi(w, h, ns)
    v.depth[:, :, 0, 0] = np.float32(z_front)
    v.depth[:, :, 0, 1] = np.float32(z_back)
    a = np.float32(alpha)
    v.rgba[:, :, 0, :3] = (np.asarray(chat, np.float32) * a).astype(np.float32)
    v.rgba[:, :, 0, 3] = a
    v.counts[:] = 1
    return v


def single_vdi(w, h, ns, ix, iy, z_front, z_back, chat=(0.3, 0.9, 0.6), alpha=0.6) -> VdiArrays:
    """One list (ix, iy) holds one supersegment; every other list is empty."""
    v = _empty_vdi(w, h, ns)
    v.depth[iy, ix, 0] = (z_front, z_back)
    a = np.float32(alpha)
    v.rgba[iy, ix, 0, :3] = (np.asarray(chat, np.float32) * a).astype(np.float32)
    v.rgba[iy, ix, 0, 3] = a
    v.counts[iy, ix] = 1
    return v


def ndc_z_of_view_depth(proj: np.ndarray, depth: float) -> float:
    """NDC z of a point at view-space distance ``depth`` in front of the camera."""
    ze = -depth
    zc = proj[2, 2] * ze + proj[2, 3]
    wc = proj[3, 2] * ze + proj[3, 3]
    return zc / wc
