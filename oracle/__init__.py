"""Python handle on the FP64 CPU oracle (``vdi_oracle.c``).

TEST INFRASTRUCTURE, NOT PRODUCT: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It never
imports the CUDA package and the CUDA package never imports it.

``build()`` compiles the C source with gcc (``-ffp-contract=off`` so that the
FP64 arithmetic is evaluated exactly as written, OpenMP for the pixel loops).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vdi_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    srcs = [_SRC] + [os.path.join(_HERE, f) for f in sorted(os.listdir(_HERE))
                     if f.endswith(".c") and f != "vdi_oracle.c"]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fvisibility=hidden", "-Wall", "-Wno-unknown-pragmas", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcVdi(C.Structure):
    _fields_ = [("w", C.c_int), ("h", C.c_int), ("ns", C.c_int),
                ("view_o", C.c_double * 16), ("proj_o", C.c_double * 16),
                ("bmin", C.c_double * 3), ("bmax", C.c_double * 3), ("u", C.c_double),
                ("rgba", C.c_void_p), ("depth", C.c_void_p), ("counts", C.c_void_p)]


class OrcView(C.Structure):
    _fields_ = [("view", C.c_double * 16), ("proj", C.c_double * 16), ("W", C.c_int), ("H", C.c_int)]


class OrcVolume(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dtype", C.c_int),
                ("data", C.c_void_p), ("bmin", C.c_double * 3), ("bmax", C.c_double * 3)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        L.orc_render_exact.argtypes = [P, P, P, C.c_int, P, P, P, P, C.c_int]
        L.orc_render_sampled.argtypes = [P, P, C.c_double, P, C.c_int, P, C.c_int]
        L.orc_render_direct.argtypes = [P, P]
        L.orc_grid_edges.argtypes = [P, C.c_int, P]
        L.orc_grid_counts.argtypes = [P, C.c_int, C.c_int, P]
        L.orc_render_preview.argtypes = [P, P, C.c_int, C.c_int, C.c_int, P, P, C.c_int, P, P, C.c_int]
        L.orc_render_preview_alt.argtypes = [P, P, C.c_int, C.c_int, C.c_int, P, P, C.c_int, P, P, P, C.c_int]
        L.orc_render_exact_ndc.argtypes = [P, P, P, C.c_int, P, P, P, P, C.c_int]
        L.orc_touch_exact.argtypes = [P, P, P, C.c_int, C.c_int, P, P, P, P]
        L.orc_upsample.argtypes = [P, C.c_int, C.c_int, P, C.c_int, C.c_int]
        L.orc_first_index.argtypes = [P, P, C.c_int, C.c_float, C.c_float, C.c_int]
        L.orc_first_index.restype = C.c_int
        L.orc_generate.argtypes = [P, P, C.c_int, P, P, C.c_int, C.c_int, C.c_int, C.c_double,
                                   C.c_double, C.c_double, C.c_int, C.c_int, P, P, P, P, C.c_int]
        L.orc_dvr.argtypes = [P, P, C.c_int, P, P, C.c_int, C.c_int, C.c_double, C.c_double,
                              C.c_int, P, P, C.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _cm(m):
    m = np.asarray(m, np.float64)
    if m.shape == (4, 4):
        m = np.ascontiguousarray(m.T).reshape(16)
    return (C.c_double * 16)(*m.tolist())


class Scene:
    """A VDI in ABI layout plus its original camera, box and length unit."""

    def __init__(self, vdi, view_o, proj_o, bmin, bmax, u, use_counts=True):
        self.rgba = np.ascontiguousarray(vdi.rgba, np.float32)
        self.depth = np.ascontiguousarray(vdi.depth, np.float32)
        self.counts = np.ascontiguousarray(vdi.counts, np.int32) if use_counts else None
        self.w, self.h, self.ns = vdi.w, vdi.h, vdi.ns
        s = OrcVdi()
        s.w, s.h, s.ns = vdi.w, vdi.h, vdi.ns
        s.view_o, s.proj_o = _cm(view_o), _cm(proj_o)
        s.bmin = (C.c_double * 3)(*map(float, bmin))
        s.bmax = (C.c_double * 3)(*map(float, bmax))
        s.u = float(u)
        s.rgba, s.depth, s.counts = _ptr(self.rgba), _ptr(self.depth), _ptr(self.counts)
        self.s = s


def _view(view, proj, W, H):
    v = OrcView()
    v.view, v.proj, v.W, v.H = _cm(view), _cm(proj), int(W), int(H)
    return v


def _pix(pix, W, H):
    if pix is None:
        return None, W * H
    p = np.ascontiguousarray(pix, np.int32)
    return p, len(p)


def render_exact(scene, view, proj, W, H, pix=None, nthreads=None):
    """Returns (rgba[n,4] f64, n_lists[n] i32, n_segs[n] i32, flags[n] u8)."""
    nthreads = nthreads or os.cpu_count()
    p, n = _pix(pix, W, H)
    out = np.zeros((n, 4), np.float64)
    nl = np.zeros(n, np.int32)
    ns = np.zeros(n, np.int32)
    fl = np.zeros(n, np.uint8)
    v = _view(view, proj, W, H)
    rc = lib().orc_render_exact(C.byref(scene.s), C.byref(v), _ptr(p), n, _ptr(out), _ptr(nl),
                                _ptr(ns), _ptr(fl), nthreads)
    assert rc == 0
    return out, nl, ns, fl


def render_sampled(scene, view, proj, W, H, h_world, pix=None, nthreads=None):
    nthreads = nthreads or os.cpu_count()
    p, n = _pix(pix, W, H)
    out = np.zeros((n, 4), np.float64)
    v = _view(view, proj, W, H)
    rc = lib().orc_render_sampled(C.byref(scene.s), C.byref(v), float(h_world), _ptr(p), n,
                                  _ptr(out), nthreads)
    assert rc == 0
    return out


def render_direct(scene):
    out = np.zeros((scene.h * scene.w, 4), np.float64)
    assert lib().orc_render_direct(C.byref(scene.s), _ptr(out)) == 0
    return out


def grid_edges(scene, nz):
    e = np.zeros(nz + 1, np.float32)
    lib().orc_grid_edges(C.byref(scene.s), nz, _ptr(e))
    return e


def grid_counts(scene, T=8, nz=20):
    gw, gh = -(-scene.w // T), -(-scene.h // T)
    g = np.zeros((nz, gh, gw), np.uint32)
    lib().orc_grid_counts(C.byref(scene.s), T, nz, _ptr(g))
    return g


def render_preview(scene, view, proj, W, H, d_r, T=8, nz=20, grid=None, pix=None, nthreads=None):
    """D_R preview at W x H.  Returns (rgba[n,4] f64, flags[n] u8)."""
    nthreads = nthreads or os.cpu_count()
    if grid is None:
        grid = grid_counts(scene, T, nz)
    grid = np.ascontiguousarray(grid, np.uint32)
    p, n = _pix(pix, W, H)
    out = np.zeros((n, 4), np.float64)
    fl = np.zeros(n, np.uint8)
    v = _view(view, proj, W, H)
    rc = lib().orc_render_preview(C.byref(scene.s), C.byref(v), int(d_r), int(T), int(nz),
                                  _ptr(grid), _ptr(p), n, _ptr(out), _ptr(fl), nthreads)
    assert rc == 0
    return out, fl


def render_preview_alt(scene, view, proj, W, H, d_r, T, nz, grid, pix, alt, nthreads=None):
    """D_R preview of the pixels ``pix`` with near-tie decisions flipped: pixel q
    flips the decisions whose bits are set in ``alt[q]`` (alt = 0: the plain
    rule).  Returns (rgba[n,4] f64, number of tie decisions each ray met)."""
    nthreads = nthreads or os.cpu_count()
    grid = np.ascontiguousarray(grid, np.uint32)
    p = np.ascontiguousarray(pix, np.int32)
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(alt, np.uint32), p.shape), np.uint32)
    out = np.zeros((len(p), 4), np.float64)
    nt = np.zeros(len(p), np.int32)
    v = _view(view, proj, W, H)
    rc = lib().orc_render_preview_alt(C.byref(scene.s), C.byref(v), int(d_r), int(T), int(nz), _ptr(grid), _ptr(p),
                                      len(p), _ptr(a), _ptr(out), _ptr(nt), nthreads)
    assert rc == 0
    return out, nt


def render_exact_ndc(scene, view, proj, xy, nthreads=None):
    """Exact render of rays through V_N NDC points xy[n, 2].  Returns
    (rgba[n,4] f64, n_lists, n_segs, flags) as render_exact."""
    nthreads = nthreads or os.cpu_count()
    xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    n = len(xy)
    out = np.zeros((n, 4), np.float64)
    nl = np.zeros(n, np.int32)
    ns = np.zeros(n, np.int32)
    fl = np.zeros(n, np.uint8)
    v = _view(view, proj, 1, 1)
    rc = lib().orc_render_exact_ndc(C.byref(scene.s), C.byref(v), _ptr(xy), n, _ptr(out), _ptr(nl), _ptr(ns),
                                    _ptr(fl), nthreads)
    assert rc == 0
    return out, nl, ns, fl


def touch_exact(scene, view, proj, W, H, pix=None):
    """Replay of the exact render's access rule (Section 4.2, Algorithm 2) over
    the rays of ``pix`` (all pixels if None).  Returns (depth[h*w, nsp, 2],
    colour[h*w, nsp], range[h*w]) boolean masks of what the rays read, and the
    per-ray flags of reads that turn on a near-tie decision."""
    nsp = scene.ns + (scene.ns & 1)
    nl = scene.w * scene.h
    p, n = _pix(pix, W, H)
    dm = np.zeros((nl, nsp, 2), np.uint8)
    cm = np.zeros((nl, nsp), np.uint8)
    rm = np.zeros(nl, np.uint8)
    fl = np.zeros(n, np.uint8)
    v = _view(view, proj, W, H)
    rc = lib().orc_touch_exact(C.byref(scene.s), C.byref(v), _ptr(p), n, nsp, _ptr(dm), _ptr(cm), _ptr(rm), _ptr(fl))
    assert rc == 0
    return dm.astype(bool), cm.astype(bool), rm.astype(bool), fl


def upsample(lo, w0, h0, W, H):
    lo = np.ascontiguousarray(lo, np.float64).reshape(h0 * w0, 4)
    hi = np.zeros((H * W, 4), np.float64)
    lib().orc_upsample(_ptr(lo), w0, h0, _ptr(hi), W, H)
    return hi


def first_index(f, b, d_entry, d_exit, increasing=True):
    f = np.ascontiguousarray(f, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    return lib().orc_first_index(_ptr(f), _ptr(b), len(f), float(d_entry), float(d_exit),
                                 1 if increasing else 0)


class Volume:
    """A scalar volume filling the box [bmin, bmax]; data[z, y, x] of uint8, uint16 or float32."""

    def __init__(self, data, bmin, bmax):
        self.data = np.ascontiguousarray(data)
        dt = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float32): 2}[self.data.dtype]
        v = OrcVolume()
        v.nz, v.ny, v.nx = self.data.shape
        v.dtype = dt
        v.data = self.data.ctypes.data_as(C.c_void_p)
        v.bmin = (C.c_double * 3)(*map(float, bmin))
        v.bmax = (C.c_double * 3)(*map(float, bmax))
        self.v = v


def generate(volume, knots, view, proj, w, h, ns, tau, step, u, fp32=False, nthreads=None, adaptive=False,
             with_tau=False):
    """VDI generation (Eq. 1 with fixed gamma = tau, or with ``adaptive`` the
    per-ray gamma of Algorithm 3).  Returns VdiArrays-like (rgba, depth,
    counts), plus the gamma each list used with ``with_tau``."""
    nthreads = nthreads or os.cpu_count()
    knots = np.ascontiguousarray(knots, np.float32)
    rgba = np.zeros((h, w, ns, 4), np.float32)
    depth = np.zeros((h, w, ns, 2), np.float32)
    counts = np.zeros((h, w), np.int32)
    taus = np.zeros((h, w), np.float32)
    rc = lib().orc_generate(C.byref(volume.v), _ptr(knots), len(knots), _ptr(_cmarr(view)), _ptr(_cmarr(proj)),
                            w, h, ns, float(tau), float(step), float(u), 1 if fp32 else 0, 1 if adaptive else 0,
                            _ptr(rgba), _ptr(depth), _ptr(counts), _ptr(taus), nthreads)
    assert rc == 0, "unsupported camera or transfer function"
    return (rgba, depth, counts, taus) if with_tau else (rgba, depth, counts)


def dvr(volume, knots, view, proj, w, h, step, u, fp32=False, nthreads=None, with_flags=False):
    """Emission-absorption DVR through the V_O pixel centres at the generation samples.

    With ``with_flags`` also returns per-ray flags marking rays whose sample
    count floor(L / step) sits within 1e-4 of a rounding boundary."""
    nthreads = nthreads or os.cpu_count()
    knots = np.ascontiguousarray(knots, np.float32)
    out = np.zeros((h * w, 4), np.float64)
    fl = np.zeros(h * w, np.uint8)
    rc = lib().orc_dvr(C.byref(volume.v), _ptr(knots), len(knots), _ptr(_cmarr(view)), _ptr(_cmarr(proj)), w, h,
                       float(step), float(u), 1 if fp32 else 0, _ptr(out), _ptr(fl), nthreads)
    assert rc == 0
    return (out, fl) if with_flags else out


def _cmarr(m):
    m = np.asarray(m, np.float64)
    if m.shape == (4, 4):
        m = m.T
    return np.ascontiguousarray(m).reshape(16)
