"""vdi_stats: what a resident VDI holds (bytes by array against the closed
forms of its layout and the paper's sizes, Sections 5 and 6.3) and the totals
of its last counted frame (rays that met a list, lists passed through,
supersegment pieces composited) against the per-ray counters of the same
frame and the FP64 oracle's."""
import math
import os

import numpy as np
import pytest

import vdi_synth as S
from helpers import random_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


@pytest.mark.parametrize("fmt", [0, 1])
def test_stats_sizes(V, ctx, fmt):
    w, h, ns, T, nz = 45, 27, 7, 8, 12
    case = random_case(w, h, ns, seed=5)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, fmt, T=T, nz=nz), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        st = V.vdi_stats(vdi)
        nl, nsp = w * h, ns + (ns & 1)
        L = st.layout
        assert (st.w, st.h, st.n_s, st.colour_fmt, st.grid_tile) == (w, h, ns, fmt, T)
        assert L.n_s_stored == nsp and (L.grid_w, L.grid_h, L.grid_nz) == (math.ceil(w / T), math.ceil(h / T), nz)
        assert L.depth_bytes == nsp // 2 * nl * 16  # (f, b) pairs of FP32, two slots per 16 B
        assert L.colour_bytes == (nsp * nl * 16 if fmt == 0 else nsp // 2 * nl * 16)
        assert L.grid_bytes == nz * L.grid_w * L.grid_h * 4
        assert L.paper_bytes == ns * nl * 24  # Section 5: RGBA32F + 2 x R32F per slot
        assert L.total_bytes >= L.depth_bytes + L.colour_bytes + L.grid_bytes + L.list_bytes
        got = V.vdi_get_layout(vdi)
        assert all(getattr(got, f) == getattr(L, f) for f, _ in L._fields_)
        assert st.frame_recorded == 0 and st.lists == 0
    finally:
        V.vdi_destroy(vdi)


def test_stats_grid_size_at_full_hd(V, ctx):
    """Section 6.3: the empty-space grid of a 1920 x 1080 VDI is 2.5 MiB."""
    gold = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_sizes.txt")):
        if line.strip() and not line.startswith("#"):
            k, v, unit = line.split()[:3]
            gold[k] = float(v) * 2**20
    d = V.desc(1920, 1080, 20, np.eye(4), np.eye(4), (0, 0, 0), (1, 1, 1), 1.0, V.VDI_F16)
    L = V.vdi_layout_bytes(d)
    assert abs(L.grid_bytes / gold["grid_1920x1080"] - 1) < 0.02


@pytest.mark.parametrize("no_ert", [True, False])
def test_stats_frame_totals(V, ctx, orc, no_ert):
    case = random_case(29, 17, 4, seed=3, u=0.2)
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 1), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        for (az, el, d_i) in ((20.0, 10.0, 1), (-45.0, 25.0, 1), (150.0, -15.0, 2)):
            W, H = 48, 40
            Wr, Hr = -(-W // d_i), -(-H // d_i)
            cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=az, el_deg=el)
            cam = V.camera(cn.view, cn.proj)
            out = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
            V.vdi_render_ex(vdi, cam, W, H, d_i, 1, out, no_ert=no_ert, record_stats=True)  # temporary counters
            st = V.vdi_stats(vdi)
            rl = torch.zeros((Hr, Wr), dtype=torch.int32, device="cuda")
            rs = torch.zeros((Hr, Wr), dtype=torch.int32, device="cuda")
            V.vdi_render_ex(vdi, cam, W, H, d_i, 1, out, no_ert=no_ert, ray_lists=rl, ray_segs=rs, record_stats=True)
            st2 = V.vdi_stats(vdi)
            gl, gs = rl.cpu().numpy().reshape(-1), rs.cpu().numpy().reshape(-1)
            for s in (st, st2):
                assert s.frame_recorded == 1 and (s.frame_w, s.frame_h) == (Wr, Hr)
                assert s.lists == gl.sum() and s.pieces == gs.sum() and s.rays_hit == (gl > 0).sum()
            _, nl, nsg, fl = orc.render_exact(sc, cn.view, cn.proj, Wr, Hr)
            ok = fl == 0
            assert np.array_equal(gl[ok], nl[ok])
            if no_ert:
                assert np.array_equal(gs[ok], nsg[ok])
            else:
                assert np.all(gs[ok] <= nsg[ok]) and st.pieces <= nsg.sum()  # early termination can end rays
            assert st.rays_hit > 100
        with pytest.raises(V.VdiError):  # previews are not counted
            V.vdi_render_ex(vdi, cam, W, H, 1, 2, out, record_stats=True)
    finally:
        V.vdi_destroy(vdi)
