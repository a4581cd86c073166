"""vdi_touch_bitmap -- the words of the VDI an exact render reads, whose
popcount is the roofline numerator -- against the oracle's replay of the same
access rule (Section 4.2, Algorithm 2), ray by ray and for whole frames.

Each ray is rendered alone: a 1 x 1 image whose frustum is shifted so that its
single pixel-centre ray is the ray of pixel q of the W x H view.  Its bitmap,
decoded through the layout the header documents (depth array, colour array,
grid, list ranges), must equal the oracle's replay on every ray the replay
does not flag (a read that turns on a near tie).  A whole frame's bitmap must
hold every word the unflagged rays read, and little else.
"""
import numpy as np
import pytest

import vdi_synth as S
from helpers import pixel_ndc, random_case

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


def shifted_camera(cam, W, H, q):
    """A camera whose 1 x 1 image's pixel-centre ray is pixel q's ray of ``cam`` at W x H."""
    x, y = pixel_ndc(q, W, H)
    sh = np.eye(4)
    sh[0, 3], sh[1, 3] = -x, -y  # clip x' = x - x0 w, y' = y - y0 w
    return S.Camera(cam.view, sh @ cam.proj, cam.eye)


def touch_words(V, vdi):
    L = V.vdi_get_layout(vdi)
    grid_words = (L.grid_w * L.grid_h * L.grid_nz + 3) // 4 * 4
    return L, ((L.depth_bytes + L.colour_bytes) // 4 + grid_words + L.list_bytes // 4 + 31) // 32


def decode(bm, L, nl, fmt):
    """Bitmap -> (depth[nl, nsp, 2], colour[nl, nsp], range[nl]) masks by the documented layout."""
    nsp = L.n_s_stored
    bits = np.unpackbits(np.ascontiguousarray(bm).view(np.uint8), bitorder="little")
    w = np.nonzero(bits)[0]
    D = L.depth_bytes // 4
    C = L.colour_bytes // 4
    G = (L.grid_w * L.grid_h * L.grid_nz + 3) // 4 * 4
    depth = np.zeros((nl, nsp, 2), bool)
    colour = np.zeros((nl, nsp), bool)
    rng = np.zeros(nl, bool)
    dw = w[w < D]
    rec, within = dw // 4, dw % 4
    depth[rec % nl, 2 * (rec // nl) + within // 2, within % 2] = True
    cw = w[(w >= D) & (w < D + C)] - D
    rec = cw // 4
    if fmt == 0:  # one 16-byte (r, g, b, kappa) record per slot
        colour[rec % nl, rec // nl] = True
        per_slot = 4
    else:  # two half4 records per 16 bytes
        colour[rec % nl, 2 * (rec // nl) + (cw % 4) // 2] = True
        per_slot = 2
    assert not np.any((w >= D + C) & (w < D + C + G)), "the exact path reads no grid cell"
    rw = w[w >= D + C + G] - (D + C + G)
    assert np.all(rw < 2 * nl)
    rng[rw // 2] = True
    # every slot's colour read covers its whole record, a range read both of its words
    assert len(w) == depth.sum() + per_slot * colour.sum() + 2 * rng.sum()
    return depth, colour, rng


def gpu_touch(V, vdi, cam, W, H, L, words, nl, fmt):
    bm = torch.zeros(words, dtype=torch.int32, device="cuda")
    V.vdi_touch_bitmap(vdi, V.camera(cam.view, cam.proj), W, H, bm)
    torch.cuda.synchronize()
    return decode(bm.cpu().numpy(), L, nl, fmt)


VIEWS = [(25.0, 10.0, 1.2, False), (-60.0, 25.0, 1.0, False), (150.0, -15.0, 1.1, False), (30.0, 15.0, 1.2, True),
         (0.0, 15.0, 1.4, False)]


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("ns", [5, 8])
def test_touch_bitmap_matches_oracle_replay_per_ray(V, ctx, orc, fmt, ns):
    case = random_case(20, 14, ns, seed=30 + ns, u=0.1, alpha_range=(0.05, 0.9), fill=0.9)
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, fmt), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        L, words = touch_words(V, vdi)
        nl = 20 * 14
        assert L.n_s_stored == ns + (ns & 1)
        rays = terminated = 0
        for (az, el, zoom, ortho) in VIEWS:
            W, H = 31, 23
            cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=az, el_deg=el, zoom=zoom, ortho=ortho)
            _, _, _, fl = orc.touch_exact(sc, cn.view, cn.proj, W, H)
            ref = orc.render_exact(sc, cn.view, cn.proj, W, H)[0]
            rng = np.random.default_rng(int(az) + 1000)
            cand = np.nonzero((fl == 0) & (ref[:, 3] > 0))[0]
            for q in rng.permutation(cand)[:40]:
                od, oc, orr, _ = orc.touch_exact(sc, cn.view, cn.proj, W, H, pix=[q])
                gd, gc, gr = gpu_touch(V, vdi, shifted_camera(cn, W, H, q), 1, 1, L, words, nl, fmt)
                assert np.array_equal(gr, orr), (az, q, np.nonzero(gr ^ orr))
                assert np.array_equal(gd, od), (az, q, np.argwhere(gd ^ od))
                assert np.array_equal(gc, oc), (az, q, np.argwhere(gc ^ oc))
                rays += 1
                terminated += ref[q, 3] > 1 - 2 ** -12
        assert rays > 150 and terminated > 5
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("fmt", [0, 1])
def test_touch_bitmap_of_a_frame(V, ctx, orc, fmt):
    case = random_case(24, 16, 6, seed=41, u=0.1, alpha_range=(0.05, 0.9), fill=0.9)
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, fmt), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        L, words = touch_words(V, vdi)
        nl = 24 * 16
        for (az, el, zoom, ortho) in VIEWS:
            W, H = 40, 27
            cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=az, el_deg=el, zoom=zoom, ortho=ortho)
            _, _, _, fl = orc.touch_exact(sc, cn.view, cn.proj, W, H)
            ok = np.nonzero(fl == 0)[0]
            od, oc, orr, _ = orc.touch_exact(sc, cn.view, cn.proj, W, H, pix=ok)
            ad, ac, ar, _ = orc.touch_exact(sc, cn.view, cn.proj, W, H)
            gd, gc, gr = gpu_touch(V, vdi, cn, W, H, L, words, nl, fmt)
            # every word an unflagged ray reads is in the frame's bitmap ...
            assert not np.any(od & ~gd) and not np.any(oc & ~gc) and not np.any(orr & ~gr), az
            # ... and the frame reads nothing beyond what some ray of the view reads,
            # up to the few words a flagged ray's tie decisions move
            extra = (gd & ~ad).sum() + (gc & ~ac).sum() + (gr & ~ar).sum()
            assert extra <= 4 * max(1, int((fl != 0).sum())), (az, extra)
    finally:
        V.vdi_destroy(vdi)
