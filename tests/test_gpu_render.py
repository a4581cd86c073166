"""GPU parity of the render path against the FP64 oracle, through the C ABI.

Covers the exact path (Section 4.1-4.2: list walk, Algorithm 2, Eq. 2,
compositing) for perspective and orthographic new views, depth increasing and
decreasing along rays (views beyond 90 degrees), several tiles with ragged
tails, FP32 and FP16 colour storage; bit-exact integer results (first-index
contract, per-ray list/supersegment counters on rays the oracle does not
flag, count grid, create/download round trip); and error reporting.
"""
import numpy as np
import pytest

import vdi_synth as S
from helpers import TOL, Case, check_exact, check_tolerance, exact_alternatives, random_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    import paper_2206_08660_gb300 as V

    V.load()
    return V


@pytest.fixture(scope="module")
def ctx(V):
    assert torch.cuda.is_available()
    c = V.vdi_ctx_create(0)
    yield c
    V.vdi_ctx_destroy(c)


def gpu_render(V, vdi, cam, W, H, d_i=1, d_r=1, counters=False, **kw):
    out = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    Hr, Wr = -(-H // d_i), -(-W // d_i)
    rl = rs = None
    if counters:
        rl = torch.zeros((Hr, Wr), dtype=torch.int32, device="cuda")
        rs = torch.zeros((Hr, Wr), dtype=torch.int32, device="cuda")
    V.vdi_render_ex(vdi, V.camera(cam.view, cam.proj), W, H, d_i, d_r, out, V.VDI_F32, ray_lists=rl,
                    ray_segs=rs, **kw)
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(-1, 4)
    if counters:
        return o, rl.cpu().numpy().reshape(-1), rs.cpu().numpy().reshape(-1)
    return o


VIEWS = [  # (azimuth, elevation, zoom, ortho)
    (10.0, 15.0, 1.0, False),
    (-35.0, 5.0, 1.2, False),
    (60.0, 40.0, 1.5, False),
    (150.0, -20.0, 1.0, False),  # more than 90 degrees away: depth decreases along rays
    (25.0, 30.0, 1.0, True),
    (0.0, 15.0, 1.0, False),  # the original direction
]


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("seed", [0, 1])
def test_exact_render_matches_oracle(V, ctx, orc, fmt, seed):
    case = random_case(37, 23, 5, seed=seed, u=0.15, alpha_range=(0.05, 0.8))
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, fmt), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        for (az, el, zoom, ortho) in VIEWS:
            W, H = 70, 45  # 3 x 6 tiles of 32 x 8 with ragged edges
            cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=az, el_deg=el, zoom=zoom, ortho=ortho)
            ref = orc.render_exact(sc, cn.view, cn.proj, W, H)[0]
            got = gpu_render(V, vdi, cn, W, H)
            assert ref[:, 3].max() > 0.2, "view shows nothing"
            check_tolerance(got, ref, fmt, what=f"view {az},{el}")
            assert np.all(got[:, :3] <= got[:, 3:4] + 1e-5) and np.all(got >= 0) and np.all(got[:, 3] <= 1 + 1e-6)
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("fmt", [0, 1])
def test_original_frustum_cuts_the_box(V, ctx, orc, fmt):
    """V_O zoomed in so that its frustum cuts the volume box: the render clips
    every ray to V_O's frustum as well as to the box (Section 4.1).  With this
    zoom some rays of the view along V_O's direction run exactly along a list
    boundary, where the field is discontinuous and both sides are valid
    limits; the oracle flags them, and they must match the oracle on a ray
    through the pixel centre moved by a thousandth of a pixel."""
    bmin, bmax = np.zeros(3), np.ones(3)
    vdi = S.random_vdi(37, 23, 5, seed=11, alpha_range=(0.05, 0.8))
    cam_o = S.orbit_camera(bmin, bmax, 37 / 23, az_deg=0.0, el_deg=15.0, zoom=1.8)
    case = Case(vdi, cam_o, bmin, bmax, 0.15)
    sc = case.oracle_scene(orc)
    g = V.vdi_create(ctx, case.gpu_desc(V, fmt), vdi.rgba, vdi.depth, vdi.counts)
    try:
        for (az, el, zoom, ortho) in VIEWS:
            W, H = 70, 45
            cn = S.orbit_camera(bmin, bmax, W / H, az_deg=az, el_deg=el, zoom=zoom, ortho=ortho)
            ref, _, _, fl = orc.render_exact(sc, cn.view, cn.proj, W, H)
            got = gpu_render(V, g, cn, W, H)
            assert ref[:, 3].max() > 0.2, "view shows nothing"
            frac, _ = check_exact(orc, sc, cn, W, H, got, fmt, ref, fl, what=f"view {az},{el}")
            assert frac < 0.05
    finally:
        V.vdi_destroy(g)


def test_counters_bit_exact_on_unflagged_rays(V, ctx, orc):
    case = random_case(29, 17, 4, seed=3, u=0.2)
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 0), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        total = 0
        for (az, el, zoom, ortho) in VIEWS:
            W, H = 48, 40
            cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=az, el_deg=el, zoom=zoom, ortho=ortho)
            _, nl, nsg, fl = orc.render_exact(sc, cn.view, cn.proj, W, H)
            _, gl, gs = gpu_render(V, vdi, cn, W, H, counters=True, no_ert=True)
            ok = fl == 0
            assert ok.mean() > 0.9
            assert np.array_equal(gl[ok], nl[ok]), np.nonzero(gl[ok] != nl[ok])
            assert np.array_equal(gs[ok], nsg[ok])
            total += int(nl[ok].sum())
            # a flagged ray's counters equal the plain oracle's or those of a ray
            # through its pixel centre moved by a thousandth of a pixel
            idx = np.nonzero(~ok)[0]
            if len(idx):
                _, anl, ans = exact_alternatives(orc, sc, cn, W, H, idx)
                ml = (gl[idx] == nl[idx]) | np.any(anl == gl[idx][None], axis=0)
                ms = (gs[idx] == nsg[idx]) | np.any(ans == gs[idx][None], axis=0)
                assert ml.all() and ms.all(), (idx[~ml], idx[~ms])
        assert total > 1000
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("search", [0, 1, 2])
def test_search_modes_and_warp_shapes_give_identical_images(V, ctx, search):
    case = random_case(40, 30, 6, seed=7)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 0), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        cn = S.orbit_camera(case.bmin, case.bmax, 1.0, az_deg=30, el_deg=20)
        base = gpu_render(V, vdi, cn, 64, 64)
        for ws in (0, 1, 2, 3):
            got = gpu_render(V, vdi, cn, 64, 64, search=search, warp_shape=ws)
            assert np.array_equal(got, base)
    finally:
        V.vdi_destroy(vdi)


def test_first_index_contract_bit_exact(V, ctx, orc):
    rng = np.random.default_rng(11)
    for ns in (1, 2, 5, 8, 20):
        w = 64
        case = random_case(w, 1, ns, seed=ns, fill=1.0)
        vdi = V.vdi_create(ctx, case.gpu_desc(V, 0), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
        try:
            for li in range(0, w, 7):
                n = int(case.vdi.counts[0, li])
                f = case.vdi.depth[0, li, :n, 0]
                b = case.vdi.depth[0, li, :n, 1]
                q = 4000
                pts = np.concatenate([f, b, np.float32([-1.0, 1.0])])
                d0 = np.where(rng.random(q) < 0.3, rng.choice(pts, q), rng.uniform(-1, 1, q)).astype(np.float32)
                d1 = np.where(rng.random(q) < 0.3, rng.choice(pts, q), rng.uniform(-1, 1, q)).astype(np.float32)
                inc = (rng.random(q) < 0.5).astype(np.int32)
                lo, hi = np.minimum(d0, d1), np.maximum(d0, d1)
                de = np.where(inc == 1, lo, hi).astype(np.float32)
                dx = np.where(inc == 1, hi, lo).astype(np.float32)
                seed = rng.integers(-1, ns + 1, q).astype(np.int32)
                expect = np.array([orc.first_index(f, b, de[i], dx[i], bool(inc[i])) for i in range(q)])
                for mode in (0, 1, 2):
                    res = torch.zeros(q, dtype=torch.int32, device="cuda")
                    t = lambda a: torch.from_numpy(a).cuda()
                    V.vdi_search_first(vdi, li, mode, t(de), t(dx), t(seed), t(inc), res)
                    torch.cuda.synchronize()
                    assert np.array_equal(res.cpu().numpy(), expect), (ns, li, mode)
        finally:
            V.vdi_destroy(vdi)


@pytest.mark.parametrize("fmt", [0, 1])
def test_create_download_roundtrip_and_grid(V, ctx, orc, fmt):
    case = random_case(45, 27, 7, seed=5)  # grid cells: ragged in x and y
    vdi = V.vdi_create(ctx, case.gpu_desc(V, fmt, T=8, nz=12), case.vdi.rgba, case.vdi.depth, None)
    try:
        rgba, depth, counts, grid = V.vdi_download(vdi, 45, 27, 7)
        assert np.array_equal(counts, case.vdi.counts)
        valid = np.arange(7)[None, None, :] < case.vdi.counts[:, :, None]
        assert np.array_equal(depth[valid], case.vdi.depth[valid])
        assert np.all(np.isinf(depth[~valid]))
        tol = 2e-6 if fmt == 0 else 2e-3
        assert np.abs(rgba[valid] - case.vdi.rgba[valid]).max() < tol
        assert np.all(rgba[~valid] == 0)
        ref = orc.grid_counts(case.oracle_scene(orc), 8, 12)
        assert np.array_equal(grid, ref)
    finally:
        V.vdi_destroy(vdi)


def test_empty_vdi_and_view_that_misses(V, ctx):
    case = random_case(16, 16, 4, seed=0, fill=0.0)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 0), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        cn = S.orbit_camera(case.bmin, case.bmax, 1.0, az_deg=20)
        assert np.all(gpu_render(V, vdi, cn, 40, 40) == 0)
    finally:
        V.vdi_destroy(vdi)
    case = random_case(16, 16, 4, seed=1)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 0), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        away = S.Camera(S.look_at(case.cam_o.eye, 2 * case.cam_o.eye - 0.5), case.cam_o.proj, case.cam_o.eye)
        assert np.all(gpu_render(V, vdi, away, 40, 40) == 0)
    finally:
        V.vdi_destroy(vdi)


def test_invalid_inputs_are_reported(V, ctx):
    case = random_case(8, 8, 4, seed=2, fill=1.0)
    bad = case.vdi.depth.copy()
    bad[3, 3, 0] = (0.5, 0.1)  # front behind back
    with pytest.raises(V.VdiError) as e:
        V.vdi_create(ctx, case.gpu_desc(V, 0), case.vdi.rgba, bad, case.vdi.counts)
    assert e.value.status == 4
    badc = case.vdi.rgba.copy()
    badc[2, 2, 0] = (0.9, 0.1, 0.1, 0.5)  # rgb above alpha: not premultiplied
    with pytest.raises(V.VdiError) as e:
        V.vdi_create(ctx, case.gpu_desc(V, 0), badc, case.vdi.depth, case.vdi.counts)
    assert e.value.status == 1
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 0), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        out = torch.zeros((4, 4, 4), device="cuda")
        cam = S.orbit_camera(case.bmin, case.bmax, 1.0)
        for args in [(0, 4, 1, 1), (4, 4, 0, 1), (4, 4, 1, 17)]:
            with pytest.raises(V.VdiError):
                V.vdi_render(vdi, V.camera(cam.view, cam.proj), args[0], args[1], args[2], args[3], out)
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("fmt", [0, 1])
def test_empty_space_skipping_matches_oracle(V, ctx, orc, fmt):
    """Section 4.3: cells whose count is 0 hold no supersegment, so skipping them
    leaves the image unchanged, up to where early termination lands: pieces
    split at cell boundaries can stop the ray one piece earlier, and whatever
    follows a transmittance of 2^-12 weighs at most 2^-12.  The skipping
    render also matches the FP64 oracle at the render tolerances."""
    for seed, fill in ((4, 0.3), (5, 0.9)):
        case = random_case(96, 64, 6, seed=seed, fill=fill)
        sc = case.oracle_scene(orc)
        vdi = V.vdi_create(ctx, case.gpu_desc(V, fmt, T=8, nz=16), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
        try:
            for (az, el, zoom, ortho) in VIEWS:
                cn = S.orbit_camera(case.bmin, case.bmax, 1.25, az_deg=az, el_deg=el, zoom=zoom, ortho=ortho)
                a = gpu_render(V, vdi, cn, 80, 64, ess=True)
                b = gpu_render(V, vdi, cn, 80, 64)
                assert np.abs(a - b).max() <= 2.0 ** -12, (seed, az)
                check_exact(orc, sc, cn, 80, 64, a, fmt, what=f"ESS seed {seed} view {az},{el}")
        finally:
            V.vdi_destroy(vdi)


@pytest.mark.parametrize("fmt", [0, 1])
def test_range_block_skipping_is_bit_identical(V, ctx, fmt):
    """A 4 x 4 block of lists whose merged depth range the ray misses holds no
    supersegment the ray meets, so skipping it changes no bit of the image."""
    for seed, fill in ((6, 0.2), (7, 0.8)):
        case = random_case(90, 70, 5, seed=seed, fill=fill)
        vdi = V.vdi_create(ctx, case.gpu_desc(V, fmt), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
        try:
            for (az, el, zoom, ortho) in VIEWS:
                cn = S.orbit_camera(case.bmin, case.bmax, 1.25, az_deg=az, el_deg=el, zoom=zoom, ortho=ortho)
                a = gpu_render(V, vdi, cn, 85, 66, blocks=True)
                b = gpu_render(V, vdi, cn, 85, 66)
                assert np.array_equal(a, b), (seed, az)
        finally:
            V.vdi_destroy(vdi)


@pytest.mark.parametrize("w,h,ns", [(1, 1, 1), (3, 40, 1), (40, 3, 2), (17, 11, 64), (9, 7, 63)])
def test_extreme_list_counts_and_grid_shapes(V, ctx, orc, w, h, ns):
    """One list, one-list-wide grids, N_S = 1 and the largest N_S (64, and an
    odd 63 that leaves a padding slot), rendered from several views."""
    case = random_case(w, h, ns, seed=w * 100 + ns, u=0.2, alpha_range=(0.05, 0.6), fill=1.0)
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 0), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        shown = 0.0
        for (az, el, zoom, ortho) in VIEWS:
            W, H = 41, 33
            cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=az, el_deg=el, zoom=zoom, ortho=ortho)
            ref, _, _, fl = orc.render_exact(sc, cn.view, cn.proj, W, H)
            got = gpu_render(V, vdi, cn, W, H)
            shown = max(shown, float(ref[:, 3].max()))
            check_exact(orc, sc, cn, W, H, got, 0, ref, fl, what=f"{w}x{h} N_S={ns} view {az},{el}")
        assert shown > 0.05
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 77), (77, 1), (33, 9)])
def test_tiny_and_thin_images(V, ctx, orc, W, H):
    case = random_case(24, 16, 4, seed=5, u=0.2)
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 1), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=20.0, el_deg=10.0)
        ref, _, _, fl = orc.render_exact(sc, cn.view, cn.proj, W, H)
        check_exact(orc, sc, cn, W, H, gpu_render(V, vdi, cn, W, H), 1, ref, fl, what=f"{W}x{H}")
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("zoom", [0.3, 1.0, 1.4])
@pytest.mark.parametrize("ns", [9, 20])
def test_views_from_the_original_eye(V, ctx, orc, fmt, zoom, ns):
    """A new view from V_O's eye (any field of view) takes the one-list-per-ray
    path: its image is bit-identical to the general list walk (the counter
    kernel runs the walk) and matches the oracle.  N_S = 9 and 20 with lists
    of every fill give odd and even supersegment counts and one to three
    batches of slot pairs."""
    case = random_case(40, 30, ns, seed=17, u=0.15, alpha_range=(0.05, 0.8), fill=0.9)
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, fmt), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        W, H = 83, 61
        cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=0.0, el_deg=15.0, zoom=zoom)
        np.testing.assert_allclose(cn.eye, case.cam_o.eye)
        fast = gpu_render(V, vdi, cn, W, H)
        walk, _, _ = gpu_render(V, vdi, cn, W, H, counters=True)
        assert np.array_equal(fast, walk)
        ref, _, _, fl = orc.render_exact(sc, cn.view, cn.proj, W, H)
        assert ref[:, 3].max() > 0.3
        check_exact(orc, sc, cn, W, H, fast, fmt, ref, fl, what=f"eye view zoom {zoom}")
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("w,h,ns,fmt", [(70, 27, 9, 1), (70, 27, 20, 0), (70, 27, 20, 1), (64, 16, 4, 1),
                                         (64, 16, 4, 0), (45, 27, 9, 1), (70, 27, 2, 1), (16, 6, 4, 1)])
def test_original_view_with_staged_tiles(V, ctx, orc, w, h, ns, fmt):
    """Rendering from V_O's own camera at the VDI's resolution: pixel (x, y)'s
    ray stays in list (x, y), so each 32 x 8 tile of rays reads one 32 x 8
    tile of lists, whose ranges and first slot pairs the one-list path loads
    into shared memory by TMA (even w; w = 45 takes the unstaged one-list
    path).  Ragged tiles on the right and bottom edges, and a 16 x 6 VDI
    smaller than one tile; N_S = 2, 4 (fewer slot
    pairs than a tile stages), 9 and 20 (slot pairs beyond the staged ones
    from global memory); FP32 and FP16 colour.  The image is bit-identical to
    the general list walk, matches the oracle, and its FP16 output is the
    FP32 output rounded, and 4 x 8 warps (the unstaged kernel) give the same
    image; no wait for a staged tile ran out."""
    case = random_case(w, h, ns, seed=5, u=0.15, alpha_range=(0.05, 0.8), fill=0.9)
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, fmt), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        cn = case.cam_o
        fast = gpu_render(V, vdi, cn, w, h)
        walk, _, _ = gpu_render(V, vdi, cn, w, h, counters=True)
        assert np.array_equal(fast, walk)
        # 4 x 8 warps take the unstaged one-list kernel: the same image
        assert np.array_equal(gpu_render(V, vdi, cn, w, h, warp_shape=3), fast)
        half = torch.zeros((h, w, 4), dtype=torch.float16, device="cuda")
        V.vdi_render(vdi, V.camera(cn.view, cn.proj), w, h, 1, 1, half, V.VDI_F16)
        torch.cuda.synchronize()
        assert np.array_equal(half.cpu().numpy().reshape(-1, 4), fast.astype(np.float16))
        ref, _, _, fl = orc.render_exact(sc, cn.view, cn.proj, w, h)
        assert ref[:, 3].max() > 0.3
        check_exact(orc, sc, cn, w, h, fast, fmt, ref, fl, what=f"original view {w}x{h} N_S={ns}")
        assert V.vdi_stats(vdi).device_flags == 0
    finally:
        V.vdi_destroy(vdi)


@pytest.mark.parametrize("zoom,shift,W", [(0.35, 0.0, 203), (1.0, 0.45, 203), (0.35, 3.0, 203), (0.35, 0.0, 204),
                                          (1.0, 0.45, 204)])
def test_tiles_outside_the_box_image(V, ctx, orc, zoom, shift, W):
    """The render grid dispatches the tiles that meet the box's pixel
    rectangle first and clears the others in blocks of several tiles: with the
    box small on screen, cut by the image's left and bottom edges, or out of
    the view entirely (look-at point moved sideways by shift times the eye's
    distance), every pixel and both per-ray counters still match the oracle;
    the cleared pixels are transparent and their counters zero.  The clearing
    uses bulk stores where every row is 16-byte aligned (FP32 output, FP16
    output at an even width) and plain stores otherwise (counters, FP16 at an
    odd width): the FP16 image is the FP32 one rounded either way."""
    case = random_case(31, 19, 4, seed=21, u=0.2, alpha_range=(0.05, 0.8))
    sc = case.oracle_scene(orc)
    vdi = V.vdi_create(ctx, case.gpu_desc(V, 1), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    try:
        H = 91  # 7 x 12 tiles with ragged edges
        cn = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=12.0, el_deg=10.0, zoom=zoom)
        if shift:
            centre = 0.5 * (np.asarray(case.bmin) + np.asarray(case.bmax))
            side = np.cross(centre - cn.eye, (0.0, 1.0, 0.0))
            side *= np.linalg.norm(centre - cn.eye) / np.linalg.norm(side)
            cn = S.Camera(S.look_at(cn.eye, centre + shift * side), cn.proj, cn.eye)
        ref, lists, segs, fl = orc.render_exact(sc, cn.view, cn.proj, W, H)
        out = torch.full((H, W, 4), 7.0, dtype=torch.float32, device="cuda")
        rl = torch.full((H, W), 99, dtype=torch.int32, device="cuda")
        rs = torch.full((H, W), 99, dtype=torch.int32, device="cuda")
        V.vdi_render_ex(vdi, V.camera(cn.view, cn.proj), W, H, 1, 1, out, V.VDI_F32, ray_lists=rl, ray_segs=rs)
        fast = torch.full((H, W, 4), 7.0, dtype=torch.float32, device="cuda")
        V.vdi_render(vdi, V.camera(cn.view, cn.proj), W, H, 1, 1, fast, V.VDI_F32)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(-1, 4)
        assert np.array_equal(got, fast.cpu().numpy().reshape(-1, 4))
        half = torch.full((H, W, 4), 7.0, dtype=torch.float16, device="cuda")
        V.vdi_render(vdi, V.camera(cn.view, cn.proj), W, H, 1, 1, half, V.VDI_F16)
        torch.cuda.synchronize()
        assert np.array_equal(half.cpu().numpy().reshape(-1, 4), got.astype(np.float16))
        ok = fl == 0
        check_exact(orc, sc, cn, W, H, got, 1, ref, fl, what=f"shift {shift}")
        assert np.array_equal(rl.cpu().numpy().reshape(-1)[ok], lists[ok])
        assert np.array_equal(rs.cpu().numpy().reshape(-1)[ok], segs[ok])
        seen = ref[:, 3].reshape(H, W) > 0
        if shift == 0.0:
            assert 0.01 < seen.mean() < 0.1, seen.mean()  # small on screen: most tiles are cleared
        elif shift < 1.0:
            assert seen[:, 0].any() and seen[-1, :].any() and seen.mean() < 0.4  # cut by two image edges
        else:
            assert not seen.any() and np.all(got == 0)
    finally:
        V.vdi_destroy(vdi)
