"""Batched persistent multi-view rendering (many views of several VDIs in one
launch, CUDA-graph replay, autotuned launch shape) against single-view
renders and the oracle.  Every request must come out exactly as it does when
rendered alone, whatever else is in the batch."""
import numpy as np
import pytest

import vdi_synth as S
from helpers import check_tolerance, random_case

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


@pytest.fixture(scope="module")
def vdis(V, ctx):
    cases = [random_case(48, 32, 4, seed=1), random_case(64, 40, 7, seed=2), random_case(40, 40, 12, seed=3),
             random_case(80, 45, 20, seed=4, fill=0.5)]
    fmts = [0, 1, 1, 0]
    out = [(c, V.vdi_create(ctx, c.gpu_desc(V, f), c.vdi.rgba, c.vdi.depth, c.vdi.counts)) for c, f in zip(cases, fmts)]
    yield out
    for _, v in out:
        V.vdi_destroy(v)


def make_requests(V, vdis, n, seed):
    rng = np.random.default_rng(seed)
    res = [(64, 36), (128, 72), (96, 96), (75, 53)]
    reqs, outs = [], []
    for i in range(n):
        case, vdi = vdis[int(rng.integers(0, len(vdis)))]
        W, H = res[int(rng.integers(0, len(res)))]
        d_i, d_r = [(1, 1), (1, 2), (2, 1), (2, 2), (1, 1)][int(rng.integers(0, 5))]
        fmt = int(rng.integers(0, 2))
        cam = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=float(rng.uniform(-30, 30)),
                             el_deg=float(rng.uniform(0, 30)))
        out = torch.zeros((H, W, 4), dtype=torch.float32 if fmt == 0 else torch.float16, device="cuda")
        reqs.append(V.request(vdi, V.camera(cam.view, cam.proj), W, H, d_i, d_r, out, fmt))
        outs.append((out, cam, case, vdi, W, H, d_i, d_r, fmt))
    return reqs, outs


def alone(V, vdi, cam, W, H, d_i, d_r, fmt):
    o = torch.zeros((H, W, 4), dtype=torch.float32 if fmt == 0 else torch.float16, device="cuda")
    V.vdi_render(vdi, V.camera(cam.view, cam.proj), W, H, d_i, d_r, o, fmt)
    return o


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("ws", [0, 1, 2, 3])
def test_batch_equals_each_request_alone(V, ctx, vdis, use_graph, ws):
    reqs, outs = make_requests(V, vdis, 24, seed=ws)
    for rep in range(2):  # second pass replays the cached graph
        for o in outs:
            o[0].zero_()
        V.vdi_render_batch(ctx, reqs, warp_shape=ws, use_graph=use_graph)
        torch.cuda.synchronize()
        for (out, cam, case, vdi, W, H, d_i, d_r, fmt) in outs:
            ref = alone(V, vdi, cam, W, H, d_i, d_r, fmt)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (W, H, d_i, d_r, fmt)


def test_graph_replay_with_new_views(V, ctx, vdis):
    reqs, outs = make_requests(V, vdis, 10, seed=5)
    V.vdi_render_batch(ctx, reqs, use_graph=True)
    # same shapes, new cameras: the cached graph is replayed with updated parameters
    reqs2, outs2 = make_requests(V, vdis, 10, seed=5)
    rng = np.random.default_rng(9)
    for i, (out, cam, case, vdi, W, H, d_i, d_r, fmt) in enumerate(outs2):
        cam2 = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=float(rng.uniform(-40, 40)), el_deg=5.0)
        reqs2[i].view = V.camera(cam2.view, cam2.proj)
        outs2[i] = (out, cam2, case, vdi, W, H, d_i, d_r, fmt)
    V.vdi_render_batch(ctx, reqs2, use_graph=True)
    torch.cuda.synchronize()
    for (out, cam, case, vdi, W, H, d_i, d_r, fmt) in outs2:
        assert torch.equal(out, alone(V, vdi, cam, W, H, d_i, d_r, fmt))


def test_batch_parity_with_oracle(V, ctx, orc, vdis):
    case, vdi = vdis[1]
    sc = case.oracle_scene(orc)
    reqs, refs, outs = [], [], []
    for az in (-20.0, 5.0, 25.0, 140.0):
        cam = S.orbit_camera(case.bmin, case.bmax, 1.5, az_deg=az, el_deg=10.0)
        out = torch.zeros((60, 90, 4), device="cuda")
        reqs.append(V.request(vdi, V.camera(cam.view, cam.proj), 90, 60, 1, 1, out))
        refs.append(orc.render_exact(sc, cam.view, cam.proj, 90, 60)[0])
        outs.append(out)
    V.vdi_render_batch(ctx, reqs)
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        check_tolerance(out.cpu().numpy(), ref, 1, what="batch")  # F16-colour VDI


def test_autotuner_picks_a_configuration_and_batches_use_it(V, ctx, vdis):
    reqs, outs = make_requests(V, vdis, 16, seed=11)
    best, ms = V.vdi_autotune_batch(ctx, reqs)
    assert 0 <= best.warp_shape <= 3 and best.blocks_per_sm >= 1 and best.use_graph == 1 and ms > 0
    for o in outs:
        o[0].zero_()
    V.vdi_render_batch(ctx, reqs, warp_shape=-1)
    torch.cuda.synchronize()
    for (out, cam, case, vdi, W, H, d_i, d_r, fmt) in outs:
        assert torch.equal(out, alone(V, vdi, cam, W, H, d_i, d_r, fmt))


def test_batch_rejects_bad_batches(V, ctx, vdis):
    reqs, _ = make_requests(V, vdis, 65, seed=1)
    with pytest.raises(V.VdiError):
        V.vdi_render_batch(ctx, reqs)
    with pytest.raises(V.VdiError):
        V.vdi_render_batch(ctx, [])
    reqs, _ = make_requests(V, vdis, 3, seed=1)
    reqs[1].out = None
    with pytest.raises(V.VdiError):
        V.vdi_render_batch(ctx, reqs)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_with_explicit_ray_counts(V, ctx, vdis, use_graph):
    """Requests that name their ray counts (fractional image-space scales, as the
    preview controller picks them) equal vdi_render_scaled, graph replays included."""
    rng = np.random.default_rng(9)
    reqs, outs = [], []
    for i in range(12):
        case, vdi = vdis[i % len(vdis)]
        W, H = [(96, 64), (75, 53), (128, 72)][i % 3]
        Wr, Hr = int(rng.integers(1, W + 1)), int(rng.integers(1, H + 1))
        d_r = 1 + (i % 2)
        fmt = i % 2
        cam = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=float(rng.uniform(-30, 30)), el_deg=15.0)
        out = torch.zeros((H, W, 4), dtype=torch.float32 if fmt == 0 else torch.float16, device="cuda")
        reqs.append(V.request(vdi, V.camera(cam.view, cam.proj), W, H, 1, d_r, out, fmt, Wr=Wr, Hr=Hr))
        outs.append((out, cam, vdi, W, H, Wr, Hr, d_r, fmt))
    for rep in range(2):
        for o in outs:
            o[0].zero_()
        V.vdi_render_batch(ctx, reqs, use_graph=use_graph)
        torch.cuda.synchronize()
        for (out, cam, vdi, W, H, Wr, Hr, d_r, fmt) in outs:
            ref = torch.zeros_like(out)
            V.vdi_render_scaled(vdi, V.camera(cam.view, cam.proj), W, H, Wr, Hr, d_r, ref, fmt)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (W, H, Wr, Hr, d_r, fmt)
