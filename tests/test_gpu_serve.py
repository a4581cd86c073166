"""Continuous-batching server over resident VDIs.

* Every result equals the same view rendered alone, whatever else was in flight.
* Requests submitted while batches run are admitted into later batches.
* Admission by memory: a request that can never fit the budget fails with
  VDI_ERR_OOM on its ticket; an unknown slot fails with VDI_ERR_INVALID_ARG.
* A slot replaced by a VDI whose producer stream is still busy: its requests
  wait (a bounded wait times out with VDI_ERR_TIMEOUT, then completes).
* Released results give their memory back.
* The budget is a device budget: resident VDIs and VDIs generated through the
  server are charged next to images and scratch.
"""
import time

import numpy as np
import pytest

import vdi_synth as S
from helpers import random_case

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


def make_vdi(V, ctx, seed, fmt):
    case = random_case(64, 48, 6, seed=seed, fill=0.7)
    return case, V.vdi_create(ctx, case.gpu_desc(V, fmt), case.vdi.rgba, case.vdi.depth, case.vdi.counts)


def download_image(V, srv, ticket, W, H, fmt):
    dt = torch.float32 if fmt == 0 else torch.float16
    out = torch.empty((H, W, 4), dtype=dt, device="cuda")
    V.vdi_server_read(srv, ticket, out)
    return out


def alone(V, vdi, cam, W, H, d_i, d_r, fmt):
    o = torch.zeros((H, W, 4), dtype=torch.float32 if fmt == 0 else torch.float16, device="cuda")
    V.vdi_render(vdi, V.camera(cam.view, cam.proj), W, H, d_i, d_r, o, fmt)
    torch.cuda.synchronize()
    return o


def test_results_equal_alone_under_concurrency(V, ctx):
    cases = [make_vdi(V, ctx, s, f) for s, f in ((1, 0), (2, 1), (3, 1))]
    # a second handle on the same arrays for the reference renders (the server owns the installed ones)
    refs = [V.vdi_create(ctx, c.gpu_desc(V, f), c.vdi.rgba, c.vdi.depth, c.vdi.counts)
            for (c, _), f in zip(cases, (0, 1, 1))]
    srv = V.vdi_server_create(ctx, budget_bytes=8 << 20, max_batch=6, max_inflight=2, n_slots=3)
    try:
        for i, (_, vdi) in enumerate(cases):
            V.vdi_server_set_vdi(srv, i, vdi)
        rng = np.random.default_rng(0)
        jobs = []
        for k in range(60):
            slot = int(rng.integers(0, 3))
            case = cases[slot][0]
            W, H = [(64, 36), (96, 64), (128, 72)][int(rng.integers(0, 3))]
            d_i, d_r = [(1, 1), (2, 1), (1, 2), (2, 2)][int(rng.integers(0, 4))]
            fmt = int(rng.integers(0, 2))
            cam = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=float(rng.uniform(-45, 45)), el_deg=10.0)
            t = V.vdi_server_submit(srv, V.view_request(slot, V.camera(cam.view, cam.proj), W, H, d_i, d_r, fmt))
            jobs.append((t, slot, cam, W, H, d_i, d_r, fmt))
            if k % 7 == 3:
                time.sleep(0.002)  # arrivals while batches are in flight
        for (t, slot, cam, W, H, d_i, d_r, fmt) in jobs:
            info = V.vdi_server_wait(srv, t, timeout_s=20.0)
            assert info.status == 0
            got = download_image(V, srv, t, W, H, fmt)
            ref = alone(V, refs[slot], cam, W, H, d_i, d_r, fmt)
            assert torch.equal(got, ref), (slot, W, H, d_i, d_r, fmt)
            V.vdi_server_release(srv, t)
        st = V.vdi_server_stats(srv)
        assert st.completed == 60 and st.failed == 0 and st.bytes_in_use == 0
        assert st.batches >= 10  # the 8 MiB budget and max_batch split the stream into many batches
    finally:
        V.vdi_server_destroy(srv)
        for r in refs:
            V.vdi_destroy(r)


def test_admission_errors_land_on_tickets(V, ctx):
    case, vdi = make_vdi(V, ctx, 4, 0)
    srv = V.vdi_server_create(ctx, budget_bytes=1 << 20, max_batch=4, max_inflight=1, n_slots=2)
    try:
        V.vdi_server_set_vdi(srv, 0, vdi)
        cam = V.camera(case.cam_o.view, case.cam_o.proj)
        too_big = V.vdi_server_submit(srv, V.view_request(0, cam, 1024, 1024, 1, 1, 0))  # 16 MiB > 1 MiB
        no_vdi = V.vdi_server_submit(srv, V.view_request(1, cam, 32, 32))
        ok = V.vdi_server_submit(srv, V.view_request(0, cam, 32, 32))
        assert V.vdi_server_wait(srv, too_big, 10.0).status == 2  # VDI_ERR_OOM
        assert V.vdi_server_wait(srv, no_vdi, 10.0).status == 1  # VDI_ERR_INVALID_ARG
        assert V.vdi_server_wait(srv, ok, 10.0).status == 0
        with pytest.raises(V.VdiError):
            V.vdi_server_submit(srv, V.view_request(0, cam, 0, 32))
    finally:
        V.vdi_server_destroy(srv)


def test_replacement_waits_for_its_producer_and_bounded_wait_times_out(V, ctx):
    case, vdi = make_vdi(V, ctx, 5, 1)
    case2, vdi2 = make_vdi(V, ctx, 6, 1)
    ref2 = V.vdi_create(ctx, case2.gpu_desc(V, 1), case2.vdi.rgba, case2.vdi.depth, case2.vdi.counts)
    srv = V.vdi_server_create(ctx, budget_bytes=32 << 20, max_batch=8, max_inflight=2, n_slots=1)
    side = torch.cuda.Stream()
    try:
        V.vdi_server_set_vdi(srv, 0, vdi)
        cam = S.orbit_camera(case.bmin, case.bmax, 1.0, az_deg=15.0)
        t0 = V.vdi_server_submit(srv, V.view_request(0, V.camera(cam.view, cam.proj), 64, 64))
        assert V.vdi_server_wait(srv, t0, 10.0).status == 0
        with torch.cuda.stream(side):
            torch.cuda._sleep(int(3e9))  # the producer stream stays busy for about a second
        V.vdi_server_set_vdi(srv, 0, vdi2, side)
        t1 = V.vdi_server_submit(srv, V.view_request(0, V.camera(cam.view, cam.proj), 64, 64))
        with pytest.raises(V.VdiError) as e:
            V.vdi_server_wait(srv, t1, 0.05)
        assert e.value.status == 5  # VDI_ERR_TIMEOUT: still waiting for the new VDI
        info = V.vdi_server_wait(srv, t1, 20.0)
        assert info.status == 0
        assert torch.equal(download_image(V, srv, t1, 64, 64, 1), alone(V, ref2, cam, 64, 64, 1, 1, 1))
    finally:
        V.vdi_server_destroy(srv)
        V.vdi_destroy(ref2)


def test_preview_controller_session_through_the_server(V, ctx):
    """A client keeps a frame-time target with the preview controller: each
    request carries the ray counts the controller chose from the previous
    request's service time, and every result equals vdi_render_scaled at those
    counts."""
    case, vdi = make_vdi(V, ctx, 7, 1)
    ref_vdi = V.vdi_create(ctx, case.gpu_desc(V, 1), case.vdi.rgba, case.vdi.depth, case.vdi.counts)
    srv = V.vdi_server_create(ctx, 1 << 28, 4, 2, 1)
    try:
        V.vdi_server_set_vdi(srv, 0, vdi)
        W, H = 320, 200
        cam = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=10.0, el_deg=15.0)
        t = V.vdi_server_submit(srv, V.view_request(0, V.camera(cam.view, cam.proj), W, H, 1, 2, V.VDI_F16))
        info = V.vdi_server_wait(srv, t, 30.0)
        V.vdi_server_release(srv, t)
        # a target below the full-resolution service time pulls the scale down
        pi = V.PiController(0.5 * (info.t_done - info.t_start) * 1e3, W, H, scale_min=0.2)
        s, Wr, Hr = pi.current()
        seen = set()
        for k in range(12):
            cam = S.orbit_camera(case.bmin, case.bmax, W / H, az_deg=10.0 + 2.0 * k, el_deg=15.0)
            t = V.vdi_server_submit(srv, V.view_request(0, V.camera(cam.view, cam.proj), W, H, 1, 2,
                                                        V.VDI_F16, Wr=Wr, Hr=Hr))
            info = V.vdi_server_wait(srv, t, 30.0)
            assert info.status == 0
            got = download_image(V, srv, t, W, H, 1)
            V.vdi_server_release(srv, t)
            ref = torch.zeros((H, W, 4), dtype=torch.float16, device="cuda")
            V.vdi_render_scaled(ref_vdi, V.camera(cam.view, cam.proj), W, H, Wr, Hr, 2, ref, V.VDI_F16)
            torch.cuda.synchronize()
            assert torch.equal(got, ref), (k, Wr, Hr)
            seen.add((Wr, Hr))
            s, Wr, Hr = pi.update((info.t_done - info.t_start) * 1e3)
        assert len(seen) >= 2 and min(w for w, _ in seen) < W  # the controller moved the ray counts
        with pytest.raises(V.VdiError):
            V.vdi_server_submit(srv, V.view_request(0, V.camera(cam.view, cam.proj), W, H, 1, 1, V.VDI_F16,
                                                    Wr=W + 1, Hr=H))
    finally:
        V.vdi_server_destroy(srv)
        V.vdi_destroy(ref_vdi)


def test_budget_is_a_device_budget(V, ctx):
    """Resident VDIs count against the server's budget next to images: a VDI
    that does not fit is refused (the caller keeps it), a request that cannot
    fit beside the resident VDIs fails at once, and generation through the
    server charges the new VDI before allocating it (a replacement frees the
    slot's old VDI when nothing else reads it)."""
    case, a = make_vdi(V, ctx, 7, 1)
    _, b = make_vdi(V, ctx, 8, 1)
    _, c = make_vdi(V, ctx, 9, 1)
    B = V.vdi_get_layout(a).total_bytes
    srv = V.vdi_server_create(ctx, budget_bytes=2 * B + (64 << 10), max_batch=4, max_inflight=1, n_slots=3)
    try:
        V.vdi_server_set_vdi(srv, 0, a)
        V.vdi_server_set_vdi(srv, 1, b)
        assert V.vdi_server_stats(srv).vdi_bytes == 2 * B
        with pytest.raises(V.VdiError) as e:
            V.vdi_server_set_vdi(srv, 2, c)
        assert e.value.status == 2  # VDI_ERR_OOM; the caller still owns c
        V.vdi_destroy(c)
        cam = V.camera(case.cam_o.view, case.cam_o.proj)
        small = V.vdi_server_submit(srv, V.view_request(0, cam, 64, 48, out_fmt=V.VDI_F16))  # 24 KiB
        assert V.vdi_server_wait(srv, small, 10.0).status == 0
        V.vdi_server_release(srv, small)
        # with nothing in flight or unreleased, 512 KiB can never fit beside the two VDIs
        big = V.vdi_server_submit(srv, V.view_request(0, cam, 256, 256, out_fmt=V.VDI_F16))
        assert V.vdi_server_wait(srv, big, 10.0).status == 2

        # generation through the server: a 32 x 24 VDI replaces slot 0's 64 x 48 one
        vol = S.blobs_volume(24, seed=3)
        bmin, bmax = np.zeros(3), np.ones(3)
        kn = S.tf_knots("dense")
        vd = torch.from_numpy(vol).cuda()
        cam_o = S.orbit_camera(bmin, bmax, 32 / 24, el_deg=15)
        args = (vd, bmin, bmax, kn, V.camera(cam_o.view, cam_o.proj))
        side = torch.cuda.Stream()
        V.vdi_server_generate(srv, 0, *args, 32, 24, 4, 0.02, 1 / 24, 1 / 24, V.VDI_F16, stream=side)
        direct = V.vdi_generate(ctx, *args, 32, 24, 4, 0.02, 1 / 24, 1 / 24, V.VDI_F16)
        small_bytes = V.vdi_get_layout(direct).total_bytes
        assert small_bytes < B and V.vdi_server_stats(srv).vdi_bytes == B + small_bytes
        cn = S.orbit_camera(bmin, bmax, 1.0, az_deg=20.0, el_deg=15.0)
        t = V.vdi_server_submit(srv, V.view_request(0, V.camera(cn.view, cn.proj), 48, 48, out_fmt=V.VDI_F16))
        assert V.vdi_server_wait(srv, t, 20.0).status == 0
        assert torch.equal(download_image(V, srv, t, 48, 48, 1), alone(V, direct, cn, 48, 48, 1, 1, 1))
        V.vdi_server_release(srv, t)
        # a VDI too large for what is left is refused before anything is generated
        with pytest.raises(V.VdiError) as e:
            V.vdi_server_generate(srv, 2, *args, 128, 96, 8, 0.02, 1 / 24, 1 / 24, V.VDI_F32, stream=side)
        assert e.value.status == 2
        assert V.vdi_server_stats(srv).vdi_bytes == B + small_bytes
        V.vdi_destroy(direct)
        torch.cuda.synchronize()
    finally:
        V.vdi_server_destroy(srv)
