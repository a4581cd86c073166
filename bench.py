#!/usr/bin/env python
"""Benchmark: VDI raycasting frames/s at 1920x1080 on the large mixing-layer workload.

Workload ("large"): a 1024^3 uint8 mixing-layer volume (tanh interface at mid
height perturbed by 64 Fourier modes) -> GPU vdi_generate at 1920x1080,
N_S = 20, FP16 colour / FP32 depth.  One step renders the resident VDI at
1920x1080 from new views rotated 10, 20 and 30 degrees about the volume's
vertical axis, plus the previews (D_I, D_R) = (2, 2) and (4, 4) at 30 degrees:
5 frames.  L2 is flushed between steps (a 256 MiB write, then a 256 MiB read
of another buffer, so the frame neither finds its data in L2 nor writes back
the flush's dirty lines); each step's kernels are timed with CUDA events on
the launching stream.

Also reported: the HBM roofline of the exact-render kernel (unique VDI bytes
one frame needs, from the instrumented touch bitmap, divided by the kernel's
event-timed duration), nvidia-smi clocks during the timed region, an
end-to-end number through the public API with images read back to pinned host
memory, and the FP64 CPU oracle timed on a bounded sample of the same frames.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import vdi_synth as S  # noqa: E402

METRIC = "VDI raycast frames/s & Grays/s at 1920x1080 (HBM roofline %); serving p50/p99 ms"

WORKLOADS = {
    "large": dict(name="mixing-layer 1024^3 u8 -> VDI 1920x1080 N_S=20 FP16 colour; renders 1920x1080 at "
                       "10/20/30 deg + previews (D_I,D_R)=(2,2),(4,4) at 30 deg",
                  n=1024, vol="mixing", dtype=np.uint8, tf="interface", w=1920, h=1080, ns=20, tau=0.01, fmt=1,
                  W=1920, H=1080, el=25.0, zoom=1.0,
                  frames=[(10.0, 1, 1), (20.0, 1, 1), (30.0, 1, 1), (30.0, 2, 2), (30.0, 4, 4)]),
    "plain": dict(name="value-noise 256^3 u16 -> VDI 1280x720 N_S=20 FP32; renders 1280x720 at 0/5/15/30 deg, zoom 1.2",
                  n=256, vol="noise", dtype=np.uint16, tf="sparse", w=1280, h=720, ns=20, tau=0.01, fmt=0,
                  W=1280, H=720, el=20.0, zoom=1.2,
                  frames=[(0.0, 1, 1), (5.0, 1, 1), (15.0, 1, 1), (30.0, 1, 1)]),
    "tiny": dict(name="blobs 64^3 f32 -> VDI 128x128 N_S=8 FP32; render 128x128 at 10 deg",
                 n=64, vol="blobs", dtype=np.float32, tf="dense", w=128, h=128, ns=8, tau=0.02, fmt=0,
                 W=128, H=128, el=15.0, zoom=1.0, frames=[(10.0, 1, 1)]),
}


def make_volume(wl, seed=0):
    if wl["vol"] == "mixing":
        return S.mixing_layer_volume(wl["n"], seed=seed, dtype=wl["dtype"])
    if wl["vol"] == "noise":
        return S.value_noise_volume(wl["n"], seed=seed, dtype=wl["dtype"])
    return S.blobs_volume(wl["n"], seed=seed)


def cameras(wl, bmin, bmax):
    cam_o = S.orbit_camera(bmin, bmax, wl["w"] / wl["h"], az_deg=0.0, el_deg=wl["el"])
    views = [S.orbit_camera(bmin, bmax, wl["W"] / wl["H"], az_deg=az, el_deg=wl["el"], zoom=wl["zoom"])
             for (az, _, _) in wl["frames"]]
    return cam_o, views


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def render_kernel_hash() -> str:
    h = hashlib.sha1()
    for fn in ("vdi_render.cu", "vdi_march.cuh", "vdi_internal.cuh", "vdi_preview.cuh", "vdi_tma.cuh"):
        with open(os.path.join(ROOT, "paper_2206_08660_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def recorded_traffic(workload: str):
    """DRAM bytes per exact-render launch from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", f"render_exact_{workload}.md")
    if not os.path.exists(p):
        return None
    want = render_kernel_hash()
    for line in open(p):
        if line.startswith("traffic_bytes_per_launch:"):
            parts = line.split()
            if len(parts) >= 4 and parts[2] == "kernel_hash" and parts[3] == want:
                return int(parts[1])
    return None


def recorded_instructions(workload: str):
    """Warp instructions per exact-render launch of each step frame (ncu
    smsp__inst_executed.sum) from the committed summary, if it was taken on the
    current kernel source; else None.  Line format:
    warp_instructions_per_launch: <deg>=<count> ... kernel_hash <hash>"""
    p = os.path.join(ROOT, "profiles", f"render_exact_{workload}.md")
    if not os.path.exists(p):
        return None
    want = render_kernel_hash()
    for line in open(p):
        if line.startswith("warp_instructions_per_launch:"):
            parts = line.split()
            if len(parts) >= 4 and parts[-2] == "kernel_hash" and parts[-1] == want:
                return {k: int(v) for k, v in (x.split("=") for x in parts[1:-2])}
    return None


def issue_peak():
    """Warp instructions per second the GPU can issue: 4 schedulers per SM, one
    instruction per scheduler and cycle, at the maximum SM clock."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return sms * 4 * mhz * 1e6, sms, mhz


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms; only samples
    taken between mark_start() and mark_stop() are kept."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def wait_ready(self, timeout=15.0):
        t = time.monotonic()
        while self.proc is not None and not self.lines and time.monotonic() - t < timeout:
            time.sleep(0.05)

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_stop(self):
        self.t1 = time.monotonic()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t0", -1e30), getattr(self, "t1", 1e30)
        for (ts, ln) in self.lines:
            if not (t0 - 0.1 <= ts <= t1 + 0.25):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu), or the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.machine()


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over the ranks of the default process group (x itself
    when there is none): the benchmark's time per step is the slowest rank's."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, step_ms: float, world: int) -> float:
    """Units per second of the whole job when every rank does the same work per step (weak scaling)."""
    return world * units_per_rank_step / (step_ms / 1e3)


class OracleLeg:
    """The FP64 CPU oracle on the same workload, for the CPU baseline and the
    reference arm.  The oracle renders its own VDI, made by the oracle's FP32
    generation (which matches the GPU's supersegments bit for bit)."""

    def __init__(self, wl, vol, bmin, bmax, u, cam_o, views):
        import oracle

        self.o = oracle
        kn = S.tf_knots(wl["tf"])
        rgba, depth, counts = oracle.generate(oracle.Volume(vol, bmin, bmax), kn, cam_o.view, cam_o.proj, wl["w"],
                                              wl["h"], wl["ns"], wl["tau"], u, u, fp32=True)
        self.sc = oracle.Scene(S.VdiArrays(wl["w"], wl["h"], wl["ns"], rgba, depth, counts), cam_o.view, cam_o.proj,
                               bmin, bmax, u)
        # the count grid is built once per VDI (as vdi_create / vdi_generate do on the
        # GPU) with the renderer's default cell shape: 8 x 8 lists by 20 slabs
        self.grid = oracle.grid_counts(self.sc, 8, 20)
        self.wl, self.views = wl, views
        self.threads = os.cpu_count() or 1

    def run(self, R, rng):
        """R random rays of every frame; returns (seconds measured, seconds extrapolated to full frames)."""
        measured = full = 0.0
        for (az, d_i, d_r), cn in zip(self.wl["frames"], self.views):
            Wr, Hr = -(-self.wl["W"] // d_i), -(-self.wl["H"] // d_i)
            # a whole frame when the sample would hold as many rays, else a random sample
            pix = None if R >= Wr * Hr else rng.integers(0, Wr * Hr, size=R).astype(np.int32)
            n = Wr * Hr if pix is None else len(pix)
            t = time.perf_counter()
            if d_r == 1:
                self.o.render_exact(self.sc, cn.view, cn.proj, Wr, Hr, pix=pix, nthreads=self.threads)
            else:
                self.o.render_preview(self.sc, cn.view, cn.proj, Wr, Hr, d_r, 8, 20, grid=self.grid, pix=pix,
                                      nthreads=self.threads)
            dt = time.perf_counter() - t
            measured += dt
            full += dt / n * (Wr * Hr)
        return measured, full

    def rays_for_budget(self, budget_s, rng, probe=2048):
        """Rays per frame so that one run() takes about budget_s seconds."""
        self.run(256, rng)  # first touch of the scene and thread start-up, untimed
        m, _ = self.run(probe, rng)
        return int(max(probe, probe * budget_s / max(m, 1e-6)))

    def rays_per_step(self):
        """Rays of one whole step (every frame at its rendered resolution)."""
        return sum((-(-self.wl["W"] // d_i)) * (-(-self.wl["H"] // d_i)) for (_, d_i, _) in self.wl["frames"])

    def sample_text(self, R):
        sizes = [(-(-self.wl["W"] // d_i)) * (-(-self.wl["H"] // d_i)) for (_, d_i, _) in self.wl["frames"]]
        if all(R >= s for s in sizes):
            return (f"whole frames: all {len(self.wl['frames'])} frames of the step at their full ray counts "
                    f"({'/'.join(str(s) for s in sorted(set(sizes)))}); oracle VDI from the oracle's own FP32 "
                    f"generation, count grid built once")
        counts = sorted({min(R, s) for s in sizes})
        n = str(counts[0]) if len(counts) == 1 else "/".join(str(c) for c in counts)
        return (f"{n} rays from each of the {len(self.wl['frames'])} frames per step (a whole frame where the "
                f"sample reaches its ray count, else drawn at random with repetition), extrapolated to full frames; "
                f"oracle VDI from the oracle's own FP32 generation, count grid built once")


SERVING = dict(n_vdis=8, w=1920, h=1080, ns=24, tau=0.01, vol_n=512, rate=240.0, seconds=8.0, replace_every=2.0,
               high_rate=2000.0, high_seconds=3.0,
               budget=24 << 30, max_batch=32, max_inflight=3,
               res=[(640, 360), (1280, 720), (1280, 720), (1920, 1080)], max_dev=45.0, seed=7)


def serving_leg(V, torch, ctx, dev, cfg=SERVING):
    """Continuous-batching server under Poisson arrivals, p50/p99 latency and throughput.

    8 resident 1920x1080 N_S=24 FP16 VDIs (from a seeded 512^3 uint8 noise volume
    seen from 8 directions); arrivals at `rate` requests/s; resolution mix
    360p:720p:1080p = 1:2:1; deviation U[0, 45] deg; D_I, D_R in {1, 2}; every
    2 s one slot gets a freshly generated VDI from a side stream.  Also measures
    saturated throughput of the same request mix through the server (batched,
    FP16 colour) and through one vdi_render per request on FP32-colour VDIs."""
    import threading as th

    rng = np.random.default_rng(cfg["seed"])
    vol = S.value_noise_volume(cfg["vol_n"], seed=cfg["seed"], dtype=np.uint8)
    bmin, bmax = S.bbox_for_dims(vol.shape)
    u = 1.0 / cfg["vol_n"]
    vol_d = torch.from_numpy(vol).to(dev)
    kn = S.tf_knots("sparse")
    az0 = [45.0 * k for k in range(cfg["n_vdis"])]
    cams_o = [S.orbit_camera(bmin, bmax, cfg["w"] / cfg["h"], az_deg=a, el_deg=20.0) for a in az0]

    def gen(k, fmt, az=None, stream=None):
        c = cams_o[k] if az is None else S.orbit_camera(bmin, bmax, cfg["w"] / cfg["h"], az_deg=az, el_deg=20.0)
        return V.vdi_generate(ctx, vol_d, bmin, bmax, kn, V.camera(c.view, c.proj), cfg["w"], cfg["h"], cfg["ns"],
                              cfg["tau"], u, u, fmt, stream=stream), c

    def make_requests(n):
        reqs = []
        for _ in range(n):
            slot = int(rng.integers(0, cfg["n_vdis"]))
            W, H = cfg["res"][int(rng.integers(0, len(cfg["res"])))]
            dev_deg = float(rng.uniform(0.0, cfg["max_dev"])) * (1 if rng.random() < 0.5 else -1)
            cam = S.orbit_camera(bmin, bmax, W / H, az_deg=az0[slot] + dev_deg, el_deg=20.0)
            d_i, d_r = int(rng.integers(1, 3)), int(rng.integers(1, 3))
            reqs.append((slot, V.camera(cam.view, cam.proj), W, H, d_i, d_r))
        return reqs

    srv = V.vdi_server_create(ctx, cfg["budget"], cfg["max_batch"], cfg["max_inflight"], cfg["n_vdis"])
    side = torch.cuda.Stream()
    try:
        for k in range(cfg["n_vdis"]):
            V.vdi_server_set_vdi(srv, k, gen(k, V.VDI_F16)[0])
        torch.cuda.synchronize()
        # warm-up: every resolution / preview combination once
        for (slot, cam, W, H, d_i, d_r) in make_requests(32):
            t = V.vdi_server_submit(srv, V.view_request(slot, cam, W, H, d_i, d_r))
            V.vdi_server_wait(srv, t, 30.0)
            V.vdi_server_release(srv, t)

        def run_open_loop(rate, seconds, replace):
            """Poisson arrivals at `rate` requests/s for `seconds`; with `replace`, one
            slot's VDI is regenerated through the server every replace_every seconds."""
            n = int(rate * seconds)
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
            reqs = make_requests(n)
            tickets = [None] * n
            lat, fails = [], 0
            st0 = V.vdi_server_stats(srv)
            t_start = time.monotonic()

            def submitter():
                for i in range(n):
                    d = t_start + arrivals[i] - time.monotonic()
                    if d > 0:
                        time.sleep(d)
                    slot, cam, W, H, d_i, d_r = reqs[i]
                    tickets[i] = V.vdi_server_submit(srv, V.view_request(slot, cam, W, H, d_i, d_r))

            def replacer():
                k = 0
                while replace:
                    # one replacement every replace_every seconds while requests still arrive
                    t_next = t_start + (k + 1) * cfg["replace_every"]
                    if t_next - t_start >= arrivals[-1]:
                        break
                    time.sleep(max(0.0, t_next - time.monotonic()))
                    slot = k % cfg["n_vdis"]
                    # generation through the server: the new VDI's bytes are charged to
                    # the device budget before it is allocated on the side stream
                    c = S.orbit_camera(bmin, bmax, cfg["w"] / cfg["h"], az_deg=az0[slot] + 5.0 * (k + 1), el_deg=20.0)
                    with torch.cuda.stream(side):
                        V.vdi_server_generate(srv, slot, vol_d, bmin, bmax, kn, V.camera(c.view, c.proj), cfg["w"],
                                              cfg["h"], cfg["ns"], cfg["tau"], u, u, V.VDI_F16, stream=side)
                    k += 1

            ts, tr = th.Thread(target=submitter), th.Thread(target=replacer)
            ts.start()
            tr.start()
            for i in range(n):
                while tickets[i] is None:
                    time.sleep(0.0002)
                info = V.vdi_server_wait(srv, tickets[i], 30.0)
                if info.status != 0:
                    fails += 1
                else:
                    lat.append((info.t_done - info.t_submit) * 1e3)
                V.vdi_server_release(srv, tickets[i])
            wall = time.monotonic() - t_start  # first arrival to the last result read
            ts.join()
            tr.join()
            st = V.vdi_server_stats(srv)
            lat = np.array(lat)
            return {"offered_rps": rate, "requests": n, "failed": fails,
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "throughput_rps": len(lat) / wall,
                    "mean_batch": (st.batched_requests - st0.batched_requests) / max(st.batches - st0.batches, 1),
                    "vdi_replacements": int(st.vdi_installs - st0.vdi_installs),
                    "resident_vdi_bytes_at_end": int(st.vdi_bytes), "budget_bytes": cfg["budget"]}

        # ---- open loop: Poisson arrivals at the configured rate, then at a rate near the
        # server's saturation, where requests that arrive while batches run share launches
        open_loop = run_open_loop(cfg["rate"], cfg["seconds"], True)
        open_loop_high = run_open_loop(cfg["high_rate"], cfg["high_seconds"], True)
        # ---- saturated throughput, same request mix: batched server (FP16) ...
        sat = make_requests(512)
        torch.cuda.synchronize()
        t0 = time.monotonic()
        ids = [V.vdi_server_submit(srv, V.view_request(*r)) for r in sat]
        for t in ids:
            V.vdi_server_wait(srv, t, 60.0)
            V.vdi_server_release(srv, t)
        batched_rps = len(sat) / (time.monotonic() - t0)
    finally:
        V.vdi_server_destroy(srv)
    # ... against one vdi_render per request on FP32-colour VDIs
    vdis32 = [gen(k, V.VDI_F32)[0] for k in range(cfg["n_vdis"])]
    outs = {}
    for (slot, cam, W, H, d_i, d_r) in sat:
        outs.setdefault((W, H), torch.empty((H, W, 4), dtype=torch.float32, device=dev))
    for (slot, cam, W, H, d_i, d_r) in sat[:16]:
        V.vdi_render(vdis32[slot], cam, W, H, d_i, d_r, outs[(W, H)], V.VDI_F32)
    torch.cuda.synchronize()
    t0 = time.monotonic()
    for (slot, cam, W, H, d_i, d_r) in sat:
        V.vdi_render(vdis32[slot], cam, W, H, d_i, d_r, outs[(W, H)], V.VDI_F32)
    torch.cuda.synchronize()
    single_rps = len(sat) / (time.monotonic() - t0)
    # accuracy of the FP16-colour VDIs against the FP32 ones on the same requests
    errs = []
    for k in range(4):
        v16 = gen(k, V.VDI_F16)[0]
        for (slot, cam, W, H, d_i, d_r) in [r for r in sat if r[0] == k][:4]:
            a = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
            b = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
            V.vdi_render(v16, cam, W, H, d_i, d_r, a, V.VDI_F32)
            V.vdi_render(vdis32[k], cam, W, H, d_i, d_r, b, V.VDI_F32)
            torch.cuda.synchronize()
            errs.append((a - b).abs().amax(dim=2).flatten().cpu().numpy())
        V.vdi_destroy(v16)
    e = np.concatenate(errs) if errs else np.zeros(1)
    fp16_vs_fp32 = {"max": float(e.max()), "q999": float(np.quantile(e, 0.999)), "requests": len(errs)}
    for v in vdis32:
        V.vdi_destroy(v)
    del vol_d
    torch.cuda.empty_cache()
    return {"workload": "8 resident 1920x1080 N_S=24 FP16 VDIs (512^3 u8 noise), Poisson 240 req/s, "
                        "360p:720p:1080p = 1:2:1, deviation U[0,45] deg, D_I,D_R in {1,2}, one VDI replaced "
                        "every 2 s from a side stream, 24 GB budget",
            "open_loop": open_loop,
            "open_loop_high_rate": open_loop_high,
            "fp16_vs_fp32_pixel_error": fp16_vs_fp32,
            "saturated": {"batched_fp16_server_rps": batched_rps, "one_view_per_launch_fp32_rps": single_rps,
                          "requests": len(sat)}}


BATCHED = dict(specs=[(640, 360, 8), (1280, 720, 16), (1920, 1080, 20), (1920, 1080, 32)], vol_n=512, n_req=64,
               res=[(640, 360), (1280, 720), (1920, 1080)], max_dev=30.0, tau=0.01, seed=3, reps=20)


def batched_config_leg(V, torch, ctx, dev, stream, flush_l2, peak, cfg=BATCHED):
    """The batched workload: 4 resident FP16-colour VDIs (640x360 N_S=8, 1280x720
    N_S=16, 1920x1080 N_S=20, 1920x1080 N_S=32, each generated from a seeded
    512^3 uint8 noise volume), 64 view requests of mixed resolution (360p..1080p)
    and deviation U[-30, 30] deg, rendered in one persistent launch replayed from
    a CUDA graph with the autotuned configuration.  L2 flushed between launches.
    Roofline numerator: per VDI, the union of the words its requests read (one
    touch bitmap accumulated over them)."""
    rng = np.random.default_rng(cfg["seed"])
    kn = S.tf_knots("sparse")
    vdis, boxes, az0 = [], [], []
    for k, (w, h, ns) in enumerate(cfg["specs"]):
        vol = S.value_noise_volume(cfg["vol_n"], seed=100 + k, dtype=np.uint8)
        bmin, bmax = S.bbox_for_dims(vol.shape)
        u = 1.0 / cfg["vol_n"]
        cam_o = S.orbit_camera(bmin, bmax, w / h, az_deg=90.0 * k, el_deg=20.0)
        vd = torch.from_numpy(vol).to(dev)
        vdis.append(V.vdi_generate(ctx, vd, bmin, bmax, kn, V.camera(cam_o.view, cam_o.proj), w, h, ns, cfg["tau"],
                                   u, u, V.VDI_F16, stream=stream))
        torch.cuda.synchronize()
        del vd
        boxes.append((bmin, bmax))
        az0.append(90.0 * k)
    reqs, jobs, rays = [], [], 0
    for i in range(cfg["n_req"]):
        k = int(rng.integers(0, len(vdis)))
        W, H = cfg["res"][int(rng.integers(0, len(cfg["res"])))]
        bmin, bmax = boxes[k]
        cn = S.orbit_camera(bmin, bmax, W / H, az_deg=az0[k] + float(rng.uniform(-cfg["max_dev"], cfg["max_dev"])),
                            el_deg=20.0)
        cam = V.camera(cn.view, cn.proj)
        out = torch.empty((H, W, 4), dtype=torch.float16, device=dev)
        reqs.append(V.request(vdis[k], cam, W, H, 1, 1, out, V.VDI_F16))
        jobs.append((k, cam, W, H))
        rays += W * H
    best, tuned_ms = V.vdi_autotune_batch(ctx, reqs, stream)
    for _ in range(3):
        V.vdi_render_batch(ctx, reqs, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(cfg["reps"])]
    for r in range(cfg["reps"]):
        flush_l2(r)
        ev[r][0].record(stream)
        V.vdi_render_batch(ctx, reqs, stream=stream)
        ev[r][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    # unique bytes per VDI over its requests
    touched = 0
    for k, v in enumerate(vdis):
        L = V.vdi_get_layout(v)
        grid_words = (L.grid_w * L.grid_h * L.grid_nz + 3) // 4 * 4
        words = ((L.depth_bytes + L.colour_bytes) // 4 + grid_words + L.list_bytes // 4 + 31) // 32
        bm = torch.zeros(words, dtype=torch.int32, device=dev)
        for (kk, cam, W, H) in jobs:
            if kk == k:
                V.vdi_touch_bitmap(v, cam, W, H, bm, stream)
        torch.cuda.synchronize()
        touched += int(np.unpackbits(bm.cpu().numpy().view(np.uint8)).sum()) * 4
    for v in vdis:
        V.vdi_destroy(v)
    achieved = touched / (ms / 1e3) / 1e9
    return {"workload": "4 resident FP16 VDIs (640x360 N_S=8, 1280x720 N_S=16, 1920x1080 N_S=20, 1920x1080 N_S=32; "
                        "512^3 u8 noise), 64 requests 360p..1080p, deviation U[-30,30] deg, one persistent launch "
                        "from a CUDA graph, autotuned",
            "ms_per_launch": ms, "frames_per_s": cfg["n_req"] / (ms / 1e3), "grays_per_s": rays / (ms / 1e3) / 1e9,
            "warp_shape": int(best.warp_shape), "blocks_per_sm": int(best.blocks_per_sm),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "algorithmic_bytes_per_launch": touched},
            "note": "CUDA events around each launch, L2 flushed between launches; rays = sum of request pixels"}


def preview_control_leg(V, torch, vdi, wl, bmin, bmax, stream, frames=240, target_ms=0.3, d_r=1):
    """The preview-rate PI controller (Section 4.4) in a session: the view orbits
    0 -> 45 -> 0 degrees over `frames` frames at the display resolution; each
    frame is rendered at the scale the controller chose from the previous
    frame's measured time (vdi_render_scaled), D_R fixed.  Every 20th frame is
    scored (SSIM) against the full-resolution exact render of the same view."""
    W, H = wl["W"], wl["H"]
    pi = V.PiController(target_ms, W, H)
    out = torch.empty((H, W, 4), dtype=torch.float16, device="cuda")
    full = torch.empty((H, W, 4), dtype=torch.float16, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times, scales, ssims = [], [], []
    s, Wr, Hr = pi.current()
    for k in range(frames):
        az = 45.0 * (1.0 - abs(1.0 - 2.0 * k / (frames - 1)))
        cn = S.orbit_camera(bmin, bmax, W / H, az_deg=az, el_deg=wl["el"], zoom=wl["zoom"])
        cam = V.camera(cn.view, cn.proj)
        e0.record(stream)
        V.vdi_render_scaled(vdi, cam, W, H, Wr, Hr, d_r, out, V.VDI_F16, stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        times.append(ms)
        scales.append(s)
        if k % 20 == 10:
            V.vdi_render(vdi, cam, W, H, 1, 1, full, V.VDI_F16, stream)
            ssims.append(V.vdi_image_quality(out, full, V.VDI_F16, stream)[0])
        s, Wr, Hr = pi.update(ms)
    t = np.array(times[20:])
    return {"target_ms": target_ms, "frames": frames, "d_r": d_r, "path": "orbit 0 -> 45 -> 0 deg",
            "frame_ms_mean": float(t.mean()), "frame_ms_p95": float(np.percentile(t, 95)),
            "within_20pct": float(np.mean(np.abs(t - target_ms) <= 0.2 * target_ms)),
            "scale_mean": float(np.mean(scales)), "scale_min": float(np.min(scales)),
            "ssim_vs_full_mean": float(np.mean(ssims)), "ssim_vs_full_min": float(np.min(ssims)),
            "note": "CUDA-event frame times with a sync per frame (the controller needs each measurement); "
                    "statistics exclude the first 20 frames"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-quality", action="store_true", help="skip the DVR / SSIM quality study")
    ap.add_argument("--frames", default=None,
                    help="override the step's frames, e.g. '0:1:1,10:1:1' (degrees:D_I:D_R); for profiling")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.frames:
        wl["frames"] = [tuple(float(x) if i == 0 else int(x) for i, x in enumerate(f.split(":")))
                        for f in args.frames.split(",")]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    vol = make_volume(wl)
    bmin, bmax = S.bbox_for_dims(vol.shape)
    u = 1.0 / max(vol.shape)
    cam_o, views = cameras(wl, bmin, bmax)
    frames_per_step = len(wl["frames"])
    config = {"workload": wl["name"], "vdi": f"{wl['w']}x{wl['h']} N_S={wl['ns']} "
                                             f"{'FP16' if wl['fmt'] else 'FP32'} colour, FP32 depth",
              "frames_per_step": frames_per_step, "image": f"{wl['W']}x{wl['H']}",
              "l2": "flushed between steps (256 MiB write, then 256 MiB read of another buffer)", "out_fmt": "f16", "search": "Algorithm 2"}

    if args.impl == "reference":
        if rank != 0:
            return
        leg = OracleLeg(wl, vol, bmin, bmax, u, cam_o, views)
        rng = np.random.default_rng(0)
        # each step is a bounded sample of the step's frames: about one second of
        # oracle work per frame, the whole run near two and a half minutes
        per_step = min(10.0, max(1.0 * frames_per_step, 150.0 / max(1, args.steps + args.warmup)))
        R = leg.rays_for_budget(per_step, rng)
        measured, full = [], []
        for i in range(args.warmup + args.steps):
            m, f = leg.run(R, rng)
            if i >= args.warmup:
                measured.append(m)
                full.append(f)
        # the metric: frames/s of whole frames at the sample's rays/s; ms_per_step is the
        # measured time of one sampled step (what the timed region really took)
        val = frames_per_step / float(np.mean(full))
        ms = 1e3 * float(np.mean(measured))
        cores, sample = leg.threads, leg.sample_text(R)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": "frames/s", "n_gpus": world,
                          "note": "the FP64 oracle on rank 0's host cores; the other ranks do no work; each step "
                                  "renders a random sample of every frame's rays and value extrapolates its rays/s "
                                  "to whole frames",
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": config,
                          "measured_s_per_step": float(np.mean(measured)),
                          "extrapolated_s_per_full_step": float(np.mean(full)),
                          "rays_per_s": leg.rays_per_step() / float(np.mean(full)),
                          "cpu_baseline": {"value": val, "unit": "frames/s", "cores": cores, "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": val, "unit": "frames/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch

    import paper_2206_08660_gb300 as V

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    V.load()
    ctx = V.vdi_ctx_create(local_rank)
    stream = torch.cuda.current_stream()
    kn = S.tf_knots(wl["tf"])
    vol_d = torch.from_numpy(vol).to(dev)
    t = time.perf_counter()
    vdi = V.vdi_generate(ctx, vol_d, bmin, bmax, kn, V.camera(cam_o.view, cam_o.proj), wl["w"], wl["h"], wl["ns"],
                         wl["tau"], u, u, wl["fmt"])
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t

    def timed_generate(**kw):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = V.vdi_generate(ctx, vol_d, bmin, bmax, kn, V.camera(cam_o.view, cam_o.proj), wl["w"], wl["h"],
                           wl["ns"], wl["tau"], u, u, wl["fmt"], stream=stream, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        counts = V.vdi_download(g, wl["w"], wl["h"], wl["ns"])[2]
        V.vdi_destroy(g)
        hit = counts > 0
        return ms, float(counts[hit].mean()) if hit.any() else 0.0

    generation = {}
    if rank == 0 and not args.no_serving:
        gen_ms, seg_fixed = timed_generate()
        ada_ms, seg_ada = timed_generate(adaptive=True)
        generation = {"fixed_tau_ms": gen_ms, "adaptive_ms": ada_ms, "mean_supersegments_fixed": seg_fixed,
                      "mean_supersegments_adaptive": seg_ada,
                      "note": "one vdi_generate of the workload's VDI, CUDA events; adaptive = Algorithm 3"}
    layout = V.vdi_get_layout(vdi)
    cams = [V.camera(c.view, c.proj) for c in views]
    W, H = wl["W"], wl["H"]
    outs = [torch.empty((H, W, 4), dtype=torch.float16, device=dev) for _ in wl["frames"]]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2
    flush_r = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def flush_l2(k, dirty_only=False):
        # the write evicts every line the frames used; the read then evicts the
        # write's dirty lines, so the next frame starts on a cold, clean L2
        flush.fill_(float(k))
        if not dirty_only:
            flush_r.sum()

    def step(evs=None):
        for i, (az, d_i, d_r) in enumerate(wl["frames"]):
            if evs is not None:
                evs[i][0].record(stream)
            V.vdi_render(vdi, cams[i], W, H, d_i, d_r, outs[i], V.VDI_F16, stream)
            if evs is not None:
                evs[i][1].record(stream)

    clk = ClockSampler(local_rank)  # started before the warm-up so its start-up cost is not timed
    clk.wait_ready()
    for i in range(args.warmup):
        flush_l2(i)
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps, events per frame
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
            for _ in wl["frames"]] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk.mark_start()
    for k in range(args.steps):
        flush_l2(k)
        step(evs[k])
    torch.cuda.synchronize()
    clk.mark_stop()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    frame_ms = np.array([[evs[k][i][0].elapsed_time(evs[k][i][1]) for i in range(frames_per_step)]
                         for k in range(args.steps)])
    step_ms = max_over_ranks(float(frame_ms.sum(axis=1).mean()), dev)
    fps = whole_job_rate(frames_per_step, step_ms, world)
    rays = sum((-(-W // d)) * (-(-H // d)) for (_, d, _) in wl["frames"])
    grays = whole_job_rate(rays, step_ms, world) / 1e9

    # ---- roofline of the exact-render kernel (frames with d_i = d_r = 1)
    exact = [i for i, (_, d_i, d_r) in enumerate(wl["frames"]) if d_i == 1 and d_r == 1]
    touched = [V.touched_bytes(vdi, cams[i], W, H) for i in exact]
    exact_ms = frame_ms[:, exact].mean(axis=0) if exact else np.zeros(0)
    achieved = float(np.sum(touched) / (np.sum(exact_ms) / 1e3) / 1e9) if exact else 0.0
    peak, peak_src = peaks()
    traffic = recorded_traffic(args.workload)
    # the same kernel against the instruction-issue roofline: it re-reads each
    # unique byte from L1/L2 for about twenty rays and is bound by issue, not HBM
    instr = recorded_instructions(args.workload)
    roofline_issue = None
    if exact and instr and all(f"{wl['frames'][i][0]:g}deg" in instr for i in exact):
        ipeak, sms, mhz = issue_peak()
        inst = float(sum(instr[f"{wl['frames'][i][0]:g}deg"] for i in exact))
        ia = inst / (np.sum(exact_ms) / 1e3)
        roofline_issue = {"bound": "issue", "achieved": ia, "peak": ipeak, "unit": "warp instructions/s",
                          "frac": ia / ipeak, "instructions_per_step": inst,
                          "peak_derivation": f"{sms} SMs x 4 schedulers x 1 instruction/cycle x {mhz:g} MHz",
                          "source": "ncu smsp__inst_executed.sum per launch (profiles/render_exact_"
                                    f"{args.workload}.md) / event-timed duration"}

    # ---- the same kernel near the original view (0 and 5 degrees), where a frame
    # streams most of the VDI rather than walking many lists
    near = {}
    for az in (0.0, 5.0):
        cn = S.orbit_camera(bmin, bmax, W / H, az_deg=az, el_deg=wl["el"], zoom=wl["zoom"])
        cam_n = V.camera(cn.view, cn.proj)
        tb = V.touched_bytes(vdi, cam_n, W, H)
        def time_near(dirty_only):
            evn = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(13)]
            for rep in range(13):
                flush_l2(rep, dirty_only)
                evn[rep][0].record(stream)
                V.vdi_render(vdi, cam_n, W, H, 1, 1, outs[0], V.VDI_F16, stream)
                evn[rep][1].record(stream)
            torch.cuda.synchronize()
            return float(np.mean([a.elapsed_time(b) for a, b in evn[3:]]))
        ms_n = time_near(False)
        near[f"{az:g}deg"] = {"ms": ms_n, "algorithmic_bytes": int(tb), "GBps": tb / (ms_n / 1e3) / 1e9,
                              "frac": tb / (ms_n / 1e3) / 1e9 / peaks()[0],
                              "ms_after_write_only_flush": time_near(True)}

    # ---- ablations on the exact frames (not part of the timed step): empty-space
    # skipping off, and the baseline first-supersegment searches of Fig. 4
    def time_variant(**kw):
        ms = []
        for i in exact:
            evs_v = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(8)]
            for rep in range(8):
                flush_l2(rep)
                evs_v[rep][0].record(stream)
                V.vdi_render_ex(vdi, cams[i], W, H, 1, 1, outs[i], V.VDI_F16, stream=stream, **kw)
                evs_v[rep][1].record(stream)
            torch.cuda.synchronize()
            ms.append(float(np.mean([a.elapsed_time(b) for a, b in evs_v[3:]])))
        return [round(m, 4) for m in ms]

    ablation = {"exact_frames_deg": [wl["frames"][i][0] for i in exact],
                "default_ms": time_variant(),
                "ess_ms": time_variant(ess=True),
                "range_blocks_ms": time_variant(blocks=True),
                "binary_search_ms": time_variant(search=V.VDI_SEARCH_BINARY),
                "linear_search_ms": time_variant(search=V.VDI_SEARCH_LINEAR),
                "note": "ms per exact frame, CUDA events, L2 flushed before each repetition"}

    # ---- the same step as one batched persistent launch (vdi_render_batch, CUDA graph,
    # autotuned): throughput of the five views rendered together
    breqs = [V.request(vdi, cams[i], W, H, d_i, d_r, outs[i], V.VDI_F16)
             for i, (az, d_i, d_r) in enumerate(wl["frames"])]
    best, _ = V.vdi_autotune_batch(ctx, breqs, stream)
    for _ in range(3):
        V.vdi_render_batch(ctx, breqs, stream=stream)
    bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(50)]
    for k in range(50):
        flush_l2(k)
        bev[k][0].record(stream)
        V.vdi_render_batch(ctx, breqs, stream=stream)
        bev[k][1].record(stream)
    torch.cuda.synchronize()
    bms = float(np.mean([a.elapsed_time(b) for a, b in bev]))
    batched_step = {"ms_per_step": bms, "frames_per_s": frames_per_step / (bms / 1e3),
                    "warp_shape": int(best.warp_shape), "blocks_per_sm": int(best.blocks_per_sm),
                    "note": "the step's five views in one vdi_render_batch call (persistent launch replayed from "
                            "a CUDA graph, autotuned), L2 flushed between steps; not the headline, which renders "
                            "one view per call"}

    # ---- the batched workload: 4 resident VDIs, 64 mixed requests, one graph launch
    batched_config = {}
    if rank == 0 and not args.no_serving:
        batched_config = batched_config_leg(V, torch, ctx, dev, stream, flush_l2, peak)

    # ---- end to end through the public API: render + read back to pinned host memory
    # Each frame's image is read back on a copy stream while the next frame
    # renders (a viewer's double buffering); the step ends when every image
    # is on the host.
    host = [torch.empty((H, W, 4), dtype=torch.float16, pin_memory=True) for _ in wl["frames"]]
    cam_bytes = 2 * 16 * 8
    e2e_steps = max(3, min(args.steps, 100))
    copy_stream = torch.cuda.Stream()
    done = [torch.cuda.Event() for _ in wl["frames"]]
    torch.cuda.synchronize()
    t = time.perf_counter()
    for k in range(e2e_steps):
        for i, (az, d_i, d_r) in enumerate(wl["frames"]):
            V.vdi_render(vdi, V.camera(views[i].view, views[i].proj), W, H, d_i, d_r, outs[i], V.VDI_F16, stream)
            done[i].record(stream)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(done[i])
                host[i].copy_(outs[i], non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t) / e2e_steps
    e2e = {"value": world * frames_per_step / e2e_s, "unit": "frames/s",
           "h2d_bytes_per_step": cam_bytes * frames_per_step,
           "d2h_bytes_per_step": int(sum(o.numel() * o.element_size() for o in outs))}

    # ---- quality study (Section 6, Fig. 9): each frame against GPU DVR from the same view
    quality = {}
    if rank == 0 and not args.no_quality:
        ref = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
        img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
        rows, dvr_ms = [], []
        q_frames = [(0.0, 1, 1)] + list(wl["frames"])
        for (az, d_i, d_r) in q_frames:
            cn = S.orbit_camera(bmin, bmax, W / H, az_deg=az, el_deg=wl["el"], zoom=wl["zoom"])
            cq = V.camera(cn.view, cn.proj)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            V.vdi_dvr(ctx, vol_d, bmin, bmax, kn, cq, W, H, u, u, ref, V.VDI_F32, stream)
            e1.record(stream)
            V.vdi_render(vdi, cq, W, H, d_i, d_r, img, V.VDI_F32, stream)
            torch.cuda.synchronize()
            dvr_ms.append(e0.elapsed_time(e1))
            s_v, p_v = V.vdi_image_quality(img, ref, V.VDI_F32, stream)
            rows.append({"frame": f"{az:g}deg_di{d_i}_dr{d_r}", "ssim_vs_dvr": s_v, "psnr_vs_dvr": p_v})
        quality = {"frames": rows, "dvr_ms_mean": float(np.mean(dvr_ms)),
                   "note": "SSIM / PSNR over RGB (7x7 windows, data range 1) of each VDI frame against GPU DVR "
                           "of the volume from the same view at a 1-voxel step (vdi_dvr, vdi_image_quality)"}
    del vol_d
    torch.cuda.empty_cache()
    control = {}
    if rank == 0 and not args.no_quality:
        control = {"dr1_target0.5ms": preview_control_leg(V, torch, vdi, wl, bmin, bmax, stream, target_ms=0.5, d_r=1),
                   "dr2_target0.25ms": preview_control_leg(V, torch, vdi, wl, bmin, bmax, stream, target_ms=0.25,
                                                           d_r=2)}

    launches_per_step = sum(1 if d_i == 1 else 2 for (_, d_i, _) in wl["frames"])
    result = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "grays_per_s": grays,
        "exact_frames_per_s": (world * len(exact) / (float(np.sum(exact_ms)) / 1e3)) if exact else None,
        "frame_ms": {f"{az:g}deg_di{d_i}_dr{d_r}": float(m) for (az, d_i, d_r), m in
                     zip(wl["frames"], frame_ms.mean(axis=0))},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "kernel": "render_kernel (exact path)",
                     "algorithmic_bytes_per_launch": [int(b) for b in touched],
                     "frac_per_frame": {f"{wl['frames'][i][0]:g}deg": float(tb / (ms / 1e3) / 1e9 / peak)
                                        for i, tb, ms in zip(exact, touched, exact_ms)}},
        "roofline_issue": roofline_issue,
        "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "ablation": ablation,
        "roofline_near_original_view": near, "batched_step": batched_step, "batched_workload": batched_config,
        "vdi_generate_ms": gen_s * 1e3, "generation": generation, "quality": quality, "preview_control": control, "vdi_bytes": int(layout.depth_bytes + layout.colour_bytes),
    }
    if not args.no_serving:
        srv = serving_leg(V, torch, ctx, dev)
        result["serving"] = srv
        result["serving_p50_ms"] = srv["open_loop"]["p50_ms"]
        result["serving_p99_ms"] = srv["open_loop"]["p99_ms"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            leg = OracleLeg(wl, vol, bmin, bmax, u, cam_o, views)
            rng = np.random.default_rng(0)
            R = leg.rays_for_budget(args.cpu_budget, rng)
            measured, full = leg.run(R, rng)
            # one core on a tenth of the sample, for the per-core rate
            threads = leg.threads
            leg.threads = 1
            R1 = max(256, R // 10)
            _, full1 = leg.run(R1, rng)
            leg.threads = threads
            result["cpu_baseline"] = {"value": frames_per_step / full, "unit": "frames/s", "cores": leg.threads,
                                      "kind": "oracle", "sample": leg.sample_text(R),
                                      "cpu_model": cpu_model(), "rays_per_s": rays / full,
                                      "one_core_frames_per_s": frames_per_step / full1,
                                      "one_core_sample": f"{R1} random rays from each frame, one thread",
                                      "measured_s": measured, "extrapolated_s_per_step": full}
        except Exception as e:  # the oracle must not take the GPU number down with it
            result["cpu_baseline"] = {"value": None, "unit": "frames/s", "cores": os.cpu_count(),
                                      "kind": "oracle", "sample": f"failed: {e}"}
    V.vdi_destroy(vdi)
    V.vdi_ctx_destroy(ctx)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
