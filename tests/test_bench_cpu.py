"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
one-line JSON contract: runs on the tiny workload without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "frames/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1 and d["data"] == "synthetic"
    # ms_per_step is the measured time of a sampled step; value extrapolates its rays/s to
    # whole frames (on the tiny workload a step's sample has a whole frame's ray count)
    assert d["value"] > 0 and abs(d["extrapolated_s_per_full_step"] * d["value"] - 1.0) < 1e-9
    assert abs(d["ms_per_step"] - 1e3 * d["measured_s_per_step"]) < 1e-6 * d["ms_per_step"]
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) < 1e-6 * d["ms_per_step"]
    assert d["rays_per_s"] > 0
    assert d["config"]["workload"].startswith("blobs 64^3")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_two_ranks_prints_once():
    """Launched like the multi-GPU benchmark (torchrun, two ranks, rendezvous on
    127.0.0.1): rank 0 alone runs the oracle and prints the line; the other rank
    exits 0 without work."""
    import random

    port = str(random.randint(29600, 29999))
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", port, os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "1", "--gpus", "2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
