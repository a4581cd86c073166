"""The preview-rate PI controller (Section 4.4) on the host, against a
synthetic plant whose frame time grows with the number of rays rendered:
T(s) = t0 + c s^2 for image-space scale s (no GPU needed).

* It settles at the scale whose frame time meets the target (integral action
  leaves no steady error), from above and from below.
* It respects its bounds and does not wind up: after a stretch where even the
  smallest scale is too slow, or the full scale is fast enough, it recovers
  within a few frames once the load changes.
* Under frame-time noise the mean frame time stays on target.
* Ray counts are round(s W) x round(s H), and bad configurations are refused.
"""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def V():
    import paper_2206_08660_gb300 as V

    V.load()
    return V


def plant(t0, c):
    return lambda s: t0 + c * s * s


def run(pi, T, frames, noise=None):
    s, _, _ = pi.current()
    hist = []
    for k in range(frames):
        t = T(s) * (1.0 if noise is None else noise[k])
        hist.append((s, t))
        s, _, _ = pi.update(t)
    return hist


def test_settles_on_the_target(V):
    target = 1.0
    T = plant(0.1, 2.5)  # s* = 0.6
    s_star = math.sqrt((target - 0.1) / 2.5)
    for start in (1.0, 0.2):
        pi = V.PiController(target, 1920, 1080, scale_start=start)
        hist = run(pi, T, 60)
        tail = hist[-10:]
        assert all(abs(t - target) / target < 0.01 for _, t in tail), tail
        assert abs(tail[-1][0] - s_star) < 0.01


def test_bounds_and_no_wind_up(V):
    target = 1.0
    pi = V.PiController(target, 1920, 1080, scale_min=0.1)
    slow = plant(1.5, 2.0)  # even s = 0.1 misses the target
    hist = run(pi, slow, 80)
    assert all(0.1 <= s <= 1.0 for s, _ in hist)
    assert all(abs(s - 0.1) < 1e-12 for s, _ in hist[30:])  # pinned at the lower bound
    # load drops: the controller leaves the bound at once and settles
    T = plant(0.1, 2.5)
    hist2 = run(pi, T, 40)
    assert hist2[3][0] > 0.2
    assert abs(hist2[-1][1] - target) / target < 0.01
    # a plant that is fast enough at full scale pins the scale at 1 without wind-up
    pi = V.PiController(target, 1920, 1080)
    run(pi, plant(0.1, 0.2), 80)
    assert pi.current()[0] == 1.0
    hist3 = run(pi, plant(0.1, 2.5), 40)
    assert hist3[2][0] < 0.95  # reacts within two frames once frames get slow
    assert abs(hist3[-1][1] - target) / target < 0.01


def test_noisy_frame_times_average_on_target(V):
    rng = np.random.default_rng(0)
    noise = rng.uniform(0.9, 1.1, 400)
    pi = V.PiController(2.0, 1920, 1080)
    hist = run(pi, plant(0.2, 4.0), 400, noise)
    mean_t = np.mean([t for _, t in hist[100:]])
    assert abs(mean_t - 2.0) / 2.0 < 0.03


def test_ray_counts_and_invalid_configs(V):
    pi = V.PiController(1.0, 1919, 1081, scale_start=0.5)
    s, w, h = pi.current()
    assert (w, h) == (math.floor(0.5 * 1919 + 0.5), math.floor(0.5 * 1081 + 0.5))  # halves round up
    s, w, h = pi.update(1.0)  # on target: the scale stays
    assert s == 0.5
    bad = [dict(target_ms=0.0), dict(scale_min=0.0), dict(scale_max=1.5), dict(scale_start=0.05),
           dict(kp=-1.0)]
    for kw in bad:
        args = dict(target_ms=1.0, W=64, H=64)
        args.update(kw)
        with pytest.raises(V.VdiError):
            V.PiController(**args)
    with pytest.raises(V.VdiError):
        pi.update(float("nan"))
