"""Pins of the oracle's image-quality measures (SSIM and PSNR, Section 6)
against closed forms of their definitions.

* Identical images: SSIM = 1, PSNR = +inf.
* A constant offset d: PSNR = 10 log10(1 / d^2).
* Two constant images: every window has zero variance, so SSIM reduces to the
  luminance term (2 a b + C1) / (a^2 + b^2 + C1) per channel.
* A single bright pixel in an empty image: exactly the 7 x 7 windows that
  contain it differ, each with mu_b = v / 49 and s_b^2 = v^2 (1 - 1/49) / 48,
  which fixes the window size, the border rule (only windows inside the
  image), the sample-variance divisor and C1, C2 at once.
"""
import numpy as np

from oracle import quality as Q

C1, C2 = 0.01 ** 2, 0.03 ** 2  # (K1 L)^2, (K2 L)^2 with K1 = 0.01, K2 = 0.03, L = 1


def rgba(h, w, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, (h, w, 4))
    a[..., :3] *= a[..., 3:4]
    return a


def test_identical_images():
    a = rgba(20, 30, 0)
    assert abs(Q.ssim(a, a) - 1.0) < 1e-12
    assert Q.psnr(a, a) == float("inf")


def test_psnr_of_a_constant_offset():
    a = rgba(16, 16, 1)
    for d in (0.5, 0.1, 0.01):
        b = a.copy()
        b[..., :3] += d
        assert abs(Q.psnr(b, a) - 10 * np.log10(1 / d ** 2)) < 1e-9
    # alpha is not part of the measure
    b = a.copy()
    b[..., 3] = 0
    assert Q.psnr(b, a) == float("inf")


def test_ssim_of_two_constant_images():
    a = np.zeros((12, 15, 4))
    b = np.zeros((12, 15, 4))
    ca, cb = (0.2, 0.5, 0.9), (0.3, 0.5, 0.1)
    for c in range(3):
        a[..., c], b[..., c] = ca[c], cb[c]
    expect = np.mean([(2 * x * y + C1) / (x * x + y * y + C1) for x, y in zip(ca, cb)])
    assert abs(Q.ssim(a, b) - expect) < 1e-12


def test_single_bright_pixel():
    H, W, v = 24, 20, 0.8
    a = np.zeros((H, W, 4))
    b = np.zeros((H, W, 4))
    b[11, 9, 1] = v  # green channel only, at least 6 pixels from every border
    n = 49
    mu = v / n
    var = (v * v - n * mu * mu) / (n - 1)
    s_hit = (C1 / (mu * mu + C1)) * (C2 / (var + C2))
    windows = (H - 6) * (W - 6)
    expect = (3 * windows - 49 + 49 * s_hit) / (3 * windows)
    assert abs(Q.ssim(a, b) - expect) < 1e-12
    # the same pixel on the border: only the windows inside the image that contain it count
    b2 = np.zeros((H, W, 4))
    b2[0, 0, 1] = v
    assert abs(Q.ssim(a, b2) - (3 * windows - 1 + s_hit) / (3 * windows)) < 1e-12


def test_ssim_is_symmetric_and_drops_with_noise():
    a = rgba(32, 32, 2)
    rng = np.random.default_rng(3)
    prev = 1.0
    for s in (0.01, 0.05, 0.2):
        b = np.clip(a + rng.normal(0, s, a.shape), 0, 1)
        v = Q.ssim(a, b)
        assert abs(v - Q.ssim(b, a)) < 1e-12
        assert v < prev
        prev = v
