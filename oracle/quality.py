"""Image quality measures of the paper's evaluation (Section 6 and its
supplement), written out from their definitions in FP64 with numpy.

TEST INFRASTRUCTURE, NOT PRODUCT: only tests, the smoke check and the CPU
legs of bench.py use this module.

* SSIM (Wang, Bovik, Sheikh and Simoncelli, 2004) per channel over every
  7 x 7 window that lies inside the image: with the window means mu, the
  sample variances s^2 and sample covariance s_ab (sums of squared deviations
  divided by 49 - 1),
      SSIM = (2 mu_a mu_b + C1)(2 s_ab + C2) / ((mu_a^2 + mu_b^2 + C1)(s_a^2 + s_b^2 + C2)),
  C1 = (0.01 L)^2, C2 = (0.03 L)^2, data range L = 1; the image's SSIM is the
  mean over windows and over the R, G, B channels.
* PSNR = 10 log10(L^2 / MSE), the MSE over every pixel and the R, G, B
  channels.

Images are [H, W, 4] premultiplied RGBA (channels beyond the third are not
used).
"""
import numpy as np

WIN = 7
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def _windows(x):
    """All 7 x 7 windows of a 2-D array, shape [H - 6, W - 6, 7, 7]."""
    return np.lib.stride_tricks.sliding_window_view(x, (WIN, WIN))


def ssim_map(a, b):
    """Per-window, per-channel SSIM, shape [3, H - 6, W - 6]."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    out = []
    n = WIN * WIN
    for c in range(3):
        wa, wb = _windows(a[..., c]), _windows(b[..., c])
        ma, mb = wa.mean(axis=(2, 3)), wb.mean(axis=(2, 3))
        da, db = wa - ma[..., None, None], wb - mb[..., None, None]
        va = (da * da).sum(axis=(2, 3)) / (n - 1)
        vb = (db * db).sum(axis=(2, 3)) / (n - 1)
        vab = (da * db).sum(axis=(2, 3)) / (n - 1)
        out.append(((2 * ma * mb + C1) * (2 * vab + C2)) / ((ma * ma + mb * mb + C1) * (va + vb + C2)))
    return np.stack(out)


def ssim(a, b):
    return float(ssim_map(a, b).mean())


def psnr(a, b):
    a = np.asarray(a, np.float64)[..., :3]
    b = np.asarray(b, np.float64)[..., :3]
    mse = float(((a - b) ** 2).mean())
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)
