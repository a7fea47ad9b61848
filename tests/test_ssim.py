"""SSIM (Wang et al. 2004, the quality index of the paper's Sec. 5) as
bench.ssim computes it, against its definition evaluated window by window."""
import numpy as np

import bench


def brute_ssim(x, y, L, win=11, sigma=1.5):
    r = win // 2
    g = np.exp(-(np.arange(-r, r + 1) ** 2) / (2.0 * sigma * sigma))
    w = np.outer(g, g)
    w /= w.sum()
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    vals = []
    for i in range(x.shape[0] - win + 1):
        for j in range(x.shape[1] - win + 1):
            a, b = x[i:i + win, j:j + win], y[i:i + win, j:j + win]
            ma, mb = (w * a).sum(), (w * b).sum()
            va, vb = (w * (a - ma) ** 2).sum(), (w * (b - mb) ** 2).sum()
            cab = (w * (a - ma) * (b - mb)).sum()
            vals.append(((2 * ma * mb + c1) * (2 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2)))
    return float(np.mean(vals))


def test_ssim_matches_window_definition():
    rng = np.random.default_rng(3)
    x = rng.random((20, 23))
    y = x + 0.1 * rng.standard_normal(x.shape)
    assert abs(bench.ssim(x, y, L=1.0) - brute_ssim(x, y, 1.0)) < 1e-12


def test_ssim_identity_symmetry_and_range():
    rng = np.random.default_rng(4)
    x = rng.random((32, 32))
    y = rng.random((32, 32))
    assert abs(bench.ssim(x, x) - 1.0) < 1e-12
    assert abs(bench.ssim(x, y, L=1.0) - bench.ssim(y, x, L=1.0)) < 1e-12
    assert abs(bench.ssim(x, y, L=1.0)) < 0.1          # independent images: near zero
    assert bench.ssim(x, x + 0.05, L=1.0) < 1.0 - 1e-3   # a shift of the mean lowers it
