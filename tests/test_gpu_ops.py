"""GPU parity of the operator kernels against the FP64 oracle (element by
element), through the C-ABI."""
import numpy as np
import pytest

from oracle import operators as O
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from helpers import dev_to_img, dev_to_planes, img_to_dev, planes_to_dev, rel

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(7)


def _torch_dtype(prec):
    import torch
    return torch.float64 if prec == "fp64" else torch.float32


TOL = {"fp64": 1e-13, "fp32": 2e-6}


def oracle_op(psf, m, level, wavelet):
    A = O.KronOp.from_psf(m, psf)
    for _ in range(level):
        A = A.coarsen(wavelet)
    return A


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("wavelet", ["haar", "db4"])
@pytest.mark.parametrize("psfname", ["gauss9", "gauss15", "motion21", "random5"])
@pytest.mark.parametrize("m", [128, 64, 16])
def test_blur_levels(prec, wavelet, psfname, m):
    import torch
    psf = {"gauss9": I.gaussian_psf(2.0, 9), "gauss15": I.gaussian_psf(3.0, 15),
           "motion21": I.motion_psf(21.0, 30.0, 21), "random5": RNG.random((5, 5))}[psfname]
    S = psf.shape[0]
    if S >= m:
        pytest.skip("PSF larger than the image")
    dt = _torch_dtype(prec)
    for level in range(0, 3):
        mi = m >> level
        if mi < 4:
            break
        A = oracle_op(psf, m, level, wavelet)
        X = RNG.standard_normal((mi, mi))
        for tr in (False, True):
            xd = img_to_dev(X, dt)
            yd = torch.empty_like(xd)
            api.apply_blur(psf, m, xd, yd, level=level, wavelet=wavelet, transpose=tr)
            torch.cuda.synchronize()
            ref = A.applyT(X) if tr else A.apply(X)
            assert rel(dev_to_img(yd, mi), ref) < TOL[prec], (level, tr)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("m", [8, 32, 256])
def test_L_Lt(prec, m):
    import torch
    dt = _torch_dtype(prec)
    X = RNG.standard_normal((m, m))
    q = torch.empty(2 * m * m, device="cuda", dtype=dt)
    api.apply_L(m, img_to_dev(X, dt), q)
    qx, qy, padx, pady = dev_to_planes(q, m)
    rx, ry = O.L_apply(X)
    assert rel(qx, rx) < TOL[prec] and rel(qy, ry) < TOL[prec]
    assert not np.any(padx) and not np.any(pady)
    ax, ay = RNG.standard_normal((m - 1, m)), RNG.standard_normal((m, m - 1))
    xo = torch.empty(m * m, device="cuda", dtype=dt)
    api.apply_Lt(m, planes_to_dev(ax, ay, dt), xo)
    assert rel(dev_to_img(xo, m), O.Lt_apply(ax, ay)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("wavelet", ["haar", "db4"])
@pytest.mark.parametrize("m", [4, 16, 128])
def test_transfers(prec, wavelet, m):
    import torch
    if wavelet == "db4" and m < 8:
        pytest.skip("coarse grid smaller than the filter")
    dt = _torch_dtype(prec)
    X = RNG.standard_normal((m, m))
    y = torch.empty((m // 2) ** 2, device="cuda", dtype=dt)
    api.restrict(m, img_to_dev(X, dt), y, wavelet=wavelet)
    assert rel(dev_to_img(y, m // 2), O.restrict(X, wavelet)) < TOL[prec]
    Y = RNG.standard_normal((m // 2, m // 2))
    x = torch.empty(m * m, device="cuda", dtype=dt)
    api.prolong(m // 2, img_to_dev(Y, dt), x, wavelet=wavelet)
    assert rel(dev_to_img(x, m), O.prolong(Y, wavelet)) < TOL[prec]
    mc = m // 2
    qx, qy = RNG.standard_normal((mc - 1, mc)), RNG.standard_normal((mc, mc - 1))
    qf = torch.empty(2 * m * m, device="cuda", dtype=dt)
    api.aux_prolong(mc, planes_to_dev(qx, qy, dt), qf, wavelet=wavelet)
    fx, fy, padx, pady = dev_to_planes(qf, m)
    rx, ry = O.aux_prolong(qx, qy, wavelet)
    assert rel(fx, rx) < TOL[prec] and rel(fy, ry) < TOL[prec]
    assert not np.any(padx) and not np.any(pady)


def test_blur_full_size_sampled():
    """m = 4096, sigma = 6 on 31 x 31, the launch the largest workloads use:
    sampled outputs against the explicit-loop definition."""
    import torch
    m = 4096
    psf = I.gaussian_psf(6.0, 31)
    X = RNG.random((m, m)).astype(np.float32).astype(np.float64)
    xd = img_to_dev(X, torch.float32)
    yd = torch.empty_like(xd)
    api.apply_blur(psf, m, xd, yd)
    Y = dev_to_img(yd, m)
    R = 15
    for (r, c) in [(0, 0), (m - 1, m - 1), (5, m - 3), (1234, 777), (m // 2, m // 2), (4000, 20)]:
        s = 0.0
        for p in range(-R, R + 1):
            for q in range(-R, R + 1):
                if 0 <= r - p < m and 0 <= c - q < m:
                    s += psf[p + R, q + R] * X[r - p, c - q]
        assert abs(Y[r, c] - s) < 2e-6 * max(1.0, abs(s))
