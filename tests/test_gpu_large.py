"""Full-size checks at m = 2048 (the large workload: Gaussian sigma = 6 on
31 x 31 and the 21-pixel motion blur at 30 degrees, 5-level Db4 cycles):
the blur element by element against the oracle, five LSQR iterations against
the oracle's, and one complete V-cycle in BF16 and FP32 storage compared with
each other and with the phantom (the oracle's full solve at this size is out
of reach; these are the properties that hold at any size)."""
import numpy as np
import pytest

from oracle import operators as O
from oracle import solvers as S
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from helpers import dev_to_img, img_to_dev, planes_to_dev, rel

pytestmark = pytest.mark.gpu
M = 2048


def oracle_op(name):
    if name == "gauss31":
        g = I.gaussian_factor(6.0, 31)
        return O.KronOp.from_factors(M, g, g), np.outer(g, g)
    P = I.motion_psf(21.0, 30.0, 21)
    return O.KronOp.from_psf(M, P), P


@pytest.mark.parametrize("name", ["gauss31", "motion21"])
def test_blur_m2048(name):
    import torch
    A, psf = oracle_op(name)
    X = I.phantom(M, 40, 20, 5)
    y = torch.empty(M * M, device="cuda", dtype=torch.float32)
    api.apply_blur(psf, M, img_to_dev(X, torch.float32), y)
    assert rel(dev_to_img(y, M), A.apply(X)) < 2e-6
    api.apply_blur(psf, M, img_to_dev(X, torch.float32), y, transpose=True)
    assert rel(dev_to_img(y, M), A.applyT(X)) < 2e-6


def test_lsqr_m2048_five_iterations():
    import torch
    A, psf = oracle_op("gauss31")
    x_true = I.phantom(M, 40, 20, 6)
    b = I.add_noise(A.apply(x_true), I.noise_direction(M, 106), 0.01)
    x0 = 0.9 * x_true
    qx, qy = O.L_apply(x0)
    c = S.mm_surrogate(qx, qy, 0.03)
    o = S.opts_with(lsqr_maxit=5, lsqr_atol=0.0, lsqr_btol=0.0)
    x_ref, its_ref = S.Subproblem(A, b, c=c).solve(1e-3, x0, o)
    xo = torch.empty(M * M, device="cuda", dtype=torch.float32)
    its = api.lsqr_solve(psf, M, "mm", 1e-3, img_to_dev(b, torch.float32), img_to_dev(x0, torch.float32),
                         planes_to_dev(*c, torch.float32), None, xo, lsqr_maxit=5, lsqr_atol=0.0, lsqr_btol=0.0)
    assert its == its_ref == 5
    assert rel(dev_to_img(xo, M), x_ref) < 1e-5


def test_solve_m2048_bf16_and_fp32():
    A, psf = oracle_op("gauss31")
    x_true = I.phantom(M, 40, 20, 7)
    b = I.add_noise(A.apply(x_true), I.noise_direction(M, 107), 0.01)
    r32 = api.deblur_solve(b, psf, "mm", "db4", 5, "X", precision="fp32")
    r16 = api.deblur_solve(b, psf, "mm", "db4", 5, "X", precision="bf16")
    e32, e16 = rel(r32["x"], x_true), rel(r16["x"], x_true)
    assert e32 < 0.5 and abs(e16 - e32) < 0.02 * max(e32, 1e-3) + 5e-3, (e32, e16)
    assert rel(r16["x"], r32["x"]) < 5e-2
    assert all(mu > 0 for mu in r32["mu"]) and len(r32["iters"]) == 5
