"""GPU GCV selection (projected form, Sec. 3) against the oracle's."""
import numpy as np
import pytest

from oracle import operators as O
from oracle import solvers as S
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from helpers import img_to_dev, planes_to_dev
from parity import check
from perturb import noisy

pytestmark = pytest.mark.gpu


def problem(m, sigma=2.0, Sz=9, seed=0):
    x_true = I.phantom(m, 12, 6, seed)
    g = I.gaussian_factor(sigma, Sz)
    A = O.KronOp.from_factors(m, g, g)
    b = I.add_noise(A.apply(x_true), I.noise_direction(m, 100 + seed), 0.01)
    return A, b, x_true, np.outer(g, g)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["plain", "irls", "mm", "sb"])
@pytest.mark.parametrize("m", [16, 32, 64])
def test_gcv_matches_oracle(prec, kind, m):
    """m = 16 (256 pixels) runs the exact mode, m = 32, 64 the projected one."""
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    A, b, x_true, psf = problem(m)
    x0 = 0.8 * x_true + 0.02
    qx, qy = O.L_apply(x0)
    a0 = a1 = None
    if kind == "irls":
        a0 = S.irls_weights(qx, qy, 0.03)
    elif kind == "mm":
        a0 = S.mm_surrogate(qx, qy, 0.03)
    elif kind == "sb":
        a0 = (S.shrink(qx, 0.005), S.shrink(qy, 0.005))
        a1 = (0.5 * (qx - a0[0]), 0.5 * (qy - a0[1]))
    # the oracle sees exactly the inputs the GPU call receives (FP32 buffers
    # hold b and the planes rounded to float32)
    rnd = (lambda v: v.astype(np.float32).astype(np.float64)) if prec == "fp32" else (lambda v: v)
    b = rnd(b)
    a0 = None if a0 is None else tuple(rnd(v) for v in a0)
    a1 = None if a1 is None else tuple(rnd(v) for v in a1)
    if kind == "irls":
        sub = S.Subproblem(A, b, weights=a0)
    elif kind == "mm":
        sub = S.Subproblem(A, b, c=a0)
    elif kind == "sb":
        sub = S.Subproblem(A, b, c=(a0[0] - a1[0], a0[1] - a1[1]))
    else:
        sub = S.Subproblem(A, b)
    g_ref = sub.gcv(S.opts_with())
    spread = max(abs(noisy(lambda: sub.gcv(S.opts_with()), prec, seed) - g_ref) / g_ref
                 for seed in (12345, 777, 4242))
    solver = {"plain": "mm", "irls": "irls", "mm": "mm", "sb": "sb"}[kind]
    g = api.gcv_select(psf, m, solver, img_to_dev(b, dt),
                       None if a0 is None else planes_to_dev(*a0, dt),
                       None if a1 is None else planes_to_dev(*a1, dt))
    check(f"gcv[{prec}-{kind}-m{m}]", "gamma", abs(g - g_ref) / g_ref, 1e-2, spread, detail=(g, g_ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["plain", "mm"])
def test_gcv_exact_mode_tiny_level(prec, kind):
    """8 x 8 level with a 5 x 5 PSF: exact mode on both sides; the minimiser
    lies at the small-gamma end, where only a cancellation-free numerator is
    meaningful."""
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    A, b, x_true, psf = problem(8, 1.2, 5)
    a0 = None
    if kind == "mm":
        qx, qy = O.L_apply(0.8 * x_true)
        a0 = S.mm_surrogate(qx, qy, 0.03)
    if prec == "fp32":          # the oracle sees the float32-rounded inputs the GPU receives
        b = b.astype(np.float32).astype(np.float64)
        a0 = None if a0 is None else tuple(v.astype(np.float32).astype(np.float64) for v in a0)
    sub = S.Subproblem(A, b, c=a0)
    g_ref = sub.gcv(S.opts_with())
    spread = max(abs(noisy(lambda: sub.gcv(S.opts_with()), prec, seed) - g_ref) / g_ref
                 for seed in (12345, 777, 4242))
    g = api.gcv_select(psf, 8, "mm", img_to_dev(b, dt), None if a0 is None else planes_to_dev(*a0, dt))
    tol = 1e-6 if prec == "fp64" else 1e-2
    check(f"gcv_exact[{prec}-{kind}-m8]", "gamma", abs(g - g_ref) / g_ref, tol, spread, detail=(g, g_ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["plain", "irls", "mm", "sb"])
def test_gcv_exact_mode_m32(prec, kind):
    """32 x 32 level (1024 pixels, the largest exact level the options allow)
    with the exact mode on both sides (Sec. 3: the GCV function of the whole
    pencil, trace from its eigenvalues). Here the projected rule would be off
    by 0.2 % (plain), 15 % (MM) and 85 % (IRLS), so the test tells the two
    modes apart. FP64: both sides stop Brent's search within tolx = 1e-5 in
    log10 gamma, so they agree to 2 * ln(10) * 1e-5 < 1e-4 relative."""
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    m = 32
    A, b, x_true, psf = problem(m)
    qx, qy = O.L_apply(0.8 * x_true + 0.02)
    a0 = a1 = None
    if kind == "irls":
        a0 = S.irls_weights(qx, qy, 0.03)
    elif kind == "mm":
        a0 = S.mm_surrogate(qx, qy, 0.03)
    elif kind == "sb":
        a0 = (S.shrink(qx, 0.005), S.shrink(qy, 0.005))
        a1 = (0.5 * (qx - a0[0]), 0.5 * (qy - a0[1]))
    rnd = (lambda v: v.astype(np.float32).astype(np.float64)) if prec == "fp32" else (lambda v: v)
    b = rnd(b)
    a0 = None if a0 is None else tuple(rnd(v) for v in a0)
    a1 = None if a1 is None else tuple(rnd(v) for v in a1)
    if kind == "irls":
        sub = S.Subproblem(A, b, weights=a0)
    elif kind == "mm":
        sub = S.Subproblem(A, b, c=a0)
    elif kind == "sb":
        sub = S.Subproblem(A, b, c=(a0[0] - a1[0], a0[1] - a1[1]))
    else:
        sub = S.Subproblem(A, b)
    o = S.opts_with(gcv_exact_max_n=1024)
    g_ref = sub.gcv(o)
    spread = max(abs(noisy(lambda: sub.gcv(o), prec, seed) - g_ref) / g_ref for seed in (12345, 777, 4242))
    solver = {"plain": "mm", "irls": "irls", "mm": "mm", "sb": "sb"}[kind]
    g = api.gcv_select(psf, m, solver, img_to_dev(b, dt),
                       None if a0 is None else planes_to_dev(*a0, dt),
                       None if a1 is None else planes_to_dev(*a1, dt), exact_max_pixels=1024)
    tol = 1e-4 if prec == "fp64" else 1e-2
    check(f"gcv_exact[{prec}-{kind}-m32]", "gamma", abs(g - g_ref) / g_ref, tol, spread, detail=(g, g_ref))
