"""GPU LSQR (persistent cooperative kernel) against the oracle's LSQR on the
augmented problem of Eq. (augmented), for the IRLS, MM and SB forms."""
import numpy as np
import pytest

from oracle import operators as O
from oracle import solvers as S
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from helpers import dev_to_img, img_to_dev, planes_to_dev, rel
from parity import check
from perturb import noisy

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(11)


def problem(m, sigma=2.0, Sz=9, seed=0):
    x_true = I.phantom(m, 12, 6, seed)
    g = I.gaussian_factor(sigma, Sz)
    A = O.KronOp.from_factors(m, g, g)
    b = I.add_noise(A.apply(x_true), I.noise_direction(m, 100 + seed), 0.01)
    return A, b, x_true, np.outer(g, g)


def aux_for(solver, x, m):
    qx, qy = O.L_apply(x)
    if solver == "irls":
        return S.irls_weights(qx, qy, 0.03), None
    if solver == "mm":
        return S.mm_surrogate(qx, qy, 0.03), None
    d = (S.shrink(qx, 0.005), S.shrink(qy, 0.005))
    g = (qx - d[0] + 0.001 * RNG.standard_normal(qx.shape), qy - d[1])
    return d, g


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("solver", ["irls", "mm", "sb"])
@pytest.mark.parametrize("m", [16, 64, 128])
def test_lsqr_matches_oracle(prec, solver, m):
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    A, b, x_true, psf = problem(m)
    x0 = 0.9 * x_true
    a0, a1 = aux_for(solver, x0, m)
    if prec == "fp32":
        # the oracle sees the float32-rounded values the GPU buffers hold
        f32 = lambda v: v.astype(np.float32).astype(np.float64)
        b, x0 = f32(b), f32(x0)
        a0 = tuple(f32(v) for v in a0)
        a1 = None if a1 is None else tuple(f32(v) for v in a1)
    gamma = 2e-4
    o = S.opts_with()
    sub = S.Subproblem(A, b, weights=a0 if solver == "irls" else None,
                       c=None if solver == "irls" else (a0 if solver == "mm" else (a0[0] - a1[0], a0[1] - a1[1])))
    x_ref, its_ref = sub.solve(gamma, x0, o)
    xo = torch.empty(m * m, device="cuda", dtype=dt)
    its = api.lsqr_solve(psf, m, solver, gamma, img_to_dev(b, dt), img_to_dev(x0, dt),
                         planes_to_dev(*a0, dt), None if a1 is None else planes_to_dev(*a1, dt), xo)
    x = dev_to_img(xo, m)
    target = 1e-10 if prec == "fp64" else 1e-4   # FP32 parity target: 1e-4 relative
    name = f"lsqr[{prec}-{solver}-m{m}]"
    compare_at_iteration(name, sub, gamma, x0, o, prec, its, its_ref, x, x_ref, target)


@pytest.mark.parametrize("direct", [1, 0], ids=["direct", "bands"])
@pytest.mark.parametrize("Sz,sigma", [(3, 0.8), (15, 3.0), (31, 6.0)], ids=["S3", "S15", "S31"])
@pytest.mark.parametrize("solver", ["irls", "mm", "sb"])
def test_lsqr_level0_forms_match_oracle(direct, Sz, sigma, solver):
    """Level 0 of a separable PSF in FP32, applied by the direct Toeplitz
    path (TMA-loaded zero-filled windows, fine_direct = 1) and by the band
    form (fine_direct = 0), each against the oracle: m = 128 (16 tiles, the
    halo crossing the image border on every side), PSF sides 3, 15 and 31
    (the 8-, 16- and 32-tap unrolled convolutions)."""
    import torch
    m = 128
    A, b, x_true, psf = problem(m, sigma, Sz, seed=2)
    x0 = 0.9 * x_true
    a0, a1 = aux_for(solver, x0, m)
    f32 = lambda v: v.astype(np.float32).astype(np.float64)
    b, x0 = f32(b), f32(x0)
    a0 = tuple(f32(v) for v in a0)
    a1 = None if a1 is None else tuple(f32(v) for v in a1)
    gamma = 2e-4
    o = S.opts_with()
    sub = S.Subproblem(A, b, weights=a0 if solver == "irls" else None,
                       c=None if solver == "irls" else (a0 if solver == "mm" else (a0[0] - a1[0], a0[1] - a1[1])))
    x_ref, its_ref = sub.solve(gamma, x0, o)
    dt = torch.float32
    xo = torch.empty(m * m, device="cuda", dtype=dt)
    its = api.lsqr_solve(psf, m, solver, gamma, img_to_dev(b, dt), img_to_dev(x0, dt), planes_to_dev(*a0, dt),
                         None if a1 is None else planes_to_dev(*a1, dt), xo, fine_direct=direct)
    compare_at_iteration(f"lsqr_level0[{'direct' if direct else 'bands'}-S{Sz}-{solver}]", sub, gamma, x0, o,
                         "fp32", its, its_ref, dev_to_img(xo, m), x_ref, 1e-4)


def compare_at_iteration(name, sub, gamma, x0, o, prec, its, its_ref, x, x_ref, target):
    """Iteration count against the oracle's, with the oracle's own spread of
    it under rounding noise; then x. The stopping iteration is a discrete
    decision (rules S1-S3): when the GPU stops at another iteration than the
    oracle, its iterate is compared with the oracle's iterate at the GPU's
    iteration (the oracle rerun with the stopping tolerances off and its
    iteration limit set to the GPU's count), with the spread of that
    fixed-count solve."""
    seeds = (12345, 777, 4242)
    reruns = [noisy(lambda: sub.solve(gamma, x0, o), prec, seed) for seed in seeds]
    spread_it = max(abs(k - its_ref) for _, k in reruns)
    check(name, "iters", abs(its - its_ref), 1, spread_it, detail=(its, its_ref, [k for _, k in reruns]))
    if its != its_ref:
        o = dict(o, lsqr_atol=0.0, lsqr_btol=0.0, lsqr_conlim=1e300, lsqr_maxit=its)
        x_ref, k = sub.solve(gamma, x0, o)
        assert k == its
        reruns = [noisy(lambda: sub.solve(gamma, x0, o), prec, seed) for seed in seeds]
    spread = max(rel(xs, x_ref) for xs, _ in reruns)
    check(name, "x", rel(x, x_ref), target, spread, detail=(its, its_ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("solver", ["irls", "sb"])
def test_lsqr_motion_psf_matches_oracle(prec, solver):
    """The 21-pixel motion blur at 30 degrees (non-separable): level 0 is
    applied by its direct taps, not by its separable terms."""
    import torch
    m = 64
    dt = torch.float64 if prec == "fp64" else torch.float32
    P = I.motion_psf(21.0, 30.0, 21)
    A = O.KronOp.from_psf(m, P)
    x_true = I.phantom(m, 12, 6, 3)
    b = I.add_noise(A.apply(x_true), I.noise_direction(m, 103), 0.01)
    x0 = 0.9 * x_true
    a0, a1 = aux_for(solver, x0, m)
    if prec == "fp32":
        f32 = lambda v: v.astype(np.float32).astype(np.float64)
        b, x0 = f32(b), f32(x0)
        a0 = tuple(f32(v) for v in a0)
        a1 = None if a1 is None else tuple(f32(v) for v in a1)
    gamma = 2e-4
    o = S.opts_with()
    sub = S.Subproblem(A, b, weights=a0 if solver == "irls" else None,
                       c=None if solver == "irls" else (a0[0] - a1[0], a0[1] - a1[1]))
    x_ref, its_ref = sub.solve(gamma, x0, o)
    xo = torch.empty(m * m, device="cuda", dtype=dt)
    its = api.lsqr_solve(P, m, solver, gamma, img_to_dev(b, dt), img_to_dev(x0, dt),
                         planes_to_dev(*a0, dt), None if a1 is None else planes_to_dev(*a1, dt), xo)
    compare_at_iteration(f"lsqr_motion[{prec}-{solver}-m{m}]", sub, gamma, x0, o, prec, its, its_ref,
                         dev_to_img(xo, m), x_ref, 1e-10 if prec == "fp64" else 1e-4)


def test_lsqr_cold_start_and_tiny():
    import torch
    m = 8
    A, b, _, psf = problem(m, 1.0, 5)
    o = S.opts_with(lsqr_warm_start=False)
    sub = S.Subproblem(A, b)
    x_ref, its_ref = sub.solve(1e-3, np.zeros((m, m)), o)
    xo = torch.empty(m * m, device="cuda", dtype=torch.float64)
    ones = (np.ones((m - 1, m)), np.ones((m, m - 1)))
    its = api.lsqr_solve(psf, m, "irls", 1e-3, img_to_dev(b, torch.float64), None,
                         planes_to_dev(*ones, torch.float64), None, xo, lsqr_warm_start=0)
    compare_at_iteration("lsqr_cold_m8", sub, 1e-3, np.zeros((m, m)), o, "fp64", its, its_ref,
                         dev_to_img(xo, m), x_ref, 1e-10)


def test_lsqr_zero_rhs():
    import torch
    m = 32
    _, _, _, psf = problem(m)
    z = torch.zeros(m * m, device="cuda", dtype=torch.float32)
    xo = torch.full((m * m,), 5.0, device="cuda", dtype=torch.float32)
    its = api.lsqr_solve(psf, m, "mm", 1e-3, z, z, torch.zeros(2 * m * m, device="cuda"), None, xo)
    assert its == 0 and float(xo.abs().max()) == 0.0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_autotuned_shapes_give_identical_results(prec):
    """The launch-shape autotuner runs every LSQR shape on the first solve of
    a size class and keeps the fastest; all shapes compute the same result,
    so a tuned context and an untuned one agree bit for bit."""
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    m = 128
    A, b, x_true, psf = problem(m)
    x0 = 0.9 * x_true
    qx, qy = O.L_apply(x0)
    a0 = S.mm_surrogate(qx, qy, 0.03)
    outs = []
    for tune in (True, False):
        ctx = api.Context(0)
        ctx.set_autotune(tune)
        xo = torch.empty(m * m, device="cuda", dtype=dt)
        its = api.lsqr_solve(psf, m, "mm", 2e-4, img_to_dev(b, dt), img_to_dev(x0, dt), planes_to_dev(*a0, dt),
                             None, xo, ctx=ctx)
        outs.append((its, dev_to_img(xo, m)))
        ctx.close()
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])


def test_direct_path_is_taken_and_can_be_turned_off():
    """Level 0 of a separable PSF at m >= 64 in FP32 takes the direct path in
    the LSQR solves and in the GCV Krylov blurs (counted in db_stats);
    fine_direct = 0 turns it off, and a 32 x 32 level never takes it."""
    A, b, _, psf = problem(128, 2.0, 9, seed=4)
    counts = {}
    for label, m, direct in (("on", 128, 1), ("off", 128, 0), ("small", 32, 1)):
        bb = b if m == 128 else problem(32, 2.0, 9, seed=4)[1]
        ctx = api.Context(0)
        api.deblur_solve(bb, psf, "mm", "haar", 2, "X", precision="fp32", ctx=ctx, fine_direct=direct)
        st = ctx.stats()
        ctx.close()
        counts[label] = (st["lsqr_direct_solves"], st["blur_direct_launches"], st["lsqr_launches"])
    assert counts["on"][0] > 0 and counts["on"][1] > 0, counts
    assert counts["off"][0] == 0 and counts["off"][1] == 0, counts
    assert counts["small"][0] == 0 and counts["small"][1] == 0, counts
