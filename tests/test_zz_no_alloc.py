"""db_lsqr_solve_static (no device allocation, static 16 MiB workspace)
against db_lsqr_solve on the same inputs, both in the band form of the blur
(the static entry has no tensor maps, so it never takes the direct level-0
path; the context call is asked for the same form with fine_direct = 0, so
the two do the same arithmetic). Collected last so it also runs after every
other GPU test in the same process."""
import numpy as np
import pytest

from oracle import operators as O
from oracle import solvers as S
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I
from paper_2608_17123_b300._lib import DeblurError

from helpers import dev_to_img, img_to_dev, planes_to_dev, rel

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-6}


def setup(m, solver, prec):
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    x_true = I.phantom(m, 12, 6, 3)
    g = I.gaussian_factor(2.0, 9)
    A = O.KronOp.from_factors(m, g, g)
    b = I.add_noise(A.apply(x_true), I.noise_direction(m, 7), 0.01)
    x0 = 0.9 * x_true
    qx, qy = O.L_apply(x0)
    if solver == "irls":
        a0, a1 = S.irls_weights(qx, qy, 0.03), None
    elif solver == "mm":
        a0, a1 = S.mm_surrogate(qx, qy, 0.03), None
    else:
        d = (S.shrink(qx, 0.005), S.shrink(qy, 0.005))
        a0, a1 = d, (qx - d[0], qy - d[1])
    args = (img_to_dev(b, dt), img_to_dev(x0, dt), planes_to_dev(*a0, dt),
            None if a1 is None else planes_to_dev(*a1, dt))
    return np.outer(g, g), args, dt


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("solver", ["irls", "mm", "sb"])
@pytest.mark.parametrize("m", [64, 256])
def test_static_matches_context_path(m, solver, prec):
    import torch
    psf, (b, x0, a0, a1), dt = setup(m, solver, prec)
    gamma = 3e-4
    x_ref = torch.empty(m * m, device="cuda", dtype=dt)
    its_ref = api.lsqr_solve(psf, m, solver, gamma, b, x0, a0, a1, x_ref, fine_direct=0)
    outs = []
    for _ in range(2):                       # two calls in a row
        xs = torch.empty(m * m, device="cuda", dtype=dt)
        its = api.lsqr_solve_static(psf, m, solver, gamma, b, x0, a0, a1, xs)
        outs.append((dev_to_img(xs, m), its))
    ref = dev_to_img(x_ref, m)
    for x, its in outs:
        assert its == its_ref
        assert rel(x, ref) <= TOL[prec], rel(x, ref)


def test_static_call_allocates_nothing():
    import torch
    m = 128
    psf, (b, x0, a0, _), dt = setup(m, "mm", "fp32")
    xs = torch.empty(m * m, device="cuda", dtype=dt)
    api.lsqr_solve_static(psf, m, "mm", 1e-3, b, x0, a0, None, xs)      # loads and looks up the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    api.lsqr_solve_static(psf, m, "mm", 1e-3, b, x0, a0, None, xs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_rejects_oversized():
    import torch
    m = 512
    b = torch.zeros(m * m, device="cuda", dtype=torch.float32)
    x = torch.empty(m * m, device="cuda", dtype=torch.float32)
    with pytest.raises(DeblurError, match="at most 256"):
        api.lsqr_solve_static(np.ones((3, 3)) / 9, m, "mm", 1e-3, b, None, None, None, x)
    b2 = torch.zeros(64 * 64, device="cuda", dtype=torch.float32)
    x2 = torch.empty(64 * 64, device="cuda", dtype=torch.float32)
    with pytest.raises(DeblurError, match="at most 31"):
        api.lsqr_solve_static(np.ones((33, 33)) / 33 ** 2, 64, "mm", 1e-3, b2, None, None, None, x2)
