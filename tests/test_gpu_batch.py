"""Batched solves (one scheduler step = one outer iteration of every
unfinished problem; their LSQR solves share one persistent launch) give the
same results as separate solves: same kernels and the same per-problem
arithmetic, so the comparison is to rounding (in practice bit-exact)."""
import numpy as np
import pytest

from oracle import operators as O
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from helpers import rel

pytestmark = pytest.mark.gpu


def make(m, sigma, Sz, seed, noise=0.01):
    x_true = I.phantom(m, 8, 4, seed)
    g = I.gaussian_factor(sigma, Sz)
    A = O.KronOp.from_factors(m, g, g)
    return I.add_noise(A.apply(x_true), I.noise_direction(m, 300 + seed), noise), np.outer(g, g)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_equals_separate_solves(prec):
    specs = [(64, 2.0, 9, 0, "irls", "haar", 2, "X"), (32, 1.5, 7, 1, "mm", "db4", 3, "D"),
             (128, 3.0, 15, 2, "sb", "haar", 3, "X"), (64, 1.5, 7, 3, "mm", "haar", 1, "X"),
             (32, 2.0, 9, 4, "irls", "db4", 3, "X")]
    probs = []
    for (m, sg, Sz, seed, solver, wv, lv, tr) in specs:
        b, psf = make(m, sg, Sz, seed)
        probs.append(dict(b=b, psf=psf, solver=solver, wavelet=wv, levels=lv, transfer=tr))
    batch = api.deblur_solve_batch(probs, precision=prec)
    for pr, rb in zip(probs, batch):
        rs = api.deblur_solve(pr["b"], pr["psf"], pr["solver"], pr["wavelet"], pr["levels"], pr["transfer"],
                              precision=prec)
        assert rb["iters"] == rs["iters"] and rb["inner"] == rs["inner"]
        assert rel(rb["x"], rs["x"]) <= 1e-12
        assert np.allclose(rb["mu"], rs["mu"], rtol=1e-12, atol=0)


def test_batch_of_one_and_mixed_precisionless_defaults():
    b, psf = make(64, 2.0, 9, 7)
    rb = api.deblur_solve_batch([dict(b=b, psf=psf, solver="sb", wavelet="db4", levels=2, transfer="D")])[0]
    rs = api.deblur_solve(b, psf, "sb", "db4", 2, "D")
    assert rb["iters"] == rs["iters"] and rel(rb["x"], rs["x"]) <= 1e-12


def test_batched_and_served_match_oracle():
    """Batched and served FP32 solves of three m = 32 cases against the FP64
    oracle, with the same rule as the single solves (tests/parity.py)."""
    from parity import check_solve
    from test_gpu_solve import case, references, storage_rounded
    A, b, _, psf = case(32, 1.5, 7, 6, 3, 1, 0.01)
    combos = [("irls", "haar", 2, "X"), ("mm", "db4", 3, "D"), ("sb", "haar", 2, "D")]
    b32 = storage_rounded(b, "fp32")
    probs = [dict(b=b32, psf=psf, solver=c[0], wavelet=c[1], levels=c[2], transfer=c[3]) for c in combos]
    batch = api.deblur_solve_batch(probs, precision="fp32")
    srv = api.Server(max_resident=2, max_m=32, ctx=api.Context(0))
    try:
        tickets = [srv.submit(b32, psf, *c) for c in combos]
        served = [srv.poll(t)[0] for t in tickets]
    finally:
        srv.close()
    for c, rb, rs in zip(combos, batch, served):
        r0, r1 = references(A, b, c, "fp32")
        tag = "-".join(map(str, c))
        check_solve(f"batched_m32[{tag}]", rb, r0, r1, 1e-4, rel)
        check_solve(f"served_m32[{tag}]", rs, r0, r1, 1e-4, rel)
