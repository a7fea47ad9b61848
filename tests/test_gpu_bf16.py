"""BF16 storage (the precision policy's third mode): image, iterate and
Krylov-vector storage in bfloat16, FP32 accumulation, FP64 reductions, GCV
and stopping tests. End-to-end V-cycle solves against the FP64 oracle; the
tolerance is the larger of the stated BF16 target (1e-3 relative difference)
and ten times the oracle's own spread under bfloat16 unit-roundoff noise
(largest over two perturbed reruns, tests/perturb.py)."""
import numpy as np
import pytest

from oracle import operators as O
from oracle import solvers as S
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from helpers import rel
from perturb import noisy

pytestmark = pytest.mark.gpu

COMBOS = [("irls", "haar", 2, "X"), ("mm", "db4", 2, "D"), ("sb", "haar", 2, "X")]


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


@pytest.mark.parametrize("combo", COMBOS, ids=["-".join(map(str, c)) for c in COMBOS])
def test_solve_bf16_matches_oracle(combo):
    m = 32
    x_true = I.phantom(m, 6, 3, 1)
    g = I.gaussian_factor(1.5, 7)
    A = O.KronOp.from_factors(m, g, g)
    b = I.add_noise(A.apply(x_true), I.noise_direction(m, 101), 0.01)
    # the GPU stores b in bfloat16 (double -> float -> bfloat16, round to
    # nearest even); the oracle sees the same rounded input
    b16 = to_bf16(b)
    r0 = S.mgm(b16, A, *combo)
    reruns = [noisy(lambda: S.mgm(b16, A, *combo), "bf16", seed) for seed in (12345, 777)]
    spread_x = max(rel(q["x"], r0["x"]) for q in reruns)
    r = api.deblur_solve(b16, np.outer(g, g), *combo, precision="bf16")
    d = rel(r["x"], r0["x"])
    assert d <= max(1e-3, 10 * spread_x), (d, spread_x)
    for i in range(len(r0["iters"])):
        spread_it = max(abs(q["iters"][i] - r0["iters"][i]) for q in reruns)
        assert abs(r["iters"][i] - r0["iters"][i]) <= max(1, 2 * spread_it), (i, r["iters"], r0["iters"])
        spread_mu = max(abs(q["mu"][i] - r0["mu"][i]) for q in reruns) / r0["mu"][i]
        assert abs(r["mu"][i] - r0["mu"][i]) <= max(1e-2, 10 * spread_mu) * r0["mu"][i], (i, r["mu"], r0["mu"])


def test_bf16_close_to_fp32_and_reconstructs():
    """Same solve in BF16 and FP32 storage (m = 64): the two reconstructions
    agree to BF16 storage accuracy and both recover the phantom."""
    m = 64
    x_true = I.phantom(m, 12, 6, 0)
    g = I.gaussian_factor(2.0, 9)
    A = O.KronOp.from_factors(m, g, g)
    b = I.add_noise(A.apply(x_true), I.noise_direction(m, 100), 0.01)
    r16 = api.deblur_solve(b, np.outer(g, g), "mm", "haar", 2, "X", precision="bf16")
    r32 = api.deblur_solve(b, np.outer(g, g), "mm", "haar", 2, "X", precision="fp32")
    # bfloat16 keeps 8 significant bits (unit roundoff 2^-8 = 3.9e-3); the
    # deblurring amplifies storage rounding about tenfold here
    assert rel(r16["x"], r32["x"]) < 1e-1
    # both recover the phantom about as well as the method allows here (relative
    # error near 0.3 at sigma = 2, 1 % noise); BF16 storage costs little on top
    e16, e32 = rel(r16["x"], x_true), rel(r32["x"], x_true)
    assert e32 < 0.35 and e16 < e32 + 0.05, (e16, e32)
