"""BF16 storage (the precision policy's third mode): image, auxiliary
planes and Krylov-vector storage in bfloat16, the outer iterate and the LSQR
correction in float32, FP32 accumulation, FP64 scalar recurrences, GCV and
stopping tests. End-to-end V-cycle solves against the FP64 oracle with the
tolerance rule of tests/parity.py: the BF16 target 1e-3 relative in x, 1 % in
gamma and +-1 outer iteration, or three times the oracle's own spread under
bfloat16 unit-roundoff noise where that spread exceeds the target."""
import numpy as np
import pytest

from oracle import operators as O
from oracle import solvers as S
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from helpers import rel
from parity import check_solve
from perturb import noisy

pytestmark = pytest.mark.gpu

COMBOS32 = [("irls", "haar", 2, "X"), ("mm", "db4", 2, "D"), ("sb", "haar", 2, "X")]
COMBOS64 = [(s, "db4", 3, t) for s in ("irls", "mm", "sb") for t in ("X", "D")]


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def bf16_case(m, nr, nd, sigma, S_, seed, noise_seed):
    x_true = I.phantom(m, nr, nd, seed)
    g = I.gaussian_factor(sigma, S_)
    A = O.KronOp.from_factors(m, g, g)
    b = I.add_noise(A.apply(x_true), I.noise_direction(m, noise_seed), 0.01)
    # the GPU stores b in bfloat16 (double -> float -> bfloat16, round to
    # nearest even); the oracle sees the same rounded input
    return A, to_bf16(b), np.outer(g, g), x_true


@pytest.mark.parametrize("combo", COMBOS32, ids=["-".join(map(str, c)) for c in COMBOS32])
def test_solve_bf16_matches_oracle_m32(combo):
    A, b16, psf, _ = bf16_case(32, 6, 3, 1.5, 7, 1, 101)
    r0 = S.mgm(b16, A, *combo)
    reruns = [noisy(lambda: S.mgm(b16, A, *combo), "bf16", seed) for seed in (12345, 777)]
    r = api.deblur_solve(b16, psf, *combo, precision="bf16")
    check_solve(f"bf16_m32[{'-'.join(map(str, combo))}]", r, r0, reruns, 1e-3, rel)


@pytest.mark.parametrize("combo", COMBOS64, ids=["-".join(map(str, c)) for c in COMBOS64])
def test_solve_bf16_matches_oracle_m64_three_levels(combo):
    """m = 64 (sigma = 2 on 9 x 9, 12 rectangles and 6 disks), 3-level Db4
    cycles of every solver under both transfer strategies."""
    A, b16, psf, _ = bf16_case(64, 12, 6, 2.0, 9, 0, 100)
    r0 = S.mgm(b16, A, *combo)
    reruns = [noisy(lambda: S.mgm(b16, A, *combo), "bf16", seed) for seed in (12345, 777)]
    r = api.deblur_solve(b16, psf, *combo, precision="bf16")
    check_solve(f"bf16_m64[{'-'.join(map(str, combo))}]", r, r0, reruns, 1e-3, rel)
