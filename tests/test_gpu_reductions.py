"""The reduction behind the LSQR norms (the Golub-Kahan scalars alpha and
beta of Sec. 3) against a float64 reduction of the same values.

The library keeps its sums on the FP32 pipe: every square enters exactly (the
rounding error of the float product is recovered with an FMA), partial sums
are double-float pairs (hi + lo) within a 1024-element tile, and the tile
partials are added in tile order, again as double-float pairs. Each
double-float addition is exact up to about 2 u^2 of the running sum (u =
2^-24), so the relative error of a sum of n non-negative terms is bounded by
about n * 2^-47 in the worst case (~3e-8 at n = 4.2M), and is of order
sqrt(n) * 2^-48 in practice. The tests hold it to 1e-12 on the vector sizes
of the m = 512 and m = 2048 workloads, and show that a plain float32
reduction of the same values misses that bound by orders of magnitude.
"""
import math

import numpy as np
import pytest

from paper_2608_17123_b300 import api

pytestmark = pytest.mark.gpu


def exact_sumsq(v):
    """Exact sum of the squares of float32/bfloat16 values: each square is
    exact in float64 and math.fsum adds them without rounding error."""
    d = v.astype(np.float64)
    return math.fsum((d * d).tolist())


@pytest.mark.parametrize("n", [512 * 512, 3 * 512 * 512 + 37, 2048 * 2048])
@pytest.mark.parametrize("dist", ["normal", "wide"])
def test_sumsq_float32_matches_float64(n, dist):
    import torch
    rng = np.random.default_rng(n + len(dist))
    if dist == "normal":
        x = rng.standard_normal(n).astype(np.float32)
    else:   # magnitudes over twelve decades
        x = (rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 6, n)).astype(np.float32)
    ref = exact_sumsq(x)
    got = api.sumsq(torch.from_numpy(x).cuda())
    err = abs(got - ref) / ref
    assert err <= 1e-12, err
    # a float32 running sum of float32 squares is far from this
    naive = float(np.cumsum((x * x).astype(np.float32), dtype=np.float32)[-1])
    assert abs(naive - ref) / ref > 100 * max(err, 1e-16)


def test_sumsq_bfloat16_and_float64():
    import torch
    rng = np.random.default_rng(5)
    x = rng.standard_normal(1 << 20)
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16)
    ref_b = exact_sumsq(xb.float().numpy())
    assert abs(api.sumsq(xb.cuda()) - ref_b) / ref_b <= 1e-12
    ref_d = math.fsum((x * x).tolist())
    assert abs(api.sumsq(torch.from_numpy(x).cuda()) - ref_d) / ref_d <= 1e-13
