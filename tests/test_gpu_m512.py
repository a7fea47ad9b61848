"""The m = 512 workload on the GPU (FP32 storage) against the FP64 oracle's
stored results: every solver / wavelet / transfer combination of 3-level
V-cycles (Alg. 4 with Alg. 1-3) at 1 % and 5 % noise.

The oracle's results were written by tests/golden/make_m512_oracle.py, which
calls only oracle/ and the input generator: gamma, outer and LSQR iteration
counts per level, and x at 16384 fixed pixels. x is compared on those pixels
(relative 2-norm over the sample, an estimate of the full relative
difference); the outer counts and gamma on every level. The tolerance rule
is that of tests/parity.py, with the oracle's spread (two reruns under
float32 unit-roundoff noise) stored beside its result.
"""
import json
import os

import numpy as np
import pytest

from oracle import operators as O
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from parity import check

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "m512_oracle")


def index():
    p = os.path.join(GOLD, "index.json")
    if not os.path.exists(p):
        return {"cases": {}}
    with open(p) as f:
        return json.load(f)


IDX = index()
CASES = sorted(IDX["cases"])
_B = {}


def observed(noise):
    """b of the workload at one noise level, rounded to float32 (the input
    the oracle solved)."""
    if noise not in _B:
        m = IDX["m"]
        g = I.gaussian_factor(3.0, 15)
        A = O.KronOp.from_factors(m, g, g)
        x_true = I.phantom(m, 40, 20, IDX["seed"])
        b = I.add_noise(A.apply(x_true), I.noise_direction(m, 10_000 + IDX["seed"]), noise)
        _B[noise] = (b.astype(np.float32).astype(np.float64), np.outer(g, g), x_true)
    return _B[noise]


def test_golden_index_complete():
    assert len(CASES) == 24, f"{len(CASES)} of 24 oracle cases present"


@pytest.mark.parametrize("name", CASES)
def test_m512_matches_oracle(name):
    c = IDX["cases"][name]
    b, psf, x_true = observed(c["noise"])
    r = api.deblur_solve(b, psf, c["solver"], c["wavelet"], 3, c["transfer"], precision="fp32")
    d = np.load(os.path.join(GOLD, name + ".npz"))
    idx = np.load(os.path.join(GOLD, "sample_index.npy"))
    xs = r["x"].T.reshape(-1)[idx]                     # column-major vec(X)
    xo = d["x_samples"].astype(np.float64)
    test = f"m512[{name}]"
    check(test, "x(sampled)", float(np.linalg.norm(xs - xo) / np.linalg.norm(xo)), 1e-4, c["spread_x"])
    for i in range(3):
        check(test, f"iters[{i}]", abs(r["iters"][i] - c["iters"][i]), 1, c["spread_iters"][i],
              detail=(r["iters"], c["iters"]))
        check(test, f"mu[{i}]", abs(r["mu"][i] - c["mu"][i]) / c["mu"][i], 1e-2, c["spread_mu"][i],
              detail=(list(map(float, r["mu"])), c["mu"]))
    # the reconstruction is as good as the oracle's (error against the phantom within 1 %)
    rre = float(np.linalg.norm(r["x"] - x_true) / np.linalg.norm(x_true))
    assert abs(rre - c["rre_vs_phantom"]) <= 1e-2 * c["rre_vs_phantom"], (rre, c["rre_vs_phantom"])
