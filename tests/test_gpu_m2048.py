"""The large-image workload on the GPU (BF16 storage) against the FP64
oracle's stored result: m = 2048 phantom, Gaussian sigma = 6 on 31 x 31, 1 %
noise, 5-level Daubechies-4 V-cycles (Alg. 4).

The oracle's result was written by tests/golden/make_m2048_oracle.py (oracle/
and the input generator only; one solve takes about 1.5 h on the CPU), with
reruns under the bfloat16 rounding-noise model of tests/perturb.py where they
are stored (<case>.rerun<seed>.npz). The comparison applies the rule of
tests/parity.py: the BF16 targets (x within 1e-3 relative on the stored
16384-pixel sample, outer iterations within +-1, gamma within 1 % on every
level), or three times the oracle's spread over its reruns where that spread
exceeds the target; without reruns, the targets alone.
"""
import glob
import json
import math
import os

import numpy as np
import pytest

from oracle import operators as O
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from parity import check

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "m2048_oracle")


def index():
    p = os.path.join(GOLD, "index.json")
    if not os.path.exists(p):
        return {"cases": {}}
    with open(p) as f:
        return json.load(f)


IDX = index()
CASES = sorted(IDX["cases"])


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even) through float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("name", CASES)
def test_m2048_matches_oracle(name, prec):
    """The same input (b rounded to bfloat16) solved with BF16 storage (the
    workload's precision; reruns of the oracle under bfloat16 noise give the
    spread) and with FP32 storage (no FP32 reruns exist at this size: the
    stated targets apply)."""
    c = IDX["cases"][name]
    m = IDX["m"]
    g = I.gaussian_factor(6.0, 31)
    A = O.KronOp.from_factors(m, g, g)
    R = int(round(40 * math.sqrt(m / 512)))
    x_true = I.phantom(m, R, R // 2, IDX["seed"])
    b = to_bf16(I.add_noise(A.apply(x_true), I.noise_direction(m, 10_000 + IDX["seed"]), IDX["noise"]))
    r = api.deblur_solve(b, np.outer(g, g), c["solver"], "db4", IDX["levels"], c["transfer"], precision=prec)
    d = np.load(os.path.join(GOLD, name + ".npz"))
    idx = np.load(os.path.join(GOLD, "sample_index.npy"))
    reruns = ([np.load(f) for f in sorted(glob.glob(os.path.join(GOLD, name + ".rerun*.npz")))]
              if prec == "bf16" else [])
    xs = r["x"].T.reshape(-1)[idx]
    xo = d["x_samples"].astype(np.float64)
    rel = lambda a: float(np.linalg.norm(a - xo) / np.linalg.norm(xo))
    test = f"m2048[{prec}-{name}]"
    sx = max((rel(q["x_samples"].astype(np.float64)) for q in reruns), default=0.0)
    check(test, "x(sampled)", rel(xs), 1e-3 if prec == "bf16" else 1e-4, sx)
    for i in range(IDX["levels"]):
        sit = max((abs(int(q["iters"][i]) - c["iters"][i]) for q in reruns), default=0)
        check(test, f"iters[{i}]", abs(r["iters"][i] - c["iters"][i]), 1, sit,
              detail=(r["iters"], c["iters"], [list(map(int, q["iters"])) for q in reruns]))
        smu = max((abs(float(q["mu"][i]) - c["mu"][i]) / c["mu"][i] for q in reruns), default=0.0)
        check(test, f"mu[{i}]", abs(r["mu"][i] - c["mu"][i]) / c["mu"][i], 1e-2, smu,
              detail=(list(map(float, r["mu"])), c["mu"]))
