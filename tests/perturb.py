"""Rounding-sensitivity of the oracle, used to derive parity tolerances.

The method is numerically sensitive (LSQR without reorthogonalisation stopped
at its iteration limit, GCV on small coarse levels). To know how far a
correct implementation in a given storage precision may land from the FP64
oracle, the oracle is rerun with every operator output (A, A^T, L, L^T with
weights) multiplied by (1 + eps * xi), xi ~ N(0, 1) seeded, eps = the unit
roundoff of that precision -- a model of storing each intermediate vector
in that precision (the dense blur matrix of the exact-mode GCV is perturbed
the same way). The distance between that run and the plain oracle run
is the "spread"; the tests accept a GPU result within max(target, 10 x spread).
"""
import contextlib

import numpy as np

from oracle import operators as O
from oracle import solvers as S

UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "bf16": 2.0 ** -8}


@contextlib.contextmanager
def rounding_noise(eps, seed=12345):
    rng = np.random.default_rng(seed)
    orig = {k: getattr(S.Subproblem, k) for k in ("Av", "Atv", "D", "Dt")}
    orig_dense = O.KronOp.dense

    def wrap(f):
        def g(self, x):
            y = f(self, x)
            return y * (1.0 + eps * rng.standard_normal(y.shape))
        return g

    try:
        for k, f in orig.items():
            setattr(S.Subproblem, k, wrap(f))
        def dense_noisy(self):
            y = orig_dense(self)
            return y * (1.0 + eps * rng.standard_normal(y.shape))
        O.KronOp.dense = dense_noisy  # exact-mode GCV matrices
        yield
    finally:
        for k, f in orig.items():
            setattr(S.Subproblem, k, f)
        O.KronOp.dense = orig_dense


def noisy(fn, prec, seed=12345):
    """Run fn() with rounding noise of precision `prec` injected."""
    with rounding_noise(UNIT_ROUNDOFF[prec], seed):
        return fn()
