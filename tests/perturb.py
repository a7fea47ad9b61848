"""Rounding-sensitivity of the oracle, used to derive parity tolerances.

The method is numerically sensitive (LSQR without reorthogonalisation stopped
at its iteration limit, GCV on small coarse levels). To know how far a
correct implementation in a given storage precision may land from the FP64
oracle, the oracle is rerun with unit-roundoff noise of that precision: every
operator output (A, A^T, L, L^T with weights) is multiplied by
(1 + eps * xi), xi ~ N(0, 1) seeded -- a model of storing each intermediate
vector in that precision (the dense blur matrix of the exact-mode GCV is
perturbed the same way). The blur operator itself is also perturbed once per
rerun, by a fixed diagonal factor diag(1 + eps * xi) on its output (A' = D A,
A'^T = A^T D): the model of an implementation whose operator (here, bands
computed from a factorisation of the PSF) differs from the exact one by a
fixed rounding-level perturbation, not only by independent rounding at every
application. The distance between that run and the plain oracle run is the
"spread".

BF16 storage keeps only some quantities in bfloat16 (the LSQR vectors and
the per-pixel planes: IRLS weights, MM shift, SB d and g) and the rest in
float32 (the outer iterate, the LSQR correction, the GCV Krylov basis). Its
model follows that split: bfloat16 noise on the operator outputs inside the
LSQR solves and on the per-pixel planes, float32 noise inside GCV.
"""
import contextlib

import numpy as np

from oracle import operators as O
from oracle import solvers as S

UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "bf16": 2.0 ** -8}


@contextlib.contextmanager
def rounding_noise(eps, seed=12345, eps_gcv=None, eps_planes=None):
    """eps: noise on operator outputs; eps_gcv (default eps): the same inside
    GCV; eps_planes (default none): noise on the IRLS weights, MM shift and
    SB shrinkage outputs."""
    rng = np.random.default_rng(seed)
    state = {"eps": eps}
    eps_gcv = eps if eps_gcv is None else eps_gcv
    orig = {k: getattr(S.Subproblem, k) for k in ("Av", "Atv", "D", "Dt")}
    orig_apply, orig_applyT = O.KronOp.apply, O.KronOp.applyT
    fixed = {}

    def fixed_factor(shape):
        # one fixed relative perturbation per operator output shape (level)
        if shape not in fixed:
            fixed[shape] = 1.0 + eps * rng.standard_normal(shape)
        return fixed[shape]
    orig_gcv = S.Subproblem.gcv
    orig_dense = O.KronOp.dense
    orig_fn = {k: getattr(S, k) for k in ("irls_weights", "mm_surrogate", "shrink")}

    def noise(y, e):
        return y * (1.0 + e * rng.standard_normal(np.shape(y)))

    def wrap(f):
        def g(self, x):
            return noise(f(self, x), state["eps"])
        return g

    def gcv(self, o):
        saved = state["eps"]
        state["eps"] = eps_gcv
        try:
            return orig_gcv(self, o)
        finally:
            state["eps"] = saved

    def wrap_planes(f):
        def g(*a):
            out = f(*a)
            if isinstance(out, tuple):
                return tuple(noise(v, eps_planes) for v in out)
            return noise(out, eps_planes)
        return g

    def apply_fixed(self, X):
        return orig_apply(self, X) * fixed_factor(X.shape)

    def applyT_fixed(self, Y):
        return orig_applyT(self, Y * fixed_factor(Y.shape))

    try:
        O.KronOp.apply, O.KronOp.applyT = apply_fixed, applyT_fixed
        for k, f in orig.items():
            setattr(S.Subproblem, k, wrap(f))
        S.Subproblem.gcv = gcv

        def dense_noisy(self):
            return noise(orig_dense(self), state["eps"])
        O.KronOp.dense = dense_noisy  # exact-mode GCV matrices
        if eps_planes:
            for k, f in orig_fn.items():
                setattr(S, k, wrap_planes(f))
        yield
    finally:
        O.KronOp.apply, O.KronOp.applyT = orig_apply, orig_applyT
        for k, f in orig.items():
            setattr(S.Subproblem, k, f)
        S.Subproblem.gcv = orig_gcv
        O.KronOp.dense = orig_dense
        for k, f in orig_fn.items():
            setattr(S, k, f)


def noisy(fn, prec, seed=12345):
    """Run fn() with rounding noise of precision `prec` injected."""
    if prec == "bf16":
        ctx = rounding_noise(UNIT_ROUNDOFF["bf16"], seed, eps_gcv=UNIT_ROUNDOFF["fp32"],
                             eps_planes=UNIT_ROUNDOFF["bf16"])
    else:
        ctx = rounding_noise(UNIT_ROUNDOFF[prec], seed)
    with ctx:
        return fn()
