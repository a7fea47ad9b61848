"""Oracle outer solvers (Sec. 2, Alg. 1-3) and the multilevel V-cycle
(Sec. 4, Alg. 4). Test infrastructure only. Float64.

Readings of points the paper leaves open (each is a default option here):
  * K_max = 50 outer iterations per level; RC = +inf when ||x^(k)|| = 0.
  * LSQR: atol = btol = 1e-6, conlim = 1e8, at most 100 iterations, warm
    started from x^(k) (it solves for the correction).
  * GCV mode: exact (the paper's definition) on levels with at most 256
    pixels, projected (see oracle.gcv) above; the projected Krylov basis on a
    level of a few dozen pixels is dominated by rounding noise.
  * GCV schedule: MM and SB estimate gamma at outer iterations k = 0, 1, 2
    and keep the last value; IRLS re-estimates at every outer iteration,
    except on the finest level of a cycle with three or more levels, where
    gamma comes from the unweighted pair {A, L} for k = 0, 1, 2 and from the
    weighted pair at k = 3, then stays fixed (Sec. 3, GSVD schedule).
  * Initialisation (Sec. 4.1): Approach I / coarsest level: x = 0, IRLS
    weights 1, MM shift 0, SB d = g = 0. Approach X: x = W x_coarse; the
    auxiliaries follow from their formulas on x (SB: d = shrink(Lx, tau),
    g = Lx - d). Approach D: x = 0, auxiliaries from the blockwise transfer;
    SB transfers d and g separately.
  * The auxiliary quantity a level returns for Approach D is computed from
    its final iterate: IRLS weights and MM shift by their formulas on the
    final x; SB d and g after the final update.
"""
from __future__ import annotations

import math

import numpy as np

from . import gcv as G
from . import operators as O
from .lsqr import lsqr

DEFAULTS = dict(
    tol_fine=1e-3, tol_coarse=1e-6, kmax=50,
    eps_irls=0.03, eps_mm=0.03, tau_sb=0.005,
    lsqr_atol=1e-6, lsqr_btol=1e-6, lsqr_conlim=1e8, lsqr_maxit=100,
    lsqr_warm_start=True,
    gcv_mode="auto", gcv_exact_max_n=256, gcv_grid=50, gcv_lo=-10.0, gcv_hi=2.0, gcv_tolx=1e-5,
    gcv_estimates=3, proj_dim=40, proj_dim_max=160,
    gamma_fixed=None,
)


def opts_with(**kw):
    o = dict(DEFAULTS)
    o.update(kw)
    return o


# ---- per-pixel steps --------------------------------------------------------

def irls_weights(qx, qy, eps):
    """w_i = max(|(Lx)_i|, eps)^(-1/2) (Sec. 2.1, Alg. 1)."""
    return (np.maximum(np.abs(qx), eps) ** -0.5, np.maximum(np.abs(qy), eps) ** -0.5)


def mm_surrogate(qx, qy, eps):
    """w_i = u_i (1 - (eps^2 / (u_i^2 + eps^2))^(1/2)), u = Lx (Eq. (wreg))."""
    f = lambda u: u * (1.0 - np.sqrt(eps * eps / (u * u + eps * eps)))
    return f(qx), f(qy)


def shrink(x, tau):
    """sign(x) max(|x| - tau, 0) (Sec. 2.3)."""
    return np.sign(x) * np.maximum(np.abs(x) - tau, 0.0)


# ---- the generic subproblem, Eq. (generic_sub) / Eq. (augmented) -------------

class Subproblem:
    """min ||A x - b||^2 + gamma ||D x - c||^2 with D = diag(w) L (IRLS) or L,
    as the augmented least-squares problem of Eq. (augmented)."""

    def __init__(self, A: O.KronOp, b, weights=None, c=None):
        self.A, self.b, self.m = A, b, b.shape[0]
        self.n = self.m * self.m
        self.wv = None if weights is None else O.lvec(*weights)
        self.cv = None if c is None else O.lvec(*c)

    # D and D^T on vectors
    def D(self, x):
        q = O.lvec(*O.L_apply(O.unvec(x, self.m, self.m)))
        return q if self.wv is None else self.wv * q

    def Dt(self, q):
        if self.wv is not None:
            q = self.wv * q
        return O.vec(O.Lt_apply(*O.unlvec(q, self.m)))

    def Av(self, x):
        return O.vec(self.A.apply(O.unvec(x, self.m, self.m)))

    def Atv(self, y):
        return O.vec(self.A.applyT(O.unvec(y, self.m, self.m)))

    def solve(self, gamma, x0, o):
        sg = math.sqrt(gamma)
        nA = self.n
        matvec = lambda v: np.concatenate([self.Av(v), sg * self.D(v)])
        rmatvec = lambda u: self.Atv(u[:nA]) + sg * self.Dt(u[nA:])
        x0v = O.vec(x0)
        c = self.cv if self.cv is not None else 0.0
        if o["lsqr_warm_start"]:
            r0 = np.concatenate([O.vec(self.b) - self.Av(x0v), sg * (c - self.D(x0v))])
        else:
            r0 = np.concatenate([O.vec(self.b), sg * (c * np.ones(len(self.D(x0v))))])
        delta, its = lsqr(matvec, rmatvec, r0, nA, o["lsqr_atol"], o["lsqr_btol"],
                          o["lsqr_conlim"], o["lsqr_maxit"])
        x = (x0v + delta) if o["lsqr_warm_start"] else delta
        return O.unvec(x, self.m, self.m), its

    def gcv(self, o):
        """gamma for this subproblem by GCV (Sec. 3); ``gamma_fixed`` bypasses
        the selection (used by tests that isolate the other steps)."""
        if o.get("gamma_fixed") is not None:
            return float(o["gamma_fixed"])
        bv = O.vec(self.b)
        mode = o["gcv_mode"]
        if mode == "auto":
            mode = "exact" if self.n <= o["gcv_exact_max_n"] else "projected"
        if mode == "exact":
            Ad = self.A.dense()
            Dd = O.L_dense(self.m)
            if self.wv is not None:
                Dd = self.wv[:, None] * Dd
            F = G.factors_exact(Ad, Dd, bv, self.cv, self.n)
            return G.select_gamma(F, o["gcv_lo"], o["gcv_hi"], o["gcv_grid"], o["gcv_tolx"])[0]
        rows_r, rows_c = self.A.middle_rows()
        scale = 1.0 if self.wv is None else float(np.mean(self.wv ** 2))
        trace = G.symbol_trace(rows_r, rows_c, self.m, scale)
        k = min(o["proj_dim"], self.n)
        gamma_prev = None
        while True:
            F = G.factors_projected(self.Av, self.Atv, self.D, self.Dt, bv, self.cv, k, self.n, trace)
            gamma = G.select_gamma(F, o["gcv_lo"], o["gcv_hi"], o["gcv_grid"], o["gcv_tolx"])[0]
            if gamma_prev is not None and abs(gamma - gamma_prev) <= 1e-3 * gamma_prev:
                return gamma
            if 2 * k > min(o["proj_dim_max"], self.n) or k >= self.n:
                return gamma
            gamma_prev = gamma
            k *= 2


def _rc(x_new, x):
    nx = np.linalg.norm(x)
    return math.inf if nx == 0.0 else float(np.linalg.norm(x_new - x) / nx)


# ---- Alg. 1: IRLS -----------------------------------------------------------

def irls(A, b, x0, w0, o, tol, schedule="every", trace=None):
    """IRLS (Alg. 1). ``w0``: initial weights (identity for Approach I,
    transferred for Approach D) or None (from x0). ``schedule``: 'every' or
    'twopass'. Returns (x, mu, outer iterations, lsqr iterations, q)."""
    x = x0.copy()
    mu = None
    inner = 0
    k = 0
    for k in range(o["kmax"]):
        w = w0 if (k == 0 and w0 is not None) else irls_weights(*O.L_apply(x), o["eps_irls"])
        if schedule == "every":
            mu = Subproblem(A, b, weights=w).gcv(o)
        elif k == 0:
            mu = Subproblem(A, b).gcv(o)
        elif k == 3:
            mu = Subproblem(A, b, weights=w).gcv(o)
        x_new, its = Subproblem(A, b, weights=w).solve(mu, x, o)
        inner += its
        rc = _rc(x_new, x)
        x = x_new
        if trace is not None:
            trace.append(dict(k=k, mu=mu, rc=rc, lsqr=its))
        if rc < tol:
            break
    return x, mu, k + 1, inner, irls_weights(*O.L_apply(x), o["eps_irls"])


# ---- Alg. 2: MM -------------------------------------------------------------

def mm(A, b, x0, c0, o, tol, trace=None):
    """MM with the fixed quadratic majorant (Alg. 2, Eq. (MMsolve))."""
    x = x0.copy()
    mu = None
    inner = 0
    k = 0
    for k in range(o["kmax"]):
        c = c0 if (k == 0 and c0 is not None) else mm_surrogate(*O.L_apply(x), o["eps_mm"])
        sub = Subproblem(A, b, c=c)
        if k < o["gcv_estimates"]:
            mu = sub.gcv(o)
        x_new, its = sub.solve(mu, x, o)
        inner += its
        rc = _rc(x_new, x)
        x = x_new
        if trace is not None:
            trace.append(dict(k=k, mu=mu, rc=rc, lsqr=its))
        if rc < tol:
            break
    return x, mu, k + 1, inner, mm_surrogate(*O.L_apply(x), o["eps_mm"])


# ---- Alg. 3: Split Bregman --------------------------------------------------

def sb(A, b, x0, d0, g0, o, tol, trace=None):
    """Split Bregman (Alg. 3, Eq. (Breg3)); d0/g0 are (qx, qy) pairs."""
    x = x0.copy()
    d, g = d0, g0
    lam = None
    inner = 0
    k = 0
    for k in range(o["kmax"]):
        c = (d[0] - g[0], d[1] - g[1])
        sub = Subproblem(A, b, c=c)
        if k < o["gcv_estimates"]:
            lam = sub.gcv(o)
        x_new, its = sub.solve(lam, x, o)
        inner += its
        qx, qy = O.L_apply(x_new)
        dn = (shrink(qx + g[0], o["tau_sb"]), shrink(qy + g[1], o["tau_sb"]))
        g = (g[0] + qx - dn[0], g[1] + qy - dn[1])
        d = dn
        rc = _rc(x_new, x)
        x = x_new
        if trace is not None:
            trace.append(dict(k=k, mu=lam, rc=rc, lsqr=its))
        if rc < tol:
            break
    return x, lam, k + 1, inner, (d, g)


# ---- Alg. 4: multilevel V-cycle ---------------------------------------------

def _zeros_l(m):
    return (np.zeros((m - 1, m)), np.zeros((m, m - 1)))


def level_solve(solver, A, b, init, o, tol, schedule):
    """One level of Alg. 4. ``init`` = ('I',) | ('X', x0) | ('D', q0)."""
    m = b.shape[0]
    kind = init[0]
    x0 = init[1] if kind == "X" else np.zeros((m, m))
    if solver == "irls":
        w0 = (np.ones((m - 1, m)), np.ones((m, m - 1))) if kind == "I" else (init[1] if kind == "D" else None)
        return irls(A, b, x0, w0, o, tol, schedule)
    if solver == "mm":
        c0 = init[1] if kind == "D" else None
        return mm(A, b, x0, c0, o, tol)
    if solver == "sb":
        if kind == "I":
            d0, g0 = _zeros_l(m), _zeros_l(m)
        elif kind == "X":
            qx, qy = O.L_apply(x0)
            d0 = (shrink(qx, o["tau_sb"]), shrink(qy, o["tau_sb"]))
            g0 = (qx - d0[0], qy - d0[1])
        else:
            d0, g0 = init[1]
        return sb(A, b, x0, d0, g0, o, tol)
    raise ValueError(solver)


def mgm(b, A0: O.KronOp, solver, wavelet, levels, transfer, o=None):
    """Multilevel V-cycle (Alg. 4) with levels = n + 1 >= 1 (1 = Approach I).

    Returns dict(x, mu [per level, finest first], iters, inner)."""
    o = o or dict(DEFAULTS)
    As, bs = [A0], [b]
    for _ in range(levels - 1):
        As.append(As[-1].coarsen(wavelet))
        bs.append(O.restrict(bs[-1], wavelet))
    mus, its, inner = [None] * levels, [0] * levels, [0] * levels
    init = ("I",)
    x = q = None
    for i in range(levels - 1, -1, -1):
        if i < levels - 1:
            if transfer == "X":
                init = ("X", O.prolong(x, wavelet))
            else:
                if solver == "sb":
                    (dc, gc) = q
                    init = ("D", (O.aux_prolong(*dc, wavelet), O.aux_prolong(*gc, wavelet)))
                else:
                    init = ("D", O.aux_prolong(*q, wavelet))
        tol = o["tol_coarse"] if i > 0 else o["tol_fine"]
        schedule = "twopass" if (solver == "irls" and levels >= 3 and i == 0) else "every"
        x, mu, k, nin, q = level_solve(solver, As[i], bs[i], init, o, tol, schedule)
        mus[i], its[i], inner[i] = mu, k, nin
    return dict(x=x, mu=mus, iters=its, inner=inner)
