"""Pins for the oracle's multilevel driver (Alg. 4 with Alg. 1-3 on every
level), its GCV schedule (Sec. 3) and the edge handling of the GCV search.

The multilevel reference in this file is composed from dense matrices
written out from the paper's statements, sharing nothing with oracle/ but
the input generator:
  * W1 from the printed filter taps (tests/golden/filters.txt), placed as the
    analysis display of Sec. 4 places them ((W1^T)[r, (2r + k) mod m] = h_k);
  * A^(0) the zero-boundary Kronecker blur of Sec. 5, A^(i) = W^T A^(i-1) W
    and b^(i) = W^T b^(i-1) as dense products (Alg. 4);
  * L = [I kron D; D kron I] with the forward difference D (Sec. 4.2);
  * every l2 subproblem of Alg. 1-3 solved by a dense least-squares solve of
    Eq. (augmented);
  * the initialisations of Sec. 4.1 (Approach X: x = W x_coarse, auxiliaries
    from their formulas on x, SB's d = shrink(Lx), g = Lx - d) and Sec. 4.2
    (Approach D: x = 0, the blockwise transfer of the IRLS weights, the MM
    shift, or SB's d and g separately).
gamma is fixed, so the comparison isolates the driver; the oracle's LSQR runs
to full accuracy, so the two agree to rounding. A wrong branch (say the
transferred weights reused after k = 0, or Approach D starting from W
x_coarse) moves the result by far more than the tolerance.
"""
import math
import os

import numpy as np
import pytest

from oracle import gcv as G
from oracle import operators as O
from oracle import solvers as S
from paper_2608_17123_b300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
EPS, TAU, GAMMA = 0.03, 0.005, 2e-3


def printed_taps(wavelet):
    with open(os.path.join(HERE, "golden", "filters.txt")) as f:
        for line in f:
            parts = line.split()
            if parts and parts[0] == wavelet:
                return np.array([float(v) for v in parts[1:]])
    raise KeyError(wavelet)


def w1_dense(m, wavelet):
    h = printed_taps(wavelet)
    Wt = np.zeros((m // 2, m))
    for r in range(m // 2):
        for k, hk in enumerate(h):
            Wt[r, (2 * r + k) % m] += hk
    return Wt.T


def toeplitz_dense(m, g):
    R = len(g) // 2
    T = np.zeros((m, m))
    for i in range(m):
        for j in range(m):
            if abs(i - j) <= R:
                T[i, j] = g[i - j + R]
    return T


def grad_dense(m):
    D = np.zeros((m - 1, m))
    for j in range(m - 1):
        D[j, j], D[j, j + 1] = -1.0, 1.0
    return np.vstack([np.kron(np.eye(m), D), np.kron(D, np.eye(m))])


def lsq(A, b, gamma, Dm, c):
    Ah = np.vstack([A, math.sqrt(gamma) * Dm])
    bh = np.concatenate([b, math.sqrt(gamma) * c])
    return np.linalg.lstsq(Ah, bh, rcond=None)[0]


def irls_w(q):
    return np.maximum(np.abs(q), EPS) ** -0.5


def mm_c(q):
    return q * (1.0 - np.sqrt(EPS * EPS / (q * q + EPS * EPS)))


def shrink(q):
    return np.sign(q) * np.maximum(np.abs(q) - TAU, 0.0)


def level_dense(solver, A, b, m, init, kmax):
    """kmax outer iterations of Alg. 1, 2 or 3 on one level (gamma fixed)."""
    Lm = grad_dense(m)
    nl = Lm.shape[0]
    kind = init[0]
    x = init[1] if kind == "X" else np.zeros(m * m)
    if solver == "irls":
        w0 = np.ones(nl) if kind == "I" else (init[1] if kind == "D" else None)
        for k in range(kmax):
            w = w0 if (k == 0 and w0 is not None) else irls_w(Lm @ x)
            x = lsq(A, b, GAMMA, w[:, None] * Lm, np.zeros(nl))
        return x, irls_w(Lm @ x)
    if solver == "mm":
        c0 = init[1] if kind == "D" else None
        for k in range(kmax):
            c = c0 if (k == 0 and c0 is not None) else mm_c(Lm @ x)
            x = lsq(A, b, GAMMA, Lm, c)
        return x, mm_c(Lm @ x)
    if kind == "I":
        d, g = np.zeros(nl), np.zeros(nl)
    elif kind == "X":
        q = Lm @ x
        d = shrink(q)
        g = q - d
    else:
        d, g = init[1]
    for k in range(kmax):
        x = lsq(A, b, GAMMA, Lm, d - g)
        q = Lm @ x
        d_new = shrink(q + g)
        g = g + q - d_new
        d = d_new
    return x, (d, g)


def vcycle_dense(b, A0, solver, wavelet, levels, transfer, kmax):
    As, bs, ms = [A0], [b], [int(round(math.sqrt(len(b))))]
    for _ in range(levels - 1):
        w = w1_dense(ms[-1], wavelet)
        W = np.kron(w, w)                       # vec(w X w^T) = (w kron w) vec(X)
        As.append(W.T @ As[-1] @ W)
        bs.append(W.T @ bs[-1])
        ms.append(ms[-1] // 2)
    init = ("I",)
    x = aux = None
    for i in range(levels - 1, -1, -1):
        if i < levels - 1:
            mf, mc = ms[i], ms[i + 1]
            w = w1_dense(mf, wavelet)
            if transfer == "X":
                init = ("X", np.kron(w, w) @ x)
            else:
                wt = w[: mf - 1, : mc - 1]
                P = np.zeros(((mf - 1) * mf * 2, (mc - 1) * mc * 2))
                kx = (mc - 1) * mc
                P[: (mf - 1) * mf, :kx] = np.kron(w, wt)      # Qx -> W~1 Qx W1^T
                P[(mf - 1) * mf:, kx:] = np.kron(wt, w)       # Qy -> W1 Qy W~1^T
                init = ("D", (P @ aux[0], P @ aux[1]) if solver == "sb" else P @ aux)
        x, aux = level_dense(solver, As[i], bs[i], ms[i], init, kmax)
    return x


def problem(m, wavelet, seed=3):
    x_true = I.phantom(m, 4, 2, seed)
    g = I.gaussian_factor(1.3, 5)
    A = O.KronOp.from_factors(m, g, g)
    b = I.add_noise(A.apply(x_true), I.noise_direction(m, seed + 11), 0.02)
    T = toeplitz_dense(m, g)
    return A, b, np.kron(T, T)


FIXED = S.opts_with(gamma_fixed=GAMMA, kmax=3, tol_fine=0.0, tol_coarse=0.0, lsqr_atol=1e-15,
                    lsqr_btol=1e-15, lsqr_conlim=1e20, lsqr_maxit=3000)
CASES = [(s, w, lv, t) for s in ("irls", "mm", "sb") for w in ("haar", "db4") for lv in (2, 3) for t in ("X", "D")]


@pytest.mark.parametrize("case", CASES, ids=["-".join(map(str, c)) for c in CASES])
def test_vcycle_matches_dense_composition(case):
    solver, wavelet, levels, transfer = case
    A, b, A0 = problem(16, wavelet)
    r = S.mgm(b, A, solver, wavelet, levels, transfer, FIXED)
    xd = vcycle_dense(O.vec(b), A0, solver, wavelet, levels, transfer, FIXED["kmax"])
    d = np.linalg.norm(O.vec(r["x"]) - xd) / np.linalg.norm(xd)
    assert d < 1e-10, d
    assert r["iters"] == [FIXED["kmax"]] * levels


def test_transfer_branches_are_distinguishable():
    """The pin above has teeth: the wrong initialisation on the fine level
    (Approach D started from W x_coarse instead of 0) moves the result by
    orders of magnitude more than its tolerance."""
    A, b, A0 = problem(16, "haar")
    xd_D = vcycle_dense(O.vec(b), A0, "sb", "haar", 2, "D", 3)
    xd_X = vcycle_dense(O.vec(b), A0, "sb", "haar", 2, "X", 3)
    assert np.linalg.norm(xd_D - xd_X) / np.linalg.norm(xd_D) > 1e-4


# ---- GCV schedule (Sec. 3) --------------------------------------------------

def spy_schedule(monkeypatch, solver, levels, kmax):
    """Runs a cycle with gamma fixed and records, per level, the outer
    iteration at which GCV was called and whether its pair was weighted,
    together with the weights that GCV and the following solve received."""
    events = []
    orig_gcv, orig_solve = S.Subproblem.gcv, S.Subproblem.solve

    def gcv(self, o):
        events.append(("gcv", self.m, None if self.wv is None else self.wv.copy()))
        return orig_gcv(self, o)

    def solve(self, gamma, x0, o):
        events.append(("solve", self.m, None if self.wv is None else self.wv.copy()))
        return orig_solve(self, gamma, x0, o)

    monkeypatch.setattr(S.Subproblem, "gcv", gcv)
    monkeypatch.setattr(S.Subproblem, "solve", solve)
    A, b, _ = problem(16, "haar")
    S.mgm(b, A, solver, "haar", levels, "X", dict(FIXED, kmax=kmax))
    per = {}
    for kind, m, w in events:
        lv = per.setdefault(m, {"k": 0, "gcv": []})
        if kind == "gcv":
            lv["gcv"].append((lv["k"], w))
        else:
            lv["k"] += 1
            if lv["gcv"] and lv["gcv"][-1][0] == lv["k"] - 1 and lv["gcv"][-1][1] is not None:
                # the pair GCV saw must be the pair this solve uses
                assert w is not None and np.array_equal(lv["gcv"][-1][1], w)
    return per


def test_irls_gcv_schedule_three_levels(monkeypatch):
    """IRLS, 3 levels: every coarse level estimates gamma at every outer
    iteration from the weighted pair; the fine level from the unweighted pair
    at k = 0 and the weighted pair at k = 3, and never again."""
    per = spy_schedule(monkeypatch, "irls", 3, 6)
    for m in (4, 8):
        assert [k for k, _ in per[m]["gcv"]] == list(range(6))
        assert all(w is not None for _, w in per[m]["gcv"])
    fine = per[16]["gcv"]
    assert [k for k, _ in fine] == [0, 3]
    assert fine[0][1] is None and fine[1][1] is not None


def test_irls_gcv_schedule_two_levels(monkeypatch):
    per = spy_schedule(monkeypatch, "irls", 2, 5)
    for m in (8, 16):
        assert [k for k, _ in per[m]["gcv"]] == list(range(5))


@pytest.mark.parametrize("solver", ["mm", "sb"])
def test_mm_sb_gcv_first_three_iterations(monkeypatch, solver):
    per = spy_schedule(monkeypatch, solver, 3, 6)
    for m in (4, 8, 16):
        assert [k for k, _ in per[m]["gcv"]] == [0, 1, 2]


# ---- GCV search edges (Sec. 3; the grid range is a reading) --------------------

def test_gcv_widening_below_the_grid():
    """A minimum below 1e-10 moves the lower end down by 4 decades (once)."""
    gamma, info = G.select_gamma(lambda g: (math.log10(g) + 12.3) ** 2 + 1.0)
    assert info["extended"] == 1 and abs(math.log10(gamma) + 12.3) < 1e-4


def test_gcv_widening_above_the_grid():
    gamma, info = G.select_gamma(lambda g: (math.log10(g) - 3.7) ** 2 + 1.0)
    assert info["extended"] == 1 and abs(math.log10(gamma) - 3.7) < 1e-4


def test_gcv_widening_stops_after_two_extensions():
    """A minimum beyond two extensions returns the end of the widened grid
    (t = -18), flagged by extended = 2."""
    gamma, info = G.select_gamma(lambda g: (math.log10(g) + 40.0) ** 2 + 1.0)
    assert info["extended"] == 2 and abs(math.log10(gamma) + 18.0) < 1e-4


def test_gcv_grid_tie_takes_smallest_gamma():
    """Equal grid minima: the bracket is around the smaller gamma."""
    t = np.linspace(-10.0, 2.0, 50)
    a, b = t[10], t[30]
    f = lambda g: min((math.log10(g) - a) ** 2, (math.log10(g) - b) ** 2) + 1.0
    gamma, info = G.select_gamma(f)
    assert info["j"] == 10 and abs(math.log10(gamma) - a) < 1e-4
