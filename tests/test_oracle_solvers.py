"""Pins for the oracle's LSQR, GCV and outer solvers: dense least-squares
solves, brute-force GCV, majorisation invariants, l1 KKT conditions and
Tikhonov special cases."""
import math

import numpy as np
import pytest

from oracle import gcv as G
from oracle import operators as O
from oracle import solvers as S
from paper_2608_17123_b300 import inputs as I

RNG = np.random.default_rng(99)


def small_problem(m=8, sigma=1.2, S_=5, noise=0.01, seed=0):
    x_true = I.phantom(m, 3, 2, seed)
    g = I.gaussian_factor(sigma, S_)
    A = O.KronOp.from_factors(m, g, g)
    b = I.add_noise(A.apply(x_true), I.noise_direction(m, seed + 7), noise)
    return A, b, x_true


def dense_subproblem(A, b, gamma, w=None, c=None):
    Ad = A.dense()
    Ld = O.L_dense(A.m)
    Dd = Ld if w is None else O.lvec(*w)[:, None] * Ld
    cv = np.zeros(Dd.shape[0]) if c is None else O.lvec(*c)
    Ah = np.vstack([Ad, math.sqrt(gamma) * Dd])
    bh = np.concatenate([O.vec(b), math.sqrt(gamma) * cv])
    return Ah, bh, Ad, Dd, cv


TIGHT = S.opts_with(lsqr_atol=1e-15, lsqr_btol=1e-15, lsqr_conlim=1e20, lsqr_maxit=2000)


@pytest.mark.parametrize("kind", ["plain", "weighted", "shifted"])
@pytest.mark.parametrize("warm", [True, False])
def test_lsqr_matches_dense_lstsq(kind, warm):
    A, b, _ = small_problem()
    m = A.m
    w = c = None
    if kind == "weighted":
        w = S.irls_weights(*O.L_apply(RNG.random((m, m))), 0.03)
    if kind == "shifted":
        c = (RNG.standard_normal((m - 1, m)) * 0.1, RNG.standard_normal((m, m - 1)) * 0.1)
    gamma = 3e-3
    Ah, bh, *_ = dense_subproblem(A, b, gamma, w, c)
    xd = np.linalg.lstsq(Ah, bh, rcond=None)[0]
    x0 = RNG.random((m, m))
    x, its = S.Subproblem(A, b, weights=w, c=c).solve(gamma, x0, dict(TIGHT, lsqr_warm_start=warm))
    assert np.allclose(O.vec(x), xd, rtol=0, atol=1e-9 * np.abs(xd).max())
    assert its > 1


def test_lsqr_maxit_and_zero_rhs():
    A, b, _ = small_problem()
    x, its = S.Subproblem(A, b).solve(1e-3, np.zeros((8, 8)), S.opts_with(lsqr_maxit=3))
    assert its == 3
    x, its = S.Subproblem(A, np.zeros((8, 8))).solve(1e-3, np.zeros((8, 8)), S.opts_with())
    assert its == 0 and not np.any(x)


def brute_gcv(Ad, Dd, b, c, gamma):
    n = Ad.shape[1]
    Ag = Ad.T @ Ad + gamma * Dd.T @ Dd
    xg = np.linalg.solve(Ag, Ad.T @ b + gamma * Dd.T @ c)
    num = float(np.sum((Ad @ xg - b) ** 2))
    tr = float(np.trace(Ad @ np.linalg.solve(Ag, Ad.T)))
    return num / (n - tr) ** 2


@pytest.mark.parametrize("kind", ["plain", "weighted", "shifted"])
def test_gcv_exact_factors_equal_brute_force(kind):
    A, b, _ = small_problem(m=8)
    m = A.m
    w = S.irls_weights(*O.L_apply(RNG.random((m, m))), 0.03) if kind == "weighted" else None
    c = (RNG.standard_normal((m - 1, m)) * 0.05, RNG.standard_normal((m, m - 1)) * 0.05) if kind == "shifted" else None
    _, _, Ad, Dd, cv = dense_subproblem(A, b, 1.0, w, c)
    F = G.factors_exact(Ad, Dd, O.vec(b), cv if c is not None else None, m * m)
    for gamma in [1e-8, 1e-5, 1e-3, 0.1, 10.0]:
        ref = brute_gcv(Ad, Dd, O.vec(b), cv, gamma)
        assert abs(F(gamma) - ref) <= 1e-7 * ref


@pytest.mark.parametrize("kind", ["weighted", "shifted"])
def test_gcv_exact_factors_equal_brute_force_m32(kind):
    """The same pin on a 32 x 32 level (n = 1024), the largest level the
    exact rule is run on: the factored GCV function against the plain
    definition n ||A x_gamma - b||^2 / (n - tr(influence))^2 from dense solves."""
    A, b, _ = small_problem(m=32, sigma=1.5, S_=7)
    m = A.m
    rng = np.random.default_rng(32)
    w = S.irls_weights(*O.L_apply(rng.random((m, m))), 0.03) if kind == "weighted" else None
    c = (rng.standard_normal((m - 1, m)) * 0.05, rng.standard_normal((m, m - 1)) * 0.05) if kind == "shifted" else None
    _, _, Ad, Dd, cv = dense_subproblem(A, b, 1.0, w, c)
    F = G.factors_exact(Ad, Dd, O.vec(b), cv if c is not None else None, m * m)
    for gamma in [1e-5, 1e-3, 0.1]:
        ref = brute_gcv(Ad, Dd, O.vec(b), cv, gamma)
        assert abs(F(gamma) - ref) <= 1e-7 * ref


def test_gcv_selection_matches_brute_grid():
    A, b, _ = small_problem(m=8, noise=0.05)
    _, _, Ad, Dd, cv = dense_subproblem(A, b, 1.0)
    F = G.factors_exact(Ad, Dd, O.vec(b), None, 64)
    gamma, info = G.select_gamma(F)
    t = np.linspace(-10, 2, 2001)
    vals = np.array([brute_gcv(Ad, Dd, O.vec(b), cv, 10 ** tt) for tt in t])
    tb = t[np.argmin(vals)]
    assert abs(math.log10(gamma) - tb) <= 12 / 2000 + 1e-9
    assert F(gamma) <= vals.min() * (1 + 1e-9)


@pytest.mark.parametrize("shifted", [False, True])
def test_projected_equals_exact_at_full_dimension(shifted):
    A, b, _ = small_problem(m=6)
    m = A.m
    c = (RNG.standard_normal((m - 1, m)) * 0.05, RNG.standard_normal((m, m - 1)) * 0.05) if shifted else None
    sub = S.Subproblem(A, b, c=c)
    _, _, Ad, Dd, cv = dense_subproblem(A, b, 1.0, None, c)
    Fe = G.factors_exact(Ad, Dd, O.vec(b), cv if shifted else None, m * m)
    Fp = G.factors_projected(sub.Av, sub.Atv, sub.D, sub.Dt, O.vec(b), sub.cv, m * m, m * m, None)
    for gamma in [1e-6, 1e-3, 1e-1]:
        assert abs(Fp(gamma) - Fe(gamma)) <= 1e-8 * Fe(gamma)


def test_symbol_trace_equals_dense_periodic_problem():
    """Under periodic boundary conditions the symbol trace is exact: build the
    circulant blur and the periodic gradient densely and compare."""
    m = 8
    g = I.gaussian_factor(1.1, 5)
    R = 2
    C = np.zeros((m, m))
    for i in range(m):
        for d in range(-R, R + 1):
            C[i, (i - d) % m] += g[d + R]
    Ap = np.kron(C, C)
    Dp = np.zeros((m, m))
    for j in range(m):
        Dp[j, j], Dp[j, (j + 1) % m] = -1.0, 1.0
    Lp = np.vstack([np.kron(np.eye(m), Dp), np.kron(Dp, np.eye(m))])
    row = C[m // 2]
    T = G.symbol_trace([row], [row], m, 2.5)
    for gamma in [1e-4, 1e-2, 1.0]:
        Ag = Ap.T @ Ap + gamma * 2.5 * Lp.T @ Lp
        assert abs(T(gamma) - np.trace(Ap @ np.linalg.solve(Ag, Ap.T))) < 1e-9


def test_brent_minimiser():
    x, fx = G.brent_min(lambda t: (t - 0.3) ** 2 + 1.0, -1.0, 2.0, 1e-5)
    assert abs(x - 0.3) < 1e-5 and abs(fx - 1.0) < 1e-9
    x, _ = G.brent_min(lambda t: abs(t - 0.71), 0.0, 1.0, 1e-5)
    assert abs(x - 0.71) < 2e-5
    x, _ = G.brent_min(lambda t: math.cos(t), 2.0, 4.5, 1e-6)
    assert abs(x - math.pi) < 1e-6


def test_elementwise_closed_forms():
    u = np.array([-1.0, -0.02, 0.0, 0.03, 0.5])
    assert np.allclose(S.shrink(u, 0.005), [-0.995, -0.015, 0.0, 0.025, 0.495])
    wx, _ = S.irls_weights(u[None, :], u[None, :], 0.03)
    assert np.allclose(wx[0], [1.0, 0.03 ** -0.5, 0.03 ** -0.5, 0.03 ** -0.5, 0.5 ** -0.5])
    cx, _ = S.mm_surrogate(np.array([0.03]), np.array([0.0]), 0.03)
    assert abs(cx[0] - 0.03 * (1 - 1 / math.sqrt(2))) < 1e-16


def J_mm(A, b, x, mu, eps):
    qx, qy = O.L_apply(x)
    u = np.concatenate([qx.ravel(), qy.ravel()])
    return float(np.sum((A.apply(x) - b) ** 2) + 2 * eps * mu * np.sum(np.sqrt(u * u + eps * eps)))


def J_irls(A, b, x, mu, eps):
    qx, qy = O.L_apply(x)
    u = np.abs(np.concatenate([qx.ravel(), qy.ravel()]))
    H = np.where(u <= eps, u * u / (2 * eps), u - eps / 2)
    return float(np.sum((A.apply(x) - b) ** 2) + 2 * mu * np.sum(H))


def test_mm_monotone_with_fixed_mu():
    A, b, _ = small_problem(m=10, noise=0.02)
    mu = 2e-3
    o = dict(TIGHT, gamma_fixed=mu, kmax=1)
    x = np.zeros((10, 10))
    J = [J_mm(A, b, x, mu, 0.03)]
    for _ in range(8):
        x, *_ = S.mm(A, b, x, None, o, tol=0.0)
        J.append(J_mm(A, b, x, mu, 0.03))
    assert all(J[i + 1] <= J[i] * (1 + 1e-12) for i in range(len(J) - 1)), J


def test_irls_monotone_with_fixed_mu():
    A, b, _ = small_problem(m=10, noise=0.02)
    mu = 2e-3
    o = dict(TIGHT, gamma_fixed=mu, kmax=1)
    x = RNG.random((10, 10)) * 0.1
    J = [J_irls(A, b, x, mu, 0.03)]
    for _ in range(8):
        x, *_ = S.irls(A, b, x, None, o, tol=0.0)
        J.append(J_irls(A, b, x, mu, 0.03))
    assert all(J[i + 1] <= J[i] * (1 + 1e-12) for i in range(len(J) - 1)), J


def test_sb_kkt_at_convergence():
    A, b, _ = small_problem(m=8, noise=0.02)
    lam, tau = 5e-3, 0.005
    o = dict(TIGHT, gamma_fixed=lam, kmax=3000, tau_sb=tau)
    z = (np.zeros((7, 8)), np.zeros((8, 7)))
    x, _, k, _, (d, g) = S.sb(A, b, np.zeros((8, 8)), z, z, o, tol=1e-14)
    qx, qy = O.L_apply(x)
    Lx = np.concatenate([qx.ravel(), qy.ravel()])
    dv = np.concatenate([d[0].ravel(), d[1].ravel()])
    gv = np.concatenate([g[0].ravel(), g[1].ravel()])
    assert np.max(np.abs(Lx - dv)) < 1e-7
    assert np.max(np.abs(gv)) <= tau * (1 + 1e-6)
    nz = np.abs(dv) > 1e-9
    assert np.allclose(gv[nz], tau * np.sign(dv[nz]), atol=1e-7)
    grad = A.applyT(A.apply(x) - b) + lam * O.Lt_apply(*g)
    assert np.max(np.abs(grad)) < 1e-7  # same level as ||Lx - d|| at this stop


def test_first_iterates_are_tikhonov():
    A, b, _ = small_problem(m=8)
    gamma = 1e-3
    Ah, bh, *_ = dense_subproblem(A, b, gamma)
    xt = np.linalg.lstsq(Ah, bh, rcond=None)[0]
    o = dict(TIGHT, gamma_fixed=gamma, kmax=1)
    z8 = np.zeros((8, 8))
    ones = (np.ones((7, 8)), np.ones((8, 7)))
    zl = (np.zeros((7, 8)), np.zeros((8, 7)))
    for x in (S.irls(A, b, z8, ones, o, 0.0)[0], S.mm(A, b, z8, None, o, 0.0)[0],
              S.sb(A, b, z8, zl, zl, o, 0.0)[0]):
        assert np.allclose(O.vec(x), xt, atol=1e-10)


@pytest.mark.parametrize("solver", ["irls", "mm", "sb"])
def test_single_level_cycle_is_approach_I(solver):
    A, b, _ = small_problem(m=8)
    o = S.opts_with(gamma_fixed=1e-3, kmax=4)
    r = S.mgm(b, A, solver, "haar", 1, "X", o)
    x2, mu, k, inner, _ = S.level_solve(solver, A, b, ("I",), o, o["tol_fine"], "every")
    assert np.array_equal(r["x"], x2) and r["iters"] == [k]
