"""Oracle GCV parameter selection (Sec. 3, Eq. (xgamma) and Eq. (GCV)).

Test infrastructure only. Float64.

For a subproblem min ||A x - b||^2 + gamma ||D x - c||^2 the trial solution is
x_gamma = (A^T A + gamma D^T D)^{-1} (A^T b + gamma D^T c) and

    GCV(gamma) = ||A x_gamma - b||^2 / (n - tr(A (A^T A + gamma D^T D)^{-1} A^T))^2

with n the number of pixels of the level. Both modes reduce the pair to the
same small form: a basis Y with Y^T G_A Y = diag(lam) and
Y^T (G_A + G_D) Y = I (a generalized symmetric eigen-decomposition, which
carries the same information as the GSVD of the pair the paper uses). The
numerator is then a sum of squares (see GcvFactors).

* exact mode (the paper's definition): G_A = A^T A, G_D = D^T D,
  g_A = A^T b, g_D = D^T c formed densely, exact trace
  sum_j lam_j / (lam_j + gamma (1 - lam_j)). Tiny images only.
* projected mode (an addition of this project; the paper's dense GSVD is
  infeasible beyond m ~ 64): the numerator restricted to
  span(V), V = orthonormal basis of K_k(A^T A, A^T b) (plus D^T c when
  c != 0), k = ``proj_dim`` doubled until gamma moves by less than 0.1 % or
  ``proj_dim_max`` is reached; the trace, which a k-dimensional subspace
  cannot represent (it is in the thousands for the m = 512 workloads), is
  taken for the same pair under periodic boundary conditions where it has a
  closed form (``symbol_trace``).

Selection (Sec. 3): 50 log-spaced grid points on [1e-10, 1e2] (range is a
reading; the side holding the grid minimum is extended by 4 decades, at most
twice), then Brent's minimiser on log10(gamma) between the grid neighbours of
the grid minimum. The paper refines with MATLAB's fminbnd, which is closed;
Brent's method (Brent 1973, golden section with parabolic steps) is used here.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


class GcvFactors:
    """The small diagonal form of the GCV functional.

    With a basis Y such that Y^T G_A Y = diag(lam), Y^T (G_A + G_D) Y = I,
    a = Y^T g_A and d = Y^T g_D, the trial solution in the eigenbasis is
    z_j = (a_j + gamma d_j) / (lam_j + gamma (1 - lam_j)), and the data residual
    splits into a gamma-dependent quadratic form and a constant without any
    cancellation between gamma-dependent terms:

      w0_j = a_j / (lam_j + eta),   f_j = a_j + d_j - w0_j,
      ||A x_gamma - b||^2 = gamma^2 sum_j lam_j (f_j / (lam_j + gamma (1 - lam_j)))^2 + r0^2,
      r0^2 = ||b||^2 - sum_j a_j w0_j   (b outside the resolved range of A V).

    With eta = 0 (the default, used everywhere) this is exact algebra (w0 is
    the gamma -> 0 solution); eta > 0 would count pencil directions with
    lam_j << eta as outside range(A). Note that forming A^T A squares the
    conditioning: on a level where A is numerically singular (pencil
    eigenvalues ~ 1e-16) the numerator of any Gram-matrix formulation carries
    errors of order 1e-2 against a QR-based least-squares residual.

    ``trace`` is a callable gamma -> tr(A A_gamma^# ); by default the exact
    sum_j lam_j / (lam_j + gamma (1 - lam_j)).
    """

    def __init__(self, lam, a, d, bnorm2, n, trace=None, eta=0.0):
        self.lam = np.asarray(lam, dtype=np.float64)
        self.a = np.asarray(a, dtype=np.float64)
        self.d = np.asarray(d, dtype=np.float64)
        self.n = n
        den = self.lam + eta
        self.w0 = np.where(den > 0.0, self.a / np.where(den > 0.0, den, 1.0), 0.0)
        self.f = self.a + self.d - self.w0
        self.r02 = max(float(bnorm2) - float(np.sum(self.a * self.w0)), 0.0)
        self._trace = trace

    def numerator(self, gamma: float) -> float:
        u = self.f / (self.lam + gamma * (1.0 - self.lam))
        return gamma * gamma * float(np.sum(self.lam * u * u)) + self.r02

    def trace(self, gamma: float) -> float:
        if self._trace is not None:
            return self._trace(gamma)
        return float(np.sum(self.lam / (self.lam + gamma * (1.0 - self.lam))))

    def __call__(self, gamma: float) -> float:
        return self.numerator(gamma) / (self.n - self.trace(gamma)) ** 2


EXACT_RANK_ETA = 0.0


def reduce_pair(GA, GD, gA, gD, bnorm2, n, trace=None, eta=0.0) -> GcvFactors:
    """Generalized symmetric eigenproblem GA y = lam (GA + GD) y."""
    lam, Y = sla.eigh(GA, GA + GD)
    return GcvFactors(lam, Y.T @ gA, Y.T @ gD, bnorm2, n, trace, eta)


def factors_exact(Ad, Dd, b, c, n) -> GcvFactors:
    """Exact mode (the paper's definition) from dense A (n x n), D (p x n)."""
    GA = Ad.T @ Ad
    GD = Dd.T @ Dd
    gD = Dd.T @ c if c is not None else np.zeros(Ad.shape[1])
    return reduce_pair(GA, GD, Ad.T @ b, gD, float(b @ b), n, eta=EXACT_RANK_ETA)


def _orth(x, basis):
    """Classical Gram-Schmidt against the orthonormal ``basis``, twice."""
    for _ in range(2):
        if basis:
            B = np.array(basis)
            x = x - B.T @ (B @ x)
    return x


def krylov_basis(A, At, b, k):
    """Orthonormal basis of K_k(A^T A, A^T b): Golub-Kahan / Lanczos on A^T A
    with full reorthogonalisation of V (each new direction A^T A v_j is
    orthogonalised against all previous ones, twice). Stops early on a
    breakdown (invariant subspace)."""
    v = At(b)
    nv = np.linalg.norm(v)
    V = [v / nv]
    while len(V) < k:
        t = _orth(At(A(V[-1])), V)
        nt = np.linalg.norm(t)
        if nt <= 1e-12 * nv:
            break
        V.append(t / nt)
    return V


def symbol_trace(rows_r, rows_c, m, weight_scale=1.0):
    """Trace of the influence matrix for the same pair under periodic boundary
    conditions, where the blur and L^T L are both diagonalised by the 2-D DFT:

        T(gamma) = sum_w |K(w)|^2 / (|K(w)|^2 + gamma s l(w)),

    K(j1, j2) = sum_t Kr_t(j1) Kc_t(j2) with Kr_t, Kc_t the DFTs of the middle
    rows (row m/2) of the level's 1-D Kronecker factors, i.e. of its interior
    stencil; l = 4 sin^2(pi j1/m) + 4 sin^2(pi j2/m) is the symbol of L^T L;
    s is the mean squared IRLS weight (1 for an unweighted pair)."""
    j = np.arange(m)
    K = np.zeros((m, m), dtype=np.complex128)
    for rr, rc in zip(rows_r, rows_c):
        K += np.outer(_dft_row(rr, m), _dft_row(rc, m))
    K2 = (np.abs(K) ** 2).ravel()
    l1 = 4.0 * np.sin(np.pi * j / m) ** 2
    ell = (l1[:, None] + l1[None, :]).ravel()

    def T(gamma):
        den = K2 + gamma * weight_scale * ell
        return float(np.sum(np.where(den > 0.0, K2 / np.where(den > 0.0, den, 1.0), 1.0)))
    return T


def _dft_row(row, m):
    """K(j) = sum_s row[s] exp(-2 pi i j (m/2 - s) / m): the DFT of the
    stencil t(d) = row[m/2 - d] that the middle row of a 1-D operator holds."""
    s = np.arange(m)
    j = np.arange(m)
    return np.exp(-2j * np.pi * np.outer(j, (m // 2) - s) / m) @ row


def factors_projected(A, At, Dop, Dt, b, c, k, n, trace) -> GcvFactors:
    """Projected mode (project addition): G_A = (AV)^T (AV), G_D = (DV)^T (DV),
    g_A = (AV)^T b, g_D = (DV)^T c on V = [K_k(A^T A, A^T b), orth(D^T c)],
    formed explicitly; ``trace`` supplies the denominator's trace."""
    V = krylov_basis(A, At, b, k)
    if c is not None and np.any(c):
        dtc = Dt(c)
        vc = _orth(dtc, V)
        nc = np.linalg.norm(vc)
        if nc > 1e-12 * np.linalg.norm(dtc):
            V.append(vc / nc)
    V = np.array(V).T  # n x k
    AV = np.column_stack([A(V[:, j]) for j in range(V.shape[1])])
    DV = np.column_stack([Dop(V[:, j]) for j in range(V.shape[1])])
    gD = DV.T @ c if c is not None else np.zeros(V.shape[1])
    return reduce_pair(AV.T @ AV, DV.T @ DV, AV.T @ b, gD, float(b @ b), n, trace)


def brent_min(f, a, b, tolx=1e-5, maxfev=500):
    """Brent's minimiser of f on [a, b] (golden-section search with
    successive parabolic interpolation, Brent 1973). Tolerance
    sqrt(eps)|x| + tolx/3. Returns (x, f(x))."""
    cgold = 0.5 * (3.0 - math.sqrt(5.0))
    sqeps = math.sqrt(2.220446049250313e-16)
    x = w = v = a + cgold * (b - a)
    fx = fw = fv = f(x)
    d = e = 0.0
    nfev = 1
    while nfev < maxfev:
        xm = 0.5 * (a + b)
        tol1 = sqeps * abs(x) + tolx / 3.0
        tol2 = 2.0 * tol1
        if abs(x - xm) <= tol2 - 0.5 * (b - a):
            break
        golden = True
        if abs(e) > tol1:
            r = (x - w) * (fx - fv)
            q = (x - v) * (fx - fw)
            p = (x - v) * q - (x - w) * r
            q = 2.0 * (q - r)
            if q > 0.0:
                p = -p
            q = abs(q)
            etemp = e
            e = d
            if abs(p) < abs(0.5 * q * etemp) and p > q * (a - x) and p < q * (b - x):
                d = p / q
                u = x + d
                if (u - a) < tol2 or (b - u) < tol2:
                    d = tol1 if xm >= x else -tol1
                golden = False
        if golden:
            e = (b - x) if x < xm else (a - x)
            d = cgold * e
        u = x + d if abs(d) >= tol1 else x + (tol1 if d > 0 else -tol1)
        fu = f(u)
        nfev += 1
        if fu <= fx:
            if u < x:
                b = x
            else:
                a = x
            v, fv = w, fw
            w, fw = x, fx
            x, fx = u, fu
        else:
            if u < x:
                a = u
            else:
                b = u
            if fu <= fw or w == x:
                v, fv = w, fw
                w, fw = u, fu
            elif fu <= fv or v == x or v == w:
                v, fv = u, fu
    return x, fx


def select_gamma(F, lo=-10.0, hi=2.0, npts=50, tolx=1e-5, max_ext=2):
    """Grid search + Brent refinement on t = log10(gamma) (Sec. 3).
    Returns (gamma, info) with info['extended'] the number of endpoint
    extensions."""
    f = lambda t: F(10.0 ** t)
    ext = 0
    while True:
        t = np.linspace(lo, hi, npts)
        vals = np.array([f(tj) for tj in t])
        j = int(np.argmin(vals))  # first (smallest gamma) among equal minima
        if j == 0 and ext < max_ext:
            lo -= 4.0
            ext += 1
            continue
        if j == npts - 1 and ext < max_ext:
            hi += 4.0
            ext += 1
            continue
        break
    a = t[max(j - 1, 0)]
    b = t[min(j + 1, npts - 1)]
    tb, fb = brent_min(f, a, b, tolx)
    tbest = tb if fb <= vals[j] else t[j]
    return 10.0 ** tbest, {"extended": ext, "grid_t": t, "grid_f": vals, "j": j}
