"""Oracle linear operators: blur A and its Galerkin coarsenings, gradient L,
low-pass wavelet transfers W and the blockwise auxiliary transfer.

Test infrastructure only (see the package docstring). Float64 throughout.

Images are 2-D arrays X[r, c]; vec(X) is column-major (Sec. 5), so a
Kronecker operator (Cc kron Cr) acts as X -> Cr X Cc^T and W = W1 kron W1
acts as Xc -> W1 Xc W1^T (Sec. 4, Approach X formula).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

# --------------------------------------------------------------------------
# Filters (Sec. 4, the two filter definitions after the W1^T display)
# --------------------------------------------------------------------------

def lowpass(wavelet: str) -> np.ndarray:
    """Low-pass analysis taps h_0..h_{kappa-1}: Haar (sqrt2/2, sqrt2/2) and the
    4-tap Daubechies filter (1+sqrt3, 3+sqrt3, 3-sqrt3, 1-sqrt3)/(4 sqrt2)."""
    if wavelet == "haar":
        return np.array([math.sqrt(2.0) / 2.0, math.sqrt(2.0) / 2.0])
    if wavelet == "db4":
        s3 = math.sqrt(3.0)
        return np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4.0 * math.sqrt(2.0))
    raise ValueError(wavelet)


def W1(m: int, wavelet: str) -> sp.csr_matrix:
    """1-D low-pass synthesis matrix W1 (m x m/2), the transpose of the
    analysis matrix displayed in Sec. 4: row r of W1^T holds h_k at column
    (2r + k) mod m (stride two, periodic wrap)."""
    h = lowpass(wavelet)
    if m % 2 or m < len(h):
        raise ValueError("W1 needs an even m >= filter length")
    rows, cols, vals = [], [], []
    for r in range(m // 2):
        for k, hk in enumerate(h):
            rows.append(r)
            cols.append((2 * r + k) % m)
            vals.append(hk)
    W1t = sp.coo_matrix((vals, (rows, cols)), shape=(m // 2, m)).tocsr()
    return W1t.T.tocsr()


# --------------------------------------------------------------------------
# Blur operator (Sec. 5 definition of A; coarse A^(i) per Sec. 4)
# --------------------------------------------------------------------------

def toeplitz_1d(m: int, t: np.ndarray) -> sp.csr_matrix:
    """Zero-boundary banded Toeplitz T (m x m) with centred kernel t of odd
    length: (T y)[i] = sum_d t[d + R] y[i - d], y = 0 outside [0, m)."""
    R = len(t) // 2
    rows, cols, vals = [], [], []
    for i in range(m):
        for d in range(-R, R + 1):
            j = i - d
            if 0 <= j < m and t[d + R] != 0.0:
                rows.append(i)
                cols.append(j)
                vals.append(t[d + R])
    return sp.coo_matrix((vals, (rows, cols)), shape=(m, m)).tocsr()


class KronOp:
    """A = sum_t (Cc_t kron Cr_t): acts on an image X as sum_t Cr_t X Cc_t^T.

    The fine-level blur of Sec. 5 is one such term (a Kronecker product of two
    banded Toeplitz matrices); a general PSF is the sum of one term per PSF
    column. The coarse operator A^(i+1) = W^T A^(i) W (Sec. 4, Alg. 4) of a
    Kronecker sum is again one, term by term (mixed-product property).
    """

    def __init__(self, terms):
        self.terms = [(sp.csr_matrix(cr), sp.csr_matrix(cc)) for cr, cc in terms]
        self.m = self.terms[0][0].shape[0]

    @staticmethod
    def from_factors(m: int, g_row: np.ndarray, g_col: np.ndarray) -> "KronOp":
        """PSF k = g_row g_col^T: A = T(g_col) kron T(g_row) (Sec. 5)."""
        return KronOp([(toeplitz_1d(m, g_row), toeplitz_1d(m, g_col))])

    @staticmethod
    def from_psf(m: int, P: np.ndarray) -> "KronOp":
        """General odd S x S PSF: (A X)(r,c) = sum_{p,q} P[p,q] X(r-p, c-q),
        zero outside; written as sum over columns q of T(P[:, q]) along rows
        and a shift by q along columns."""
        S = P.shape[0]
        R = S // 2
        terms = []
        for q in range(-R, R + 1):
            col = P[:, q + R]
            if not np.any(col):
                continue
            shift = np.zeros(S)
            shift[q + R] = 1.0
            terms.append((toeplitz_1d(m, col), toeplitz_1d(m, shift)))
        return KronOp(terms)

    def apply(self, X: np.ndarray) -> np.ndarray:
        Y = np.zeros_like(X)
        for cr, cc in self.terms:
            Y += cr @ (cc @ X.T).T
        return Y

    def applyT(self, Y: np.ndarray) -> np.ndarray:
        X = np.zeros_like(Y)
        for cr, cc in self.terms:
            X += cr.T @ (cc.T @ Y.T).T
        return X

    def coarsen(self, wavelet: str) -> "KronOp":
        """A^(i+1) = W^T A^(i) W with W = W1 kron W1 (Sec. 4, Alg. 4)."""
        w = W1(self.m, wavelet)
        return KronOp([(w.T @ cr @ w, w.T @ cc @ w) for cr, cc in self.terms])

    def middle_rows(self):
        """Row m/2 of each 1-D factor (the level's interior stencil), as two
        lists of dense length-m arrays (rows factors, column factors)."""
        r = self.m // 2
        return ([cr.getrow(r).toarray().ravel() for cr, _ in self.terms],
                [cc.getrow(r).toarray().ravel() for _, cc in self.terms])

    def dense(self) -> np.ndarray:
        """The n x n matrix acting on column-major vec(X) (tiny m only)."""
        return sum(sp.kron(cc, cr).toarray() for cr, cc in self.terms)


def blur_direct(X: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Explicit-loop zero-boundary convolution, the definition the other
    forms are checked against: Y(r,c) = sum_{p,q} P[p,q] X(r-p, c-q)."""
    m = X.shape[0]
    R = P.shape[0] // 2
    Y = np.zeros_like(X)
    for r in range(m):
        for c in range(m):
            s = 0.0
            for p in range(-R, R + 1):
                for q in range(-R, R + 1):
                    rr, cc = r - p, c - q
                    if 0 <= rr < m and 0 <= cc < m:
                        s += P[p + R, q + R] * X[rr, cc]
            Y[r, c] = s
    return Y


# --------------------------------------------------------------------------
# Gradient L = [I kron D; D kron I] (Sec. 4.2, computational implementation)
# --------------------------------------------------------------------------

def Dmat(m: int) -> sp.csr_matrix:
    """1-D forward difference D ((m-1) x m): D[j,j] = -1, D[j,j+1] = +1."""
    return sp.diags([-np.ones(m - 1), np.ones(m - 1)], [0, 1], shape=(m - 1, m)).tocsr()


def L_apply(X: np.ndarray):
    """L vec(X) = [vec(D X); vec(X D^T)]: returns (qx, qy), shapes
    (m-1) x m and m x (m-1)."""
    D = Dmat(X.shape[0])
    return D @ X, (D @ X.T).T


def Lt_apply(qx: np.ndarray, qy: np.ndarray) -> np.ndarray:
    """L^T [vec(qx); vec(qy)] = D^T qx + qy D."""
    D = Dmat(qx.shape[1])
    return D.T @ qx + (D.T @ qy.T).T


def L_dense(m: int) -> np.ndarray:
    D = Dmat(m).toarray()
    I = np.eye(m)
    return np.vstack([np.kron(I, D), np.kron(D, I)])


# --------------------------------------------------------------------------
# Level transfers (Sec. 4: restriction W^T, prolongation W; Sec. 4.2 blockwise)
# --------------------------------------------------------------------------

def restrict(X: np.ndarray, wavelet: str) -> np.ndarray:
    """W^T vec(X) = vec(W1^T X W1): b^(i+1) = W^T b^(i) (Alg. 4)."""
    w = W1(X.shape[0], wavelet)
    return (w.T @ (w.T @ X).T).T


def prolong(Xc: np.ndarray, wavelet: str) -> np.ndarray:
    """W vec(Xc) = vec(W1 Xc W1^T): Approach X interpolation (Sec. 4.1)."""
    w = W1(2 * Xc.shape[0], wavelet)
    return (w @ (w @ Xc).T).T


def aux_prolong(qx: np.ndarray, qy: np.ndarray, wavelet: str):
    """Approach D blockwise transfer (Sec. 4.2):
    Qx_f = W~1 Qx_c W1^T, Qy_f = W1 Qy_c W~1^T, with W~1 the first m_f - 1
    rows and m_c - 1 columns of W1 (m_f x m_c)."""
    mc = qy.shape[0]
    mf = 2 * mc
    w = W1(mf, wavelet)
    wt = w[: mf - 1, : mc - 1]
    return wt @ (w @ qx.T).T, w @ (wt @ qy.T).T


# --------------------------------------------------------------------------
# Vectorisation helpers (column-major, Sec. 5)
# --------------------------------------------------------------------------

def vec(X: np.ndarray) -> np.ndarray:
    return np.asarray(X).reshape(-1, order="F")


def unvec(x: np.ndarray, rows: int, cols: int) -> np.ndarray:
    return np.asarray(x).reshape(rows, cols, order="F")


def lvec(qx: np.ndarray, qy: np.ndarray) -> np.ndarray:
    return np.concatenate([vec(qx), vec(qy)])


def unlvec(q: np.ndarray, m: int):
    k = (m - 1) * m
    return unvec(q[:k], m - 1, m), unvec(q[k:], m, m - 1)
