"""Pins for the oracle's linear operators against definitions written out
independently (explicit loops, dense matrices, closed forms)."""
import math

import numpy as np
import pytest

from oracle import operators as O
from paper_2608_17123_b300 import inputs as I

RNG = np.random.default_rng(1234)


def dense_W1_from_display(m, h):
    """W1^T built row by row from the matrix display of Sec. 4."""
    Wt = np.zeros((m // 2, m))
    for r in range(m // 2):
        for k in range(len(h)):
            Wt[r, (2 * r + k) % m] += h[k]
    return Wt.T


def load_golden_filters():
    vals = {}
    with open("tests/golden/filters.txt") as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                name, *nums = line.split()
                vals[name] = np.array([float(x) for x in nums])
    return vals


@pytest.mark.parametrize("wavelet", ["haar", "db4"])
def test_filters_golden_and_identities(wavelet):
    h = O.lowpass(wavelet)
    gold = load_golden_filters()[wavelet]
    assert np.allclose(h, gold, rtol=0, atol=1e-15)
    assert abs(h.sum() - math.sqrt(2.0)) < 1e-15
    assert abs((h * h).sum() - 1.0) < 1e-15
    kappa = len(h)
    g = np.array([(-1) ** k * h[kappa - 1 - k] for k in range(kappa)])
    # high-pass vanishing moments: Haar 1, Db4 2 (reproduction of constants / lines)
    moments = 1 if wavelet == "haar" else 2
    for p in range(moments):
        assert abs(sum(g[k] * k ** p for k in range(kappa))) < 1e-14


@pytest.mark.parametrize("wavelet", ["haar", "db4"])
@pytest.mark.parametrize("m", [4, 8, 16])
def test_W1_orthonormal_and_perfect_reconstruction(wavelet, m):
    h = O.lowpass(wavelet)
    if m < len(h):
        return
    W = O.W1(m, wavelet).toarray()
    assert np.allclose(W, dense_W1_from_display(m, h), atol=0)
    assert np.allclose(W.T @ W, np.eye(m // 2), atol=1e-14)
    kappa = len(h)
    g = np.array([(-1) ** k * h[kappa - 1 - k] for k in range(kappa)])
    G1 = dense_W1_from_display(m, g)
    Q = np.hstack([W, G1])
    assert np.allclose(Q.T @ Q, np.eye(m), atol=1e-14)  # perfect reconstruction


def test_db4_reproduces_linear_away_from_wrap():
    m = 32
    W = O.W1(m, "db4").toarray()
    G1 = dense_W1_from_display(m, np.array([(-1) ** k * O.lowpass("db4")[3 - k] for k in range(4)]))
    lin = 0.3 + 0.7 * np.arange(m)
    detail = G1.T @ lin
    assert np.all(np.abs(detail[:-1]) < 1e-12)  # only the wrapped row sees the jump
    rec = W @ (W.T @ lin)
    assert np.allclose(rec[2:-2], lin[2:-2], atol=1e-12)


@pytest.mark.parametrize("m", [8, 13])
def test_blur_forms_equal_explicit_loop(m):
    X = RNG.standard_normal((m, m))
    P = RNG.standard_normal((5, 5))  # no symmetry
    assert np.allclose(O.KronOp.from_psf(m, P).apply(X), O.blur_direct(X, P), atol=1e-13)
    g = I.gaussian_factor(1.3, 5)
    Pg = np.outer(g, g)
    assert np.allclose(O.KronOp.from_factors(m, g, g).apply(X), O.blur_direct(X, Pg), atol=1e-14)
    # a rank-1 but non-symmetric PSF: rows factor vs column factor orientation
    gr, gc = RNG.random(5), RNG.random(3)
    gc = np.concatenate([[0.0], gc, [0.0]])
    assert np.allclose(O.KronOp.from_factors(m, gr, gc).apply(X), O.blur_direct(X, np.outer(gr, gc)), atol=1e-13)


def test_motion_psf_forms_agree():
    m = 24
    P = I.motion_psf(21.0, 30.0, 21)
    X = RNG.standard_normal((m, m))
    assert np.allclose(O.KronOp.from_psf(m, P).apply(X), O.blur_direct(X, P), atol=1e-13)


def _check_adjoint(f, ft, shape_in, shape_out, tol=1e-13):
    x = RNG.standard_normal(shape_in)
    y = RNG.standard_normal(shape_out)
    lhs = float(np.sum(f(x) * y))
    rhs = float(np.sum(x * ft(y)))
    assert abs(lhs - rhs) <= tol * max(1.0, abs(lhs))


@pytest.mark.parametrize("wavelet", ["haar", "db4"])
def test_adjoint_identities_all_levels(wavelet):
    m = 32
    P = I.motion_psf(9.0, 30.0, 9)
    g = I.gaussian_factor(2.0, 9)
    for A in (O.KronOp.from_psf(m, P), O.KronOp.from_factors(m, g, g)):
        for _ in range(3):
            mm = A.m
            _check_adjoint(A.apply, A.applyT, (mm, mm), (mm, mm))
            A = A.coarsen(wavelet)
    _check_adjoint(lambda X: O.lvec(*O.L_apply(X)), lambda q: O.Lt_apply(*O.unlvec(q, m)),
                   (m, m), (2 * m * (m - 1),))
    _check_adjoint(lambda X: O.restrict(X, wavelet), lambda Y: O.prolong(Y, wavelet),
                   (m, m), (m // 2, m // 2))


@pytest.mark.parametrize("wavelet", ["haar", "db4"])
def test_L_and_W_dense_forms(wavelet):
    m = 8
    X = RNG.standard_normal((m, m))
    # L: [I kron D; D kron I] on column-major vec (Sec. 4.2)
    assert np.allclose(O.L_dense(m) @ O.vec(X), O.lvec(*O.L_apply(X)), atol=1e-14)
    # explicit forward differences
    qx, qy = O.L_apply(X)
    assert np.allclose(qx, X[1:, :] - X[:-1, :])
    assert np.allclose(qy, X[:, 1:] - X[:, :-1])
    W = np.kron(dense_W1_from_display(m, O.lowpass(wavelet)), dense_W1_from_display(m, O.lowpass(wavelet)))
    Xc = RNG.standard_normal((m // 2, m // 2))
    assert np.allclose(W @ O.vec(Xc), O.vec(O.prolong(Xc, wavelet)), atol=1e-14)
    assert np.allclose(W.T @ O.vec(X), O.vec(O.restrict(X, wavelet)), atol=1e-14)


@pytest.mark.parametrize("wavelet", ["haar", "db4"])
def test_aux_prolong_dense(wavelet):
    mc, mf = 4, 8
    W1d = dense_W1_from_display(mf, O.lowpass(wavelet))  # mf x mc
    Wt = W1d[: mf - 1, : mc - 1]
    qx = RNG.standard_normal((mc - 1, mc))
    qy = RNG.standard_normal((mc, mc - 1))
    fx, fy = O.aux_prolong(qx, qy, wavelet)
    assert fx.shape == (mf - 1, mf) and fy.shape == (mf, mf - 1)
    assert np.allclose(fx, Wt @ qx @ W1d.T, atol=1e-14)
    assert np.allclose(fy, W1d @ qy @ Wt.T, atol=1e-14)


@pytest.mark.parametrize("wavelet", ["haar", "db4"])
def test_coarse_operator_equals_galerkin_dense(wavelet):
    m = 16
    g = I.gaussian_factor(1.5, 7)
    P = I.motion_psf(7.0, 30.0, 7)
    for A in (O.KronOp.from_factors(m, g, g), O.KronOp.from_psf(m, P)):
        Ad = A.dense()
        Wd = np.kron(dense_W1_from_display(m, O.lowpass(wavelet)), dense_W1_from_display(m, O.lowpass(wavelet)))
        Ac = A.coarsen(wavelet)
        assert np.allclose(Ac.dense(), Wd.T @ Ad @ Wd, atol=1e-14)
        Wd2 = np.kron(dense_W1_from_display(m // 2, O.lowpass(wavelet)),
                      dense_W1_from_display(m // 2, O.lowpass(wavelet)))
        assert np.allclose(Ac.coarsen(wavelet).dense(), Wd2.T @ Wd.T @ Ad @ Wd @ Wd2, atol=1e-14)


def test_haar_coarse_kernel_closed_form():
    """Haar keeps zero-BC Toeplitz structure (Sec. 4.2) with the 1-D kernel
    t'(d) = (t(2d-1) + 2 t(2d) + t(2d+1)) / 2 (derived by hand from the
    display: W1^T row r touches fine 2r and 2r+1 only, no wrap)."""
    m = 32
    g = I.gaussian_factor(2.5, 11)
    R = 5
    t = lambda d: g[d + R] if -R <= d <= R else 0.0
    Rc = (R + 1) // 2
    tc = np.array([(t(2 * d - 1) + 2 * t(2 * d) + t(2 * d + 1)) / 2.0 for d in range(-Rc, Rc + 1)])
    Ac = O.KronOp.from_factors(m, g, g).coarsen("haar")
    assert np.allclose(Ac.terms[0][0].toarray(), O.toeplitz_1d(m // 2, tc).toarray(), atol=1e-15)
    assert abs(tc.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("wavelet", ["haar", "db4"])
def test_coarse_rows_sum_to_one_in_interior(wavelet):
    m = 64
    g = I.gaussian_factor(2.0, 9)
    A = O.KronOp.from_factors(m, g, g)
    for _ in range(2):
        A = A.coarsen(wavelet)
        Y = A.apply(np.ones((A.m, A.m)))
        k = 8
        assert np.allclose(Y[k:-k, k:-k], 1.0, atol=1e-13)


def test_inputs_recipes():
    X = I.phantom(64, 12, 6, 0)
    assert X.min() >= 0 and X.max() <= 1 and len(np.unique(X)) <= 19
    assert np.array_equal(X, I.phantom(64, 12, 6, 0))
    P = I.gaussian_psf(2.0, 9)
    assert abs(P.sum() - 1) < 1e-14 and np.allclose(P, P.T) and np.allclose(P, P[::-1, ::-1])
    M = I.motion_psf(21.0, 30.0, 21)
    assert abs(M.sum() - 1) < 1e-14 and np.allclose(M, M[::-1, ::-1], atol=1e-16)
    b = np.ones((8, 8))
    xi = I.noise_direction(8, 3)
    e = I.add_noise(b, xi, 0.05) - b
    assert abs(np.linalg.norm(e) / np.linalg.norm(b) - 0.05) < 1e-14
    assert np.array_equal(I.from_colmajor(I.to_colmajor(X).ravel(), 64), X)
