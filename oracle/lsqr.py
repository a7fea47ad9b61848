"""Oracle LSQR (Paige & Saunders 1982), the Krylov solver the paper applies to
the augmented problem, Eq. (augmented) in Sec. 3.

Test infrastructure only. Float64, no reorthogonalisation.

Warm start: the outer solvers pass the right-hand side r0 = b_hat - A_hat x0
and add the returned correction to x0 (a reading of a point the paper leaves
open).

Stopping rules (Paige & Saunders, rules S1-S3, with their usual estimates):
  ||r_k||        ~ phibar_{k+1}
  ||A^T r_k||    ~ phibar_{k+1} alpha_{k+1} |c_k|
  ||A_hat||      ~ ||B_k||_F = sqrt(sum alpha_j^2 + beta_{j+1}^2)
  cond(A_hat)    ~ ||B_k||_F * ||D_k||_F,  D_k columns w_j / rho_j
  ||delta_k||    computed exactly from the iterate
  S1: ||r_k|| <= btol ||r0|| + atol ||A_hat|| ||delta_k||
  S2: ||A^T r_k|| <= atol ||A_hat|| ||r_k||
  S3: cond(A_hat) >= conlim
and at most ``maxit`` iterations.
"""
from __future__ import annotations

import math

import numpy as np


def lsqr(matvec, rmatvec, r0, n, atol=1e-6, btol=1e-6, conlim=1e8, maxit=100):
    """Return (delta, iterations) approximately minimising ||A_hat delta - r0||.

    ``matvec(v)`` applies A_hat (image -> stacked data/penalty vector),
    ``rmatvec(u)`` applies A_hat^T, ``n`` is the image-vector length.
    Vectors are 1-D float64 arrays.
    """
    n_img = n
    beta = float(np.linalg.norm(r0))
    if beta == 0.0:
        return np.zeros(n_img), 0
    u = r0 / beta
    v = rmatvec(u)
    alpha = float(np.linalg.norm(v))
    if alpha == 0.0:
        return np.zeros(n_img), 0
    v = v / alpha
    w = v.copy()
    delta = np.zeros(n_img)
    phibar, rhobar = beta, alpha
    bnorm = beta
    anorm2 = 0.0
    dnorm2 = 0.0
    it = 0
    while it < maxit:
        it += 1
        # Golub-Kahan step: beta_{i+1} u_{i+1} = A v_i - alpha_i u_i
        u = matvec(v) - alpha * u
        beta_new = float(np.linalg.norm(u))
        if beta_new > 0.0:
            u = u / beta_new
        anorm2 += alpha * alpha + beta_new * beta_new
        # alpha_{i+1} v_{i+1} = A^T u_{i+1} - beta_{i+1} v_i
        v = rmatvec(u) - beta_new * v
        alpha_new = float(np.linalg.norm(v))
        if alpha_new > 0.0:
            v = v / alpha_new
        # plane rotation eliminating the subdiagonal of B_k
        rho = math.sqrt(rhobar * rhobar + beta_new * beta_new)
        c, s = rhobar / rho, beta_new / rho
        theta = s * alpha_new
        rhobar = -c * alpha_new
        phi = c * phibar
        phibar = s * phibar
        # iterate and search-direction update
        dnorm2 += float(np.dot(w, w)) / (rho * rho)
        delta = delta + (phi / rho) * w
        w = v - (theta / rho) * w
        alpha, beta = alpha_new, beta_new
        # stopping tests
        rnorm = phibar
        arnorm = phibar * alpha * abs(c)
        anorm = math.sqrt(anorm2)
        xnorm = float(np.linalg.norm(delta))
        acond = anorm * math.sqrt(dnorm2)
        if rnorm <= btol * bnorm + atol * anorm * xnorm:
            break
        if anorm > 0.0 and rnorm > 0.0 and arnorm <= atol * anorm * rnorm:
            break
        if acond >= conlim:
            break
    return delta, it
