"""Seeded synthetic inputs for the deblurring workloads.

This module is shared by the tests, the benchmark and the CPU oracle. It holds
none of the method's arithmetic: it draws phantoms, samples point-spread
functions and draws the raw noise direction. Forming b = A x_true + e needs the
blur operator, so each side does that with its own operator.

Image convention: a 2-D numpy array ``X`` of shape (m, m) indexed ``X[r, c]``
(r = row, c = column). The C-ABI stores ``vec(X)`` column-major, element
(r, c) at ``r + c*m`` (Sec. 5 vectorises images column-wise); in numpy that is
the C-contiguous buffer of ``X.T``.

PSF convention: an (S, S) array ``P`` with odd S, centred, indexed
``P[p + R, q + R]`` for row offset p and column offset q (R = (S-1)/2), acting
as ``(A X)(r, c) = sum_{p,q} P[p+R, q+R] * X[r-p, c-q]`` with X = 0 outside
the image (zero boundary, Sec. 5).
"""
from __future__ import annotations

import math

import numpy as np


def phantom(m: int, n_rect: int, n_disk: int, seed: int) -> np.ndarray:
    """Piecewise-constant test image standing in for the paper's Voronoi and QR
    images (Sec. 5), which are not available here.

    Starts from zeros, paints ``n_rect`` axis-aligned rectangles (centre
    U[0,m)^2, sides U[m/32, m/4] with at least 2 px, clipped, intensity U[0,1])
    and then ``n_disk`` disks (centre U[0,m)^2, radius U[m/64, m/8] with at
    least 1 px, pixel-centre test, intensity U[0,1]), in that order.
    Generator: numpy PCG64 seeded with ``seed``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.zeros((m, m), dtype=np.float64)
    for _ in range(n_rect):
        cr, cc = rng.uniform(0.0, m, size=2)
        hr, hc = rng.uniform(m / 32.0, m / 4.0, size=2)
        hr, hc = max(hr, 2.0), max(hc, 2.0)
        val = rng.uniform(0.0, 1.0)
        r0, r1 = int(max(0, math.floor(cr - hr / 2))), int(min(m, math.ceil(cr + hr / 2)))
        c0, c1 = int(max(0, math.floor(cc - hc / 2))), int(min(m, math.ceil(cc + hc / 2)))
        X[r0:r1, c0:c1] = val
    rr, cc_ = np.meshgrid(np.arange(m) + 0.5, np.arange(m) + 0.5, indexing="ij")
    for _ in range(n_disk):
        cr, cc = rng.uniform(0.0, m, size=2)
        rad = max(rng.uniform(m / 64.0, m / 8.0), 1.0)
        val = rng.uniform(0.0, 1.0)
        X[(rr - cr) ** 2 + (cc_ - cc) ** 2 <= rad * rad] = val
    return X


def gaussian_factor(sigma: float, S: int) -> np.ndarray:
    """1-D Gaussian samples g(d) = exp(-d^2 / (2 sigma^2)), |d| <= (S-1)/2,
    scaled to sum 1. This is the first row of the banded Toeplitz factor in
    Sec. 5 (band = (S+1)/2), reflected to a centred kernel."""
    if S % 2 != 1 or S < 1:
        raise ValueError("PSF support must be odd")
    R = S // 2
    d = np.arange(-R, R + 1, dtype=np.float64)
    g = np.exp(-(d * d) / (2.0 * sigma * sigma))
    return g / g.sum()


def gaussian_psf(sigma: float, S: int) -> np.ndarray:
    """S x S Gaussian PSF k = g g^T (Kronecker structure of Sec. 5), sum 1."""
    g = gaussian_factor(sigma, S)
    return np.outer(g, g)


def motion_psf(length: float, angle_deg: float, S: int, samples: int = 2001) -> np.ndarray:
    """Linear motion blur (not in the paper; a workload of this project).

    A segment of the given length centred at the origin at ``angle_deg``
    (x to the right, y up) is sampled at ``samples`` equally spaced points,
    each splatted bilinearly onto the S x S grid (row offset p = -y, column
    offset q = x); the result is scaled to sum 1. It is point-symmetric.
    """
    R = S // 2
    P = np.zeros((S, S), dtype=np.float64)
    th = math.radians(angle_deg)
    t = np.linspace(-length / 2.0, length / 2.0, samples)
    xs, ys = t * math.cos(th), t * math.sin(th)
    for x, y in zip(xs, ys):
        pr, pc = -y + R, x + R
        r0, c0 = int(math.floor(pr)), int(math.floor(pc))
        fr, fc = pr - r0, pc - c0
        for dr, wr in ((0, 1.0 - fr), (1, fr)):
            for dc, wc in ((0, 1.0 - fc), (1, fc)):
                rr, cc = r0 + dr, c0 + dc
                if 0 <= rr < S and 0 <= cc < S:
                    P[rr, cc] += wr * wc
    # symmetrise the splat (equal up to rounding by construction)
    P = 0.5 * (P + P[::-1, ::-1])
    return P / P.sum()


def noise_direction(m: int, seed: int) -> np.ndarray:
    """Standard normal m x m draw (PCG64, ``seed``); the method scales it to
    the requested relative noise level, ||e|| / ||b_true|| (Sec. 5)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((m, m))


def add_noise(b_true: np.ndarray, xi: np.ndarray, level: float) -> np.ndarray:
    """b = b_true + e with e = level * ||b_true|| * xi / ||xi|| (Sec. 5)."""
    return b_true + level * np.linalg.norm(b_true) * xi / np.linalg.norm(xi)


def to_colmajor(X: np.ndarray, dtype=np.float64) -> np.ndarray:
    """C-contiguous buffer holding vec(X) (column-major), as the C-ABI expects."""
    return np.ascontiguousarray(np.asarray(X).T, dtype=dtype)


def from_colmajor(buf: np.ndarray, m: int) -> np.ndarray:
    """Inverse of :func:`to_colmajor`."""
    return np.asarray(buf, dtype=np.float64).reshape(m, m).T.copy()


# --- workload recipes -----------------------------------------------------

def problem(m: int, n_rect: int, n_disk: int, seed: int, psf: np.ndarray,
            noise: float, noise_seed: int | None = None):
    """(x_true, psf, xi, noise level) for one synthetic problem. The caller
    forms b with its own blur operator and :func:`add_noise`."""
    x_true = phantom(m, n_rect, n_disk, seed)
    xi = noise_direction(m, 10_000 + seed if noise_seed is None else noise_seed)
    return x_true, psf, xi, noise


def config_small(seed: int = 0):
    """m = 64, 12 rectangles, 6 disks, Gaussian sigma = 2 on 9 x 9, 1 % noise."""
    return problem(64, 12, 6, seed, gaussian_psf(2.0, 9), 0.01)


def config_512(seed: int = 0, noise: float = 0.01):
    """m = 512, 40 rectangles, 20 disks, Gaussian sigma = 3 on 15 x 15."""
    return problem(512, 40, 20, seed, gaussian_psf(3.0, 15), noise)


def config_large(m: int, seed: int = 0, blur: str = "gauss"):
    """m in {2048, 4096}: R = 40 sqrt(m/512) rectangles, R/2 disks, Gaussian
    sigma = 6 on 31 x 31 or 21-px motion at 30 degrees, 1 % noise."""
    R = int(round(40 * math.sqrt(m / 512)))
    psf = gaussian_psf(6.0, 31) if blur == "gauss" else motion_psf(21.0, 30.0, 21)
    return problem(m, R, R // 2, seed, psf, 0.01)
