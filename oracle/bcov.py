"""Prior covariance square root B = L L^T (oracle, FP64, dense).

Section 2.1 writes B = L L^T and works in the control variable dv with
dx = L dv; Section 3.1 takes Gaussian background-error correlations.  The
paper does not say how L is formed.  The reading used here (and by the GPU
library) is the square-root kernel of a Gaussian correlation: L is the
periodic Gaussian convolution of length l/sqrt(2),

    S_d = alpha * sum_j exp(-(d + j n)^2 / l^2),   L = diag(sigma) S,

normalised so that (S S^T)_ii = 1.  Since a Gaussian of length l/sqrt(2)
convolved with itself is a Gaussian of length l, B = L L^T is the Gaussian
correlation exp(-d^2 / (2 l^2)) scaled by sigma_i sigma_j, up to lattice
terms of relative size 2 exp(-pi^2 l^2 / 2) (5e-9 at l = 2, 1e-34 at l = 4).
S is symmetric, so L is the symmetric square root of B when sigma is
constant.  Unlike the eigen-square-root of the sampled Gaussian (whose
smallest eigenvalues sit below double rounding), this L is well defined to
rounding and its entries below 1e-18 of the peak are exactly negligible.

Test infrastructure only.
"""
import functools

import numpy as np


def ring_distance(n):
    i = np.arange(n)
    d = np.abs(i[:, None] - i[None, :])
    return np.minimum(d, n - d)


def gaussian_corr(n, ell):
    """The target correlation C_ij = exp(-d_ij^2 / (2 l^2)) on the ring."""
    d = ring_distance(n).astype(np.float64)
    return np.exp(-d * d / (2.0 * ell * ell))


def sqrt_kernel_row(n, ell):
    """First row of S: the periodised Gaussian exp(-m^2 / l^2), unit-variance normalised."""
    d = np.arange(n, dtype=np.float64)
    row = np.zeros(n)
    reach = int(np.ceil(40.0 * ell / n)) + 1
    for j in range(-reach, reach + 1):
        row += np.exp(-((d + j * n) ** 2) / (ell * ell))
    return row / np.sqrt(np.sum(row * row))


@functools.lru_cache(maxsize=8)
def _sqrt_corr_cached(n, ell):
    row = sqrt_kernel_row(n, ell)
    i = np.arange(n)
    S = row[(i[None, :] - i[:, None]) % n]     # S_ij = row[(j - i) mod n]
    S.setflags(write=False)
    return S


def sqrt_corr(n, ell):
    """S (dense n x n, symmetric circulant), S S^T = Gaussian correlation."""
    return _sqrt_corr_cached(int(n), float(ell))


def bsqrt(n, ell, sigma_b):
    """L = diag(sigma) S; sigma_b is a scalar or a length-n vector."""
    S = sqrt_corr(n, ell)
    sig = np.broadcast_to(np.asarray(sigma_b, dtype=np.float64), (n,))
    return sig[:, None] * S
