"""Prior covariance square root B = L L^T (oracle, FP64, dense).

Section 2.1 writes B = L L^T and works in the control variable dz with
dx = L dz.  The Lorenz-96 workloads take B Gaussian-correlated on the
periodic ring: C_ij = exp(-d_ij^2 / (2 l^2)) with d_ij = min(|i-j|, n-|i-j|),
and B = diag(sigma) C diag(sigma).  L is the symmetric square root of C,
scaled by sigma on the left: L = diag(sigma) S, S = f(C).

The paper does not say how L is formed.  The exact square root of a
Gaussian correlation matrix is numerically ill-posed: its smallest
eigenvalues sit far below double rounding, so any two computations of
sqrt(C) differ at the 1e-8 level there.  The reading used here (and by the
GPU library, which reaches the same S through the discrete Fourier
transform) is a regularised square root, f(c) = sqrt(c) for c >= tau and
f(c) = c / sqrt(tau) below, with tau = 1e-10 * max eigenvalue: continuous,
equal to sqrt(c) on every eigenvalue that carries information, and
insensitive to rounding noise in the tiny ones.

Test infrastructure only.
"""
import functools

import numpy as np

TAU_REL = 1e-10


def ring_distance(n):
    i = np.arange(n)
    d = np.abs(i[:, None] - i[None, :])
    return np.minimum(d, n - d)


def gaussian_corr(n, ell):
    d = ring_distance(n).astype(np.float64)
    return np.exp(-d * d / (2.0 * ell * ell))


def reg_sqrt_eigs(c):
    tau = TAU_REL * np.max(c)
    out = np.where(c >= tau, np.sqrt(np.maximum(c, tau)), c / np.sqrt(tau))
    return out


@functools.lru_cache(maxsize=8)
def _sqrt_corr_cached(n, ell):
    C = gaussian_corr(n, ell)
    lam, V = np.linalg.eigh(C)
    S = (V * reg_sqrt_eigs(lam)) @ V.T
    S = 0.5 * (S + S.T)
    S.setflags(write=False)
    return S


def sqrt_corr(n, ell):
    """S = f(C) for the Gaussian ring correlation (dense n x n, symmetric)."""
    return _sqrt_corr_cached(int(n), float(ell))


def bsqrt(n, ell, sigma_b):
    """L = diag(sigma) S; sigma_b is a scalar or a length-n vector."""
    S = sqrt_corr(n, ell)
    sig = np.broadcast_to(np.asarray(sigma_b, dtype=np.float64), (n,))
    return sig[:, None] * S
