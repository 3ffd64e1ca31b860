"""FP64 Lorenz-96 model, tangent-linear and adjoint (oracle).

Thin numpy wrappers over the plain-C integrators in ``l96.c``: Section 3.1
(the L-96 equation) and the TL/AD models that Algorithms 1-3 linearise about
the stored trajectory.  Test infrastructure only.
"""
import numpy as np

from ._clib import lib, ptr


def rhs(x, F):
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.empty_like(x)
    lib().l96_rhs(x.size, F, ptr(x), ptr(f))
    return f


def nl(x0, T, dt, F):
    """Trajectory x_t, t = 0..T, shape (T+1, n)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    n = x0.size
    traj = np.empty((T + 1, n))
    lib().l96_nl(n, T, dt, F, ptr(x0), ptr(traj))
    return traj


def tl(traj, dx0, dt, F):
    """TL states M_{0->t} dx0 for t = 0..T, shape (T+1, n)."""
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    dx0 = np.ascontiguousarray(dx0, dtype=np.float64)
    T = traj.shape[0] - 1
    n = traj.shape[1]
    out = np.empty((T + 1, n))
    lib().l96_tl(n, T, dt, F, ptr(traj), ptr(dx0), ptr(out))
    return out


def ad(traj, forcing, dt, F):
    """lam_0 of the backward recursion lam_t = M_t^T lam_{t+1} + forcing_t."""
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    forcing = np.ascontiguousarray(forcing, dtype=np.float64)
    T = traj.shape[0] - 1
    n = traj.shape[1]
    assert forcing.shape == (T + 1, n)
    lam0 = np.empty(n)
    lib().l96_ad(n, T, dt, F, ptr(traj), ptr(forcing), ptr(lam0))
    return lam0
