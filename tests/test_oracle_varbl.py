"""Pins of the oracle's Algorithm 2 (VarBL, block Lanczos from gradient samples).

Checked against what the mathematics fixes, not against the oracle itself:
with one sample the block recurrence is Algorithm 1 (pinned separately); when
the block Krylov space fills the whole space the increment is the exact
minimiser -(I + A)^-1 g (dense solve of the closed-form Hessian of a window
without model steps); the basis is orthonormal, T is the projection Q^T A Q and
the basis spans the block Krylov space; the Ritz values interlace with the
eigenvalues of A (Cauchy); the gradient samples reduce to the gradient without
perturbations and to their closed form on the linear window."""
import numpy as np
import pytest

from oracle import bcov, problem, riot as orc
from synth import configs, philox


def _linear_problem(n=24, ell=2.0, seed=11):
    rng = np.random.default_rng(seed)
    L = bcov.bsqrt(n, ell, 1.0)
    sigma = rng.uniform(0.5, 2.0, n)
    x_b = 8.0 + rng.standard_normal(n)
    y = x_b + 1.5 * rng.standard_normal(n)
    prob = orc.L96Problem(n=n, T=0, dt=0.05, F=8.0, obs_step=np.zeros(n, dtype=np.int64),
                          obs_idx=np.arange(n), y=y, sigma_o=sigma, L=L, x_b=x_b)
    A = L.T @ np.diag(1.0 / sigma ** 2) @ L
    return prob, A


def _eps(n, l, stream):
    return philox.normals(configs.BASE_SEED, stream, n * l).reshape(l, n).T


def test_samples_without_perturbation_are_the_gradient():
    cfg = configs.l96_custom("vbl_small", n=40, T=12, obs_every=2, obs_frac=0.5, ell=2.0, k=8, q=0)
    prob = problem.build(cfg)
    traj = orc.trajectory(prob, prob.x_b)
    v = 0.1 * _eps(cfg.n, 1, 50)[:, 0]
    g = orc.gradient_b(prob, traj, orc.innovation(prob, traj)) + v
    B = orc.gradient_samples(prob, prob.x_b, v, np.zeros((prob.p, 3)), np.zeros((cfg.n, 3)))
    for j in range(3):
        np.testing.assert_allclose(B[:, j], g, rtol=1e-14, atol=1e-14 * np.abs(g).max())


def test_samples_closed_form_on_the_linear_window():
    prob, A = _linear_problem()
    n, l = prob.n, 4
    eo, eb = _eps(n, l, 51), _eps(n, l, 52)
    v = 0.3 * _eps(n, 1, 53)[:, 0]
    B = orc.gradient_samples(prob, prob.x_b, v, eo, eb)
    L, s = prob.L, prob.sigma_o
    for j in range(l):
        d = prob.x_b + L @ eb[:, j] - prob.y + s * eo[:, j]
        want = L.T @ (d / s ** 2) + v + eb[:, j]
        np.testing.assert_allclose(B[:, j], want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_one_sample_is_algorithm_1():
    cfg = configs.l96_custom("vbl_small", n=40, T=12, obs_every=2, obs_frac=0.5, ell=2.0, k=8, q=0)
    prob = problem.build(cfg)
    traj = orc.trajectory(prob, prob.x_b)
    g = orc.gradient_b(prob, traj, orc.innovation(prob, traj))
    dv1, th1, _ = orc.varcg(prob, traj, g, 9)
    dv2, th2, _, _, _ = orc.varbl(prob, traj, g[:, None], 9, g)
    np.testing.assert_allclose(np.sort(th2), np.sort(th1), rtol=0, atol=1e-10 * th1.max())
    np.testing.assert_allclose(dv2, dv1, rtol=0, atol=1e-10 * np.abs(dv1).max())


@pytest.mark.parametrize("l,m", [(4, 6), (3, 8), (6, 4)])
def test_full_block_krylov_space_gives_the_minimiser(l, m):
    prob, A = _linear_problem()
    n = prob.n
    assert l * m == n
    traj = orc.trajectory(prob, prob.x_b)
    g = orc.gradient_b(prob, traj, orc.innovation(prob, traj))
    B0 = orc.gradient_samples(prob, prob.x_b, np.zeros(n), _eps(n, l, 54), _eps(n, l, 55))
    dv, lam, U, T, Q = orc.varbl(prob, traj, B0, m, g)
    exact = -np.linalg.solve(np.eye(n) + A, g)
    assert np.linalg.norm(dv - exact) <= 1e-9 * np.linalg.norm(exact)
    np.testing.assert_allclose(np.sort(lam), np.linalg.eigvalsh(A), rtol=0, atol=1e-9 * np.abs(A).max())


def test_basis_projection_krylov_span_and_interlacing():
    prob, A = _linear_problem(n=30)
    n, l, m = prob.n, 3, 4
    traj = orc.trajectory(prob, prob.x_b)
    g = orc.gradient_b(prob, traj, orc.innovation(prob, traj))
    B0 = _eps(n, l, 56)
    dv, lam, U, T, Q = orc.varbl(prob, traj, B0, m, g)
    np.testing.assert_allclose(Q.T @ Q, np.eye(l * m), atol=1e-12)
    np.testing.assert_allclose(T, Q.T @ A @ Q, rtol=0, atol=1e-10 * np.abs(A).max())
    # block tridiagonal: blocks two or more off the diagonal vanish
    for i in range(m):
        for j in range(m):
            if abs(i - j) > 1:
                assert np.abs(T[i * l:(i + 1) * l, j * l:(j + 1) * l]).max() <= 1e-10 * np.abs(A).max()
    # span(Q) = span[B0, A B0, ..., A^(m-1) B0]
    K = np.hstack([np.linalg.matrix_power(A, j) @ B0 for j in range(m)])
    Kn = K / np.linalg.norm(K, axis=0)
    assert np.linalg.norm(Kn - Q @ (Q.T @ Kn)) <= 1e-8 * np.linalg.norm(Kn)
    # Cauchy interlacing: the i-th largest Ritz value lies below the i-th largest eigenvalue of A
    ev = np.sort(np.linalg.eigvalsh(A))[::-1]
    assert np.all(lam <= ev[:lam.size] * (1 + 1e-12) + 1e-12)
    assert np.all(lam[::-1] >= ev[::-1][:lam.size] * (1 - 1e-12) - 1e-12)
    # the increment is Algorithm 2's formula on the orthonormal Ritz vectors
    np.testing.assert_allclose(U.T @ U, np.eye(l * m), atol=1e-12)


def test_invariant_krylov_space_stops_the_recurrence():
    """B0 spanned by four eigenvectors of A: the space is invariant after one block."""
    prob, A = _linear_problem()
    ev, V = np.linalg.eigh(A)
    traj = orc.trajectory(prob, prob.x_b)
    g = V[:, -4:] @ np.array([1.0, -2.0, 0.5, 3.0])
    dv, lam, U, T, Q = orc.varbl(prob, traj, V[:, -4:] @ np.diag([1.0, 2.0, 3.0, 4.0]), 5, g)
    assert T.shape == (4, 4)
    np.testing.assert_allclose(np.sort(lam), ev[-4:], rtol=1e-12)
    np.testing.assert_allclose(dv, -np.linalg.solve(np.eye(prob.n) + A, g), rtol=0, atol=1e-12 * np.abs(g).max())
