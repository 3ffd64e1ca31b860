"""Pins of the oracle's spectral preconditioner and rotation (Section 2.2
"Preconditioning", Eq. 7, Algorithm 3 with precond / rotation).

Each check rests on something other than the oracle itself: the closed form of
the Hessian of a window with no model steps (T = 0, every variable observed:
A = L^T R^-1 L), its eigendecomposition by LAPACK, the exact minimiser
-(I + A)^-1 b by a dense solve, and the algebra of the factors (inverse,
transpose).  A preconditioner built from exact eigenpairs must send the
resolved eigenvalues of A to 0 and leave the others alone; two outer loops, the
second run with rotation on exactly the unresolved complement, must land on the
exact minimiser of the linear problem."""
import numpy as np
import pytest

from oracle import bcov, problem, riot as orc
from synth import configs, philox


def _linear_problem(n=24, ell=2.0, seed=11):
    """Lorenz-96 state observed at t = 0 only (T = 0): H is the identity, so
    A = L^T R^-1 L is known in closed form and does not depend on x."""
    rng = np.random.default_rng(seed)
    L = bcov.bsqrt(n, ell, 1.0)
    sigma = rng.uniform(0.5, 2.0, n)
    x_b = 8.0 + rng.standard_normal(n)
    y = x_b + 1.5 * rng.standard_normal(n)
    prob = orc.L96Problem(n=n, T=0, dt=0.05, F=8.0, obs_step=np.zeros(n, dtype=np.int64),
                          obs_idx=np.arange(n), y=y, sigma_o=sigma, L=L, x_b=x_b)
    A = L.T @ np.diag(1.0 / sigma ** 2) @ L
    b0 = L.T @ ((x_b - y) / sigma ** 2)
    return prob, A, b0


def _eig_desc(A):
    lam, V = np.linalg.eigh(A)
    return lam[::-1], V[:, ::-1]


def test_closed_form_hessian_of_the_linear_window():
    prob, A, b0 = _linear_problem()
    traj = orc.trajectory(prob, prob.x_b)
    np.testing.assert_allclose(orc.dense_hessian(prob, traj), A, rtol=0, atol=1e-13 * np.abs(A).max())
    np.testing.assert_allclose(orc.gradient_b(prob, traj, orc.innovation(prob, traj)), b0, rtol=1e-13)


def test_factors_invert_and_transpose():
    n = 30
    rng = np.random.default_rng(3)
    pc = orc.SpectralPreconditioner(n)
    for m in (5, 8, 3):
        V, _ = np.linalg.qr(rng.standard_normal((n, m)))
        pc.push(rng.uniform(-0.5, 40.0, m), V)
    I = np.eye(n)
    P = pc.apply(I)
    np.testing.assert_allclose(pc.apply_t(I), P.T, atol=1e-13)
    np.testing.assert_allclose(pc.apply_inv(P), I, atol=1e-12)
    np.testing.assert_allclose(P @ pc.apply_inv(I), I, atol=1e-12)
    with pytest.raises(ValueError):
        pc.push(np.array([-1.0]), np.eye(n)[:, :1])


def test_exact_pairs_deflate_the_resolved_modes():
    """P'^T (I + A) P' = I on the resolved span: those eigenvalues of A_2 are 0,
    the unresolved ones are unchanged (V spans an invariant subspace)."""
    prob, A, _ = _linear_problem()
    n, m = prob.n, 7
    lam, V = _eig_desc(A)
    pc = orc.SpectralPreconditioner(n)
    pc.push(lam[:m], V[:, :m])
    Ak = pc.hessian(lambda W: A @ W)(np.eye(n))
    np.testing.assert_allclose(Ak, Ak.T, atol=1e-12 * lam[0])
    got = np.sort(np.linalg.eigvalsh(0.5 * (Ak + Ak.T)))
    want = np.sort(np.concatenate([np.zeros(m), lam[m:]]))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11 * lam[0])


def test_rotation_samples_the_unresolved_complement():
    prob, A, _ = _linear_problem()
    n, m = prob.n, 6
    lam, V = _eig_desc(A)
    pc = orc.SpectralPreconditioner(n)
    pc.push(lam[:m], V[:, :m])
    Om = philox.normals(configs.BASE_SEED, 40, n * 9).reshape(9, n).T
    rot = pc.rotate(Om)
    back = pc.apply(rot)                              # the sampled directions in the control variable
    np.testing.assert_allclose(V[:, :m].T @ back, 0.0, atol=1e-12 * np.abs(Om).max())
    np.testing.assert_allclose(back, Om - V[:, :m] @ (V[:, :m].T @ Om), atol=1e-12 * np.abs(Om).max())
    Ur = pc.rotation_basis()
    assert Ur.shape == (n, m)
    np.testing.assert_allclose(Ur @ Ur.T, V[:, :m] @ V[:, :m].T, atol=1e-12)


@pytest.mark.parametrize("m", [5, 12])
def test_two_loops_with_rotation_reach_the_minimiser(m):
    """Loop 1: the adaptive increment from the exact leading m pairs.  Loop 2:
    preconditioned, rotated, with n - m samples, so its sketch spans exactly the
    unresolved complement.  The total increment must be -(I + A)^-1 b."""
    prob, A, b0 = _linear_problem()
    n = prob.n
    lam, V = _eig_desc(A)
    exact = -np.linalg.solve(np.eye(n) + A, b0)
    dv1, _ = orc.increment(lam[:m], V[:, :m], b0)
    pc = orc.SpectralPreconditioner(n)
    pc.push(lam[:m], V[:, :m])
    x1, v1 = prob.x_b + prob.L @ dv1, dv1
    Om = philox.normals(configs.BASE_SEED, 41, n * (n - m)).reshape(n - m, n).T
    st = orc.outer_step_precond(prob, x1, v1, Om, pc, rotation=True)
    np.testing.assert_allclose(st["lam"], lam[m:], rtol=0, atol=1e-10 * lam[0])
    assert np.linalg.norm(st["v_next"] - exact) <= 1e-10 * np.linalg.norm(exact)
    np.testing.assert_allclose(st["x_next"], prob.x_b + prob.L @ exact, rtol=0, atol=1e-10 * np.abs(prob.x_b).max())


def test_full_rank_second_loop_reaches_the_minimiser_after_an_approximate_first():
    """Whatever loop 1 resolved (a rank-8 randomized estimate here), a full-rank
    loop 2 minimises the preconditioned quadratic exactly, and mapping its
    increment back by P_2 gives the exact minimiser of the original one."""
    prob, A, b0 = _linear_problem()
    n = prob.n
    exact = -np.linalg.solve(np.eye(n) + A, b0)
    Om1 = philox.normals(configs.BASE_SEED, 42, n * 8).reshape(8, n).T
    pc = orc.SpectralPreconditioner(n)
    st1 = orc.outer_step_precond(prob, prob.x_b, np.zeros(n), Om1, pc, q=1)
    pc.push(st1["lam"], st1["U"])
    Om2 = philox.normals(configs.BASE_SEED, 43, n * n).reshape(n, n).T
    st2 = orc.outer_step_precond(prob, st1["x_next"], st1["v_next"], Om2, pc)
    assert np.linalg.norm(st2["v_next"] - exact) <= 1e-9 * np.linalg.norm(exact)
    # the increment of loop 1 alone is not the minimiser (the check above is not vacuous)
    assert np.linalg.norm(st1["v_next"] - exact) > 1e-3 * np.linalg.norm(exact)


def test_first_loop_is_the_unpreconditioned_cycle():
    cfg = configs.l96_custom("pc_small", n=40, T=12, obs_every=2, obs_frac=0.5, ell=2.0, k=10, q=1)
    prob = problem.build(cfg)
    Om = cfg.sketch(0).T
    a = orc.outer_step(prob, prob.x_b, np.zeros(cfg.n), Om, q=1)
    b = orc.outer_step_precond(prob, prob.x_b, np.zeros(cfg.n), Om, orc.SpectralPreconditioner(cfg.n), q=1,
                               rotation=True)
    np.testing.assert_allclose(b["lam"], a["lam"], rtol=1e-13)
    np.testing.assert_allclose(b["dv"], a["dv"], rtol=0, atol=1e-13 * np.abs(a["dv"]).max())


def test_inverse_is_the_identity_on_the_rotated_complement():
    """P_k^{-1} z = z for every z orthogonal to all P_j V_j (induction over the factors:
    P_j^T z = z and (P_j V_j)^T z = V_j^T z), so the P_k^{-1} of the rotation only
    changes rounding.  Checked with inexact, non-orthogonal factor spans."""
    n = 40
    rng = np.random.default_rng(5)
    pc = orc.SpectralPreconditioner(n)
    for m in (6, 4, 7):
        V, _ = np.linalg.qr(rng.standard_normal((n, m)))
        pc.push(rng.uniform(0.1, 50.0, m), V)
    Ur = pc.rotation_basis()
    assert Ur.shape[1] == 17
    z = rng.standard_normal((n, 5))
    z -= Ur @ (Ur.T @ z)
    np.testing.assert_allclose(pc.apply_inv(z), z, atol=1e-12)
    np.testing.assert_allclose(pc.apply(z), z, atol=1e-12)
    np.testing.assert_allclose(pc.apply_t(z), z, atol=1e-12)
