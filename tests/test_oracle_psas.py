"""Pins of the oracle's RIOT-PSAS (Appendix, Algorithm 4: the observation-space
dual).

On a window without model steps (T = 0) observing half the variables, H is a
selection P and the dual Hessian has the closed form S P B P^T S (S =
diag(1/sigma_o)); its nonzero eigenvalues are those of the primal
A = L^T P^T S^2 P L (G G^T and G^T G, G = S P L).  At full rank (m = p) one
dual cycle lands on the primal minimiser x_b + L (-(I + A)^-1 b) (the
Sherman-Morrison-Woodbury identity), a second full-rank cycle of the linear
problem stays there (which the listing's literal x_{k-1} + B H^T dw update
does not), and on a nonlinear Lorenz-96 window the full-rank dual step equals
the primal Gauss-Newton step computed by the primal oracle (pinned
separately)."""
import numpy as np
import pytest

from oracle import bcov, l96, riot as orc
from synth import configs, philox


def _linear_problem(n=24, ell=2.0, seed=13, sig=(0.5, 2.0)):
    rng = np.random.default_rng(seed)
    L = bcov.bsqrt(n, ell, 1.0)
    idx = np.arange(0, n, 2)
    p = idx.size
    sigma = rng.uniform(sig[0], sig[1], p)
    x_b = 8.0 + rng.standard_normal(n)
    y = x_b[idx] + 1.5 * rng.standard_normal(p)
    prob = orc.L96Problem(n=n, T=0, dt=0.05, F=8.0, obs_step=np.zeros(p, dtype=np.int64), obs_idx=idx, y=y,
                          sigma_o=sigma, L=L, x_b=x_b)
    P = np.zeros((p, n))
    P[np.arange(p), idx] = 1.0
    return prob, P


def _omega(p, m, stream):
    return philox.normals(configs.BASE_SEED, stream, p * m).reshape(m, p).T


def test_dual_hessian_closed_form_and_spectrum():
    prob, P = _linear_problem()
    traj = orc.trajectory(prob, prob.x_b)
    S = np.diag(1.0 / prob.sigma_o)
    B = prob.L @ prob.L.T
    Ad = orc.dual_hvp(prob, traj, np.eye(prob.p))
    want = S @ P @ B @ P.T @ S
    np.testing.assert_allclose(Ad, want, rtol=0, atol=1e-13 * np.abs(want).max())
    A = prob.L.T @ P.T @ S @ S @ P @ prob.L
    ev_primal = np.sort(np.linalg.eigvalsh(A))[::-1][:prob.p]
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(Ad))[::-1], ev_primal, rtol=1e-10)
    # and the primal oracle's own dense Hessian agrees with the closed form (two integrator orders)
    np.testing.assert_allclose(orc.dense_hessian(prob, traj), A, rtol=0, atol=1e-13 * np.abs(A).max())


@pytest.mark.parametrize("sig,mode", [((0.5, 2.0), 1), ((0.02, 0.05), 0)])
def test_full_rank_cycle_is_the_primal_minimiser_and_a_fixed_point(sig, mode):
    """Weakly observed: some dual eigenvalues below 1 (LRU); strongly observed: all above (LRA)."""
    prob, P = _linear_problem(sig=sig)
    n, p = prob.n, prob.p
    S2 = np.diag(1.0 / prob.sigma_o ** 2)
    A = prob.L.T @ P.T @ S2 @ P @ prob.L
    b = prob.L.T @ (P.T @ (S2 @ (prob.x_b[P.argmax(axis=1)] - prob.y)))
    x_star = prob.x_b + prob.L @ (-np.linalg.solve(np.eye(n) + A, b))
    st1 = orc.psas_outer_step(prob, prob.x_b, _omega(p, p, 60))
    assert st1["mode"] == mode
    np.testing.assert_allclose(st1["bprime"], 0.0, atol=1e-15)
    np.testing.assert_allclose(st1["x_next"], x_star, rtol=0, atol=1e-10 * np.abs(x_star).max())
    st2 = orc.psas_outer_step(prob, st1["x_next"], _omega(p, p, 61))
    np.testing.assert_allclose(st2["bprime"], P @ (prob.x_b - st1["x_next"]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(st2["x_next"], x_star, rtol=0, atol=1e-10 * np.abs(x_star).max())
    # the listing's literal update would move away from the minimiser
    literal = st1["x_next"] + (st2["x_next"] - prob.x_b)
    assert np.linalg.norm(literal - x_star) > 1e-3 * np.linalg.norm(x_star - prob.x_b)


@pytest.mark.parametrize("q,exact_rr", [(0, False), (1, False), (0, True)])
def test_full_rank_dual_step_equals_the_primal_gauss_newton_step(q, exact_rr):
    """Nonlinear Lorenz-96 window, 10 observations of a 40-variable state."""
    n, T = 40, 8
    rng = np.random.default_rng(17)
    x0 = l96.nl(8.0 + rng.standard_normal(n), 300, 0.05, 8.0)[-1]
    steps = np.repeat([4, 8], 5)
    idx = np.concatenate([np.array([1, 9, 17, 25, 33]), np.array([5, 13, 21, 29, 37])])
    truth = l96.nl(x0, T, 0.05, 8.0)
    sigma = np.full(10, 0.5)
    y = truth[steps, idx] + sigma * rng.standard_normal(10)
    L = bcov.bsqrt(n, 2.0, 1.0)
    prob = orc.L96Problem(n=n, T=T, dt=0.05, F=8.0, obs_step=steps, obs_idx=idx, y=y, sigma_o=sigma, L=L,
                          x_b=x0 + L @ rng.standard_normal(n))
    st = orc.psas_outer_step(prob, prob.x_b, _omega(prob.p, prob.p, 62), q=q, exact_rr=exact_rr)
    traj = orc.trajectory(prob, prob.x_b)
    g = orc.gradient_b(prob, traj, orc.innovation(prob, traj))
    dv = orc.converged_increment(prob, traj, g)
    x_gn = prob.x_b + L @ dv
    np.testing.assert_allclose(st["x_next"], x_gn, rtol=0, atol=1e-9 * np.abs(x_gn - prob.x_b).max())
    # the dual eigenvalues are the primal ones (p nonzero of n)
    ev = np.sort(np.linalg.eigvalsh(orc.dense_hessian(prob, traj)))[::-1][:prob.p]
    np.testing.assert_allclose(st["lam"], ev, rtol=1e-8, atol=1e-10 * ev[0])


# --- the tracer-transport problem ---------------------------------------------------------

@pytest.fixture(scope="module")
def tracer():
    from oracle import advdiff as AD
    from synth import advdiff as S
    cfg = S.bc_tiny()
    prob = AD.build(cfg)
    return AD, cfg, prob


def test_tracer_dual_hessian_against_the_tangent_linear_jacobian(tracer):
    """The dual product runs the adjoint, then the TL model; G = H' L from the TL model alone
    (column by column) gives S G G^T S, and the nonzero spectrum is the primal one."""
    AD, _, prob = tracer
    traj = AD.trajectory(prob, prob.x_b)
    Ad = AD.dual_hvp(prob, traj, np.eye(prob.p))
    G = AD.tl_obs(prob, traj, prob.Lop.apply(np.eye(prob.n))).T          # (p, n)
    S = 1.0 / prob.sigma_o
    want = (S[:, None] * G) @ (G.T * S[None, :])
    np.testing.assert_allclose(Ad, want, rtol=0, atol=1e-10 * np.abs(want).max())
    r = min(prob.n, prob.p)
    ev_d = np.sort(np.linalg.eigvalsh(0.5 * (Ad + Ad.T)))[::-1][:r]
    ev_p = np.sort(np.linalg.eigvalsh(AD.hvp(prob, traj, np.eye(prob.n))))[::-1][:r]
    np.testing.assert_allclose(ev_d, ev_p, rtol=0, atol=1e-9 * ev_p[0])


def test_tracer_full_rank_dual_cycle_is_the_exact_inner_solution(tracer):
    AD, cfg, prob = tracer
    st = AD.psas_outer_step(prob, prob.x_b, _omega(prob.p, prob.p, 63))
    np.testing.assert_allclose(st["bprime"], 0.0, atol=1e-15)
    traj = st["traj"]
    g = AD.gradient_b(prob, traj, AD.innovation(prob, traj))
    dv = -orc.cg_solve(lambda v: v + AD.hvp(prob, traj, v[:, None])[:, 0], g, tol=1e-14)
    x_exact = prob.x_b + prob.Lop.apply(dv)
    dx = x_exact - prob.x_b
    np.testing.assert_allclose(st["x_next"], x_exact, rtol=0, atol=1e-8 * np.abs(dx).max())
