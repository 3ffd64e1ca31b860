"""Pins for the oracle's 4D-Var / RIOT linear algebra (CPU only).

The references here are closed forms (A = L^T L for a one-time fully
observed window, A = I in the trivial case), dense-matrix identities
(P_a = (B^-1 + G^T R^-1 G)^-1), finite differences of the non-quadratic cost,
textbook solves, and the full-rank equalities of Section 2.2: at k = n the
randomized range finder spans everything, so RIOT, CG and the exact
minimiser coincide and LRA = LRU.
"""
import numpy as np
import pytest

from synth import configs
from oracle import bcov, l96, problem, riot


def _problem_from(n, T, ell, sigma_b, obs_steps, obs_idx, sigma_o=1.0, F=8.0, dt=0.05, seed=0):
    rng = np.random.default_rng(seed)
    x0 = l96.nl(F + rng.standard_normal(n), 300, dt, F)[-1]
    st = np.repeat(np.asarray(obs_steps), len(obs_idx))
    ix = np.tile(np.asarray(obs_idx), len(obs_steps))
    L = bcov.bsqrt(n, ell, sigma_b)
    traj_true = l96.nl(x0, T, dt, F)
    y = traj_true[st, ix] + rng.standard_normal(st.size) * sigma_o
    x_b = x0 + L @ rng.standard_normal(n)
    return riot.L96Problem(n=n, T=T, dt=dt, F=F, obs_step=st, obs_idx=ix, y=y,
                           sigma_o=np.full(st.size, sigma_o), L=L, x_b=x_b)


def _sigma_vec(n):
    return 0.5 + np.arange(n) / n      # makes L = diag(sigma) S non-symmetric


def test_gaussian_sqrt_reproduces_B():
    # B = L L^T must be the Gaussian correlation exp(-d^2/(2 l^2)) scaled by
    # sigma_i sigma_j (|sigma| <= 1.5), up to the lattice term
    # 2 exp(-pi^2 l^2 / 2) and, on short rings, the periodic images
    # exp(-(n - d)^2 / (2 l^2)) that the ring distance leaves out.
    for n, ell, tol in [(40, 2.0, 5e-8), (33, 3.0, 5e-7), (64, 4.0, 5e-14)]:
        sig = _sigma_vec(n)
        L = bcov.bsqrt(n, ell, sig)
        B = sig[:, None] * bcov.gaussian_corr(n, ell) * sig[None, :]
        np.testing.assert_allclose(L @ L.T, B, rtol=0, atol=tol)
        S = bcov.sqrt_corr(n, ell)
        np.testing.assert_allclose(S, S.T, rtol=0, atol=0)
        # circulant: every row is the previous one shifted by one place
        np.testing.assert_allclose(np.roll(S[0], 5), S[5], rtol=0, atol=0)


def test_single_time_full_observation_gives_LtL():
    # T = 0, all variables observed at t = 0, R = I  =>  A = L^T L.
    n = 16
    p = _problem_from(n, 0, 2.0, _sigma_vec(n), [0], np.arange(n))
    traj = riot.trajectory(p, p.x_b)
    A = riot.dense_hessian(p, traj)
    np.testing.assert_allclose(A, p.L.T @ p.L, rtol=0, atol=1e-13)


def test_hessian_equals_GtRinvG_and_is_psd():
    n = 20
    p = _problem_from(n, 8, 2.0, _sigma_vec(n), [2, 5, 8], np.arange(0, n, 3), sigma_o=0.7)
    traj = riot.trajectory(p, p.x_b)
    A = riot.dense_hessian(p, traj)
    G = riot.tl_matrix(p, traj)
    ref = G.T @ (G * p.rinv[:, None])
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > -1e-12 * np.abs(A).max()


def test_gradient_is_derivative_of_cost():
    n = 18
    p = _problem_from(n, 10, 2.0, _sigma_vec(n), [3, 6, 10], np.arange(0, n, 2))
    rng = np.random.default_rng(9)
    v = 0.1 * rng.standard_normal(n)
    x = p.x_b + p.L @ v
    traj = riot.trajectory(p, x)
    g = riot.gradient_b(p, traj, riot.innovation(p, traj)) + v
    e = 1e-6
    fd = np.empty(n)
    for j in range(n):
        dv = np.zeros(n)
        dv[j] = e
        Jp = riot.cost(p, riot.trajectory(p, x + p.L @ dv), v + dv)
        Jm = riot.cost(p, riot.trajectory(p, x - p.L @ dv), v - dv)
        fd[j] = (Jp - Jm) / (2 * e)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


def test_trivial_hessian_identity_lru_tie():
    # L = I (vanishing correlation length), T = 0, every variable observed,
    # R = I  =>  A = I, every eigenvalue is exactly 1, Algorithm 3's switch
    # picks LRU, and dv = -(I - U U^T / 2) g = -g / 2.
    n = 12
    p = _problem_from(n, 0, 0.05, 1.0, [0], np.arange(n))
    np.testing.assert_allclose(p.L, np.eye(n), atol=1e-15)
    traj = riot.trajectory(p, p.x_b)
    Om = configs.l96_small().sketch(0, k=n, n=n).T
    lam, U, _ = riot.rsvd(p, traj, Om)
    np.testing.assert_allclose(lam, 1.0, atol=1e-12)
    g = np.random.default_rng(1).standard_normal(n)
    dv, mode = riot.increment(lam, U, g)
    assert mode == 1
    np.testing.assert_allclose(dv, -g / 2, atol=1e-12)


def test_increment_mode_rule():
    U = np.eye(4)[:, :2]
    g = np.ones(4)
    assert riot.increment(np.array([3.0, 1.0]), U, g)[1] == 1       # lambda_m = 1 -> LRU
    assert riot.increment(np.array([3.0, 1.0 + 1e-12]), U, g)[1] == 0
    dv, _ = riot.increment(np.array([3.0, 2.0]), U, g)
    np.testing.assert_allclose(dv, [-0.25, -1 / 3, 0, 0])
    dv, _ = riot.increment(np.array([3.0, 0.5]), U, g)
    np.testing.assert_allclose(dv, [-0.25, -1 / 1.5, -1, -1])


@pytest.fixture(scope="module")
def small():
    cfg = configs.l96_small()
    p = problem.build(cfg)
    traj = riot.trajectory(p, p.x_b)
    return cfg, p, traj


def test_full_rank_rsvd_matches_dense_eigh(small):
    cfg, p, traj = small
    A = riot.dense_hessian(p, traj)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (A + A.T)))[::-1]
    lam, U, _ = riot.rsvd(p, traj, cfg.sketch(0).T, q=cfg.q)
    np.testing.assert_allclose(lam, ev, rtol=1e-9, atol=1e-9 * ev[0])
    # eigenvectors: A U = U Lambda
    np.testing.assert_allclose(A @ U, U * lam, rtol=0, atol=1e-9 * ev[0])
    np.testing.assert_allclose(U.T @ U, np.eye(cfg.n), atol=1e-10)


def test_full_rank_increment_is_exact_minimiser(small):
    cfg, p, traj = small
    d = riot.innovation(p, traj)
    g = riot.gradient_b(p, traj, d)
    lam, U, _ = riot.rsvd(p, traj, cfg.sketch(0).T)
    dv, mode = riot.increment(lam, U, g)
    A = riot.dense_hessian(p, traj)
    exact = -np.linalg.solve(np.eye(cfg.n) + A, g)
    np.testing.assert_allclose(dv, exact, rtol=0, atol=1e-10 * np.abs(exact).max())
    cg = riot.converged_increment(p, traj, g)
    np.testing.assert_allclose(cg, exact, rtol=0, atol=1e-10 * np.abs(exact).max())
    # LRA and LRU coincide at full rank
    c = U.T @ g
    lra = -(U @ (c / (1 + lam)))
    lru = -(g - U @ (c * lam / (1 + lam)))
    np.testing.assert_allclose(lra, lru, atol=1e-10 * np.abs(lra).max())
    # Algorithm 1 with m = n Lanczos steps reaches the same minimiser
    dv1, _, _ = riot.varcg(p, traj, g, cfg.n)
    np.testing.assert_allclose(dv1, exact, atol=1e-8 * np.abs(exact).max())


def test_minimiser_zeroes_quadratic_gradient(small):
    cfg, p, traj = small
    d = riot.innovation(p, traj)
    v = np.zeros(cfg.n)
    g = riot.gradient_b(p, traj, d) + v
    dv = riot.converged_increment(p, traj, g)
    J0 = riot.quadratic_cost(p, traj, d, v, dv)
    rng = np.random.default_rng(3)
    for _ in range(3):
        e = 1e-3 * rng.standard_normal(cfg.n)
        assert riot.quadratic_cost(p, traj, d, v, dv + e) > J0
    assert J0 < riot.quadratic_cost(p, traj, d, v, 0 * dv)


def test_posterior_covariance_full_rank():
    n = 14
    p = _problem_from(n, 6, 1.5, _sigma_vec(n), [1, 3, 6], np.arange(0, n, 2), sigma_o=0.8)
    traj = riot.trajectory(p, p.x_b)
    Om = configs.l96_small().sketch(0, k=n, n=n).T
    lam, U, _ = riot.rsvd(p, traj, Om)
    G = riot.tl_matrix(p, traj)            # d obs / d v = H M L
    B = p.L @ p.L.T
    # in state space the observation Jacobian is H M = G L^-1
    HM = np.linalg.solve(p.L.T, G.T).T
    ref = np.linalg.inv(np.linalg.inv(B) + HM.T @ (HM * p.rinv[:, None]))
    Pa = riot.analysis_cov_dense(p.L, lam, U)
    np.testing.assert_allclose(Pa, ref, rtol=0, atol=1e-8 * np.abs(ref).max())
    # both low-rank forms agree at full rank
    LU = p.L @ U
    lra = (LU / (1 + lam)) @ LU.T
    lru = B - (LU * (lam / (1 + lam))) @ LU.T
    np.testing.assert_allclose(lra, lru, atol=1e-10 * np.abs(lra).max())


def test_power_iteration_improves_partial_rank(small):
    cfg, p, traj = small
    A = riot.dense_hessian(p, traj)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (A + A.T)))[::-1]
    Om = cfg.sketch(1, k=12).T
    lam0, _, _ = riot.rsvd(p, traj, Om, q=0)
    lam1, _, _ = riot.rsvd(p, traj, Om, q=1)
    e0 = np.abs(lam0[:4] - ev[:4]) / ev[:4]
    e1 = np.abs(lam1[:4] - ev[:4]) / ev[:4]
    assert e1.max() < e0.max()
    assert e1.max() < 1e-2
    # the exact Rayleigh-Ritz variant returns Ritz values bounded by the spectrum
    lam_rr, _, _ = riot.rsvd(p, traj, Om, q=1, exact_rr=True)
    assert np.all(lam_rr <= ev[:12] * (1 + 1e-10))


def test_outer_loop_reduces_cost_and_matches_gauss_newton(small):
    cfg, p, _ = small
    x, v = p.x_b.copy(), np.zeros(cfg.n)
    xg, vg = x.copy(), v.copy()
    Js = []
    for k in range(cfg.outer):
        st = riot.outer_step(p, x, v, cfg.sketch(k).T, q=cfg.q)
        Js.append(st["J"])
        x, v = st["x_next"], st["v_next"]
        # Gauss-Newton with the exact dense Hessian (Section 3.1 reference curve)
        tg = riot.trajectory(p, xg)
        gg = riot.gradient_b(p, tg, riot.innovation(p, tg)) + vg
        dvg = -np.linalg.solve(np.eye(cfg.n) + riot.dense_hessian(p, tg), gg)
        np.testing.assert_allclose(st["dv"], dvg, atol=1e-8 * np.abs(dvg).max())
        xg, vg = xg + p.L @ dvg, vg + dvg
    Js.append(riot.cost(p, riot.trajectory(p, x), v))
    assert Js[-1] < Js[0]
    assert Js[1] < Js[0]


def test_range_finder_meets_the_gaussian_sketch_bound(small):
    """Halko, Martinsson & Tropp (2011), Eq. (1.9): with a Gaussian sketch of k + p columns,
    ||(I - Q Q^T) A|| <= [1 + 11 sqrt(k + p) sqrt(n)] sigma_{k+1} except with probability
    at most 6 p^-p.  Eight seeded sketches with p = 6 (failure probability 1.3e-4 each)."""
    cfg, prob, traj = small
    A = riot.dense_hessian(prob, traj)
    A = 0.5 * (A + A.T)
    sv = np.sort(np.abs(np.linalg.eigvalsh(A)))[::-1]          # singular values of the PSD A
    k, p = 6, 6
    bound = (1.0 + 11.0 * np.sqrt(k + p) * np.sqrt(prob.n)) * sv[k]
    for s in range(8):
        Om = cfg.sketch(20 + s, k=k + p).T
        _, _, info = riot.rsvd(prob, traj, Om, q=0)
        Q = info["Q"]
        err = np.linalg.norm(A - Q @ (Q.T @ A), 2)
        assert err <= bound
        assert err >= sv[k + p] * (1 - 1e-10)                 # no rank-(k+p) basis does better (Eckart-Young)


def test_range_finder_error_decreases_with_nested_sketches(small):
    """Section 2.2: more samples, smaller error.  With nested sketches the ranges are nested,
    so the projection error cannot grow."""
    cfg, prob, traj = small
    A = riot.dense_hessian(prob, traj)
    Om = cfg.sketch(30, k=24).T
    errs = []
    for k in (4, 8, 12, 16, 20, 24):
        _, _, info = riot.rsvd(prob, traj, Om[:, :k], q=0)
        Q = info["Q"]
        errs.append(np.linalg.norm(A - Q @ (Q.T @ A), 2))
    assert all(b <= a * (1 + 1e-10) for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-2 * errs[0]


def test_rayleigh_ritz_values_interlace(small):
    """K = Q^T A Q (exact_rr): lambda_i(A) >= theta_i >= lambda_{n-k+i}(A) (Cauchy)."""
    cfg, prob, traj = small
    A = riot.dense_hessian(prob, traj)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (A + A.T)))[::-1]
    n = prob.n
    for k in (5, 12, 25):
        theta, _, _ = riot.rsvd(prob, traj, cfg.sketch(40, k=k).T, q=1, exact_rr=True)
        tol = 1e-10 * ev[0]
        assert np.all(theta <= ev[:k] + tol)
        assert np.all(theta >= ev[n - k:] - tol)


def test_quadratic_cost_is_the_taylor_quadratic(small):
    """J~(dv) of Eq. 3 equals J + g^T dv + 1/2 dv^T (I + A) dv exactly (a quadratic), with J
    from the nonlinear cost, g = b + v from the adjoint gradient and A dv from the Hessian
    product: the three are computed by different code (TL residuals, adjoint, both), so a
    sign, a dropped term or a wrong v in any of them breaks the identity."""
    cfg, p, traj = small
    d = riot.innovation(p, traj)
    rng = np.random.default_rng(11)
    v = 0.3 * rng.standard_normal(cfg.n)
    g = riot.gradient_b(p, traj, d) + v
    J = riot.cost(p, traj, v)
    assert riot.quadratic_cost(p, traj, d, v, np.zeros(cfg.n)) == pytest.approx(J, rel=1e-14)
    for s in (1e-3, 0.1, 2.0):
        dv = s * rng.standard_normal(cfg.n)
        want = J + g @ dv + 0.5 * dv @ dv + 0.5 * dv @ riot.hvp(p, traj, dv[:, None])[:, 0]
        assert riot.quadratic_cost(p, traj, d, v, dv) == pytest.approx(want, rel=1e-11, abs=1e-11 * J)
