"""Pins of the FP64 tracer-transport oracle (black-carbon-style inversion).

Each test checks the oracle against something other than itself: exact
conservation laws of the flux form, closed forms of special cases (constant
wind upwinding, the Neumann diffusion spectrum, RK4 on an eigenmode),
dot-product identities, Taylor expansions, finite differences and the exact
solve of the quadratic inner problem.
"""
import numpy as np
import pytest

from oracle import advdiff as A
from oracle import riot
from synth import advdiff as S


@pytest.fixture(scope="module")
def tiny():
    cfg = S.bc_tiny()
    prob = A.build(cfg)
    return cfg, prob


def _model(nx=10, ny=7, nz=5, u=None, v=None, kz=None, amp=None, T=6, nb=2):
    return A.AdvDiffModel(nx=nx, ny=ny, nz=nz, nb=nb, T=T, dt=400.0, dx=12000.0, dy=12000.0, dz=250.0,
                          u=np.zeros((ny, nx)) if u is None else u,
                          v=np.zeros((ny + 1, nx)) if v is None else v,
                          amp=np.ones(nz) if amp is None else amp,
                          kz=np.zeros(nz + 1) if kz is None else kz,
                          Eb=np.ones((nb, ny, nx)))


def test_flux_form_conserves_mass(tiny):
    _, prob = tiny
    m = prob.m
    rng = np.random.default_rng(1)
    c = rng.random((3, m.nz, m.ny, m.nx))
    tend = A.tendency(m, c)
    scale = np.abs(tend).sum()
    assert np.all(np.abs(tend.sum(axis=(1, 2, 3))) <= 1e-13 * scale)
    # T steps with a constant surface source add exactly T h sum(s)
    s = rng.random((m.ny, m.nx))
    c = np.zeros((m.nz, m.ny, m.nx))
    for _ in range(m.T):
        c = A.rk4_step(m, c, s)
    want = m.T * m.dt * s.sum()
    assert abs(c.sum() - want) <= 1e-12 * want


def test_uniform_field_stays_uniform(tiny):
    # the face winds come from a stream function: discrete divergence zero
    _, prob = tiny
    m = prob.m
    t = A.tendency(m, np.ones((m.nz, m.ny, m.nx)))
    assert np.abs(t).max() <= 1e-12 * 15.0 / m.dx


@pytest.mark.parametrize("u0", [7.5, -7.5])
def test_constant_wind_is_textbook_upwind(u0):
    nx, ny, nz = 9, 3, 2
    m = _model(nx=nx, ny=ny, nz=nz, u=np.full((ny, nx), u0))
    c = np.random.default_rng(2).random((nz, ny, nx))
    if u0 > 0:
        want = -u0 * (c - np.roll(c, 1, axis=-1)) / m.dx
    else:
        want = -u0 * (np.roll(c, -1, axis=-1) - c) / m.dx
    np.testing.assert_allclose(A.tendency(m, c), want, rtol=1e-14, atol=1e-20)


def _column_operator(m):
    ncell = m.nz * m.ny * m.nx
    E = np.eye(ncell).reshape(ncell, m.nz, m.ny, m.nx)
    return A.tendency(m, E).reshape(ncell, ncell).T


def test_vertical_diffusion_has_the_neumann_spectrum():
    nz, K = 8, 15.0
    kz = np.full(nz + 1, K)
    m = _model(nx=1, ny=1, nz=nz, kz=kz)
    Aop = _column_operator(m)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (Aop + Aop.T)))
    mm = np.arange(nz)
    want = np.sort(-4.0 * K / m.dz ** 2 * np.sin(np.pi * mm / (2 * nz)) ** 2)
    np.testing.assert_allclose(ev, want, rtol=1e-12, atol=1e-16)


def test_rk4_step_on_an_eigenmode_is_the_stability_polynomial():
    nz, K = 8, 15.0
    m = _model(nx=1, ny=1, nz=nz, kz=np.full(nz + 1, K))
    mode = 3
    l = np.arange(nz)
    phi = np.cos(np.pi * mode * (l + 0.5) / nz).reshape(nz, 1, 1)
    mu = -4.0 * K / m.dz ** 2 * np.sin(np.pi * mode / (2 * nz)) ** 2
    z = m.dt * mu
    P = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    np.testing.assert_allclose(A.rk4_step(m, phi), P * phi, rtol=1e-13, atol=1e-15)


def test_adjoint_dot_products(tiny):
    _, prob = tiny
    m = prob.m
    rng = np.random.default_rng(3)
    c = rng.standard_normal((m.nz, m.ny, m.nx))
    g = rng.standard_normal((m.nz, m.ny, m.nx))
    lhs, rhs = np.sum(A.tendency(m, c) * g), np.sum(c * A.tendency_adj(m, g))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    s = rng.standard_normal((m.ny, m.nx))
    lam = rng.standard_normal((m.nz, m.ny, m.nx))
    cb, sb = A.rk4_step_adj(m, lam)
    lhs = np.sum(A.rk4_step(m, c, s) * lam)
    rhs = np.sum(c * cb) + np.sum(s * sb)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    src = rng.standard_normal((m.nb, m.ny, m.nx))
    r = rng.standard_normal(prob.p)
    lhs = np.dot(A.run(m, prob.obs, src), r)
    rhs = np.sum(src * A.run_adj(m, prob.obs, r))
    assert abs(lhs - rhs) <= 1e-12 * np.abs(A.run(m, prob.obs, src)).sum() * np.abs(r).max()


def test_trilinear_interpolation():
    m = _model(nx=6, ny=5, nz=4)
    # grid points pick a single cell
    pos = np.array([[2.0, 3.0, 1.0], [5.0, 0.0, 0.0], [0.0, 4.0, 3.0]])
    cells, w = A.trilinear(m, pos)
    for q in range(3):
        i, j, l = pos[q].astype(int)
        k = np.argmax(w[q])
        assert w[q, k] == pytest.approx(1.0) and cells[q, k] == (l * m.ny + j) * m.nx + i
    # linear in y and z, periodic-linear in x away from the seam: reproduced exactly
    rng = np.random.default_rng(4)
    pos = np.stack([rng.uniform(0, m.nx - 1, 50), rng.uniform(0, m.ny - 1, 50), rng.uniform(0, m.nz - 1, 50)], 1)
    l, j, i = np.meshgrid(np.arange(m.nz), np.arange(m.ny), np.arange(m.nx), indexing="ij")
    field = 0.5 + 0.3 * i + 0.2 * j - 0.7 * l
    obs = A.make_obs(m, np.ones(50, dtype=int), pos)
    _, val = A.observe(m, obs, field, 1)
    np.testing.assert_allclose(val, 0.5 + 0.3 * pos[:, 0] + 0.2 * pos[:, 1] - 0.7 * pos[:, 2], rtol=1e-13)
    np.testing.assert_allclose(obs.w.sum(axis=1), 1.0, rtol=1e-15)
    # across the periodic seam the weights join cell nx-1 and cell 0
    cells, w = A.trilinear(m, np.array([[m.nx - 0.25, 1.0, 1.0]]))
    nz_cells = sorted(set(cells[0][w[0] > 0] % m.nx))
    assert nz_cells == [0, m.nx - 1]


def test_prior_square_root_reproduces_the_exponential_correlation():
    cfg = S.bc_tiny()
    Lop = A.exp_separable_sqrt(cfg.nx, cfg.ny, cfg.nblocks, cfg.dx, cfg.dy, cfg.ell, cfg.sigma_b)
    L = Lop.dense()
    B = L @ L.T
    ix = np.arange(cfg.nx)
    dxp = np.abs(ix[:, None] - ix[None, :])
    dxp = np.minimum(dxp, cfg.nx - dxp) * cfg.dx
    iy = np.arange(cfg.ny)
    dyp = np.abs(iy[:, None] - iy[None, :]) * cfg.dy
    C1 = np.kron(np.exp(-dyp / cfg.ell), np.exp(-dxp / cfg.ell))
    want = cfg.sigma_b ** 2 * np.kron(np.eye(cfg.nblocks), C1)
    np.testing.assert_allclose(B, want, atol=1e-13)
    w = np.random.default_rng(5).standard_normal((3, L.shape[0]))
    np.testing.assert_allclose(Lop.apply(w), w @ L.T, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Lop.apply_t(w), w @ L, rtol=1e-12, atol=1e-14)


def test_taylor_expansion_of_the_observed_emission_response(tiny):
    _, prob = tiny
    rng = np.random.default_rng(6)
    x = 0.3 * rng.standard_normal(prob.n)
    dx = rng.standard_normal(prob.n)
    traj = A.trajectory(prob, x)
    H0 = traj["Hx"]
    lin = A.tl_obs(prob, traj, dx)[0]
    errs = []
    for eps in (1e-2, 1e-3, 1e-4):
        H1 = A.trajectory(prob, x + eps * dx)["Hx"]
        errs.append(np.linalg.norm(H1 - H0 - eps * lin) / np.linalg.norm(eps * lin))
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.2 * errs[1] and errs[2] < 1e-3


def test_gradient_matches_finite_differences(tiny):
    _, prob = tiny
    rng = np.random.default_rng(7)
    v = 0.2 * rng.standard_normal(prob.n)

    def J(vv):
        x = prob.x_b + prob.Lop.apply(vv)
        return A.cost(prob, A.trajectory(prob, x), vv)

    x = prob.x_b + prob.Lop.apply(v)
    traj = A.trajectory(prob, x)
    g = A.gradient_b(prob, traj, A.innovation(prob, traj)) + v
    for j in rng.choice(prob.n, 6, replace=False):
        e = np.zeros(prob.n)
        e[j] = 1e-5
        fd = (J(v + e) - J(v - e)) / 2e-5
        assert fd == pytest.approx(g[j], rel=1e-6, abs=1e-8 * np.abs(g).max())


def test_hessian_is_symmetric_psd_and_equals_the_gauss_newton_product(tiny):
    _, prob = tiny
    traj = A.trajectory(prob, prob.x_b)
    H = A.hvp(prob, traj, np.eye(prob.n))
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
    assert np.linalg.eigvalsh(H).min() >= -1e-12 * np.abs(H).max()
    # A = G^T R^-1 G with G the Jacobian of the observations w.r.t. v
    G = A.tl_obs(prob, traj, prob.Lop.apply(np.eye(prob.n))).T     # (p, n)
    np.testing.assert_allclose(H, G.T @ (G * prob.rinv[:, None]), rtol=1e-10, atol=1e-12 * np.abs(H).max())


def test_full_rank_riot_increment_is_the_exact_inner_solution(tiny):
    cfg, prob = tiny
    x, v = prob.x_b.copy(), np.zeros(prob.n)
    res = A.outer_step(prob, x, v, cfg.sketch(0, k=prob.n).T, q=0)
    traj = res["traj"]
    dv_exact = -riot.cg_solve(lambda p: p + A.hvp(prob, traj, p[:, None])[:, 0], res["g"], tol=1e-14)
    assert res["mode"] == 1           # rank-deficient Hessian: the smallest Ritz value is < 1
    np.testing.assert_allclose(res["dv"], dv_exact, rtol=1e-8, atol=1e-10 * np.abs(dv_exact).max())


def test_quadratic_cost_is_the_taylor_quadratic(tiny):
    """J~(dv) of Eq. 3 on the tracer problem equals J + g^T dv + 1/2 dv^T (I + A) dv (the
    transport is linear in the emission perturbation, so the quadratic is exact): cost,
    adjoint gradient and Hessian product are independent code paths."""
    _, prob = tiny
    rng = np.random.default_rng(12)
    v = 0.2 * rng.standard_normal(prob.n)
    traj = A.trajectory(prob, prob.x_b)
    d = A.innovation(prob, traj)
    g = A.gradient_b(prob, traj, d) + v
    J = A.cost(prob, traj, v)
    assert A.quadratic_cost(prob, traj, d, v, np.zeros(prob.n)) == pytest.approx(J, rel=1e-14)
    for s in (1e-2, 0.5):
        dv = s * rng.standard_normal(prob.n)
        want = J + g @ dv + 0.5 * dv @ dv + 0.5 * dv @ A.hvp(prob, traj, dv[:, None])[:, 0]
        assert A.quadratic_cost(prob, traj, d, v, dv) == pytest.approx(want, rel=1e-11, abs=1e-11 * J)
