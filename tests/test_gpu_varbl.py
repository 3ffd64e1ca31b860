"""Algorithm 2 (VarBL, block Lanczos from gradient samples) on the GPU through
riot_varbl, against the oracle's gradient_samples + varbl with the same
perturbations.

The samples are formed through the library (one FP64 context per sample, on
observations y - sigma eps_obs_j, riot_outer_begin at x + L eps_b_j, then the
gradient plus eps_b_j); the oracle forms its own.  Tolerances: both sides run
the same block steps in FP64 with two re-orthogonalisation passes, so the Ritz
values agree to rounding (1e-9 of the largest), the increments to 1e-8
relative, and when the block Krylov space fills the space the increment is the
exact minimiser -(I + A)^-1 g (1e-8).  With FP32 Hessian products (mixed
precision, ~2e-5 of a column on this window) to 1e-4."""
import numpy as np
import pytest

from oracle import problem, riot as orc
from synth import configs, philox

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _ctx(R, prob, ell, precision, kmax, y=None):
    return R.Context(n=prob.n, T=prob.T, dt=prob.dt, F=prob.F, obs_step=prob.obs_step, obs_idx=prob.obs_idx,
                     obs_y=prob.y if y is None else y, obs_sigma=prob.sigma_o, length=ell, sigma_b=1.0,
                     precision=precision, kmax=kmax)


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


@pytest.fixture(scope="module")
def small():
    cfg = configs.l96_small()
    prob = problem.build(cfg)
    return cfg, prob, orc.trajectory(prob, prob.x_b)


def _perturbations(prob, l, seed_stream):
    eo = philox.normals(configs.BASE_SEED, seed_stream, prob.p * l).reshape(l, prob.p).T
    eb = philox.normals(configs.BASE_SEED, seed_stream + 1, prob.n * l).reshape(l, prob.n).T.copy()
    eb[:, 0] = 0.0                       # the listing's eps_b_1 = 0
    return eo, eb


def _gpu_samples(R, prob, cfg, eo, eb):
    """b_j through the library: one context per perturbed observation vector."""
    rows = []
    for j in range(eb.shape[1]):
        c = _ctx(R, prob, cfg.ell, R.RIOT_PREC_FP64, 4, y=prob.y - prob.sigma_o * eo[:, j])
        Le = torch.empty(1, prob.n, dtype=torch.float64, device=DEV)
        R.riot_bsqrt_apply(c.h, _t(eb[:, j][None, :]), Le, transpose=False, ncols=1)
        R.riot_outer_begin(c.h, _t(prob.x_b) + Le[0])
        g = torch.empty(prob.n, dtype=torch.float64, device=DEV)
        R.riot_get_state(c.h, g=g)
        rows.append(g + _t(eb[:, j]))
        c.close()
    return torch.stack(rows).contiguous()


def _run(R, prob, cfg, l, m, precision, stream):
    eo, eb = _perturbations(prob, l, stream)
    B0 = _gpu_samples(R, prob, cfg, eo, eb)
    ctx = _ctx(R, prob, cfg.ell, precision, cfg.k)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    dv = torch.empty(prob.n, dtype=torch.float64, device=DEV)
    theta, nb = R.riot_varbl(ctx.h, l, m, B0, dv)
    ctx.close()
    return theta, nb, dv.cpu().numpy(), B0.cpu().numpy().T, eo, eb


def _oracle(prob, traj, l, m, eo, eb):
    g = orc.gradient_b(prob, traj, orc.innovation(prob, traj))
    B0 = orc.gradient_samples(prob, prob.x_b, np.zeros(prob.n), eo, eb)
    dv, lam, _, _, _ = orc.varbl(prob, traj, B0, m, g)
    return dv, lam, g, B0


@pytest.mark.parametrize("l,m", [(4, 5), (2, 8), (1, 6), (8, 3)])
def test_varbl_fp64_matches_oracle(gpu_lib, small, l, m):
    R = gpu_lib
    cfg, prob, traj = small
    theta, nb, dv, B0g, eo, eb = _run(R, prob, cfg, l, m, R.RIOT_PREC_FP64, 60 + 2 * l)
    dvr, lamr, _, B0r = _oracle(prob, traj, l, m, eo, eb)
    np.testing.assert_allclose(B0g, B0r, rtol=0, atol=1e-10 * np.abs(B0r).max())
    assert nb == m and theta.size == lamr.size
    np.testing.assert_allclose(theta, lamr, rtol=0, atol=1e-9 * lamr[0])
    assert np.linalg.norm(dv - dvr) <= 1e-8 * np.linalg.norm(dvr)


def test_varbl_full_space_is_the_minimiser(gpu_lib, small):
    R = gpu_lib
    cfg, prob, traj = small
    l, m = 4, 10
    theta, nb, dv, _, eo, eb = _run(R, prob, cfg, l, m, R.RIOT_PREC_FP64, 70)
    dvr, lamr, g, _ = _oracle(prob, traj, l, m, eo, eb)
    exact = -np.linalg.solve(np.eye(cfg.n) + orc.dense_hessian(prob, traj), g)
    assert np.linalg.norm(dv - exact) <= 1e-8 * np.linalg.norm(exact)
    assert np.linalg.norm(dvr - exact) <= 1e-8 * np.linalg.norm(exact)


def test_varbl_mixed_precision(gpu_lib, small):
    R = gpu_lib
    cfg, prob, traj = small
    l, m = 4, 5
    theta, nb, dv, _, eo, eb = _run(R, prob, cfg, l, m, R.RIOT_PREC_MIXED, 72)
    dvr, lamr, _, _ = _oracle(prob, traj, l, m, eo, eb)
    assert nb == m
    np.testing.assert_allclose(theta, lamr, rtol=0, atol=1e-4 * lamr[0])
    assert np.linalg.norm(dv - dvr) <= 1e-4 * np.linalg.norm(dvr)


def test_varbl_stops_on_an_invariant_space(gpu_lib, small):
    """Four eigenvectors of A as the starting block: one block step spans an
    invariant space, the recurrence stops and the Ritz values are those eigenvalues."""
    R = gpu_lib
    cfg, prob, traj = small
    A = orc.dense_hessian(prob, traj)
    ev, V = np.linalg.eigh(0.5 * (A + A.T))
    B0 = V[:, -4:] @ np.diag([1.0, 2.0, 3.0, 4.0])
    g = orc.gradient_b(prob, traj, orc.innovation(prob, traj))
    dvr, lamr, _, _, _ = orc.varbl(prob, traj, B0, 5, g)
    ctx = _ctx(R, prob, cfg.ell, R.RIOT_PREC_FP64, cfg.k)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    dv = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    theta, nb = R.riot_varbl(ctx.h, 4, 5, _t(B0.T), dv)
    assert nb == 1 and lamr.size == 4
    np.testing.assert_allclose(theta, ev[::-1][:4], rtol=1e-9)
    assert np.linalg.norm(dv.cpu().numpy() - dvr) <= 1e-8 * np.linalg.norm(dvr)
    ctx.close()


def test_varbl_arguments_and_state(gpu_lib, small):
    R = gpu_lib
    cfg, prob, _ = small
    ctx = _ctx(R, prob, cfg.ell, R.RIOT_PREC_FP64, 16)
    B0 = torch.randn(4, cfg.n, dtype=torch.float64, device=DEV)
    with pytest.raises(R.RiotError) as e:
        R.riot_varbl(ctx.h, 4, 2, B0)
    assert e.value.status == -6                       # before riot_outer_begin
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    with pytest.raises(R.RiotError) as e:
        R.riot_varbl(ctx.h, 4, 5, B0)                 # l m = 20 > kmax = 16
    assert e.value.status == -1
    Bd = B0.clone()
    Bd[1] = Bd[0]
    with pytest.raises(R.RiotError) as e:
        R.riot_varbl(ctx.h, 4, 2, Bd)                 # dependent samples
    assert e.value.status == -4
    theta, nb = R.riot_varbl(ctx.h, 4, 4, B0)
    assert nb == 4 and theta.size == 16
    with pytest.raises(R.RiotError) as e:
        R.riot_increment(ctx.h)                       # the workspace now holds the block basis
    assert e.value.status == -6
    R.riot_precond_enable(ctx.h, 1, False)
    e0 = torch.zeros(1, cfg.n, dtype=torch.float64, device=DEV)
    e0[0, 0] = 1.0
    R.riot_precond_push_pairs(ctx.h, e0, [1.0])
    R.riot_outer_begin(ctx.h)
    with pytest.raises(R.RiotError) as e:
        R.riot_varbl(ctx.h, 4, 2, B0)                 # Algorithm 2 takes no preconditioner
    assert e.value.status == -6
    ctx.close()
