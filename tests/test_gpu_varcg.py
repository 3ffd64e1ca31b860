"""Algorithm 1 (VarCG, the Lanczos form of conjugate gradients with full
re-orthogonalisation) on the GPU through riot_varcg, against the FP64 oracle's
varcg on the same window and gradient.

Tolerances: both sides run the same m Lanczos steps in FP64 with two
re-orthogonalisation passes, so the Ritz values agree to rounding (1e-9 of the
largest) and the increments to 1e-8 relative; at m = n the Krylov space is the
whole space and the increment is the exact minimiser -(I + A)^-1 g (1e-8).
With FP32 Hessian products (mixed precision, 2e-5 of the column norm on this
window) the Ritz values and the increment agree to 1e-4."""
import numpy as np
import pytest

from oracle import problem, riot as orc
from synth import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _ctx(R, prob, ell, precision=None, kmax=64):
    if precision is None:
        precision = R.RIOT_PREC_FP64
    return R.Context(n=prob.n, T=prob.T, dt=prob.dt, F=prob.F, obs_step=prob.obs_step, obs_idx=prob.obs_idx,
                     obs_y=prob.y, obs_sigma=prob.sigma_o, length=ell, sigma_b=1.0, precision=precision, kmax=kmax)


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def small():
    cfg = configs.l96_small()
    prob = problem.build(cfg)
    return cfg, prob, orc.trajectory(prob, prob.x_b)


def _g(prob, traj, cfg):
    st = orc.outer_step(prob, prob.x_b, np.zeros(cfg.n), cfg.sketch(0).T, q=cfg.q)
    return st["g"]


@pytest.mark.parametrize("m", [8, 25, 40])
def test_varcg_fp64_matches_oracle(gpu_lib, small, m):
    R = gpu_lib
    cfg, prob, traj = small
    ctx = _ctx(R, prob, cfg.ell, kmax=cfg.k)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    g = _g(prob, traj, cfg)
    dv = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    theta, used = R.riot_varcg(ctx.h, m, dv)
    dvr, thr, _ = orc.varcg(prob, traj, g, m)
    assert used == thr.size
    np.testing.assert_allclose(np.sort(theta), np.sort(thr), rtol=0, atol=1e-9 * np.abs(thr).max())
    dvg = dv.cpu().numpy()
    assert np.linalg.norm(dvg - dvr) <= 1e-8 * np.linalg.norm(dvr)
    if m == cfg.n:
        A = orc.dense_hessian(prob, traj)
        exact = -np.linalg.solve(np.eye(cfg.n) + A, g)
        assert np.linalg.norm(dvg - exact) <= 1e-8 * np.linalg.norm(exact)
    ctx.close()


def test_varcg_mixed_precision(gpu_lib, small):
    R = gpu_lib
    cfg, prob, traj = small
    ctx = _ctx(R, prob, cfg.ell, kmax=cfg.k, precision=R.RIOT_PREC_MIXED)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    g = _g(prob, traj, cfg)
    dv = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    theta, used = R.riot_varcg(ctx.h, 10, dv)
    dvr, thr, _ = orc.varcg(prob, traj, g, 10)
    assert used == 10
    np.testing.assert_allclose(np.sort(theta), np.sort(thr), rtol=0, atol=1e-4 * np.abs(thr).max())
    assert np.linalg.norm(dv.cpu().numpy() - dvr) <= 1e-4 * np.linalg.norm(dvr)
    ctx.close()


def test_varcg_arguments_and_state(gpu_lib, small):
    R = gpu_lib
    cfg, prob, _ = small
    ctx = _ctx(R, prob, cfg.ell, kmax=8)
    with pytest.raises(R.RiotError) as e:
        R.riot_varcg(ctx.h, 4)
    assert e.value.status == -6
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    for m in (0, 9):
        with pytest.raises(R.RiotError) as e:
            R.riot_varcg(ctx.h, m)
        assert e.value.status == -1
    R.riot_rsvd(ctx.h, 8, 0, sketch_stream=configs.STREAM_SKETCH0)
    theta, used = R.riot_varcg(ctx.h, 8)
    assert used == 8 and np.all(np.diff(theta) <= 0)
    # the Lanczos basis took the inner-loop workspace: the RSVD increment needs a new riot_rsvd
    with pytest.raises(R.RiotError) as e:
        R.riot_increment(ctx.h)
    assert e.value.status == -6
    ctx.close()
