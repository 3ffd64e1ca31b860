"""The C ABI's own contract on the GPU: timeout reporting, the caller's allocator, and
the inner-loop quadratic cost (Eq. 3) that measures an increment's cost reduction.

Tolerances:
  The quadratic cost is evaluated in FP64 on either precision (one FP64
  tangent-linear integration); against the FP64 oracle it agrees to the
  rounding of the trajectory and the products: 1e-10 relative.
  Cost reduction at full rank (the small window, k = n): the reduction of an
  increment e away from the exact minimiser falls short of the exact one by
  1/2 e^T (I + A) e, which is second order in e.  An FP64 increment (relative
  error ~1e-10) and a mixed one (~1e-4: FP32 products, see the design notes)
  both leave it below 1e-6 of the exact reduction, the bound asked of the
  method against converged CG.
"""
import numpy as np
import pytest

from oracle import advdiff as A
from oracle import problem, riot as orc
from synth import advdiff as S
from synth import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _l96_ctx(R, cfg, prob, precision, kmax, **kw):
    return R.Context(n=prob.n, T=prob.T, dt=prob.dt, F=prob.F, obs_step=prob.obs_step, obs_idx=prob.obs_idx,
                     obs_y=prob.y, obs_sigma=prob.sigma_o, length=cfg.ell, sigma_b=cfg.sigma_b,
                     precision=precision, kmax=kmax, **kw)


def _bc_ctx(R, cfg, prob, precision, kmax):
    m = prob.m
    return R.Context(nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, nblocks=cfg.nblocks, T=cfg.T, dt=cfg.dt, dx=cfg.dx,
                     dy=cfg.dy, dz=cfg.dz, u=m.u, v=m.v, amp=m.amp, kz=m.kz, emis_b=m.Eb,
                     obs_step=prob.obs.step, obs_pos=prob.obs.pos, obs_y=prob.y, obs_sigma=prob.sigma_o,
                     length=cfg.ell, sigma_b=cfg.sigma_b, precision=precision, kmax=kmax)


@pytest.fixture(scope="module")
def small():
    cfg = configs.l96_small()
    prob = problem.build(cfg)
    return cfg, prob, orc.trajectory(prob, prob.x_b)


def test_forced_wait_timeout_is_reported_and_the_context_recovers(gpu_lib, small):
    """A wait bound of 0 polls makes every block of the Hessian kernel give up on its first
    stage copy: the call must return RIOT_ETIMEOUT (the kernel still waits for the copies
    it started before its blocks exit), and after the default bound is restored the same
    context must give the right products and a clean inner loop."""
    R = gpu_lib
    cfg, prob, traj = small
    ctx = _l96_ctx(R, cfg, prob, R.RIOT_PREC_MIXED, kmax=cfg.k)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    W = cfg.sketch(1, k=8).astype(np.float32)
    Wt = _t(W, torch.float32)
    Y = torch.empty_like(Wt)
    R.riot_set_wait_limit(ctx.h, 0)
    for fn in (R.riot_hessian_apply, R.riot_hessian_apply_noalloc):
        with pytest.raises(R.RiotError) as e:
            fn(ctx.h, Wt, Y)
        assert e.value.status == -5 and "bounded device wait" in str(e.value)
    R.riot_set_wait_limit(ctx.h, -1)
    R.riot_hessian_apply(ctx.h, Wt, Y)
    ref = orc.hvp(prob, traj, W.astype(np.float64).T).T
    got = Y.double().cpu().numpy()
    assert (np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < 2e-5
    lam = R.riot_rsvd(ctx.h, cfg.k, cfg.q, Omega=_t(cfg.sketch(0), torch.float32))
    assert np.all(np.isfinite(lam))
    ctx.close()


def test_workspace_comes_from_the_torch_caching_allocator(gpu_lib, small):
    """With the binding's default allocator callback the context's workspace is memory of
    PyTorch's caching allocator (and goes back to it); without it the library allocates
    with cudaMalloc and torch sees nothing."""
    import gc
    R = gpu_lib
    cfg, prob, _ = small
    gc.collect()   # tensors of earlier tests must not be freed inside the measurement
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    ctx = _l96_ctx(R, cfg, prob, R.RIOT_PREC_FP64, kmax=cfg.k)
    held = torch.cuda.memory_allocated() - base
    # at least the k-column blocks W, Y, Q, U of the context (4 n k doubles)
    assert held >= 4 * cfg.n * cfg.k * 8
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    R.riot_rsvd(ctx.h, cfg.k, cfg.q, Omega=_t(cfg.sketch(0)))
    ctx.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    ctx = _l96_ctx(R, cfg, prob, R.RIOT_PREC_FP64, kmax=cfg.k, torch_allocator=False)
    assert torch.cuda.memory_allocated() == base
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quadratic_cost_l96(gpu_lib, small, precision):
    R = gpu_lib
    cfg, prob, traj = small
    prec = R.RIOT_PREC_FP64 if precision == "fp64" else R.RIOT_PREC_MIXED
    ctx = _l96_ctx(R, cfg, prob, prec, kmax=cfg.k)
    rng = np.random.default_rng(21)
    v = 0.3 * rng.standard_normal(cfg.n)
    J = R.riot_outer_begin(ctx.h, _t(prob.x_b), _t(v))
    d = orc.innovation(prob, traj)
    assert R.riot_quadratic_cost(ctx.h) == pytest.approx(J, rel=1e-12)
    for s in (1e-2, 1.0):
        dv = s * rng.standard_normal(cfg.n)
        want = orc.quadratic_cost(prob, traj, d, v, dv)
        assert R.riot_quadratic_cost(ctx.h, _t(dv)) == pytest.approx(want, rel=1e-10)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quadratic_cost_tracer(gpu_lib, precision):
    R = gpu_lib
    cfg = S.bc_tiny()
    prob = A.build(cfg)
    prec = R.RIOT_PREC_FP64 if precision == "fp64" else R.RIOT_PREC_MIXED
    ctx = _bc_ctx(R, cfg, prob, prec, kmax=8)
    rng = np.random.default_rng(22)
    v = 0.2 * rng.standard_normal(prob.n)
    J = R.riot_outer_begin(ctx.h, _t(prob.x_b), _t(v))
    traj = A.trajectory(prob, prob.x_b)
    d = A.innovation(prob, traj)
    assert R.riot_quadratic_cost(ctx.h) == pytest.approx(J, rel=1e-12)
    dv = 0.1 * rng.standard_normal(prob.n)
    assert R.riot_quadratic_cost(ctx.h, _t(dv)) == pytest.approx(A.quadratic_cost(prob, traj, d, v, dv), rel=1e-10)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_rank_cost_reduction_matches_converged_cg(gpu_lib, small, precision):
    """The small window at full rank (k = n): the cost reduction J~(0) - J~(dv) of the
    library's increment is within 1e-6 of the converged-CG reduction (CG on (I + A) dv = -g
    to a relative residual of 1e-13, the oracle)."""
    R = gpu_lib
    cfg, prob, traj = small
    prec = R.RIOT_PREC_FP64 if precision == "fp64" else R.RIOT_PREC_MIXED
    dt = torch.float64 if precision == "fp64" else torch.float32
    ctx = _l96_ctx(R, cfg, prob, prec, kmax=cfg.k)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    R.riot_rsvd(ctx.h, cfg.k, cfg.q, Omega=_t(cfg.sketch(0), dt))
    dv = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    R.riot_increment(ctx.h, dv)
    red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    d = orc.innovation(prob, traj)
    g = orc.gradient_b(prob, traj, d)
    v = np.zeros(cfg.n)
    dvs = orc.converged_increment(prob, traj, g)
    red_cg = orc.quadratic_cost(prob, traj, d, v, v) - orc.quadratic_cost(prob, traj, d, v, dvs)
    assert red_cg > 0
    assert abs(red - red_cg) <= 1e-6 * red_cg, (red, red_cg)
    ctx.close()


def test_deflated_full_rank_cost_reduction_matches_converged_cg(gpu_lib, small):
    """The deflated eigendecomposition on the small window (level 0 at full rank, k = n = 40):
    level 0 keeps every eigenvalue down to 2^-24 lambda_1 = 1.7e-4, so the deflated operator's
    largest eigenvalue is below 1 and level 1 adds nothing; the increment (LRU, the dropped
    directions taken at lambda = 0) has its cost reduction within 1e-6 of converged CG."""
    R = gpu_lib
    cfg, prob, traj = small
    ctx = _l96_ctx(R, cfg, prob, R.RIOT_PREC_MIXED, kmax=2 * cfg.k)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    lam = R.riot_rsvd_deflated(ctx.h, [cfg.k, cfg.k], 0, sketch_stream=3)
    lam_o = np.linalg.eigvalsh(orc.dense_hessian(prob, traj))[::-1]
    assert lam.size == int(np.sum(lam_o >= 2.0 ** -24 * lam_o[0])) or abs(lam.size - np.sum(lam_o >= 2.0 ** -24 * lam_o[0])) <= 2
    assert lam[-1] > 2.0 ** -24 * lam[0] * 0.5
    dv = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    R.riot_increment(ctx.h, dv)
    red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    d = orc.innovation(prob, traj)
    g = orc.gradient_b(prob, traj, d)
    v = np.zeros(cfg.n)
    dvs = orc.converged_increment(prob, traj, g)
    red_cg = orc.quadratic_cost(prob, traj, d, v, v) - orc.quadratic_cost(prob, traj, d, v, dvs)
    assert abs(red - red_cg) <= 1e-6 * red_cg, (red, red_cg)
    ctx.close()
