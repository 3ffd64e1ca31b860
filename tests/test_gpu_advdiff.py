"""GPU parity of the tracer-transport inversion against the FP64 oracle (through the C ABI).

Tolerances:
  FP64 library vs FP64 oracle: same operations in a different order (the
  library forms five upwind coefficients per column and the transposed ones
  for the adjoint, the oracle forms face fluxes and their reverse mode), so
  results agree to rounding: 1e-11 relative for forecasts and observations,
  1e-10 for Hessian products and gradients, 1e-8 for eigenvalues.
  FP32 Hessian products: the transport is linear and stable (RK4 inside its
  stability region, upwinding dissipative), so the error of a column stays a
  small multiple of 2^-24 per step; 2e-5 of the column norm is required.
"""
import numpy as np
import pytest

from oracle import advdiff as A
from oracle import riot as orc
from synth import advdiff as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _ctx(R, cfg, prob, precision, kmax=64, y=None, sigma=None):
    m = prob.m
    return R.Context(nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, nblocks=cfg.nblocks, T=cfg.T, dt=cfg.dt, dx=cfg.dx,
                     dy=cfg.dy, dz=cfg.dz, u=m.u, v=m.v, amp=m.amp, kz=m.kz, emis_b=m.Eb,
                     obs_step=prob.obs.step, obs_pos=prob.obs.pos,
                     obs_y=prob.y if y is None else y, obs_sigma=prob.sigma_o if sigma is None else sigma,
                     length=cfg.ell, sigma_b=cfg.sigma_b, precision=precision, kmax=kmax)


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _cfg(name):
    if name == "small":
        return S.bc_small()
    if name == "tiny":
        return S.bc_tiny()
    if name == "ragged":   # two x tiles with a ragged second one, y not a multiple of the tile, nz > 8
        return S.AdvDiffConfig(name="ragged", nx=45, ny=7, nz=12, T=10, nblocks=3, n_hotspots=4, n_tracks=3,
                               pts_per_track=40, k=16, q=1, alt_lo=100.0, alt_hi=1200.0)
    if name == "deep":     # the 30-level column of the full grid on a small area
        return S.AdvDiffConfig(name="deep", nx=20, ny=9, nz=30, T=8, nblocks=2, n_hotspots=3, n_tracks=3,
                               pts_per_track=30, k=16, q=0, alt_lo=100.0, alt_hi=1500.0)
    raise KeyError(name)


@pytest.fixture(scope="module", params=["small", "tiny", "ragged", "deep"])
def case(request):
    cfg = _cfg(request.param)
    prob = A.build(cfg)
    return cfg, prob


def test_observations_of_a_forecast(gpu_lib, case):
    # with y = 0 and sigma = 1 the innovation is H(x) and J = 1/2 |H(x)|^2
    R = gpu_lib
    cfg, prob = case
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_FP64, kmax=4, y=np.zeros(prob.p), sigma=np.ones(prob.p))
    x = 0.3 * np.random.default_rng(1).standard_normal(prob.n)
    J = R.riot_outer_begin(ctx.h, _t(x))
    d = torch.empty(prob.p, dtype=torch.float64, device=DEV)
    R.riot_get_innovation(ctx.h, d)
    ref = A.trajectory(prob, x)["Hx"]
    np.testing.assert_allclose(d.cpu().numpy(), ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    assert J == pytest.approx(0.5 * float(ref @ ref), rel=1e-11)
    ctx.close()


def test_cost_and_gradient(gpu_lib, case):
    R = gpu_lib
    cfg, prob = case
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_FP64, kmax=4)
    rng = np.random.default_rng(2)
    x = prob.x_b + 0.1 * rng.standard_normal(prob.n)
    v = 0.2 * rng.standard_normal(prob.n)
    J = R.riot_outer_begin(ctx.h, _t(x), _t(v))
    g = torch.empty(prob.n, dtype=torch.float64, device=DEV)
    R.riot_get_state(ctx.h, g=g)
    traj = A.trajectory(prob, x)
    want = A.gradient_b(prob, traj, A.innovation(prob, traj)) + v
    np.testing.assert_allclose(g.cpu().numpy(), want, rtol=1e-10, atol=1e-10 * np.abs(want).max())
    assert J == pytest.approx(A.cost(prob, traj, v), rel=1e-11)
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_hessian_products(gpu_lib, case, precision, tol):
    R = gpu_lib
    cfg, prob = case
    prec = R.RIOT_PREC_FP64 if precision == "fp64" else R.RIOT_PREC_MIXED
    dt = torch.float64 if precision == "fp64" else torch.float32
    ncols = 9
    ctx = _ctx(R, cfg, prob, prec, kmax=4)     # more columns than kmax: sliced batches
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    W = np.random.default_rng(3).standard_normal((ncols, prob.n))
    if dt == torch.float32:
        W = W.astype(np.float32).astype(np.float64)
    Wt = _t(W, dt)
    Y = torch.empty_like(Wt)
    R.riot_hessian_apply(ctx.h, Wt, Y)
    traj = A.trajectory(prob, prob.x_b)
    ref = A.hvp(prob, traj, W.T).T
    got = Y.double().cpu().numpy()
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= tol, err
    Y2 = torch.empty_like(Wt)
    R.riot_hessian_apply(ctx.h, Wt, Y2, add_identity=True)
    got2 = Y2.double().cpu().numpy()
    err2 = np.linalg.norm(got2 - ref - W, axis=1) / np.linalg.norm(ref + W, axis=1)
    assert err2.max() <= tol
    ctx.close()


def test_prior_square_root(gpu_lib):
    R = gpu_lib
    cfg = _cfg("ragged")
    prob = A.build(cfg)
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_FP64, kmax=4)
    W = np.random.default_rng(4).standard_normal((5, prob.n))
    out = torch.empty(5, prob.n, dtype=torch.float64, device=DEV)
    R.riot_bsqrt_apply(ctx.h, _t(W), out, ncols=5)
    np.testing.assert_allclose(out.cpu().numpy(), prob.Lop.apply(W), rtol=1e-11, atol=1e-12)
    R.riot_bsqrt_apply(ctx.h, _t(W), out, transpose=True, ncols=5)
    np.testing.assert_allclose(out.cpu().numpy(), prob.Lop.apply_t(W), rtol=1e-11, atol=1e-12)
    ctx.close()


@pytest.mark.parametrize("which,k,q", [("tiny", 20, 0), ("small", 32, 1)])
def test_rsvd_increment_and_covariance_fp64(gpu_lib, which, k, q):
    R = gpu_lib
    cfg = _cfg(which)
    prob = A.build(cfg)
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_FP64, kmax=k)
    x = prob.x_b.copy()
    R.riot_outer_begin(ctx.h, _t(x))
    Om = cfg.sketch(0, k=k)
    lam = R.riot_rsvd(ctx.h, k, q, Omega=_t(Om))
    dv = torch.empty(prob.n, dtype=torch.float64, device=DEV)
    mode = R.riot_increment(ctx.h, dv)
    res = A.outer_step(prob, x, np.zeros(prob.n), Om.T, q=q)
    np.testing.assert_allclose(lam, res["lam"], rtol=1e-8, atol=1e-9 * res["lam"][0])
    assert mode == res["mode"]
    np.testing.assert_allclose(dv.cpu().numpy(), res["dv"], rtol=1e-7, atol=1e-8 * np.abs(res["dv"]).max())
    xs = torch.empty(prob.n, dtype=torch.float64, device=DEV)
    R.riot_get_state(ctx.h, x=xs)
    np.testing.assert_allclose(xs.cpu().numpy(), res["x_next"], rtol=1e-9, atol=1e-9)
    m = k // 2
    LU = torch.empty(m, prob.n, dtype=torch.float64, device=DEV)
    coef, cmode = R.riot_analysis_cov_lowrank(ctx.h, m, LU)
    LUo, coefo, modeo = orc.analysis_cov_lowrank(prob.L, res["lam"][:m], res["U"][:, :m])
    assert cmode == modeo
    np.testing.assert_allclose(coef, coefo, rtol=1e-8)
    # columns are determined up to sign; compare the covariance they build
    Pg = (LU.cpu().numpy().T * coef) @ LU.cpu().numpy()
    Po = (LUo * coefo) @ LUo.T
    np.testing.assert_allclose(Pg, Po, atol=1e-7 * np.abs(Po).max())
    ctx.close()


def test_rsvd_mixed_leading_eigenvalues(gpu_lib):
    R = gpu_lib
    cfg = _cfg("small")
    prob = A.build(cfg)
    k, q = 32, 1
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_MIXED, kmax=k)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    Om = cfg.sketch(0, k=k)
    lam = R.riot_rsvd(ctx.h, k, q, Omega=_t(Om, torch.float32))
    res = A.outer_step(prob, prob.x_b, np.zeros(prob.n), Om.astype(np.float32).astype(np.float64).T, q=q)
    lead = res["lam"] > 1e-3 * res["lam"][0]
    np.testing.assert_allclose(lam[lead], res["lam"][lead], rtol=1e-3)
    ctx.close()


def test_rsvd_mixed_increment_and_cost_reduction(gpu_lib):
    """The mixed tracer inner loop (16 x 12 x 6 box, k = 32, q = 1) against the FP64 oracle on
    the FP32-rounded sketch.  Every retained eigenvalue is above the FP32 floor here, so both
    sides use all 32 pairs.  FP32 products carry an error of at most eps = 16 sqrt(8T) 2^-24
    of A's scale (the product bound of these tests, 1.3e-5 at T = 24), so the eigenpairs, the
    adaptive weights and the increment move by at most about eps lambda_1 relative; the cost
    reduction, second order in the increment's error, is held to 1e-4."""
    R = gpu_lib
    cfg = _cfg("small")
    prob = A.build(cfg)
    k, q = 32, 1
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_MIXED, kmax=k)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    Om = cfg.sketch(0, k=k)
    lam = R.riot_rsvd(ctx.h, k, q, Omega=_t(Om, torch.float32))
    dv = torch.empty(prob.n, dtype=torch.float64, device=DEV)
    mode = R.riot_increment(ctx.h, dv)
    assert R.riot_increment_pairs(ctx.h) == k
    red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    res = A.outer_step(prob, prob.x_b, np.zeros(prob.n), Om.astype(np.float32).astype(np.float64).T, q=q)
    eps = 16 * np.sqrt(8 * cfg.T) * 2.0 ** -24
    assert mode == res["mode"]
    dvo = res["dv"]
    err = np.linalg.norm(dv.cpu().numpy() - dvo) / np.linalg.norm(dvo)
    assert err <= eps * res["lam"][0], (err, eps * res["lam"][0])
    z = np.zeros(prob.n)
    d = A.innovation(prob, res["traj"])
    red_o = A.quadratic_cost(prob, res["traj"], d, z, z) - A.quadratic_cost(prob, res["traj"], d, z, dvo)
    assert red_o > 0 and abs(red - red_o) <= 1e-4 * red_o, (red, red_o)
    ctx.close()


def test_full_grid_properties(gpu_lib):
    """The 192 x 192 x 30 grid of the benchmark workload (shortened window):
    FP64 observations against the oracle, and symmetry of the FP32 Hessian
    in the launch configuration the benchmark times."""
    R = gpu_lib
    full = S.bc_large()
    cfg = S.AdvDiffConfig(name="full_grid_T24", T=24, nblocks=4, k=8, q=0, alt_lo=100.0, alt_hi=1500.0)
    prob = A.build(cfg)
    assert prob.m.nx == full.nx and prob.m.ny == full.ny and prob.m.nz == full.nz
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_FP64, kmax=2, y=np.zeros(prob.p), sigma=np.ones(prob.p))
    x = 0.2 * np.random.default_rng(5).standard_normal(prob.n)
    R.riot_outer_begin(ctx.h, _t(x))
    d = torch.empty(prob.p, dtype=torch.float64, device=DEV)
    R.riot_get_innovation(ctx.h, d)
    ref = A.trajectory(prob, x)["Hx"]
    np.testing.assert_allclose(d.cpu().numpy(), ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    ctx.close()
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_MIXED, kmax=128, sigma=np.ones(prob.p))
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    W = torch.tensor(np.random.default_rng(6).standard_normal((2, prob.n)), dtype=torch.float32, device=DEV)
    Y = torch.empty_like(W)
    R.riot_hessian_apply(ctx.h, W, Y)
    a = float((W[0].double() @ Y[1].double()).item())
    b = float((W[1].double() @ Y[0].double()).item())
    assert abs(a - b) <= 1e-4 * max(abs(a), abs(b))
    assert float((W[0].double() @ Y[0].double()).item()) > 0
    ctx.close()


def test_bad_descriptors_are_rejected(gpu_lib):
    R = gpu_lib
    cfg, prob = _cfg("tiny"), None
    prob = A.build(cfg)
    bad_pos = prob.obs.pos.copy()
    bad_pos[0, 1] = cfg.ny   # beyond the last row centre
    with pytest.raises(R.RiotError) as e:
        R.riot_setup_advdiff(nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, nblocks=cfg.nblocks, T=cfg.T, dt=cfg.dt, dx=cfg.dx,
                             dy=cfg.dy, dz=cfg.dz, u=prob.m.u, v=prob.m.v, amp=prob.m.amp, kz=prob.m.kz,
                             emis_b=prob.m.Eb, obs_step=prob.obs.step, obs_pos=bad_pos, obs_y=prob.y,
                             obs_sigma=prob.sigma_o, length=cfg.ell, sigma_b=cfg.sigma_b)
    assert e.value.status == -1
    v_bad = prob.m.v.copy()
    v_bad[0, 0] = 1.0        # flow through a wall
    with pytest.raises(R.RiotError):
        R.riot_setup_advdiff(nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, nblocks=cfg.nblocks, T=cfg.T, dt=cfg.dt, dx=cfg.dx,
                             dy=cfg.dy, dz=cfg.dz, u=prob.m.u, v=v_bad, amp=prob.m.amp, kz=prob.m.kz,
                             emis_b=prob.m.Eb, obs_step=prob.obs.step, obs_pos=prob.obs.pos, obs_y=prob.y,
                             obs_sigma=prob.sigma_o, length=cfg.ell, sigma_b=cfg.sigma_b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_grid_products_against_the_oracle(gpu_lib, precision):
    """Two Hessian-vector products on the full 192 x 192 x 30 grid (240 steps, 8000 observations,
    n = 147 456) against the FP64 oracle's, sampled at 512 seeded positions per column
    (tests/golden/bc_large_products.json, written by the oracle alone; unit sigma_o).  FP64: the
    operations differ only in order, 1e-10 of the column norm as on the small grids.  FP32: the
    transport is linear and dissipative, so rounding errors add like a random walk over the 8T
    stages of the forward and backward passes: 16 sqrt(8T) 2^-24 = 4.2e-5 (the same derivation as
    the Lorenz-96 products, without a trajectory term)."""
    import json
    import os
    R = gpu_lib
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bc_large_products.json")) as f:
        gold = json.load(f)
    cfg = S.bc_large()
    m = A.model_from_config(cfg)
    step, pos = cfg.tracks()
    obs = A.make_obs(m, step, pos)
    p = step.size
    Lop = A.exp_separable_sqrt(cfg.nx, cfg.ny, cfg.nblocks, cfg.dx, cfg.dy, cfg.ell, cfg.sigma_b)
    x_b = Lop.apply(cfg.background_perturbation())
    prec = R.RIOT_PREC_FP64 if precision == "fp64" else R.RIOT_PREC_MIXED
    ctx = R.Context(nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, nblocks=cfg.nblocks, T=cfg.T, dt=cfg.dt, dx=cfg.dx,
                    dy=cfg.dy, dz=cfg.dz, u=m.u, v=m.v, amp=m.amp, kz=m.kz, emis_b=m.Eb, obs_step=obs.step,
                    obs_pos=obs.pos, obs_y=np.zeros(p), obs_sigma=np.ones(p), length=cfg.ell,
                    sigma_b=cfg.sigma_b, precision=prec, kmax=2)
    assert gold["n"] == ctx.n and gold["p"] == p
    R.riot_outer_begin(ctx.h, _t(x_b))
    cols = gold["columns"]
    W = cfg.sketch(0, k=cols)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Wt = _t(W, dt)
    Y = torch.empty_like(Wt)
    R.riot_hessian_apply(ctx.h, Wt, Y)
    got = Y.double().cpu().numpy()
    idx = np.asarray(gold["sample_index"])
    vals = gold["values"] if precision == "fp64" else gold["values_f32_input"]
    norms = gold["norm"] if precision == "fp64" else gold["norm_f32_input"]
    tol = 1e-10 if precision == "fp64" else 16 * np.sqrt(8 * cfg.T) * 2.0 ** -24
    for j in range(cols):
        ref = np.asarray(vals[j])
        assert np.linalg.norm(got[j, idx] - ref) <= tol * np.linalg.norm(ref), (j, np.linalg.norm(got[j, idx] - ref) / np.linalg.norm(ref))
        assert abs(np.linalg.norm(got[j]) - norms[j]) <= tol * norms[j]
    ctx.close()
