"""GPU parity of the large Lorenz-96 window that the benchmark times (n = 4096, F = 8, T = 200
steps of dt = 0.05, 1024 observed variables every 4 steps: p = 51 200, k = 512, q = 1)
against the FP64 oracle run on the same sketch, through the C ABI.

Tolerances (derived, not picked):
  FP32 Hessian products: each RK4 stage rounds every variable a few times
  (gamma = 4 roundings on the longest path: the difference, two FMAs, the stage
  combination); along a tangent-linear or adjoint solution the rounding error
  grows with the solution itself, so relative errors add up over the 8T stages
  of the forward and backward passes like a random walk: sqrt(8T) gamma 2^-24,
  times 4 for safety, i.e. 16 sqrt(8T) 2^-24 = 3.8e-5 at T = 200, plus the
  FP64 trajectory's own spread below (the FP32 stage coefficients are rounded
  from the library's FP64 trajectory, which differs from the oracle's).
  FP64: the window is chaotic (ten time units of Lorenz-96): a one-ulp change
  of the initial state moves the trajectory's end by 2.6e-7 and the answer of
  the FP64 oracle itself by the spreads in tests/golden/l96_large_sensitivity.json
  (written by the oracle alone).  Two correct FP64 programs round differently at
  every step, so the library is held to 10 x those spreads: products, every
  eigenvalue, the increment and the cost reduction.  The eigenvalues that the
  FP64 problem determines to better than 1e-4 (494 of 512) are also held to the
  1e-3 asked of the leading eigenvalues.  The increment is not determined to
  1e-4 by the FP64 problem at all (spread 2.3e-3): the cost reduction it
  achieves is (spread 1.5e-6).
"""
import json
import os

import numpy as np
import pytest

from oracle import problem, riot as orc
from oracle.pool import HvpPool
from synth import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"
HERE = os.path.dirname(os.path.abspath(__file__))
U32 = 2.0 ** -24


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _ctx(R, cfg, prob, precision):
    return R.Context(n=prob.n, T=prob.T, dt=prob.dt, F=prob.F, obs_step=prob.obs_step, obs_idx=prob.obs_idx,
                     obs_y=prob.y, obs_sigma=prob.sigma_o, length=cfg.ell, sigma_b=cfg.sigma_b,
                     precision=precision, kmax=cfg.k)


@pytest.fixture(scope="module")
def large():
    cfg = configs.l96_large()
    prob = problem.build(cfg)
    traj = orc.trajectory(prob, prob.x_b)
    with open(os.path.join(HERE, "golden", "l96_large_sensitivity.json")) as f:
        sens = json.load(f)
    return cfg, prob, traj, sens


@pytest.fixture(scope="module")
def oracle_loop(large):
    """The oracle's inner loop on the benchmark's sketch (1024 products on a spawned pool), its
    increment and cost reduction, and 16 products of sketch 5 (FP64 and FP32-rounded input)."""
    cfg, prob, traj, _ = large
    d = orc.innovation(prob, traj)
    g = orc.gradient_b(prob, traj, d)
    W16 = cfg.sketch(5, k=16).T
    W16f = W16.astype(np.float32).astype(np.float64)
    with HvpPool(cfg) as pool:
        Y16 = pool.apply(W16)
        Y16f = pool.apply(W16f)
        lam, U, _ = orc.rsvd(prob, traj, cfg.sketch(0).T, q=cfg.q, apply=pool.apply)
        Omf = cfg.sketch(0).astype(np.float32).astype(np.float64).T
        lamf, Uf, _ = orc.rsvd(prob, traj, Omf, q=cfg.q, apply=pool.apply)
    z = np.zeros(prob.n)
    J0 = orc.quadratic_cost(prob, traj, d, z, z)
    out = {"W16": W16, "Y16": Y16, "W16f": W16f, "Y16f": Y16f, "J0": J0}
    out["lamf_pairs"] = (lamf, Uf)
    for tag, (l_, U_) in {"": (lam, U), "f": (lamf, Uf)}.items():
        dv, mode = orc.increment(l_, U_, g)
        out.update({"lam" + tag: l_, "dv" + tag: dv, "mode" + tag: mode,
                    "red" + tag: J0 - orc.quadratic_cost(prob, traj, d, z, dv)})
    return out


def _rel_cols(got, ref):
    return np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)


def test_large_window_products_fp64(gpu_lib, large, oracle_loop):
    R = gpu_lib
    cfg, prob, _, sens = large
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_FP64)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    W = _t(oracle_loop["W16"].T)
    Y = torch.empty_like(W)
    R.riot_hessian_apply(ctx.h, W, Y)
    err = _rel_cols(Y.cpu().numpy().T, oracle_loop["Y16"])
    assert err.max() <= 10 * max(sens["hvp_col_rel_spread"]), (err.max(), max(sens["hvp_col_rel_spread"]))
    ctx.close()


def test_large_window_products_fp32(gpu_lib, large, oracle_loop):
    R = gpu_lib
    cfg, prob, _, sens = large
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_MIXED)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    W = _t(oracle_loop["W16f"].T, torch.float32)
    Y = torch.empty_like(W)
    R.riot_hessian_apply(ctx.h, W, Y)
    err = _rel_cols(Y.double().cpu().numpy().T, oracle_loop["Y16f"])
    # FP32 rounding of the products plus the FP64 trajectory's own spread (the FP32 stage
    # coefficients come from the library's FP64 trajectory, not the oracle's)
    tol = 16 * np.sqrt(8 * cfg.T) * U32 + 10 * max(sens["hvp_col_rel_spread"])
    assert err.max() <= tol, (err.max(), tol)
    ctx.close()


def test_large_window_inner_loop_fp64(gpu_lib, large, oracle_loop):
    R = gpu_lib
    cfg, prob, _, sens = large
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_FP64)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    lam = R.riot_rsvd(ctx.h, cfg.k, cfg.q, Omega=_t(cfg.sketch(0)))
    dv = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    mode = R.riot_increment(ctx.h, dv)
    red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    ref = oracle_loop
    spread = np.asarray(sens["eig_rel_spread"])
    rel = np.abs(lam - ref["lam"]) / np.abs(ref["lam"])
    well = spread < 1e-4
    assert well.sum() >= 480
    assert rel[well].max() <= 1e-3, rel[well].max()
    assert np.all(rel <= np.maximum(1e-3, 10 * spread)), np.max(rel / np.maximum(1e-3, 10 * spread))
    assert mode == ref["mode"] == 0
    dv_err = np.linalg.norm(dv.cpu().numpy() - ref["dv"]) / np.linalg.norm(ref["dv"])
    assert dv_err <= 10 * sens["dv_rel_spread"], dv_err
    assert abs(red - ref["red"]) <= 10 * sens["reduction_rel_spread"] * ref["red"], (red, ref["red"])
    ctx.close()


def test_large_window_inner_loop_mixed(gpu_lib, large, oracle_loop):
    """Mixed precision (FP32 products).  An FP32 product carries an absolute error of about
    2^-24 lambda_1 |w|, so the mixed path retains the m pairs with lambda >= 2^-24 lambda_1.
    The leading eigenvalues, those a perturbation of 2^-24 lambda_1 moves by at most 1e-3
    (lambda >= 1e3 2^-24 lambda_1, as for the batch kernel), are held to 1e-3 (measured 7e-6);
    every retained eigenvalue to 1e-2 (measured 2e-3 at 1.6 times the floor, an absolute error
    of 2e-10 lambda_1: the FP32 rounding of the products, which moves with the order of the
    FP64 arithmetic around them).  The increment is LRA as in the oracle, and its cost
    reduction equals, to 1e-3, that of the oracle's own increment restricted to its leading m
    pairs.  (Against the full rank-512 increment it is smaller: the pairs below the FP32 floor
    carry the rest of the reduction at this window.)"""
    R = gpu_lib
    cfg, prob, traj, _ = large
    ctx = _ctx(R, cfg, prob, R.RIOT_PREC_MIXED)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    lam = R.riot_rsvd(ctx.h, cfg.k, cfg.q, Omega=_t(cfg.sketch(0), torch.float32))
    dv = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    mode = R.riot_increment(ctx.h, dv)
    m = R.riot_increment_pairs(ctx.h)
    red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    ref = oracle_loop
    assert m == int(np.sum(lam >= U32 * lam[0])) and 64 <= m < cfg.k
    rel = np.abs(lam[:m] - ref["lamf"][:m]) / ref["lamf"][:m]
    lead = lam[:m] >= 1e3 * U32 * lam[0]
    assert lead.sum() >= 32
    assert rel[lead].max() <= 1e-3, rel[lead].max()
    assert rel.max() <= 1e-2, rel.max()
    assert mode == 0
    # the oracle's increment on its own leading m pairs, and its cost reduction
    lam_o, U_o = ref["lamf_pairs"]
    d = orc.innovation(prob, traj)
    g = orc.gradient_b(prob, traj, d)
    dv_m, mode_m = orc.increment(lam_o[:m], U_o[:, :m], g)
    z = np.zeros(cfg.n)
    red_m = orc.quadratic_cost(prob, traj, d, z, z) - orc.quadratic_cost(prob, traj, d, z, dv_m)
    assert mode_m == 0
    assert abs(red - red_m) <= 1e-3 * red_m, (red, red_m, ref["redf"])
    ctx.close()


def test_large_window_deflated_mixed_reaches_the_fp64_reduction(gpu_lib, large, oracle_loop):
    """The deflated two-level eigendecomposition (FP32 products only: 256 columns, then 320 on
    the operator deflated by the pairs level 0 kept, one power iteration each) resolves the
    spectrum about as far down as the FP64 path: its increment reaches at least 0.95 of the
    cost reduction of the oracle's rank-512 FP64 increment (0.99 to 1.01 measured on this
    window with two sketches; the plain mixed path reaches 0.39), its leading eigenvalues agree
    with the oracle's to the 1e-3 asked of them, and the increment is LRA."""
    R = gpu_lib
    cfg, prob, _, _ = large
    ctx = R.Context(n=prob.n, T=prob.T, dt=prob.dt, F=prob.F, obs_step=prob.obs_step, obs_idx=prob.obs_idx,
                    obs_y=prob.y, obs_sigma=prob.sigma_o, length=cfg.ell, sigma_b=cfg.sigma_b,
                    precision=R.RIOT_PREC_MIXED, kmax=576)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    lam = R.riot_rsvd_deflated(ctx.h, [256, 320], cfg.q, sketch_stream=40, kmax=576)
    m = lam.size
    assert m >= 450 and np.all(np.diff(lam) <= 0)
    dv = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    mode = R.riot_increment(ctx.h, dv)
    assert mode == 0 and R.riot_increment_pairs(ctx.h) == m
    red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    ref = oracle_loop
    assert red >= 0.95 * ref["red"], (red, ref["red"])
    lead = 128
    rel = np.abs(lam[:lead] - ref["lam"][:lead]) / ref["lam"][:lead]
    assert rel.max() <= 1e-3, rel.max()
    ctx.close()
