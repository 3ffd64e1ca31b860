"""riot_hessian_apply_noalloc: the Hessian apply for callers that cannot allocate.

Some callers run where the library must not call cudaMalloc when the
Hessian is applied (a memory pool or budget fixed at start-up, or a context
built with a small kmax).  This entry point keeps the tangent-linear
residuals in a fixed static device array instead; it must give the same
result as riot_hessian_apply, call after call, must leave the device's free
memory unchanged, and must refuse columns that do not fit the array.  This
file is collected last on purpose.

Comparison: on the Lorenz-96 model both entry points run the same kernel on
every column with arithmetic that does not depend on how the columns are
sliced (one observation per slot and step in these windows, so the adjoint's
shared-memory accumulation has a single term per slot): the results must be
bitwise equal.  The tracer model scatters observations into the adjoint field
with atomic additions whose order varies between launches, so there the two
agree to the rounding of that order: 1e-6 relative in FP32, 1e-13 in FP64.
"""
import numpy as np
import pytest

from oracle import advdiff as A
from oracle import problem
from synth import advdiff as S
from synth import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _ctx(R, prob, ell, precision, kmax, F=None):
    return R.Context(n=prob.n, T=prob.T, dt=prob.dt, F=prob.F if F is None else F, obs_step=prob.obs_step,
                     obs_idx=prob.obs_idx, obs_y=prob.y, obs_sigma=prob.sigma_o, length=ell, sigma_b=1.0,
                     precision=precision, kmax=kmax)


def _check_twice(R, ctx, W, ref, tol):
    for call in range(2):
        Y = torch.full_like(W, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        R.riot_hessian_apply_noalloc(ctx.h, W, Y)
        torch.cuda.synchronize()
        if call == 1:   # nothing was allocated on the device by the second call
            assert torch.cuda.mem_get_info()[0] == free0
        got = Y.double().cpu().numpy()
        if tol == 0.0:
            np.testing.assert_array_equal(got, ref)
        else:
            err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
            assert err.max() <= tol, err.max()


@pytest.mark.parametrize("which,precision,ncols", [
    ("small", "fp64", 37),
    ("small", "mixed", 40),
    ("large", "mixed", 100),    # 200 kB of residuals per column: two slices of the array
    ("unstable", "mixed", 24),  # FP32 products scaled by a power of two (the window's growth passes 2^96)
])
def test_noalloc_equals_hessian_apply_twice(gpu_lib, which, precision, ncols):
    R = gpu_lib
    if which == "unstable":
        # F = 10 over 300 steps: |A w| / |w| near 1e30, above the 2^96 where the FP32 path scales
        cfg = configs.l96_custom("unstable", n=64, T=300, obs_every=4, obs_frac=0.25, ell=4.0, k=ncols, q=0,
                                 F=10.0, spinup=200)
    else:
        cfg = configs.l96_small() if which == "small" else configs.l96_large()
    prob = problem.build(cfg)
    prec = R.RIOT_PREC_FP64 if precision == "fp64" else R.RIOT_PREC_MIXED
    dt = torch.float64 if precision == "fp64" else torch.float32
    ctx = _ctx(R, prob, cfg.ell, prec, kmax=max(ncols, 1))
    R.riot_outer_begin(ctx.h, torch.tensor(prob.x_b, device=DEV))
    W = torch.tensor(cfg.sketch(3, k=ncols), dtype=dt, device=DEV)
    Y_ref = torch.empty_like(W)
    R.riot_hessian_apply(ctx.h, W, Y_ref)
    ref = Y_ref.double().cpu().numpy()
    assert np.all(np.isfinite(ref))
    if which == "unstable":   # the products are far beyond the FP32 range without the scaling
        assert np.abs(ref).max() > 1e30
    _check_twice(R, ctx, W, ref, 0.0)
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 1e-6)])
def test_noalloc_tracer_matches_hessian_apply_twice(gpu_lib, precision, tol):
    R = gpu_lib
    cfg = S.bc_tiny()
    prob = A.build(cfg)
    m = prob.m
    prec = R.RIOT_PREC_FP64 if precision == "fp64" else R.RIOT_PREC_MIXED
    dt = torch.float64 if precision == "fp64" else torch.float32
    ctx = R.Context(nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, nblocks=cfg.nblocks, T=cfg.T, dt=cfg.dt, dx=cfg.dx,
                    dy=cfg.dy, dz=cfg.dz, u=m.u, v=m.v, amp=m.amp, kz=m.kz, emis_b=m.Eb,
                    obs_step=prob.obs.step, obs_pos=prob.obs.pos, obs_y=prob.y, obs_sigma=prob.sigma_o,
                    length=cfg.ell, sigma_b=cfg.sigma_b, precision=prec, kmax=4)
    R.riot_outer_begin(ctx.h, torch.tensor(prob.x_b, device=DEV))
    W = torch.tensor(np.random.default_rng(5).standard_normal((9, prob.n)), dtype=dt, device=DEV)
    Y_ref = torch.empty_like(W)
    R.riot_hessian_apply(ctx.h, W, Y_ref)
    _check_twice(R, ctx, W, Y_ref.double().cpu().numpy(), tol)
    ctx.close()


def test_noalloc_rejects_columns_larger_than_the_array(gpu_lib):
    # every variable observed at every one of 600 steps of an n = 4096 window:
    # 2 461 696 observations x 8 bytes = 19.7 MB per column > 16 MiB
    R = gpu_lib
    n, T = 4096, 600
    st = np.repeat(np.arange(T + 1), n).astype(np.int32)
    ix = np.tile(np.arange(n), T + 1).astype(np.int32)
    ctx = R.Context(n=n, T=T, dt=0.05, F=8.0, obs_step=st, obs_idx=ix, obs_y=np.zeros(st.size),
                    obs_sigma=np.ones(st.size), length=4.0, precision=R.RIOT_PREC_FP64, kmax=1)
    R.riot_outer_begin(ctx.h, torch.full((n,), 8.0, dtype=torch.float64, device=DEV))
    W = torch.zeros(1, n, dtype=torch.float64, device=DEV)
    with pytest.raises(R.RiotError) as e:
        R.riot_hessian_apply_noalloc(ctx.h, W, W.clone())
    assert e.value.status == -1 and "static array" in str(e.value)
    ctx.close()
