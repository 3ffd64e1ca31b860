"""riot_hessian_apply_noalloc: the Hessian apply for callers that cannot allocate.

Some callers run where the library must not call cudaMalloc when the
Hessian is applied (a memory pool or budget fixed at start-up, or a context
built with a small kmax).  This entry point keeps the tangent-linear
residuals in a fixed static device array instead; it must give the same
result as riot_hessian_apply, call after call, and must refuse columns that
do not fit the array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import problem
from synth import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _ctx(R, prob, ell, precision, kmax):
    return R.Context(n=prob.n, T=prob.T, dt=prob.dt, F=prob.F, obs_step=prob.obs_step, obs_idx=prob.obs_idx,
                     obs_y=prob.y, obs_sigma=prob.sigma_o, length=ell, sigma_b=1.0, precision=precision,
                     kmax=kmax)


@pytest.mark.parametrize("which,precision,ncols,tol", [
    ("small", "fp64", 37, 1e-10),     # tolerance of the FP64 Hessian tests
    ("small", "mixed", 40, 2e-5),     # tolerance of the FP32 Hessian tests
    ("large", "mixed", 100, 2e-5),    # 200 kB of residuals per column: two slices of the array
])
def test_noalloc_matches_hessian_apply_twice(gpu_lib, which, precision, ncols, tol):
    R = gpu_lib
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
    for _ in range(2):
        Y = torch.full_like(W, float("nan"))
        R.riot_hessian_apply_noalloc(ctx.h, W, Y)
        torch.cuda.synchronize()
        got = Y.double().cpu().numpy()
        err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= tol, err.max()
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
