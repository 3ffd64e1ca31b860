"""RIOT-PSAS (Appendix, Algorithm 4) on the GPU through riot_psas, against the
oracle's psas_outer_step on the same window and sketches.

The dual cycle runs in FP64 on either precision (the observation space is the
small side), so both sides compute the same quantities in another order
(CholeskyQR for Householder, the normal equations for the solve for K, a
scattered adjoint forcing): eigenvalues agree to 1e-9 of the largest and the
updated states to 1e-9 of the increment at full rank, 1e-7 below it, where
the solve for K amplifies rounding by the conditioning of Q^T W.  The windows
keep the smallest retained eigenvalue away from 1 (the adaptive switch)."""
import numpy as np
import pytest

from oracle import bcov, l96, riot as orc
from synth import configs, philox

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _window(n, T, steps, per_step, sigma, seed, ell=2.0):
    rng = np.random.default_rng(seed)
    x0 = l96.nl(8.0 + rng.standard_normal(n), 300, 0.05, 8.0)[-1]
    st, ix = [], []
    for s in steps:
        st.append(np.full(per_step, s))
        ix.append(np.sort(rng.choice(n, per_step, replace=False)))
    st, ix = np.concatenate(st), np.concatenate(ix)
    truth = l96.nl(x0, T, 0.05, 8.0)
    sig = np.full(st.size, sigma)
    y = truth[st, ix] + sig * rng.standard_normal(st.size)
    L = bcov.bsqrt(n, ell, 1.0)
    return orc.L96Problem(n=n, T=T, dt=0.05, F=8.0, obs_step=st, obs_idx=ix, y=y, sigma_o=sig, L=L,
                          x_b=x0 + L @ rng.standard_normal(n)), ell


def _ctx(R, prob, ell, precision, kmax, exact_rr=False):
    return R.Context(n=prob.n, T=prob.T, dt=prob.dt, F=prob.F, obs_step=prob.obs_step, obs_idx=prob.obs_idx,
                     obs_y=prob.y, obs_sigma=prob.sigma_o, length=ell, sigma_b=1.0, precision=precision, kmax=kmax,
                     exact_rr=exact_rr)


def _omega(p, m, stream):
    return philox.normals(configs.BASE_SEED, stream, p * m).reshape(m, p)      # row j = column j


def _cycles(R, ctx, prob, m, q, streams):
    xs, out = [], []
    x = torch.empty(prob.n, dtype=torch.float64, device=DEV)
    for c, stream in enumerate(streams):
        J = R.riot_outer_begin(ctx.h, _t(prob.x_b)) if c == 0 else R.riot_outer_begin(ctx.h)
        lam, mode = R.riot_psas(ctx.h, m, q, Omega=_t(_omega(prob.p, m, stream)))
        R.riot_get_state(ctx.h, x=x)
        out.append({"J": J, "lam": lam, "mode": mode, "x": x.cpu().numpy().copy()})
    return out


def _oracle_cycles(prob, m, q, streams, exact_rr=False):
    x, out = prob.x_b.copy(), []
    for stream in streams:
        st = orc.psas_outer_step(prob, x, _omega(prob.p, m, stream).T, q=q, exact_rr=exact_rr)
        out.append(st)
        x = st["x_next"]
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("q", [0, 1])
def test_full_rank_cycles_match_oracle(gpu_lib, precision, q):
    R = gpu_lib
    prob, ell = _window(40, 8, [4, 8], 5, 0.5, 17)
    m = prob.p
    ref = _oracle_cycles(prob, m, q, [80, 81])
    ctx = _ctx(R, prob, ell, R.RIOT_PREC_FP64 if precision == "fp64" else R.RIOT_PREC_MIXED, m)
    got = _cycles(R, ctx, prob, m, q, [80, 81])
    for c, (a, b) in enumerate(zip(got, ref)):
        assert abs(b["lam"][-1] - 1.0) > 0.05
        assert abs(a["J"] - b["J"]) <= 1e-9 * b["J"], c
        np.testing.assert_allclose(a["lam"], b["lam"], rtol=0, atol=1e-9 * b["lam"][0], err_msg=str(c))
        assert a["mode"] == b["mode"], c
        dx = b["x_next"] - prob.x_b
        np.testing.assert_allclose(a["x"], b["x_next"], rtol=0, atol=1e-9 * np.abs(dx).max(), err_msg=str(c))
    ctx.close()


@pytest.mark.parametrize("q,exact_rr,m", [(1, False, 30), (0, True, 30), (1, False, 48)])
def test_partial_rank_cycle_matches_oracle(gpu_lib, q, exact_rr, m):
    """p = 125 observations of 256 variables; m = 30 retains eigenvalues above 1 (LRA), m = 48
    reaches below (LRU)."""
    R = gpu_lib
    prob, ell = _window(256, 20, [4, 8, 12, 16, 20], 25, 1.0, 23, ell=4.0)
    ref = _oracle_cycles(prob, m, q, [82], exact_rr=exact_rr)[0]
    assert abs(ref["lam"][-1] - 1.0) > 0.05
    ctx = _ctx(R, prob, ell, R.RIOT_PREC_FP64, m, exact_rr=exact_rr)
    got = _cycles(R, ctx, prob, m, q, [82])[0]
    np.testing.assert_allclose(got["lam"], ref["lam"], rtol=0, atol=1e-8 * ref["lam"][0])
    assert got["mode"] == ref["mode"]
    dx = ref["x_next"] - prob.x_b
    np.testing.assert_allclose(got["x"], ref["x_next"], rtol=0, atol=1e-7 * np.abs(dx).max())
    ctx.close()


def test_psas_arguments_and_state(gpu_lib):
    R = gpu_lib
    prob, ell = _window(40, 8, [4, 8], 5, 0.5, 17)
    ctx = _ctx(R, prob, ell, R.RIOT_PREC_FP64, 16)
    with pytest.raises(R.RiotError) as e:
        R.riot_psas(ctx.h, 4)
    assert e.value.status == -6                       # before riot_outer_begin
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    with pytest.raises(R.RiotError) as e:
        R.riot_psas(ctx.h, prob.p + 1)                # m > p
    assert e.value.status == -1
    with pytest.raises(R.RiotError) as e:
        R.riot_psas(ctx.h, 4, q=65)
    assert e.value.status == -1
    lam, mode = R.riot_psas(ctx.h, 6, 1, sketch_stream=5)    # a drawn sketch
    assert lam.size == 6 and np.all(np.diff(lam) <= 0) and mode in (0, 1)
    ctx.close()


# --- the tracer-transport problem ---------------------------------------------------------

def _bc_ctx(R, cfg, prob, precision, kmax, exact_rr=False):
    m = prob.m
    return R.Context(nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, nblocks=cfg.nblocks, T=cfg.T, dt=cfg.dt, dx=cfg.dx,
                     dy=cfg.dy, dz=cfg.dz, u=m.u, v=m.v, amp=m.amp, kz=m.kz, emis_b=m.Eb,
                     obs_step=prob.obs.step, obs_pos=prob.obs.pos, obs_y=prob.y, obs_sigma=prob.sigma_o,
                     length=cfg.ell, sigma_b=cfg.sigma_b, precision=precision, kmax=kmax, exact_rr=exact_rr)


def _bc_oracle_cycles(AD, prob, m, q, streams, exact_rr=False):
    x, out = prob.x_b.copy(), []
    for stream in streams:
        st = AD.psas_outer_step(prob, x, _omega(prob.p, m, stream).T, q=q, exact_rr=exact_rr)
        out.append(st)
        x = st["x_next"]
    return out


@pytest.fixture(scope="module")
def bc_small():
    from oracle import advdiff as AD
    from synth import advdiff as S
    cfg = S.bc_small()
    return AD, cfg, AD.build(cfg)


@pytest.mark.parametrize("precision,m,q,exact_rr,streams", [
    ("fp64", 16, 1, False, [90, 91]),     # lambda_16 = 2.9: LRA
    ("fp64", 48, 1, False, [92]),         # lambda_48 = 0.05: LRU
    ("mixed", 48, 1, False, [92]),        # the dual runs in FP64 on a mixed context too
    ("fp64", 24, 0, True, [93]),
])
def test_tracer_cycles_match_oracle(gpu_lib, bc_small, precision, m, q, exact_rr, streams):
    """The tracer window of 384 controls and 240 observations (rank of A_dual about 120):
    eigenvalues to 1e-8 of the largest and the updated controls to 1e-7 of the increment,
    as on the Lorenz-96 windows below full rank.  The second cycle starts from the state the
    first one left (the outer loop's linearisation moves with x: E = E_b exp(x))."""
    R = gpu_lib
    AD, cfg, prob = bc_small
    ref = _bc_oracle_cycles(AD, prob, m, q, streams, exact_rr=exact_rr)
    prec = R.RIOT_PREC_FP64 if precision == "fp64" else R.RIOT_PREC_MIXED
    ctx = _bc_ctx(R, cfg, prob, prec, kmax=max(m, 48), exact_rr=exact_rr)
    got = _cycles(R, ctx, prob, m, q, streams)
    for c, (a, b) in enumerate(zip(got, ref)):
        assert abs(b["lam"][-1] - 1.0) > 0.05
        np.testing.assert_allclose(a["lam"], b["lam"], rtol=0, atol=1e-8 * b["lam"][0], err_msg=str(c))
        assert a["mode"] == b["mode"], c
        dx = b["x_next"] - (prob.x_b if c == 0 else ref[c - 1]["x_next"])
        np.testing.assert_allclose(a["x"], b["x_next"], rtol=0, atol=1e-7 * np.abs(dx).max(), err_msg=str(c))
    ctx.close()
