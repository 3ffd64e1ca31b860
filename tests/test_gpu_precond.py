"""Spectral preconditioner and rotation (Section 2.2, Eq. 7, Algorithm 3 with
precond = true) on the GPU through riot_precond_* / riot_rsvd /
riot_increment, against the oracle's SpectralPreconditioner and
outer_step_precond run on the same window with the same sketches.

Chained loops (FP64 contexts).  Every loop is the oracle's FP64 computation in
another order (CholeskyQR instead of Householder, a projection for the rotation
instead of an SVD basis, P_k^-1 left out on the rotated complement where it is
the identity); loop-1 quantities agree to ~1e-9 as in the unpreconditioned
parity tests and three chained loops are held to 1e-8 (cost), 1e-7 (gradient;
eigenvalues, relative to the largest) and 1e-6 (increments, states).  Each loop pushes its pairs with
positive eigenvalue (the solve for K of Algorithm 3 returns trailing Ritz values
below -1 on the flattened spectrum of a preconditioned loop, where Eq. 7's
factor is undefined); the counts agree because no value lies near 0 on this
window.

One loop preconditioned by given exact pairs (the leading eigenpairs of the
oracle's dense Hessian, pushed into both sides): the preconditioned Hessian is
then well conditioned, so the mixed path can be held to 2e-3 (leading
eigenvalues) and 3e-3 (increment); FP32 products with 2e-5 noise move them by
2e-6 and 7e-5 in the oracle.  With n = 1024, k = m = 128 the factor products
and the rotation run on the tensor-core FP32 GEMMs.  The windows keep the
smallest retained eigenvalue away from 1, where the adaptive switch flips."""
import numpy as np
import pytest

from oracle import problem, riot as orc
from synth import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _ctx(R, prob, ell, precision, kmax):
    return R.Context(n=prob.n, T=prob.T, dt=prob.dt, F=prob.F, obs_step=prob.obs_step, obs_idx=prob.obs_idx,
                     obs_y=prob.y, obs_sigma=prob.sigma_o, length=ell, sigma_b=1.0, precision=precision, kmax=kmax)


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _fp64_window():
    return configs.l96_custom("pc_n40", n=40, T=20, obs_every=1, obs_frac=0.5, obs_layout="even", ell=2.0, k=12,
                              q=1)


def _oracle_loops(prob, cfg, loops, rotation, f32_sketch):
    pc = orc.SpectralPreconditioner(cfg.n)
    x, v = prob.x_b.copy(), np.zeros(cfg.n)
    out = []
    for it in range(loops):
        Om = cfg.sketch(it).T
        if f32_sketch:
            Om = Om.astype(np.float32).astype(np.float64)
        st = orc.outer_step_precond(prob, x, v, Om, pc, q=cfg.q, rotation=rotation)
        out.append(st)
        m = int(np.sum(st["lam"] > 0))
        pc.push(st["lam"][:m], st["U"][:, :m])
        x, v = st["x_next"], st["v_next"]
    return out, pc


def _gpu_loops(R, ctx, cfg, prob, loops, dtype):
    out = []
    for it in range(loops):
        J = R.riot_outer_begin(ctx.h, _t(prob.x_b)) if it == 0 else R.riot_outer_begin(ctx.h)
        g = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
        R.riot_get_state(ctx.h, g=g)
        lam = R.riot_rsvd(ctx.h, cfg.k, cfg.q, Omega=_t(cfg.sketch(it), dtype))
        dv = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
        mode = R.riot_increment(ctx.h, dv)
        R.riot_precond_push(ctx.h, int(np.sum(lam > 0)))
        out.append({"J": J, "g": g.cpu().numpy(), "lam": lam, "dv": dv.cpu().numpy(), "mode": mode})
    x = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    v = torch.empty(cfg.n, dtype=torch.float64, device=DEV)
    R.riot_get_state(ctx.h, x=x, v=v)
    return out, x.cpu().numpy(), v.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("rotation", [True, False])
def test_preconditioned_loops_fp64_track_oracle(gpu_lib, rotation):
    R = gpu_lib
    cfg = _fp64_window()
    prob = problem.build(cfg)
    loops = 3
    ref, pc = _oracle_loops(prob, cfg, loops, rotation, f32_sketch=False)
    for st in ref:
        assert abs(st["lam"][-1] - 1.0) > 0.05
        assert np.abs(st["lam"]).min() > 0.05
    ctx = _ctx(R, prob, cfg.ell, R.RIOT_PREC_FP64, cfg.k)
    R.riot_precond_enable(ctx.h, loops * cfg.k, rotation)
    got, x, v = _gpu_loops(R, ctx, cfg, prob, loops, torch.float64)
    assert R.riot_precond_count(ctx.h) == loops
    for it, (a, b) in enumerate(zip(got, ref)):
        assert int(np.sum(a["lam"] > 0)) == int(np.sum(b["lam"] > 0)), it
        assert abs(a["J"] - b["J"]) <= 1e-8 * b["J"], it
        assert _rel(a["g"], b["g"]) <= 1e-7, it
        np.testing.assert_allclose(a["lam"], b["lam"], rtol=0, atol=1e-7 * b["lam"][0], err_msg=str(it))
        assert a["mode"] == b["mode"], it
        assert _rel(a["dv"], b["dv"]) <= 1e-6, it
    np.testing.assert_allclose(x, ref[-1]["x_next"], rtol=0, atol=1e-6 * np.abs(ref[-1]["x_next"]).max())
    np.testing.assert_allclose(v, ref[-1]["v_next"], rtol=0, atol=1e-6 * np.abs(ref[-1]["v_next"]).max())
    # the factors themselves: P_k, P_k^T and P_k^-1 on the identity
    I = torch.eye(cfg.n, dtype=torch.float64, device=DEV)
    Y = torch.empty_like(I)
    for op, f in ((R.PRECOND_P, pc.apply), (R.PRECOND_PT, pc.apply_t), (R.PRECOND_PINV, pc.apply_inv)):
        R.riot_precond_apply(ctx.h, I, Y, op)
        want = f(np.eye(cfg.n))                      # column j of op(P) = row j of Y
        np.testing.assert_allclose(Y.cpu().numpy().T, want, rtol=0, atol=1e-6 * np.abs(want).max())
    ctx.close()


def _exact_pairs_window(n, k):
    cfg = configs.l96_custom("pc_exact_n%d" % n, n=n, T=20, obs_every=4, obs_frac=0.25, ell=4.0, k=k, q=1)
    prob = problem.build(cfg)
    A = orc.dense_hessian(prob, orc.trajectory(prob, prob.x_b))
    lam, V = np.linalg.eigh(0.5 * (A + A.T))
    return cfg, prob, lam[::-1], V[:, ::-1]


@pytest.mark.parametrize("precision,n,k,m,tol_lam,tol_dv", [
    ("fp64", 512, 64, 16, 1e-9, 1e-8),
    ("mixed", 1024, 128, 128, 2e-3, 3e-3),
])
def test_loop_preconditioned_by_given_pairs(gpu_lib, precision, n, k, m, tol_lam, tol_dv):
    R = gpu_lib
    cfg, prob, lam_e, V_e = _exact_pairs_window(n, k)
    mixed = precision == "mixed"
    pc = orc.SpectralPreconditioner(n)
    pc.push(lam_e[:m], V_e[:, :m])
    Om = cfg.sketch(0).T
    if mixed:
        Om = Om.astype(np.float32).astype(np.float64)
    ref = orc.outer_step_precond(prob, prob.x_b, np.zeros(n), Om, pc, q=cfg.q, rotation=True)
    assert abs(ref["lam"][-1] - 1.0) > 0.05
    ctx = _ctx(R, prob, cfg.ell, R.RIOT_PREC_MIXED if mixed else R.RIOT_PREC_FP64, k)
    R.riot_precond_enable(ctx.h, m, True)
    R.riot_precond_push_pairs(ctx.h, _t(V_e[:, :m].T), lam_e[:m])
    J = R.riot_outer_begin(ctx.h, _t(prob.x_b))
    assert abs(J - ref["J"]) <= 1e-9 * ref["J"]
    lam = R.riot_rsvd(ctx.h, k, cfg.q, Omega=_t(cfg.sketch(0), torch.float32 if mixed else torch.float64))
    dv = torch.empty(n, dtype=torch.float64, device=DEV)
    mode = R.riot_increment(ctx.h, dv)
    lead = ref["lam"] > 0.1 * ref["lam"][0]
    assert lead.sum() >= 10
    assert (np.abs(lam[lead] - ref["lam"][lead]) / ref["lam"][lead]).max() < tol_lam
    assert mode == ref["mode"]
    assert _rel(dv.cpu().numpy(), ref["dv"]) <= tol_dv
    x = torch.empty(n, dtype=torch.float64, device=DEV)
    R.riot_get_state(ctx.h, x=x)
    dx = ref["x_next"] - prob.x_b
    np.testing.assert_allclose(x.cpu().numpy() - prob.x_b, dx, rtol=0, atol=tol_dv * np.abs(dx).max())
    ctx.close()


def test_precond_call_order_and_errors(gpu_lib):
    R = gpu_lib
    cfg = _fp64_window()
    prob = problem.build(cfg)
    ctx = _ctx(R, prob, cfg.ell, R.RIOT_PREC_FP64, cfg.k)
    with pytest.raises(R.RiotError) as e:
        R.riot_precond_push(ctx.h, 4)
    assert e.value.status == -6                       # before riot_precond_enable
    with pytest.raises(R.RiotError) as e:
        R.riot_precond_enable(ctx.h, cfg.n + 1, True)
    assert e.value.status == -1
    R.riot_precond_enable(ctx.h, cfg.k + 4, True)
    R.riot_outer_begin(ctx.h, _t(prob.x_b))
    with pytest.raises(R.RiotError) as e:
        R.riot_precond_push(ctx.h, 4)
    assert e.value.status == -6                       # no inner loop yet
    R.riot_rsvd(ctx.h, cfg.k, 0, Omega=_t(cfg.sketch(0)))
    with pytest.raises(R.RiotError) as e:
        R.riot_precond_push(ctx.h, 4)
    assert e.value.status == -6                       # no increment yet
    R.riot_increment(ctx.h)
    with pytest.raises(R.RiotError) as e:
        R.riot_precond_push(ctx.h, cfg.k + 1)
    assert e.value.status == -1
    R.riot_precond_push(ctx.h, cfg.k)
    with pytest.raises(R.RiotError) as e:
        R.riot_precond_push(ctx.h, cfg.k)
    assert e.value.status == -6                       # one push per outer loop
    assert R.riot_precond_count(ctx.h) == 1
    with pytest.raises(R.RiotError) as e:
        R.riot_rsvd(ctx.h, cfg.k, 0)
    assert e.value.status == -6                       # the gradient must be formed with the new P_k first
    with pytest.raises(R.RiotError) as e:
        R.riot_increment(ctx.h)
    assert e.value.status == -6
    R.riot_outer_begin(ctx.h)
    with pytest.raises(R.RiotError) as e:
        R.riot_varcg(ctx.h, 4)
    assert e.value.status == -6
    with pytest.raises(R.RiotError) as e:              # rotation: k + 12 resolved columns > n = 40
        R.riot_rsvd(ctx.h, 29, 0)
    assert e.value.status == -1
    lam = R.riot_rsvd(ctx.h, cfg.k, 0, Omega=_t(cfg.sketch(1)))
    assert np.all(lam[:4] > 0)
    R.riot_increment(ctx.h)
    R.riot_precond_push(ctx.h, 4)
    R.riot_outer_begin(ctx.h)
    R.riot_rsvd(ctx.h, 4, 0, Omega=_t(cfg.sketch(2, k=4)))
    V = torch.zeros(1, cfg.n, dtype=torch.float64, device=DEV)
    V[0, 0] = 1.0
    with pytest.raises(R.RiotError) as e:
        R.riot_precond_push_pairs(ctx.h, V, [2.0])
    assert e.value.status == -6                       # inside an inner loop
    R.riot_increment(ctx.h)
    with pytest.raises(R.RiotError) as e:
        R.riot_precond_push(ctx.h, 4)
    assert e.value.status == -1                       # storage for k + 4 columns is full
    R.riot_precond_enable(ctx.h, 4, False)
    with pytest.raises(R.RiotError) as e:
        R.riot_precond_push_pairs(ctx.h, V, [-1.0])
    assert e.value.status == -8                       # I + A_k must be positive definite
    R.riot_precond_push_pairs(ctx.h, V, [3.0])         # P = I + (1/2 - 1) e_0 e_0^T
    X = torch.ones(2, cfg.n, dtype=torch.float64, device=DEV)
    Y = torch.empty_like(X)
    R.riot_precond_apply(ctx.h, X, Y, R.PRECOND_PINV)
    want = np.ones(cfg.n)
    want[0] = 2.0
    np.testing.assert_array_equal(Y.cpu().numpy(), np.stack([want, want]))
    R.riot_precond_enable(ctx.h, 0, False)            # off: the plain loop and Algorithm 1 again
    assert R.riot_precond_count(ctx.h) == 0
    R.riot_outer_begin(ctx.h)
    theta, used = R.riot_varcg(ctx.h, 4)
    assert used == 4
    # enabling after an inner loop keeps that loop's pairs available to push
    lam = R.riot_rsvd(ctx.h, cfg.k, 0, Omega=_t(cfg.sketch(0)))
    R.riot_increment(ctx.h)
    R.riot_precond_enable(ctx.h, cfg.k, True)
    R.riot_precond_push(ctx.h, int(np.sum(lam > 0)))
    with pytest.raises(R.RiotError) as e:
        R.riot_rsvd(ctx.h, 4, 0)
    assert e.value.status == -6
    R.riot_outer_begin(ctx.h)
    R.riot_rsvd(ctx.h, 4, 0, Omega=_t(cfg.sketch(3, k=4)))
    ctx.close()
