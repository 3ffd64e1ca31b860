"""The learned sketch proposal on the GPU: network forward, loss and gradients
against the FP64 oracle, Adam, the trajectory input, the Rayleigh-residual
gate of riot_rsvd_proposal, and what a trained network gains over the
Gaussian sketch on held-out windows.

Tolerances: the network runs in FP32 (tanh from the CUDA math library, sums
of up to width * ksize terms), so outputs match the FP64 oracle to ~1e-6 of
their scale (1e-5 is required); gradients are sums over batch * n positions
and are compared as vectors (relative 2-norm error 1e-4).  BF16 inference
rounds weights and activations to 8 significant bits: 3e-2."""
import numpy as np
import pytest

from oracle import sketchnet as N
from synth import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _setup(R, c_in=4, width=8, m=6, n=40, B=3, seed=11):
    params = N.init_params(c_in, width, m, seed)
    flat32 = N.flatten(params).astype(np.float32)
    shapes = [W.shape for W, _ in params]
    params64 = N.unflatten(flat32.astype(np.float64), shapes)
    rng = np.random.default_rng(seed + 1)
    xs = rng.standard_normal((B, c_in, n)).astype(np.float32)
    Us = np.ascontiguousarray(np.stack([np.linalg.qr(rng.standard_normal((n, 3)))[0].T
                                        for _ in range(B)]).astype(np.float32))
    net = R.riot_sketchnet_create(c_in, width, m, n_max=n, batch_max=B, r_max=3)
    R.riot_sketchnet_set_params(net, torch.tensor(flat32, device=DEV))
    return net, params64, shapes, xs, Us


def test_forward_matches_oracle(gpu_lib):
    R = gpu_lib
    net, params, _, xs, _ = _setup(R)
    B, _, n = xs.shape
    Z = torch.empty(B, 6, n, dtype=torch.float32, device=DEV)
    R.riot_sketchnet_forward(net, torch.tensor(xs, device=DEV), Z)
    for b in range(B):
        ref, _ = N.forward(params, xs[b].astype(np.float64))
        np.testing.assert_allclose(Z[b].cpu().numpy(), ref, atol=1e-5 * np.abs(ref).max())
    R.riot_sketchnet_forward(net, torch.tensor(xs, device=DEV), Z, bf16=True)
    ref, _ = N.forward(params, xs[0].astype(np.float64))
    assert np.abs(Z[0].cpu().numpy() - ref).max() <= 3e-2 * np.abs(ref).max()
    R.riot_sketchnet_destroy(net)


def test_loss_and_gradient_match_oracle(gpu_lib):
    R = gpu_lib
    net, params, _, xs, Us = _setup(R)
    mu = 0.3
    g = torch.empty(R.riot_sketchnet_num_params(net), dtype=torch.float32, device=DEV)
    L = R.riot_sketchnet_loss_grad(net, torch.tensor(xs, device=DEV), torch.tensor(Us, device=DEV), mu, g)
    Lo, go = N.batch_loss_grad(params, [x.astype(np.float64) for x in xs],
                               [U.T.astype(np.float64) for U in Us], mu)
    assert L == pytest.approx(Lo, rel=1e-5)
    gg = g.cpu().numpy().astype(np.float64)
    gof = N.flatten(go)
    assert np.linalg.norm(gg - gof) <= 1e-4 * np.linalg.norm(gof)
    R.riot_sketchnet_destroy(net)


def test_adam_steps_follow_the_oracle(gpu_lib):
    R = gpu_lib
    net, params, shapes, xs, Us = _setup(R, seed=21)
    mu, lr = 0.3, 1e-2
    xt, Ut = torch.tensor(xs, device=DEV), torch.tensor(Us, device=DEV)
    p = N.flatten(params)
    opt = N.Adam(p.size, lr)
    losses, losses_o = [], []
    for _ in range(5):
        losses.append(R.riot_sketchnet_train_step(net, xt, Ut, mu, lr))
        Lo, go = N.batch_loss_grad(N.unflatten(p, shapes), [x.astype(np.float64) for x in xs],
                                   [U.T.astype(np.float64) for U in Us], mu)
        losses_o.append(Lo)
        p = opt.step(p, N.flatten(go))
    np.testing.assert_allclose(losses, losses_o, rtol=1e-4)
    out = torch.empty(p.size, dtype=torch.float32, device=DEV)
    R.riot_sketchnet_get_params(net, out)
    np.testing.assert_allclose(out.cpu().numpy(), p, atol=2e-5 * np.abs(p).max())
    R.riot_sketchnet_destroy(net)


def test_input_snapshots(gpu_lib):
    R = gpu_lib
    T, n, C = 37, 50, 8
    traj = np.random.default_rng(3).standard_normal((T + 1, n)) * 3.0 + 2.0
    x = torch.empty(C, n, dtype=torch.float32, device=DEV)
    R.riot_sketchnet_input(torch.tensor(traj, device=DEV), T, n, C, x)
    np.testing.assert_allclose(x.cpu().numpy(), N.snapshot_input(traj, C), rtol=1e-5, atol=1e-6)


def _l96_window(R, n, T, k, seed, F=12.0):
    from paper_1906_01413_gb300 import workloads
    cfg = configs.L96Config(name="ls", n=n, F=F, T=T, obs_every=2, obs_frac=0.5, obs_layout="random", ell=4.0,
                            k=k, q=1, spinup=300, seed=seed)
    ctx, xb, _ = workloads.l96_twin(R, torch, cfg, DEV, R.RIOT_PREC_MIXED, k)
    R.riot_outer_begin(ctx.h, xb)
    return cfg, ctx


def test_proposal_gate(gpu_lib):
    R = gpu_lib
    n, T, k, m = 96, 30, 32, 8
    cfg, ctx = _l96_window(R, n, T, k, configs.BASE_SEED + 900)
    lam_g = R.riot_rsvd(ctx.h, k, 1, sketch_stream=5)
    U = torch.empty(k, n, dtype=torch.float64, device=DEV)
    R.riot_get_state(ctx.h, U=U)
    # no proposal: identical to riot_rsvd
    lam0, rho0, used0 = R.riot_rsvd_proposal(ctx.h, k, 1, None, 0, sketch_stream=5)
    assert used0 == 0 and rho0 == -1.0
    np.testing.assert_array_equal(lam0, lam_g)
    # random directions are far from invariant: rejected, and the result is the Gaussian one
    P = torch.randn(m, n, dtype=torch.float32, device=DEV)
    lam1, rho1, used1 = R.riot_rsvd_proposal(ctx.h, k, 1, P, m, rho_max=1e-2, sketch_stream=5)
    assert used1 == 0 and rho1 > 1e-2
    np.testing.assert_array_equal(lam1, lam_g)
    # the leading Ritz vectors themselves are (nearly) invariant: kept
    P = U[:m].float().contiguous()
    lam2, rho2, used2 = R.riot_rsvd_proposal(ctx.h, k, 1, P, m, rho_max=1e-2, sketch_stream=5)
    assert used2 == 1 and rho2 < 1e-2
    np.testing.assert_allclose(lam2[:4], lam_g[:4], rtol=1e-3)
    ctx.close()


def test_trained_network_captures_held_out_eigenvectors(gpu_lib):
    """Windows of the same size with different seeds: a network trained on 32
    of them must capture more of the leading eigenvector subspace of 6 unseen
    windows than its untrained initial state and than random directions."""
    R = gpu_lib
    n, T, k, m, C, width = 128, 40, 48, 12, 8, 16
    xs, Us = [], []
    for w in range(38):
        cfg, ctx = _l96_window(R, n, T, k, configs.BASE_SEED + 3000 + w)
        R.riot_rsvd(ctx.h, k, 1, sketch_stream=2)
        U = torch.empty(k, n, dtype=torch.float64, device=DEV)
        R.riot_get_state(ctx.h, U=U)
        traj = torch.empty(T + 1, n, dtype=torch.float64, device=DEV)
        R.riot_get_trajectory(ctx.h, traj)
        x = torch.empty(C, n, dtype=torch.float32, device=DEV)
        R.riot_sketchnet_input(traj, T, n, C, x)
        xs.append(x)
        Us.append(U[:m].float())
        ctx.close()
    X = torch.stack(xs).contiguous()
    Ut = torch.stack(Us).contiguous()
    ntr = 32
    params = N.init_params(C, width, m, seed=5)
    flat = torch.tensor(N.flatten(params).astype(np.float32), device=DEV)
    net = R.riot_sketchnet_create(C, width, m, n_max=n, batch_max=8, r_max=m)
    R.riot_sketchnet_set_params(net, flat)

    def capture(xb, ub):
        Z = torch.empty(xb.shape[0], m, n, dtype=torch.float32, device=DEV)
        R.riot_sketchnet_forward(net, xb.contiguous(), Z)
        out = []
        for b in range(xb.shape[0]):
            Q, _ = torch.linalg.qr(Z[b].double().T)
            out.append(float((ub[b].double() @ Q).pow(2).sum()) / m)
        return float(np.mean(out))

    held_x, held_u = X[ntr:], Ut[ntr:]
    before = capture(held_x, held_u)
    rng = np.random.default_rng(0)
    for step in range(400):
        idx = torch.tensor(rng.choice(ntr, 8, replace=False), device=DEV)
        R.riot_sketchnet_train_step(net, X[idx].contiguous(), Ut[idx].contiguous(), 0.1, 3e-3)
    after = capture(held_x, held_u)
    random = m / n
    R.riot_sketchnet_destroy(net)
    print("held-out capture: untrained %.3f, trained %.3f, random %.3f" % (before, after, random))
    assert after > before and after > 1.5 * random
