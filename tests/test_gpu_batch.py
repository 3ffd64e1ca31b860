"""Batches of Lorenz-96 windows: one persistent Hessian launch per application,
the inner loops of all windows captured as one CUDA graph.

Every window of a batch must end exactly where the same window ends when run
alone through riot_rsvd + riot_increment: the batch kernel runs the same
per-column arithmetic (only the grouping of columns into CTAs differs) and
the rest of the inner loop is the same code, so eigenvalues, increments and
updated states are compared to 1e-12 (FP64 quantities built from identical
FP32 Hessian blocks).
"""
import numpy as np
import pytest

from synth import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _windows():
    # uneven sizes: every chunk width (E = 4, 8, 16), ragged chunks, k from 8 to n
    spec = [(40, 30, 40), (100, 21, 16), (333, 17, 64), (1000, 12, 128), (4096, 6, 64), (5001, 5, 32),
            (8192, 4, 48), (61, 9, 8)]
    out = []
    for i, (n, T, k) in enumerate(spec):
        out.append(configs.L96Config(name="bw%d" % i, n=n, F=8.0 + i, T=T, obs_every=2, obs_frac=0.3,
                                     obs_layout="random", ell=4.0, k=k, q=1, spinup=200,
                                     seed=configs.BASE_SEED + 500 + i))
    return out


def _make(R, cfgs):
    from paper_1906_01413_gb300 import workloads
    ctxs, xbs = [], []
    for c in cfgs:
        ctx, xb, _ = workloads.l96_twin(R, torch, c, DEV, R.RIOT_PREC_MIXED, c.k)
        R.riot_outer_begin(ctx.h, xb)
        ctxs.append(ctx)
        xbs.append(xb)
    return ctxs, xbs


def _state(R, ctx, n, k):
    lam = torch.empty(k, dtype=torch.float64, device=DEV)
    x = torch.empty(n, dtype=torch.float64, device=DEV)
    v = torch.empty(n, dtype=torch.float64, device=DEV)
    R.riot_get_state(ctx.h, x=x, v=v, lam=lam)
    return lam.cpu().numpy(), x.cpu().numpy(), v.cpu().numpy()


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_windows_run_alone(gpu_lib, use_graph):
    R = gpu_lib
    cfgs = _windows()
    q = 1
    # alone
    ctxs, _ = _make(R, cfgs)
    alone = []
    for c, ctx in zip(cfgs, ctxs):
        R.riot_rsvd(ctx.h, c.k, q, sketch_stream=configs.STREAM_SKETCH0)
        R.riot_increment(ctx.h)
        alone.append(_state(R, ctx, c.n, c.k))
    for ctx in ctxs:
        ctx.close()
    # batched
    ctxs, _ = _make(R, cfgs)
    b = R.riot_batch_create([ctx.h for ctx in ctxs], [c.k for c in cfgs], q)
    st = R.riot_batch_run(b, len(cfgs), sketch_stream=configs.STREAM_SKETCH0, use_graph=use_graph)
    assert st == [0] * len(cfgs)
    for i, (c, ctx) in enumerate(zip(cfgs, ctxs)):
        lam, x, v = _state(R, ctx, c.n, c.k)
        np.testing.assert_allclose(lam, alone[i][0], rtol=1e-12, err_msg=c.name)
        np.testing.assert_allclose(x, alone[i][1], rtol=1e-12, atol=1e-12, err_msg=c.name)
        np.testing.assert_allclose(v, alone[i][2], rtol=1e-12, atol=1e-12, err_msg=c.name)
    R.riot_batch_destroy(b)
    for ctx in ctxs:
        ctx.close()


def test_graph_replays_follow_new_outer_loops(gpu_lib):
    """After riot_outer_begin at the updated states, a replay of the captured
    graph runs the next inner loop: it must equal a fresh eager run."""
    R = gpu_lib
    cfgs = _windows()[:5]
    q = 1
    runs = {}
    for mode in ("graph", "eager"):
        ctxs, _ = _make(R, cfgs)
        b = R.riot_batch_create([ctx.h for ctx in ctxs], [c.k for c in cfgs], q)
        for outer in range(2):
            if outer:
                for ctx in ctxs:
                    R.riot_outer_begin(ctx.h)
            R.riot_batch_run(b, len(cfgs), sketch_stream=configs.STREAM_SKETCH0, use_graph=(mode == "graph"))
        runs[mode] = [_state(R, ctx, c.n, c.k) for c, ctx in zip(cfgs, ctxs)]
        R.riot_batch_destroy(b)
        for ctx in ctxs:
            ctx.close()
    for a, e in zip(runs["graph"], runs["eager"]):
        for u, w in zip(a, e):
            np.testing.assert_allclose(u, w, rtol=1e-12, atol=1e-12)


def test_autotuned_shape_gives_the_same_products(gpu_lib):
    R = gpu_lib
    cfgs = _windows()
    ctxs, _ = _make(R, cfgs)
    b = R.riot_batch_create([ctx.h for ctx in ctxs], [c.k for c in cfgs], 0)
    P, S, ms = R.riot_batch_autotune(b)
    assert P in (0, 32, 16, 8, 4, 2) and S in (2, 3, 4) and ms > 0
    outs = []
    for cfg_ in ((P, S), (1, 2), (0, 4)):
        R.riot_batch_set_config(b, *cfg_)
        st = R.riot_batch_run(b, len(cfgs), sketch_stream=7, use_graph=False)
        assert st == [0] * len(cfgs)
        # the eigenpairs depend on the stored trajectory only, not on the updated x, v
        outs.append([_state(R, ctx, c.n, c.k)[0] for c, ctx in zip(cfgs, ctxs)])
    for o in outs[1:]:
        for a, e in zip(o, outs[0]):
            np.testing.assert_array_equal(a, e)
    R.riot_batch_destroy(b)
    for ctx in ctxs:
        ctx.close()


def test_batch_rejects_bad_windows(gpu_lib):
    R = gpu_lib
    cfgs = _windows()[:2]
    ctxs, _ = _make(R, cfgs)
    with pytest.raises(R.RiotError):
        R.riot_batch_create([ctxs[0].h, ctxs[0].h], [8, 8], 1)          # same context twice
    with pytest.raises(R.RiotError):
        R.riot_batch_create([ctxs[0].h], [cfgs[0].n + 1], 1)            # k > n
    for ctx in ctxs:
        ctx.close()


def test_window_beyond_the_fp32_range(gpu_lib):
    """F = 16 over 300 steps: the tangent-linear growth squared exceeds the
    FP32 range, so the mixed path forms 2^-c A with a power-of-two c chosen
    at riot_outer_begin.  Its leading eigenvalues must match the FP64 path."""
    R = gpu_lib
    from paper_1906_01413_gb300 import workloads
    cfg = configs.L96Config(name="strong", n=64, F=16.0, T=300, obs_every=4, obs_frac=0.5, obs_layout="random",
                            ell=4.0, k=16, q=1, spinup=300, seed=configs.BASE_SEED + 77)
    lams = {}
    for prec in (R.RIOT_PREC_MIXED, R.RIOT_PREC_FP64):
        ctx, xb, _ = workloads.l96_twin(R, torch, cfg, DEV, prec, cfg.k)
        R.riot_outer_begin(ctx.h, xb)
        lams[prec] = R.riot_rsvd(ctx.h, cfg.k, cfg.q, sketch_stream=3)
        ctx.close()
    lm, l64 = lams[R.RIOT_PREC_MIXED], lams[R.RIOT_PREC_FP64]
    assert l64[0] > 1e39            # beyond what an unscaled FP32 product can hold
    assert np.all(np.isfinite(lm))
    np.testing.assert_allclose(lm[:4], l64[:4], rtol=1e-3)


def test_window_beyond_any_fp32_scaling_is_refused(gpu_lib):
    """F = 16 over 600 steps: the Hessian reaches ~2^390, beyond what one
    power-of-two scaling of FP32 products can hold.  The mixed path must say so
    at riot_outer_begin (RIOT_ENONFINITE) instead of returning garbage; the
    FP64 path handles the window."""
    R = gpu_lib
    from paper_1906_01413_gb300 import workloads
    cfg = configs.L96Config(name="stronger", n=48, F=16.0, T=600, obs_every=8, obs_frac=0.5, obs_layout="random",
                            ell=4.0, k=8, q=1, spinup=300, seed=configs.BASE_SEED + 78)
    ctx, xb, _ = workloads.l96_twin(R, torch, cfg, DEV, R.RIOT_PREC_MIXED, cfg.k)
    with pytest.raises(R.RiotError) as e:
        R.riot_outer_begin(ctx.h, xb)
    assert e.value.status == -8 and "FP64" in str(e.value)
    ctx.close()
    ctx, xb, _ = workloads.l96_twin(R, torch, cfg, DEV, R.RIOT_PREC_FP64, cfg.k)
    R.riot_outer_begin(ctx.h, xb)
    lam = R.riot_rsvd(ctx.h, cfg.k, cfg.q, sketch_stream=3)
    assert np.all(np.isfinite(lam)) and lam[0] > 1e70
    ctx.close()


def _oracle_windows():
    # three uneven windows small enough for the oracle: every chunk width the batch kernel
    # sees below 512 variables, ragged chunks, different T and k
    spec = [(61, 9, 8, 10.0), (150, 30, 48, 9.0), (333, 17, 64, 12.0)]
    return [configs.L96Config(name="ow%d" % i, n=n, F=F, T=T, obs_every=2, obs_frac=0.3, obs_layout="random",
                              ell=4.0, k=k, q=1, spinup=200, seed=configs.BASE_SEED + 700 + i)
            for i, (n, T, k, F) in enumerate(spec)]


def test_batch_kernel_matches_the_oracle(gpu_lib):
    """One graph-captured batch inner loop of three uneven windows (one persistent Hessian
    launch per application) against the FP64 oracle run on the same FP32 sketches.  The FP32
    products' error is of order 2^-24 lambda_1, so by Weyl's inequality the eigenvalues with
    lambda >= 1000 2^-24 lambda_1 are held to the 1e-3 asked of the leading eigenvalues (the
    ones nearer the 2^-24 lambda_1 floor, still kept by the mixed increment, can be off by
    about a percent); the increment of each window, over the pairs it kept, has its cost
    reduction within 1e-3 of that of the oracle's increment restricted to the same pairs
    (second order in the increment's error)."""
    from oracle import problem, riot as orc
    from synth import philox
    R = gpu_lib
    cfgs = _oracle_windows()
    probs = [problem.build(c) for c in cfgs]
    ctxs = []
    for c, p in zip(cfgs, probs):
        ctx = R.Context(n=p.n, T=p.T, dt=p.dt, F=p.F, obs_step=p.obs_step, obs_idx=p.obs_idx, obs_y=p.y,
                        obs_sigma=p.sigma_o, length=c.ell, sigma_b=c.sigma_b, precision=R.RIOT_PREC_MIXED, kmax=c.k)
        R.riot_outer_begin(ctx.h, torch.tensor(p.x_b, device=DEV))
        ctxs.append(ctx)
    b = R.riot_batch_create([ctx.h for ctx in ctxs], [c.k for c in cfgs], 1)
    st = R.riot_batch_run(b, len(cfgs), sketch_stream=configs.STREAM_SKETCH0, use_graph=True)
    assert st == [0] * len(cfgs)
    for c, p, ctx in zip(cfgs, probs, ctxs):
        lam, _, v = _state(R, ctx, c.n, c.k)
        m = R.riot_increment_pairs(ctx.h)
        dv = torch.tensor(v, device=DEV)          # v started at 0: v = the increment
        red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
        # the oracle on the same sketch: seed 0, stream STREAM_SKETCH0, FP32-rounded
        Om = philox.normals(0, configs.STREAM_SKETCH0, c.n * c.k).reshape(c.k, c.n)
        Om = Om.astype(np.float32).astype(np.float64).T
        traj = orc.trajectory(p, p.x_b)
        lo, Uo, _ = orc.rsvd(p, traj, Om, q=1)
        assert m == int(np.sum(lam >= 2.0 ** -24 * lam[0]))
        lead = lo >= 1e3 * 2.0 ** -24 * lo[0]
        assert lead.sum() >= 4
        rel = np.abs(lam[lead] - lo[lead]) / np.abs(lo[lead])
        assert rel.max() <= 1e-3, (c.name, rel.max())
        d = orc.innovation(p, traj)
        g = orc.gradient_b(p, traj, d)
        dvo, mode_o = orc.increment(lo[:m], Uo[:, :m], g)
        z = np.zeros(c.n)
        red_o = orc.quadratic_cost(p, traj, d, z, z) - orc.quadratic_cost(p, traj, d, z, dvo)
        assert abs(red - red_o) <= 1e-3 * abs(red_o), (c.name, red, red_o)
    R.riot_batch_destroy(b)
    for ctx in ctxs:
        ctx.close()
