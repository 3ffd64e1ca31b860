"""Synthetic twin experiments built on the GPU with the library itself.

Helpers for benchmarks and tests: they turn a seeded workload description
(``synth``) into a ready context by running the library's own forecasts (a
truth, its observations plus noise, a background).  No oracle code is used.
"""
import numpy as np

from synth import advdiff as bc_synth


def l96_twin(R, torch, cfg, dev, precision, kmax):
    """Lorenz-96: truth spun up on the attractor, observations of the truth
    plus noise, background = truth + L eps_b.  Returns (context, x_b, p)."""
    n, T = cfg.n, cfg.T
    x_init = torch.tensor(cfg.F + cfg.truth_sd * cfg.truth_perturbation(), device=dev)
    x0 = torch.empty(n, dtype=torch.float64, device=dev)
    R.riot_l96_forecast(n, cfg.spinup, cfg.dt, cfg.F, x_init, x0, store_all=False)
    traj = torch.empty(T + 1, n, dtype=torch.float64, device=dev)
    R.riot_l96_forecast(n, T, cfg.dt, cfg.F, x0, traj)
    st, ix = cfg.obs_layout_arrays()
    sig = np.full(st.size, cfg.sigma_o)
    y = traj[torch.tensor(st, device=dev), torch.tensor(ix, device=dev)].cpu().numpy() + sig * cfg.obs_noise(st.size)
    ctx = R.Context(n=n, T=T, dt=cfg.dt, F=cfg.F, obs_step=st, obs_idx=ix, obs_y=y, obs_sigma=sig,
                    length=cfg.ell, sigma_b=cfg.sigma_b, precision=precision, kmax=kmax, seed=cfg.seed)
    eps = torch.tensor(cfg.background_perturbation(), device=dev)
    xb = torch.empty(n, dtype=torch.float64, device=dev)
    R.riot_bsqrt_apply(ctx.h, eps, xb)
    xb += x0
    return ctx, xb, st.size


def bc_twin(R, torch, cfg, dev, precision, kmax):
    """Tracer-transport inversion: observations of the truth (x = 0, E = E_b)
    from an FP64 forecast, sigma_o = 20 % of the value with a floor of 5 % of
    the median, background x_b = L eps_b.  Returns (context, x_b, p)."""
    n = cfg.n
    u, v = cfg.winds()
    step, pos = cfg.tracks()
    p = int(step.size)
    common = dict(nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, nblocks=cfg.nblocks, T=cfg.T, dt=cfg.dt, dx=cfg.dx, dy=cfg.dy,
                  dz=cfg.dz, u=u, v=v, amp=cfg.amplitude(), kz=cfg.kz(), emis_b=cfg.background_emissions(),
                  obs_step=step, obs_pos=pos, length=cfg.ell, sigma_b=cfg.sigma_b)
    c0 = R.Context(obs_y=np.zeros(p), obs_sigma=np.ones(p), precision=R.RIOT_PREC_FP64, kmax=1, **common)
    R.riot_outer_begin(c0.h, torch.zeros(n, dtype=torch.float64, device=dev))
    d = torch.empty(p, dtype=torch.float64, device=dev)
    R.riot_get_innovation(c0.h, d)
    y_true = d.cpu().numpy()
    sig = cfg.obs_rel * np.maximum(y_true, cfg.obs_floor_frac * np.median(y_true))
    y = y_true + sig * cfg.obs_noise(p)
    eps = torch.tensor(cfg.background_perturbation(), device=dev)
    xb = torch.empty_like(eps)
    R.riot_bsqrt_apply(c0.h, eps, xb)
    c0.close()
    ctx = R.Context(obs_y=y, obs_sigma=sig, precision=precision, kmax=kmax, seed=cfg.seed, **common)
    return ctx, xb, p


__all__ = ["l96_twin", "bc_twin", "bc_synth"]
