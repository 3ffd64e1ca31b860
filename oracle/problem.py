"""Synthetic Lorenz-96 OSSE built in FP64 from the seeded draws (oracle).

Recipe (Section 3.1 experiment, resized to the workloads' N, F, window and
observation network): the truth starts at F + N(0, sd^2) and is spun up on
the attractor; observations are the truth at the observed (step, index)
pairs plus sigma_o N(0, 1) noise; the background is truth + L eps_b.
Test infrastructure only.
"""
import numpy as np

from . import bcov, l96
from .riot import L96Problem


def truth_initial(cfg):
    x = cfg.F + cfg.truth_sd * cfg.truth_perturbation()
    if cfg.spinup > 0:
        x = l96.nl(x, cfg.spinup, cfg.dt, cfg.F)[-1]
    return x


def build(cfg, with_truth=False):
    n = cfg.n
    x_true = truth_initial(cfg)
    traj_true = l96.nl(x_true, cfg.T, cfg.dt, cfg.F)
    st, ix = cfg.obs_layout_arrays()
    p = st.size
    sigma = np.full(p, cfg.sigma_o)
    y = traj_true[st, ix] + sigma * cfg.obs_noise(p)
    L = bcov.bsqrt(n, cfg.ell, cfg.sigma_b)
    x_b = x_true + L @ cfg.background_perturbation()
    prob = L96Problem(n=n, T=cfg.T, dt=cfg.dt, F=cfg.F, obs_step=st, obs_idx=ix, y=y,
                      sigma_o=sigma, L=L, x_b=x_b)
    if with_truth:
        return prob, x_true
    return prob
