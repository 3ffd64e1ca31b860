"""Seeded synthetic workloads shaped like the paper's Lorenz-96 experiments.

Each workload is a plain description (sizes, physical parameters, seeds) plus
the raw random draws that the experiment needs.  Turning the draws into a
truth trajectory, observations and a background (which needs the model and
the prior square root) is done by whoever consumes them: the FP64 oracle in
tests, the CUDA library in the benchmark.

Stream numbers used with ``synth.philox`` (one independent stream each):
  1 truth perturbation, 2 observed indices, 3 observation noise,
  4 background perturbation, 16 + j the sketch of outer iteration j.
"""
from dataclasses import dataclass, field

import numpy as np

from . import philox

BASE_SEED = 20190604
STREAM_TRUTH = 1
STREAM_OBS_IDX = 2
STREAM_OBS_NOISE = 3
STREAM_BKG = 4
STREAM_SKETCH0 = 16


@dataclass
class L96Config:
    name: str
    n: int
    F: float = 8.0
    dt: float = 0.05
    T: int = 20
    spinup: int = 1000
    truth_sd: float = 0.1          # x0 = F + N(0, 0.01): variance 0.01
    obs_every: int = 1             # observation steps: obs_every, 2*obs_every, ..., T
    obs_frac: float = 0.5          # fraction of variables observed
    obs_layout: str = "even"       # "even": indices 0,2,4,...; "random": fixed random subset
    sigma_o: float = 1.0
    sigma_b: float = 1.0
    ell: float = 2.0               # Gaussian correlation length (grid cells)
    k: int = 40                    # sketch columns
    q: int = 0                     # power iterations
    outer: int = 3
    seed: int = BASE_SEED
    extra: dict = field(default_factory=dict)

    # -- raw draws -------------------------------------------------------------
    def truth_perturbation(self):
        return philox.normals(self.seed, STREAM_TRUTH, self.n)

    def obs_indices(self):
        m = max(1, int(round(self.obs_frac * self.n)))
        if self.obs_layout == "even":
            return np.arange(0, self.n, 2, dtype=np.int64)[:m]
        return philox.choose_indices(self.seed, STREAM_OBS_IDX, self.n, m)

    def obs_steps(self):
        return np.arange(self.obs_every, self.T + 1, self.obs_every, dtype=np.int64)

    def obs_layout_arrays(self):
        """(step, idx) of every observation, sorted by step then index."""
        steps = self.obs_steps()
        idx = self.obs_indices()
        st = np.repeat(steps, idx.size)
        ix = np.tile(idx, steps.size)
        return st, ix

    def obs_noise(self, p):
        return philox.normals(self.seed, STREAM_OBS_NOISE, p)

    def background_perturbation(self):
        return philox.normals(self.seed, STREAM_BKG, self.n)

    def sketch(self, outer_iter, k=None, n=None):
        """Gaussian sketch, column-major (k columns of length n), float64."""
        k = self.k if k is None else k
        n = self.n if n is None else n
        z = philox.normals(self.seed, STREAM_SKETCH0 + outer_iter, k * n)
        return z.reshape(k, n)   # row j = column j of Omega


def l96_small():
    """Lorenz-96 N=40, F=8, dt=0.05, 20-step window, every 2nd variable
    observed at every step, sigma_o=1, Gaussian B (sigma_b=1, length 2),
    full-rank sketch k=40, q=0, 3 outer loops, FP64 throughout."""
    return L96Config(name="l96_n40_T20_k40", n=40, T=20, obs_every=1, obs_frac=0.5,
                     obs_layout="even", ell=2.0, k=40, q=0, outer=3)


def l96_large():
    """Lorenz-96 N=4096, F=8, dt=0.05, 200-step window, 25% of variables at
    fixed random indices observed every 4 steps, sigma_o=1, Gaussian B
    (sigma_b=1, length 4), k=512 Gaussian sketch columns, q=1, 5 outer loops."""
    return L96Config(name="l96_n4096_T200_k512", n=4096, T=200, obs_every=4, obs_frac=0.25,
                     obs_layout="random", ell=4.0, k=512, q=1, outer=5)


def l96_custom(name, n, T, obs_every, obs_frac, ell, k, q, F=8.0, outer=1,
               obs_layout="random", spinup=1000, seed=BASE_SEED):
    return L96Config(name=name, n=n, F=F, T=T, obs_every=obs_every, obs_frac=obs_frac,
                     obs_layout=obs_layout, ell=ell, k=k, q=q, outer=outer,
                     spinup=spinup, seed=seed)


STREAM_BATCH = 10


def batch_windows(nwin=96, seed=BASE_SEED, n_max=8192):
    """Independent Lorenz-96 windows of uneven size for batched inner loops:
    n log-uniform in [40, n_max], F uniform in [8, 16], T uniform in
    {50, ..., 300}, k drawn from {16, 64, 128, 256, 512} and clipped to n,
    observation density uniform in [0.1, 0.5] at fixed random indices every 4
    steps, Gaussian B (sigma_b = 1, length 4), q = 1.  Window w draws its own
    truth, observations and background from seed + 1000 + w."""
    u = philox.uniforms(seed, STREAM_BATCH, 5 * nwin).reshape(nwin, 5)
    ks = np.array([16, 64, 128, 256, 512])
    out = []
    for w in range(nwin):
        n = int(round(np.exp(np.log(40.0) + u[w, 0] * (np.log(n_max) - np.log(40.0)))))
        n = min(max(n, 40), n_max)
        F = 8.0 + 8.0 * u[w, 1]
        T = 50 + int(u[w, 2] * 251)
        k = int(min(ks[min(int(u[w, 3] * 5), 4)], n))
        frac = 0.1 + 0.4 * u[w, 4]
        out.append(L96Config(name="batch_w%02d_n%d_T%d_k%d" % (w, n, T, k), n=n, F=F, T=min(T, 300), obs_every=4,
                             obs_frac=frac, obs_layout="random", ell=4.0, k=k, q=1, outer=1,
                             seed=seed + 1000 + w))
    return out
