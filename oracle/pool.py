"""The oracle's Hessian-vector products over a pool of spawned processes (test infrastructure).

The sketch columns of a product block are independent (Algorithm 3, "do in parallel"), so the
columns of one call are split into chunks and each chunk is applied by ``riot.hvp`` in a worker
process that built the same problem from its seeded description.  Nothing here changes the
arithmetic of a product: every column is computed by the plain FP64 oracle alone.

Workers are started with the ``spawn`` method, so a pool is safe to open after the parent
process has initialised CUDA.
"""
import multiprocessing as mp
import os

import numpy as np

_STATE = {}
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _init(cfg, x_scale, x_seed):
    from . import problem, riot
    prob = problem.build(cfg)
    x = perturbed_state(prob.x_b, x_scale, x_seed)
    _STATE["pt"] = (prob, riot.trajectory(prob, x))


def _apply(cols):
    from . import riot
    prob, traj = _STATE["pt"]
    return riot.hvp(prob, traj, cols)


def perturbed_state(x, scale, seed):
    """x (1 + scale * xi), xi seeded N(0, 1): scale = 2^-52 moves each variable by about one ulp."""
    if scale == 0.0:
        return np.array(x, dtype=np.float64)
    return x * (1.0 + scale * np.random.default_rng(seed).standard_normal(x.size))


class HvpPool:
    """``with HvpPool(cfg, workers) as pool: Y = pool.apply(W)`` for W (n, m)."""

    def __init__(self, cfg, workers=None, x_scale=0.0, x_seed=7):
        self.workers = workers or max(1, len(os.sched_getaffinity(0)))
        # one BLAS thread per worker: the children read these when they start
        saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        os.environ.update({k: "1" for k in _THREAD_VARS})
        try:
            self._pool = mp.get_context("spawn").Pool(self.workers, initializer=_init,
                                                      initargs=(cfg, x_scale, x_seed))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def apply(self, W):
        W = np.asarray(W, dtype=np.float64)
        chunks = [c for c in np.array_split(np.arange(W.shape[1]), 4 * self.workers) if c.size]
        parts = self._pool.map(_apply, [np.ascontiguousarray(W[:, c]) for c in chunks])
        return np.concatenate(parts, axis=1)

    def close(self):
        self._pool.close()
        self._pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self._pool.terminate()
        self._pool.join()
