"""Write bc_large_products.json: FP64 oracle Hessian-vector products on the full tracer grid
(192 x 192 x 30 cells, 240 steps, 4 emission blocks: n = 147 456 controls, 8000 observations
along 20 tracks) of two sketch columns, and of the same columns rounded to FP32 (the input of
the mixed-precision path), sampled at 512 seeded positions per column, with their norms.

The window is the large tracer workload with sigma_o = 1 for every observation (the Hessian
A = L^T H'^T R^-1 H' L does not depend on y, and with unit sigma_o it needs no truth run), at
the control x = x_b = L eps_b; the sketch columns are Philox stream 16 of the workload seed.
Calls only the oracle (about ten minutes on one core):

    python tests/golden/make_bc_large_products.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import advdiff as A  # noqa: E402
from synth import advdiff as S  # noqa: E402
from synth import philox  # noqa: E402

COLS = 2
SAMPLES = 512
SAMPLE_STREAM = 99


def problem(cfg):
    """The large tracer window with unit observation errors (no truth run)."""
    m = A.model_from_config(cfg)
    step, pos = cfg.tracks()
    obs = A.make_obs(m, step, pos)
    p = step.size
    Lop = A.exp_separable_sqrt(cfg.nx, cfg.ny, cfg.nblocks, cfg.dx, cfg.dy, cfg.ell, cfg.sigma_b)
    x_b = Lop.apply(cfg.background_perturbation())
    return A.AdvDiffProblem(m=m, obs=obs, y=np.zeros(p), sigma_o=np.ones(p), Lop=Lop, x_b=x_b)


def main():
    cfg = S.bc_large()
    prob = problem(cfg)
    traj = {"E": A.emissions(prob, prob.x_b)}          # the Hessian needs only E = E_b exp(x)
    W = cfg.sketch(0, k=COLS)                          # (COLS, n)
    W32 = W.astype(np.float32).astype(np.float64)
    Y = A.hvp(prob, traj, np.concatenate([W, W32]).T).T   # (2 COLS, n)
    idx = np.sort(philox.choose_indices(cfg.seed, SAMPLE_STREAM, prob.n, SAMPLES))
    out = {"workload": cfg.name + " with sigma_o = 1, x = x_b, sketch stream 16 (outer iteration 0)",
           "n": int(prob.n), "p": int(prob.p), "columns": COLS, "sample_stream": SAMPLE_STREAM,
           "sample_index": [int(i) for i in idx],
           "norm": [float(np.linalg.norm(Y[j])) for j in range(COLS)],
           "values": [[float(v) for v in Y[j, idx]] for j in range(COLS)],
           "norm_f32_input": [float(np.linalg.norm(Y[COLS + j])) for j in range(COLS)],
           "values_f32_input": [[float(v) for v in Y[COLS + j, idx]] for j in range(COLS)]}
    with open(os.path.join(HERE, "bc_large_products.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")
    print("norms", out["norm"])


if __name__ == "__main__":
    main()
