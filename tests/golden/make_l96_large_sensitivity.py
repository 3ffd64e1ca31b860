"""Write l96_large_sensitivity.json: how far the FP64 answer of the large Lorenz-96 window
(n = 4096, T = 200, k = 512, q = 1) moves when the initial state moves by about one ulp.

Two runs of the FP64 oracle (Algorithm 3: sketch, Y = A Omega, one power iteration,
Householder QR, K, LAPACK eigh, Ritz vectors, adaptive increment; Eq. 3 for the cost) on the
same sketch, one at x_b and one at x_b (1 + 2^-52 xi), xi seeded N(0, 1).  Any two correct
FP64 programs differ at least this much (their roundings differ at every step, not once), so
the spreads recorded here are the scale of the tolerances of the large-window parity tests.
Calls only the oracle.  Takes about two minutes on eight cores:

    python tests/golden/make_l96_large_sensitivity.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import problem, riot as orc  # noqa: E402
from oracle.pool import HvpPool, perturbed_state  # noqa: E402
from synth import configs  # noqa: E402

SCALE = 2.0 ** -52
SEED = 7
PRODUCT_COLS = 16


def run(cfg, prob, scale):
    x = perturbed_state(prob.x_b, scale, SEED)
    traj = orc.trajectory(prob, x)
    d = orc.innovation(prob, traj)
    g = orc.gradient_b(prob, traj, d)
    with HvpPool(cfg, x_scale=scale, x_seed=SEED) as pool:
        Y16 = pool.apply(cfg.sketch(5, k=PRODUCT_COLS).T)
        lam, U, _ = orc.rsvd(prob, traj, cfg.sketch(0).T, q=cfg.q, apply=pool.apply)
    dv, mode = orc.increment(lam, U, g)
    z = np.zeros(prob.n)
    red = orc.quadratic_cost(prob, traj, d, z, z) - orc.quadratic_cost(prob, traj, d, z, dv)
    return {"traj_end": traj[-1], "Y16": Y16, "lam": lam, "dv": dv, "mode": int(mode), "reduction": red}


def main():
    cfg = configs.l96_large()
    prob = problem.build(cfg)
    a = run(cfg, prob, 0.0)
    b = run(cfg, prob, SCALE)
    rel = lambda u, v: float(np.linalg.norm(u - v) / np.linalg.norm(u))
    out = {
        "workload": "l96_n4096_F8_T200_obs25pct_every4_k512_q1 (sketch of outer loop 0; products: sketch 5, 16 columns)",
        "perturbation": "x_b * (1 + 2^-52 xi), xi = numpy default_rng(7) N(0, 1)",
        "traj_end_rel_spread": rel(a["traj_end"], b["traj_end"]),
        "hvp_col_rel_spread": [rel(a["Y16"][:, j], b["Y16"][:, j]) for j in range(PRODUCT_COLS)],
        "eig_rel_spread": [float(v) for v in np.abs(a["lam"] - b["lam"]) / np.abs(a["lam"])],
        "dv_rel_spread": rel(a["dv"], b["dv"]),
        "reduction": [a["reduction"], b["reduction"]],
        "reduction_rel_spread": abs(a["reduction"] - b["reduction"]) / abs(a["reduction"]),
        "modes": [a["mode"], b["mode"]],
        "lambda_1": float(a["lam"][0]),
        "lambda_k": float(a["lam"][-1]),
    }
    with open(os.path.join(HERE, "l96_large_sensitivity.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print({k: v for k, v in out.items() if not isinstance(v, list)})


if __name__ == "__main__":
    main()
