"""Seeded initial weights of the learned sketch network (random draws only).

Glorot-uniform weights U(-l, l), l = sqrt(6 / ((C_in + C_out) K)), and zero
biases, laid out as the network's flat parameter vector: per layer
W[C_out][C_in][K] then b[C_out].  Drawn from Philox stream 11.
"""
import numpy as np

from . import philox
from .configs import BASE_SEED

STREAM_NET_INIT = 11


def initial_params(c_in, width, m, depth=4, ksize=5, seed=BASE_SEED):
    chans = [c_in] + [width] * (depth - 1) + [m]
    sizes = [(chans[l + 1], chans[l]) for l in range(depth)]
    total_w = sum(co * ci * ksize for co, ci in sizes)
    u = philox.uniforms(seed, STREAM_NET_INIT, total_w)
    out, o = [], 0
    for co, ci in sizes:
        lim = np.sqrt(6.0 / ((ci + co) * ksize))
        cnt = co * ci * ksize
        out.append(lim * (2.0 * u[o:o + cnt] - 1.0))
        out.append(np.zeros(co))
        o += cnt
    return np.concatenate(out)
