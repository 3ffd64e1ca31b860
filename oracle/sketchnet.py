"""FP64 oracle of the learned sketch proposal (test infrastructure only).

A small periodic 1-D convolutional network maps snapshots of the background
trajectory of a Lorenz-96 window to m proposed sketch directions; it is
trained on the leading Hessian eigenvectors that RIOT itself produced for
other windows (the paper's sketch is purely Gaussian, Algorithm 3; this is an
extension of its randomized range finder, Section 2.2, with the Gaussian
sketch kept as the fallback that decides).

Network (all layers periodic in the ring index i, kernel width K = 2h + 1):
  h_0 = input (C_in, n)
  h_l = tanh(conv(h_{l-1}; W_l, b_l)),  l = 1 .. L-1
  Z   = conv(h_{L-1}; W_L, b_L)                         (m, n): m directions
  conv(x; W, b)[o, i] = b[o] + sum_c sum_d W[o, c, d] x[c, (i + d - h) mod n]

Loss for one window with target eigenvectors U (n, r), orthonormal columns,
on the directions as columns X = Z^T (n, m):
  L1 = ||X - U U^T X||_F^2 / ||X||_F^2          (energy outside span U)
  S  = X^T X / s,  s = ||X||_F^2 / m             (scale-free Gram)
  L2 = ||S - I||_F^2 / m^2                       (keeps the directions apart)
  L  = L1 + mu L2,   averaged over the windows of a batch.
Optimiser: Adam (Kingma & Ba) with bias correction.

Inputs: C_in snapshots of the trajectory at steps floor(j T / C_in),
j = 0 .. C_in - 1, standardised by their common mean and standard deviation.
"""
import numpy as np


def layer_shapes(c_in, width, m, depth=4, ksize=5):
    chans = [c_in] + [width] * (depth - 1) + [m]
    return [(chans[l + 1], chans[l], ksize) for l in range(depth)]


def init_params(c_in, width, m, seed, depth=4, ksize=5):
    """Glorot-uniform weights from a numpy generator seeded with `seed`, zero biases.
    Returns a list of (W, b) pairs."""
    rng = np.random.default_rng(seed)
    params = []
    for (co, ci, k) in layer_shapes(c_in, width, m, depth, ksize):
        lim = np.sqrt(6.0 / (ci * k + co * k))
        params.append((rng.uniform(-lim, lim, (co, ci, k)), np.zeros(co)))
    return params


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflatten(vec, shapes):
    out, o = [], 0
    for (co, ci, k) in shapes:
        W = vec[o:o + co * ci * k].reshape(co, ci, k)
        o += co * ci * k
        b = vec[o:o + co]
        o += co
        out.append((W, b))
    return out


def conv(x, W, b):
    """Periodic conv: x (C_in, n), W (C_out, C_in, K), b (C_out,) -> (C_out, n)."""
    K = W.shape[2]
    h = K // 2
    out = np.zeros((W.shape[0], x.shape[1])) + b[:, None]
    for d in range(K):
        out += W[:, :, d] @ np.roll(x, -(d - h), axis=1)
    return out


def conv_backward(x, W, gout):
    """Gradients of conv w.r.t. its input, weights and bias given d(out) = gout."""
    K = W.shape[2]
    h = K // 2
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for d in range(K):
        xs = np.roll(x, -(d - h), axis=1)            # xs[c, i] = x[c, i + d - h]
        gW[:, :, d] = gout @ xs.T
        gx += np.roll(W[:, :, d].T @ gout, d - h, axis=1)
    return gx, gW, gout.sum(axis=1)


def forward(params, x):
    """Returns (Z (m, n), activations list [h_0, ..., h_{L-1}])."""
    acts = [x]
    h = x
    for l, (W, b) in enumerate(params):
        z = conv(h, W, b)
        if l < len(params) - 1:
            h = np.tanh(z)
            acts.append(h)
        else:
            h = z
    return h, acts


def loss_and_grad_z(Z, U, mu):
    """L and dL/dZ for one window (Z (m, n), U (n, r))."""
    X = Z.T
    m = X.shape[1]
    R = X - U @ (U.T @ X)
    b = float(np.sum(X * X))
    L1 = float(np.sum(R * R)) / b
    s = b / m
    S = X.T @ X / s
    E = S - np.eye(m)
    L2 = float(np.sum(E * E)) / (m * m)
    gX1 = (2.0 * R - 2.0 * L1 * X) / b
    trES = float(np.sum(E * S))
    gX2 = (4.0 / (m * m * s)) * (X @ E - (trES / m) * X)
    return L1 + mu * L2, (gX1 + mu * gX2).T, (L1, L2)


def backward(params, acts, gZ):
    """Parameter gradients from dL/dZ by the chain rule through the layers."""
    grads = [None] * len(params)
    g = gZ
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        gx, gW, gb = conv_backward(acts[l], W, g)
        grads[l] = (gW, gb)
        if l > 0:
            g = gx * (1.0 - acts[l] * acts[l])        # through tanh of layer l-1's output
    return grads


def batch_loss_grad(params, xs, Us, mu):
    """Mean loss and gradients over a batch of windows."""
    tot = 0.0
    acc = None
    for x, U in zip(xs, Us):
        Z, acts = forward(params, x)
        L, gZ, _ = loss_and_grad_z(Z, U, mu)
        g = backward(params, acts, gZ)
        tot += L
        acc = g if acc is None else [(a[0] + c[0], a[1] + c[1]) for a, c in zip(acc, g)]
    nb = len(xs)
    return tot / nb, [(gW / nb, gb / nb) for gW, gb in acc]


class Adam:
    def __init__(self, nparams, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(nparams)
        self.v = np.zeros(nparams)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, p, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return p - self.lr * mh / (np.sqrt(vh) + self.eps)


def snapshot_input(traj, c_in):
    """C_in standardised snapshots of a trajectory (T+1, n) at steps floor(j T / C_in)."""
    T = traj.shape[0] - 1
    idx = [(j * T) // c_in for j in range(c_in)]
    x = traj[idx]
    return (x - x.mean()) / x.std()


def rayleigh_residual(Q, AQ):
    """rho = ||AQ - Q (Q^T A Q)||_F / ||AQ||_F for Q with orthonormal columns."""
    R = AQ - Q @ (Q.T @ AQ)
    return float(np.linalg.norm(R) / np.linalg.norm(AQ))
