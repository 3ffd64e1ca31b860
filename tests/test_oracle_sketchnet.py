"""Pins of the FP64 learned-sketch oracle: finite differences for every
gradient, the adjoint identity of the periodic convolution, translation
equivariance of the network, the loss at its closed-form extremes, Adam on a
quadratic, and the Rayleigh residual of an invariant subspace."""
import numpy as np
import pytest

from oracle import sketchnet as N


def _net(seed=0, c_in=3, width=4, m=3, n=16):
    params = N.init_params(c_in, width, m, seed)
    rng = np.random.default_rng(seed + 1)
    x = rng.standard_normal((c_in, n))
    U, _ = np.linalg.qr(rng.standard_normal((n, 2)))
    return params, x, U


def test_conv_backward_is_the_adjoint_of_conv():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 11))
    W = rng.standard_normal((5, 3, 5))
    b = np.zeros(5)
    g = rng.standard_normal((5, 11))
    gx, gW, _ = N.conv_backward(x, W, g)
    assert np.sum(N.conv(x, W, b) * g) == pytest.approx(np.sum(x * gx), rel=1e-12)
    assert np.sum(N.conv(x, W, b) * g) == pytest.approx(np.sum(W * gW), rel=1e-12)


def test_network_is_translation_equivariant():
    params, x, _ = _net()
    Z, _ = N.forward(params, x)
    Z3, _ = N.forward(params, np.roll(x, 3, axis=1))
    np.testing.assert_allclose(Z3, np.roll(Z, 3, axis=1), rtol=1e-12, atol=1e-12)


def test_loss_extremes():
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((20, 4)))
    # directions inside span U, mutually orthogonal with equal norms: both terms vanish
    L, _, (L1, L2) = N.loss_and_grad_z((U[:, :3] * 2.0).T, U, mu=1.0)
    assert L1 == pytest.approx(0.0, abs=1e-15) and L2 == pytest.approx(0.0, abs=1e-15)
    # directions orthogonal to span U: all energy outside
    V = np.linalg.qr(np.concatenate([U, rng.standard_normal((20, 3))], axis=1))[0][:, 4:]
    L, _, (L1, _) = N.loss_and_grad_z(V.T, U, mu=0.0)
    assert L1 == pytest.approx(1.0, rel=1e-12)
    # one unit direction repeated m times: s = 1, S is all ones, ||S - I||^2 = m^2 - m
    m = 3
    Z = np.tile(U[:, 0], (m, 1))
    _, _, (_, L2) = N.loss_and_grad_z(Z, U, mu=1.0)
    assert L2 == pytest.approx((m * m - m) / (m * m), rel=1e-12)


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    U, _ = np.linalg.qr(rng.standard_normal((12, 3)))
    Z = rng.standard_normal((4, 12))
    L, gZ, _ = N.loss_and_grad_z(Z, U, mu=0.7)
    for _ in range(10):
        i, j = rng.integers(0, 4), rng.integers(0, 12)
        E = np.zeros_like(Z)
        E[i, j] = 1e-6
        fd = (N.loss_and_grad_z(Z + E, U, 0.7)[0] - N.loss_and_grad_z(Z - E, U, 0.7)[0]) / 2e-6
        assert fd == pytest.approx(gZ[i, j], rel=1e-6, abs=1e-9)


def test_parameter_gradients_match_finite_differences():
    params, x, U = _net(seed=5)
    rng = np.random.default_rng(6)
    x2 = rng.standard_normal(x.shape)
    U2, _ = np.linalg.qr(rng.standard_normal(U.shape))
    shapes = [W.shape for W, _ in params]
    mu = 0.5
    L, grads = N.batch_loss_grad(params, [x, x2], [U, U2], mu)
    p = N.flatten(params)
    g = N.flatten(grads)
    for idx in rng.choice(p.size, 25, replace=False):
        e = np.zeros_like(p)
        e[idx] = 1e-6
        Lp = N.batch_loss_grad(N.unflatten(p + e, shapes), [x, x2], [U, U2], mu)[0]
        Lm = N.batch_loss_grad(N.unflatten(p - e, shapes), [x, x2], [U, U2], mu)[0]
        fd = (Lp - Lm) / 2e-6
        assert fd == pytest.approx(g[idx], rel=1e-6, abs=1e-9), idx


def test_adam_minimises_a_quadratic():
    rng = np.random.default_rng(7)
    D = np.diag(rng.uniform(0.5, 3.0, 6))
    target = rng.standard_normal(6)
    p = np.zeros(6)
    opt = N.Adam(6, lr=0.05)
    for _ in range(2000):
        p = opt.step(p, 2 * D @ (p - target))
    np.testing.assert_allclose(p, target, atol=1e-3)


def test_rayleigh_residual():
    rng = np.random.default_rng(8)
    M = rng.standard_normal((15, 15))
    A = M @ M.T
    w, V = np.linalg.eigh(A)
    Q = V[:, -4:]
    assert N.rayleigh_residual(Q, A @ Q) < 1e-12
    # a rotated basis of the same invariant subspace still has rho = 0
    Rq, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    assert N.rayleigh_residual(Q @ Rq, A @ Q @ Rq) < 1e-12
    # two eigenvectors mixed at 45 degrees, eigenvalues a, c: rho^2 = (a - c)^2 / (2 (a^2 + c^2))
    q = (V[:, -1] + V[:, 0]) / np.sqrt(2)
    a, c = w[-1], w[0]
    want = np.sqrt((a - c) ** 2 / (2 * (a * a + c * c)))
    assert N.rayleigh_residual(q[:, None], (A @ q)[:, None]) == pytest.approx(want, rel=1e-10)


def test_snapshot_input_is_standardised():
    traj = np.random.default_rng(9).standard_normal((21, 10)) * 3 + 2
    x = N.snapshot_input(traj, 4)
    assert x.shape == (4, 10)
    assert abs(x.mean()) < 1e-12 and x.std() == pytest.approx(1.0)
    np.testing.assert_allclose(x[1], (traj[5] - traj[[0, 5, 10, 15]].mean()) / traj[[0, 5, 10, 15]].std())
