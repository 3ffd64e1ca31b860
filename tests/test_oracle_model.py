"""Pins for the oracle's Lorenz-96 model, TL and AD (CPU only).

Each test checks the oracle against something other than itself: a closed
form, an invariant of the equations, finite differences, or a published
known-answer vector.
"""
import os

import numpy as np
import pytest

from synth import philox
from oracle import l96

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(np.array(v[:4]), np.array(v[4:6]))
        assert [int(o) for o in out] == v[6:10]


def test_normals_stream_offsets_and_moments():
    z = philox.normals(7, 3, 200003)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    np.testing.assert_array_equal(philox.normals(7, 3, 11, first=5), z[5:16])
    # Box-Muller pairs share the radius: z0^2 + z1^2 = -2 ln u0
    u = philox.uniforms(7, 3, 8)
    np.testing.assert_allclose(z[0] ** 2 + z[1] ** 2, -2 * np.log(u[0]), rtol=1e-13)


def test_choose_indices_distinct_sorted():
    ix = philox.choose_indices(1, 2, 100, 37)
    assert ix.size == 37 and np.all(np.diff(ix) > 0) and ix.min() >= 0 and ix.max() < 100


def test_l96_energy_identity():
    # sum_i x_i (x_{i+1} - x_{i-2}) x_{i-1} telescopes to zero, so
    # sum_i x_i f_i = -sum x_i^2 + F sum x_i.
    rng = np.random.default_rng(0)
    for n in (4, 5, 40, 97):
        x = rng.standard_normal(n) * 3
        f = l96.rhs(x, 8.0)
        assert abs(x @ f - (-(x @ x) + 8.0 * x.sum())) < 1e-12 * (1 + np.abs(x).max() ** 3 * n)


def test_l96_tendency_matches_definition_pointwise():
    rng = np.random.default_rng(1)
    n = 11
    x = rng.standard_normal(n)
    f = l96.rhs(x, 3.5)
    for i in range(n):
        ref = (x[(i + 1) % n] - x[(i - 2) % n]) * x[(i - 1) % n] - x[i] + 3.5
        assert abs(f[i] - ref) < 1e-14


def test_rk4_closed_form_on_uniform_state():
    # A uniform state c obeys dx/dt = F - x, so one RK4 step is
    # x+ = F + (c - F) R(-dt) with R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24.
    F, c, dt = 8.0, 3.25, 0.05
    traj = l96.nl(np.full(9, c), 3, dt, F)
    z = -dt
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    for t in range(4):
        np.testing.assert_allclose(traj[t], F + (c - F) * R ** t, rtol=0, atol=1e-14)


def test_rk4_fourth_order():
    rng = np.random.default_rng(2)
    x0 = 8.0 + rng.standard_normal(20)
    Tt = 0.4
    ref = l96.nl(x0, 1280, Tt / 1280, 8.0)[-1]
    e1 = np.linalg.norm(l96.nl(x0, 20, Tt / 20, 8.0)[-1] - ref)
    e2 = np.linalg.norm(l96.nl(x0, 40, Tt / 40, 8.0)[-1] - ref)
    assert 13.0 < e1 / e2 < 19.0


def _traj(n=30, T=15, dt=0.05, F=8.0, seed=3):
    rng = np.random.default_rng(seed)
    x0 = l96.nl(F + rng.standard_normal(n), 200, dt, F)[-1]
    return l96.nl(x0, T, dt, F), dt, F


def test_tl_taylor():
    traj, dt, F = _traj()
    rng = np.random.default_rng(4)
    dx = rng.standard_normal(traj.shape[1])
    tl = l96.tl(traj, dx, dt, F)[-1]
    prev = None
    for eps in [1e-1, 1e-2, 1e-3, 1e-4, 1e-5]:
        pert = l96.nl(traj[0] + eps * dx, traj.shape[0] - 1, dt, F)[-1]
        ratio = np.linalg.norm(pert - traj[-1]) / np.linalg.norm(eps * tl)
        err = abs(ratio - 1.0)
        if prev is not None and eps >= 1e-4:
            assert err < 0.2 * prev      # |ratio - 1| = O(eps)
        prev = err
    assert prev < 1e-4


def test_tl_matches_central_differences_everywhere():
    traj, dt, F = _traj(n=12, T=6)
    rng = np.random.default_rng(5)
    dx = rng.standard_normal(12)
    eps = 1e-5
    tl = l96.tl(traj, dx, dt, F)
    fp = l96.nl(traj[0] + eps * dx, 6, dt, F)
    fm = l96.nl(traj[0] - eps * dx, 6, dt, F)
    np.testing.assert_allclose(tl, (fp - fm) / (2 * eps), rtol=0, atol=1e-7 * np.abs(tl).max())


@pytest.mark.parametrize("n,T", [(30, 15), (7, 40), (64, 1), (5, 0)])
def test_adjoint_dot_product(n, T):
    traj, dt, F = _traj(n=n, T=T)
    rng = np.random.default_rng(6)
    dx = rng.standard_normal(n)
    forcing = rng.standard_normal((T + 1, n))
    lhs = float(np.sum(l96.tl(traj, dx, dt, F) * forcing))
    rhs = float(dx @ l96.ad(traj, forcing, dt, F))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


def test_adjoint_is_transpose_of_tl_matrix():
    n, T = 9, 4
    traj, dt, F = _traj(n=n, T=T)
    M = np.stack([l96.tl(traj, e, dt, F)[-1] for e in np.eye(n)], axis=1)
    forcing = np.zeros((T + 1, n))
    Mt = np.empty((n, n))
    for j in range(n):
        forcing[-1] = 0
        forcing[-1, j] = 1.0
        Mt[:, j] = l96.ad(traj, forcing, dt, F)
    np.testing.assert_allclose(Mt, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
