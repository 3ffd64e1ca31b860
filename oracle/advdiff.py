"""FP64 oracle of the black-carbon-style source inversion (test infrastructure only).

The paper's large experiments (Section 3.2) invert surface black-carbon
emissions with a chemical transport model and aircraft observations.  This
module restates that setting on a synthetic linear tracer model, written
plainly in numpy and vectorised over sketch columns:

  * grid: nx x ny x nz cells, x periodic, solid walls in y, zero flux at the
    bottom and top; cell (i, j, l) centred at (i, j, l) in cell units;
  * transport dc/dt = A c + s: first-order upwind advection in flux form by
    the steady horizontal face winds amp(l) * (u, v), plus vertical diffusion
    with diffusivity Kz on the interior faces; s is the surface source
    E / dz in the bottom layer;
  * time stepping: classical RK4 with the source held for the whole step;
  * emissions E = E_b exp(x) with the control x the log scaling of each
    surface cell in each emission block (step t uses block t * nb // T);
  * observations: trilinear interpolation of the tracer at (x, y, z) at the
    end of step `step` (periodic in x);
  * prior: B = L L^T with L = sigma_b (S_y kron S_x) per block, S the
    symmetric square roots of exponential correlations exp(-d / ell)
    (periodic distance in x).

The tangent-linear model is the same linear transport driven by
dE = E dx; the adjoint is written out as the reverse-mode transpose of each
flux and RK4 stage (not as a second forward model), so that the dot-product
test pins it.  The RIOT linear algebra (randomized eigendecomposition,
adaptive increment, covariance) is the generic code of ``oracle.riot``.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class AdvDiffModel:
    nx: int
    ny: int
    nz: int
    nb: int
    T: int
    dt: float
    dx: float
    dy: float
    dz: float
    u: np.ndarray      # (ny, nx)    x-face i-1/2 of row j, amplitude 1
    v: np.ndarray      # (ny+1, nx)  y-face j-1/2 of column i (rows 0, ny: walls)
    amp: np.ndarray    # (nz,)       level scaling of the winds
    kz: np.ndarray     # (nz+1,)     diffusivity at face l-1/2 (ends unused)
    Eb: np.ndarray     # (nb, ny, nx) background emissions

    def block(self, t):
        return (t * self.nb) // self.T


def model_from_config(cfg):
    u, v = cfg.winds()
    return AdvDiffModel(nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, nb=cfg.nblocks, T=cfg.T, dt=cfg.dt,
                        dx=cfg.dx, dy=cfg.dy, dz=cfg.dz, u=u, v=v, amp=cfg.amplitude(), kz=cfg.kz(),
                        Eb=cfg.background_emissions())


# --- transport operator ---------------------------------------------------------------

def _face_winds(m):
    a = m.amp[:, None, None]
    return a * m.u[None], a * m.v[None]


def tendency(m, c):
    """A c for c of shape (..., nz, ny, nx): upwind flux-form advection plus
    vertical diffusion, no source."""
    U, V = _face_winds(m)
    # x: flux through face i-1/2 takes the upwind cell (i-1 when U > 0, i when U < 0)
    fx = np.maximum(U, 0.0) * np.roll(c, 1, axis=-1) + np.minimum(U, 0.0) * c
    out = -(np.roll(fx, -1, axis=-1) - fx) / m.dx
    # y: faces j-1/2, j = 0..ny; no tracer beyond the walls
    zrow = np.zeros(c.shape[:-2] + (1, m.nx))
    cS = np.concatenate([zrow, c], axis=-2)          # cell j-1 for face j
    cN = np.concatenate([c, zrow], axis=-2)          # cell j for face j
    fy = np.maximum(V, 0.0) * cS + np.minimum(V, 0.0) * cN
    out = out - (fy[..., 1:, :] - fy[..., :-1, :]) / m.dy
    # z: diffusive flux through face l-1/2 = -Kz (c_l - c_{l-1}) / dz, zero at the ends
    K = m.kz[1:m.nz][:, None, None]
    fz = -K * (c[..., 1:, :, :] - c[..., :-1, :, :]) / m.dz        # faces 1..nz-1
    zl = np.zeros(c.shape[:-3] + (1, m.ny, m.nx))
    fz = np.concatenate([zl, fz, zl], axis=-3)                      # faces 0..nz
    out = out - (fz[..., 1:, :, :] - fz[..., :-1, :, :]) / m.dz
    return out


def tendency_adj(m, g):
    """A^T g: the reverse-mode transpose of `tendency`, operation by operation."""
    U, V = _face_winds(m)
    cb = np.zeros_like(g)
    # z part: out -= (fz[l+1] - fz[l]) / dz  ->  fz_bar[l] = (g[l] - g[l-1]) / dz
    zl = np.zeros(g.shape[:-3] + (1, m.ny, m.nx))
    gp = np.concatenate([zl, g, zl], axis=-3)                       # g[-1] = g[nz] = 0
    fzb = (gp[..., 1:, :, :] - gp[..., :-1, :, :]) / m.dz            # faces 0..nz
    fzb_in = fzb[..., 1:m.nz, :, :]                                  # faces 1..nz-1
    K = m.kz[1:m.nz][:, None, None]
    # fz[l] = -K (c_l - c_{l-1}) / dz
    t = -K * fzb_in / m.dz
    cb[..., 1:, :, :] += t
    cb[..., :-1, :, :] -= t
    # y part: out -= (fy[j+1] - fy[j]) / dy
    zrow = np.zeros(g.shape[:-2] + (1, m.nx))
    gpy = np.concatenate([zrow, g, zrow], axis=-2)                  # g[-1] = g[ny] = 0
    fyb = (gpy[..., 1:, :] - gpy[..., :-1, :]) / m.dy                # faces 0..ny
    cSb = np.maximum(V, 0.0) * fyb                                  # d fy / d cS
    cNb = np.minimum(V, 0.0) * fyb                                  # d fy / d cN
    cb += cSb[..., 1:, :]                                           # cS[j] = c[j-1]
    cb += cNb[..., :-1, :]                                          # cN[j] = c[j]
    # x part: out = -(fx[i+1] - fx[i]) / dx  ->  fx_bar[i] = (g[i] - g[i-1]) / dx
    fxb = (g - np.roll(g, 1, axis=-1)) / m.dx
    cb += np.roll(np.maximum(U, 0.0) * fxb, -1, axis=-1)            # fx[i] uses c[i-1]
    cb += np.minimum(U, 0.0) * fxb
    return cb


def _with_source(m, k, s):
    if s is not None:
        k = k.copy()
        k[..., 0, :, :] += s
    return k


def rk4_step(m, c, s=None):
    """One classical RK4 step of dc/dt = A c + s (s: surface source (..., ny, nx) or None)."""
    h = m.dt
    k1 = _with_source(m, tendency(m, c), s)
    k2 = _with_source(m, tendency(m, c + 0.5 * h * k1), s)
    k3 = _with_source(m, tendency(m, c + 0.5 * h * k2), s)
    k4 = _with_source(m, tendency(m, c + h * k3), s)
    return c + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def rk4_step_adj(m, lam):
    """Reverse mode of `rk4_step` at the adjoint lam of its output.
    Returns (adjoint of c, adjoint of the surface source s)."""
    h = m.dt
    cb = lam.copy()
    k1b = (h / 6.0) * lam
    k2b = (h / 3.0) * lam
    k3b = (h / 3.0) * lam
    k4b = (h / 6.0) * lam
    sb = np.zeros(lam.shape[:-3] + (m.ny, m.nx))
    # k4 = A (c + h k3) + s
    sb += k4b[..., 0, :, :]
    u3b = tendency_adj(m, k4b)
    cb += u3b
    k3b = k3b + h * u3b
    # k3 = A (c + h/2 k2) + s
    sb += k3b[..., 0, :, :]
    u2b = tendency_adj(m, k3b)
    cb += u2b
    k2b = k2b + 0.5 * h * u2b
    # k2 = A (c + h/2 k1) + s
    sb += k2b[..., 0, :, :]
    u1b = tendency_adj(m, k2b)
    cb += u1b
    k1b = k1b + 0.5 * h * u1b
    # k1 = A c + s
    sb += k1b[..., 0, :, :]
    cb += tendency_adj(m, k1b)
    return cb, sb


# --- observation operator ----------------------------------------------------------------

def trilinear(m, pos):
    """Cells (p, 8) as (l, j, i) flat indices and weights (p, 8) of trilinear
    interpolation at pos (p, 3) = (x, y, z) in cell units.  x is periodic;
    y must lie in [0, ny-1] and z in [0, nz-1]."""
    pos = np.asarray(pos, dtype=np.float64)
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    fx0 = np.floor(x)
    i0 = np.mod(fx0, m.nx).astype(np.int64)
    i1 = np.mod(i0 + 1, m.nx)
    wx = x - fx0
    j0 = np.minimum(np.floor(y), m.ny - 2).astype(np.int64)
    wy = y - j0
    l0 = np.minimum(np.floor(z), m.nz - 2).astype(np.int64)
    wz = z - l0
    cells, wts = [], []
    for dl, fz in ((0, 1 - wz), (1, wz)):
        for dj, fy in ((0, 1 - wy), (1, wy)):
            for ii, fxx in ((i0, 1 - wx), (i1, wx)):
                cells.append(((l0 + dl) * m.ny + (j0 + dj)) * m.nx + ii)
                wts.append(fz * fy * fxx)
    return np.stack(cells, axis=1), np.stack(wts, axis=1)


@dataclass
class AdvDiffObs:
    step: np.ndarray    # (p,) 1..T, nondecreasing
    pos: np.ndarray     # (p, 3)
    cells: np.ndarray   # (p, 8)
    w: np.ndarray       # (p, 8)


def make_obs(m, step, pos):
    cells, w = trilinear(m, pos)
    return AdvDiffObs(step=np.asarray(step, dtype=np.int64), pos=np.asarray(pos, dtype=np.float64),
                      cells=cells, w=w)


def observe(m, obs, c, t):
    """Values (..., p_t) of the observations at step t from c (..., nz, ny, nx)."""
    sel = np.nonzero(obs.step == t)[0]
    flat = c.reshape(c.shape[:-3] + (-1,))
    return sel, np.sum(flat[..., obs.cells[sel]] * obs.w[sel], axis=-1)


def observe_adj(m, obs, r, t, lam):
    """lam += H_t^T r for the observations of step t (r: (..., p) full length)."""
    sel = np.nonzero(obs.step == t)[0]
    if sel.size == 0:
        return lam
    flat = lam.reshape((-1, m.nz * m.ny * m.nx)).copy()
    vals = (r[..., sel, None] * obs.w[sel]).reshape(flat.shape[0], -1)     # (batch, p_t * 8)
    np.add.at(flat, (slice(None), obs.cells[sel].reshape(-1)), vals)
    return flat.reshape(lam.shape)


# --- window integrations ------------------------------------------------------------------

def run(m, obs, src):
    """Integrate from c = 0 with the surface source fields src (..., nb, ny, nx)
    (already divided by dz) and return the observed values (..., p)."""
    lead = src.shape[:-3]
    c = np.zeros(lead + (m.nz, m.ny, m.nx))
    out = np.zeros(lead + (obs.step.size,))
    for t in range(m.T):
        c = rk4_step(m, c, src[..., m.block(t), :, :])
        sel, val = observe(m, obs, c, t + 1)
        out[..., sel] = val
    return out


def run_final(m, src, T=None):
    """Tracer field after T steps (default the window) from c = 0."""
    lead = src.shape[:-3]
    c = np.zeros(lead + (m.nz, m.ny, m.nx))
    for t in range(m.T if T is None else T):
        c = rk4_step(m, c, src[..., m.block(t), :, :])
    return c


def run_adj(m, obs, r):
    """Adjoint of `run`: the source adjoint (..., nb, ny, nx) of the
    observation-space forcing r (..., p)."""
    lead = r.shape[:-1]
    lam = np.zeros(lead + (m.nz, m.ny, m.nx))
    sb = np.zeros(lead + (m.nb, m.ny, m.nx))
    for t in range(m.T - 1, -1, -1):
        lam = observe_adj(m, obs, r, t + 1, lam)
        lam, s_t = rk4_step_adj(m, lam)
        sb[..., m.block(t), :, :] += s_t
    return sb


# --- prior square root ----------------------------------------------------------------------

def exp_corr(n, ell_cells, periodic):
    i = np.arange(n)
    d = np.abs(i[:, None] - i[None, :]).astype(np.float64)
    if periodic:
        d = np.minimum(d, n - d)
    return np.exp(-d / ell_cells)


def sym_sqrt(C):
    """Symmetric square root via the eigendecomposition (eigenvalues below 0 set to 0)."""
    w, Z = np.linalg.eigh(C)
    return (Z * np.sqrt(np.maximum(w, 0.0))) @ Z.T


@dataclass
class ExpSeparableSqrt:
    Sx: np.ndarray     # (nx, nx)
    Sy: np.ndarray     # (ny, ny)
    sigma_b: float
    nb: int

    def apply(self, W):
        """L W for W (..., n) with n = nb * ny * nx (block, row, column order)."""
        ny, nx = self.Sy.shape[0], self.Sx.shape[0]
        F = np.asarray(W, dtype=np.float64).reshape(W.shape[:-1] + (self.nb, ny, nx))
        out = self.sigma_b * np.einsum("ab,...bc,dc->...ad", self.Sy, F, self.Sx)
        return out.reshape(W.shape)

    def apply_t(self, W):
        ny, nx = self.Sy.shape[0], self.Sx.shape[0]
        F = np.asarray(W, dtype=np.float64).reshape(W.shape[:-1] + (self.nb, ny, nx))
        out = self.sigma_b * np.einsum("ba,...bc,cd->...ad", self.Sy, F, self.Sx)
        return out.reshape(W.shape)

    def dense(self):
        L1 = self.sigma_b * np.kron(self.Sy, self.Sx)
        return np.kron(np.eye(self.nb), L1)


def exp_separable_sqrt(nx, ny, nb, dx, dy, ell, sigma_b):
    Sx = sym_sqrt(exp_corr(nx, ell / dx, periodic=True))
    Sy = sym_sqrt(exp_corr(ny, ell / dy, periodic=False))
    return ExpSeparableSqrt(Sx=Sx, Sy=Sy, sigma_b=sigma_b, nb=nb)


# --- 4D-Var problem ---------------------------------------------------------------------------

@dataclass
class AdvDiffProblem:
    m: AdvDiffModel
    obs: AdvDiffObs
    y: np.ndarray
    sigma_o: np.ndarray
    Lop: ExpSeparableSqrt
    x_b: np.ndarray

    @property
    def n(self):
        return self.m.nb * self.m.ny * self.m.nx

    @property
    def p(self):
        return self.y.size

    @property
    def rinv(self):
        return 1.0 / (self.sigma_o * self.sigma_o)

    @property
    def L(self):
        return self.Lop.dense()


def emissions(prob, x):
    """E = E_b exp(x), (nb, ny, nx)."""
    return prob.m.Eb * np.exp(np.asarray(x).reshape(prob.m.nb, prob.m.ny, prob.m.nx))


def trajectory(prob, x):
    """The outer-loop quantities at control x: emissions and H(x)."""
    E = emissions(prob, x)
    Hx = run(prob.m, prob.obs, E / prob.m.dz)
    return {"E": E, "Hx": Hx}


def innovation(prob, traj):
    return traj["Hx"] - prob.y


def cost(prob, traj, v):
    d = innovation(prob, traj)
    return 0.5 * float(np.sum(d * d * prob.rinv)) + 0.5 * float(np.dot(v, v))


def _source_adj_to_control(prob, traj, sb):
    """Adjoint of x -> E/dz, i.e. multiply by E/dz, flattened to (..., n)."""
    g = sb * (traj["E"] / prob.m.dz)
    return g.reshape(g.shape[:-3] + (prob.n,))


def gradient_b(prob, traj, d):
    """b = L^T H'^T R^-1 d (one adjoint run)."""
    sb = run_adj(prob.m, prob.obs, d * prob.rinv)
    return prob.Lop.apply_t(_source_adj_to_control(prob, traj, sb))


def hvp(prob, traj, W):
    """A W for the columns of W (n, m): L^T H'^T R^-1 H' L W, vectorised over columns."""
    W = np.atleast_2d(np.asarray(W, dtype=np.float64).T).T
    dx = prob.Lop.apply(W.T)                                       # (m, n)
    dE = dx.reshape(-1, prob.m.nb, prob.m.ny, prob.m.nx) * traj["E"]
    r = run(prob.m, prob.obs, dE / prob.m.dz) * prob.rinv
    sb = run_adj(prob.m, prob.obs, r)
    return prob.Lop.apply_t(_source_adj_to_control(prob, traj, sb)).T


def tl_obs(prob, traj, dx):
    """H' dx: observation-space tangent-linear response (dx in control-increment
    space of x, not v)."""
    dE = np.asarray(dx).reshape(-1, prob.m.nb, prob.m.ny, prob.m.nx) * traj["E"]
    return run(prob.m, prob.obs, dE / prob.m.dz)


def quadratic_cost(prob, traj, d, v, dv):
    """Inner-loop quadratic cost of Eq. 3 with Algorithm 3's sign of d and the
    accumulated control v: J~(dv) = 1/2 ||R^-1/2 (d + H' L dv)||^2 + 1/2 ||v + dv||^2,
    H' the tangent-linear observation operator at the trajectory's emissions."""
    r = d + tl_obs(prob, traj, prob.Lop.apply(np.asarray(dv)[None, :]))[0]
    return 0.5 * float(np.sum(r * r * prob.rinv)) + 0.5 * float(np.dot(v + dv, v + dv))


def build(cfg, with_truth=False):
    """Twin experiment: truth x = 0 (E = E_b), y = H(truth) + sigma_o eps with
    sigma_o = rel * max(y_true, floor_frac * median(y_true)), background
    x_b = L eps_b."""
    m = model_from_config(cfg)
    step, pos = cfg.tracks()
    obs = make_obs(m, step, pos)
    y_true = run(m, obs, m.Eb / m.dz)
    floor = cfg.obs_floor_frac * np.median(y_true)
    sigma = cfg.obs_rel * np.maximum(y_true, floor)
    y = y_true + sigma * cfg.obs_noise(y_true.size)
    Lop = exp_separable_sqrt(cfg.nx, cfg.ny, cfg.nblocks, cfg.dx, cfg.dy, cfg.ell, cfg.sigma_b)
    x_b = Lop.apply(cfg.background_perturbation())
    prob = AdvDiffProblem(m=m, obs=obs, y=y, sigma_o=sigma, Lop=Lop, x_b=x_b)
    if with_truth:
        return prob, np.zeros(prob.n)
    return prob


def outer_step(prob, x, v, Omega, q=0, exact_rr=False):
    """One cycle of Algorithm 3 on the tracer problem (generic RIOT algebra)."""
    from . import riot
    traj = trajectory(prob, x)
    d = innovation(prob, traj)
    J = cost(prob, traj, v)
    b = gradient_b(prob, traj, d)
    g = b + v
    lam, U, info = riot.rsvd(prob, traj, Omega, q=q, exact_rr=exact_rr,
                             apply=lambda W: hvp(prob, traj, W))
    dv, mode = riot.increment(lam, U, g)
    return {"traj": traj, "J": J, "b": b, "g": g, "lam": lam, "U": U, "dv": dv, "mode": mode,
            "x_next": x + prob.Lop.apply(dv), "v_next": v + dv, "info": info}


def dual_hvp(prob, traj, W):
    """A_dual W = S H' B H'^T S W for the columns of W (p, m), S = diag(1 / sigma_o) (Appendix,
    Algorithm 4): one adjoint run from the forcing S w, the source adjoint to the control,
    B = L L^T, one tangent-linear run; vectorised over columns."""
    W = np.atleast_2d(np.asarray(W, dtype=np.float64).T).T
    s = 1.0 / prob.sigma_o
    sb = run_adj(prob.m, prob.obs, (s[:, None] * W).T)                  # (m, nb, ny, nx)
    z = prob.Lop.apply(prob.Lop.apply_t(_source_adj_to_control(prob, traj, sb)))
    return s[:, None] * tl_obs(prob, traj, z).T


def psas_outer_step(prob, x, Omega, q=0, exact_rr=False):
    """One cycle of Algorithm 4 on the tracer problem: d = y - H(x), b' = H'(x_b - x), the
    randomized eigendecomposition of A_dual on the sketch Omega (p, m), the adaptive weights,
    x_next = x_b + B H'^T dw (the reading of the state update taken for the Lorenz-96 dual)."""
    from . import riot
    traj = trajectory(prob, x)
    d = prob.y - traj["Hx"]
    bprime = tl_obs(prob, traj, prob.x_b - x)[0]
    lam, U, info = riot.rsvd(prob, traj, Omega, q=q, exact_rr=exact_rr,
                             apply=lambda W: dual_hvp(prob, traj, W))
    dw, mode = riot.psas_weights(lam, U, prob.sigma_o, d, bprime)
    sb = run_adj(prob.m, prob.obs, dw[None, :])
    x_next = prob.x_b + prob.Lop.apply(prob.Lop.apply_t(_source_adj_to_control(prob, traj, sb)))[0]
    return {"traj": traj, "d": d, "bprime": bprime, "lam": lam, "U": U, "dw": dw, "mode": mode,
            "x_next": x_next, "info": info}
