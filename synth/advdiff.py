"""Seeded synthetic black-carbon-style source inversion (inputs only).

A linear tracer is carried by steady, level-scaled horizontal winds and mixed
vertically on a box grid (x periodic, walls in y, zero flux at the bottom and
top).  The control is the log of a scaling of the surface emissions, one
field per emission time block; aircraft-like tracks sample the tracer.  This
is the seeded stand-in for the paper's black-carbon inversions (Section 3.2:
a ~1e5 surface emission control, aircraft observations), which rely on data
and a transport model that are not available here.

Everything below is a raw input of that experiment (grid, winds, diffusivity,
background emissions, flight tracks, random draws).  Running the transport
model, forming observations from a truth and building the prior square root
is left to the consumer: the FP64 oracle in tests, the CUDA library in the
benchmark.

Philox streams (base seed 20190604): 5 stream-function modes, 6 emission
field, 7 flight tracks, 8 observation noise, 9 background, 16 + j sketch of
outer iteration j.
"""
from dataclasses import dataclass

import numpy as np

from . import philox
from .configs import BASE_SEED

STREAM_WIND = 5
STREAM_EMIS = 6
STREAM_TRACKS = 7
STREAM_NOISE = 8
STREAM_BKG = 9
STREAM_SKETCH0 = 16


@dataclass
class AdvDiffConfig:
    name: str
    nx: int = 192
    ny: int = 192
    nz: int = 30
    T: int = 240
    nblocks: int = 4
    dx: float = 12000.0          # m (also dy)
    dz: float = 250.0            # m
    umax: float = 15.0           # m/s, largest face speed at amplitude 1
    cfl: float = 0.5             # dt = cfl * dx / umax
    nmodes: int = 8              # Fourier modes of the stream function
    kz_max: float = 20.0         # m^2/s at the lowest interior face
    kz_scale: float = 1500.0     # m, e-folding height of Kz
    n_hotspots: int = 50
    n_tracks: int = 20
    pts_per_track: int = 400
    alt_lo: float = 500.0        # m
    alt_hi: float = 6000.0       # m
    sigma_b: float = 0.5
    ell: float = 50000.0         # m, exponential correlation length
    obs_rel: float = 0.2         # sigma_o = 0.2 * max(y_true, floor)
    obs_floor_frac: float = 0.05  # floor = 0.05 * median(y_true)
    k: int = 1024
    q: int = 1
    seed: int = BASE_SEED

    @property
    def dy(self):
        return self.dx

    @property
    def dt(self):
        return self.cfl * self.dx / self.umax

    @property
    def n(self):
        """Control size: one log-scaling per surface cell and emission block."""
        return self.nblocks * self.ny * self.nx

    @property
    def ncells(self):
        return self.nz * self.ny * self.nx

    # -- winds ------------------------------------------------------------------
    def stream_function(self):
        """psi at the cell corners, shape (ny + 1, nx): a sum of seeded modes
        A sin(pi m_y y / Ly) cos(2 pi m_x x / Lx + phi), zero on both walls,
        scaled so that the largest face speed is umax."""
        w = philox.uniforms(self.seed, STREAM_WIND, 4 * self.nmodes).reshape(self.nmodes, 4)
        amp = philox.normals(self.seed, STREAM_WIND + 100, self.nmodes)
        mx = 1 + np.floor(3 * w[:, 0]).astype(int)
        my = 1 + np.floor(3 * w[:, 1]).astype(int)
        phi = 2 * np.pi * w[:, 2]
        X = np.arange(self.nx) / self.nx
        Y = np.arange(self.ny + 1) / self.ny
        psi = np.zeros((self.ny + 1, self.nx))
        for m in range(self.nmodes):
            psi += amp[m] * np.sin(np.pi * my[m] * Y)[:, None] * np.cos(2 * np.pi * mx[m] * X + phi[m])[None, :]
        psi[0, :] = 0.0
        psi[-1, :] = 0.0
        u, v = self._faces(psi)
        s = self.umax / max(np.abs(u).max(), np.abs(v).max())
        return psi * s

    def _faces(self, psi):
        u = -(psi[1:, :] - psi[:-1, :]) / self.dy                # (ny, nx): x-face i-1/2 of row j
        v = (np.roll(psi, -1, axis=1) - psi) / self.dx            # (ny+1, nx): y-face j-1/2 of column i
        return u, v

    def winds(self):
        """Face velocities (m/s) at amplitude 1: u (ny, nx) on the x-faces i-1/2,
        v (ny + 1, nx) on the y-faces j-1/2 (rows 0 and ny are the walls, v = 0)."""
        u, v = self._faces(self.stream_function())
        v[0, :] = 0.0
        v[-1, :] = 0.0
        return u, v

    def amplitude(self):
        """Level scaling of the horizontal winds, (nz,), in (0, 1]."""
        z = np.arange(self.nz)
        return 0.5 + 0.5 * z / max(self.nz - 1, 1)

    def kz(self):
        """Vertical diffusivity (m^2/s) at the faces l - 1/2, l = 0..nz (ends zero)."""
        k = np.zeros(self.nz + 1)
        zf = np.arange(1, self.nz) * self.dz
        k[1:self.nz] = self.kz_max * np.exp(-zf / self.kz_scale)
        return k

    # -- emissions ----------------------------------------------------------------
    def background_emissions(self):
        """E_b >= 0, (nblocks, ny, nx): log-normal cell noise plus Gaussian hot
        spots, modulated per time block."""
        nyx = self.ny * self.nx
        g = philox.normals(self.seed, STREAM_EMIS, nyx).reshape(self.ny, self.nx)
        base = 0.01 * np.exp(0.5 * g)
        w = philox.uniforms(self.seed, STREAM_EMIS + 100, 4 * self.n_hotspots).reshape(-1, 4)
        xs, ys = w[:, 0] * self.nx, w[:, 1] * self.ny
        rad = 1.0 + 3.0 * w[:, 2]
        amp = 0.1 * (0.5 + 1.5 * w[:, 3])
        X = np.arange(self.nx) + 0.0
        Y = np.arange(self.ny) + 0.0
        for h in range(self.n_hotspots):
            dxp = np.abs(X - xs[h])
            dxp = np.minimum(dxp, self.nx - dxp)
            dyp = Y - ys[h]
            base += amp[h] * np.exp(-(dyp[:, None] ** 2 + dxp[None, :] ** 2) / (2 * rad[h] ** 2))
        cycle = np.array([0.7, 1.2, 1.3, 0.8])
        fac = cycle[np.arange(self.nblocks) % 4]
        return base[None, :, :] * fac[:, None, None]

    # -- observations ---------------------------------------------------------------
    def tracks(self):
        """(step, pos) of every observation, sorted by step: pos (p, 3) are
        (x, y, z) in cell units (cell (i, j, l) is centred at (i, j, l)),
        x periodic in [0, nx), y in [0.5, ny - 1.5], z within the altitude band."""
        ntr, npt = self.n_tracks, self.pts_per_track
        w = philox.uniforms(self.seed, STREAM_TRACKS, ntr * 17).reshape(ntr, 17)
        zlo = max(0.0, self.alt_lo / self.dz - 0.5)
        zhi = min(self.nz - 1.0, self.alt_hi / self.dz - 0.5)
        steps, pos = [], []
        s = (np.arange(npt) + 0.5) / npt
        for t in range(ntr):
            ts = 1 + int(w[t, 0] * (self.T // 2))
            td = max(1, self.T // 4 + int(w[t, 1] * (self.T // 4)))
            td = min(td, self.T - ts)
            wp = w[t, 2:17].reshape(5, 3)
            wx = wp[:, 0] * self.nx
            wy = 0.5 + wp[:, 1] * (self.ny - 2.0)
            wz = zlo + wp[:, 2] * (zhi - zlo)
            leg = s * 4.0
            li = np.minimum(np.floor(leg).astype(int), 3)
            f = leg - li
            px = np.mod(wx[li] * (1 - f) + wx[li + 1] * f, self.nx)
            py = wy[li] * (1 - f) + wy[li + 1] * f
            pz = wz[li] * (1 - f) + wz[li + 1] * f
            steps.append(ts + np.rint(s * td).astype(np.int64))
            pos.append(np.stack([px, py, pz], axis=1))
        step = np.concatenate(steps)
        pos = np.concatenate(pos)
        order = np.argsort(step, kind="stable")
        return np.clip(step[order], 1, self.T), pos[order]

    def obs_noise(self, p):
        return philox.normals(self.seed, STREAM_NOISE, p)

    def background_perturbation(self):
        return philox.normals(self.seed, STREAM_BKG, self.n)

    def sketch(self, outer_iter, k=None):
        k = self.k if k is None else k
        return philox.normals(self.seed, STREAM_SKETCH0 + outer_iter, k * self.n).reshape(k, self.n)


def bc_large():
    """192 x 192 x 30 box (12 km, 250 m), 240 steps of 400 s, four emission
    blocks (147 456 controls), 20 tracks x 400 points (8000 observations),
    exponential B (50 km, sigma_b 0.5), k = 1024, q = 1."""
    return AdvDiffConfig(name="bc_192x192x30_T240_k1024")


def bc_small():
    """A small box with the same recipe for parity tests: 16 x 12 x 6 cells,
    24 steps, 2 blocks (384 controls), 4 tracks x 60 points."""
    return AdvDiffConfig(name="bc_16x12x6_T24", nx=16, ny=12, nz=6, T=24, nblocks=2, n_hotspots=6,
                         n_tracks=4, pts_per_track=60, k=48, q=1)


def bc_tiny():
    """Smallest box with every feature (full-rank tests): 8 x 6 x 4 cells,
    12 steps, 2 blocks (96 controls), 4 tracks x 50 points."""
    return AdvDiffConfig(name="bc_8x6x4_T12", nx=8, ny=6, nz=4, T=12, nblocks=2, n_hotspots=3,
                         n_tracks=4, pts_per_track=50, k=96, q=0)
