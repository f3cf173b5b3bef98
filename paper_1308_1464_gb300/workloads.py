"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle's tests.

This module holds no arithmetic of the wave-propagation method: it only draws
initial states.  Every random number comes from the SplitMix64 generator
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014; output function as in Vigna's public-domain splitmix64.c) used as
a counter-based generator: draw ``k`` of stream ``s`` under seed ``seed`` is
``mix(base(seed, s) + (k + 1) * GOLDEN)``, so any subset of a workload can be
regenerated without the rest.

The paper measures only synthetic grids (§3, Table 3, Fig. 1-3: 1024^2 and
2048^2 grids with no named dataset), so these generators are the workloads.
Arrays are float64, interior cells only, shape ``(meqn, my, mx)``; cell
centres are at ``x_lo + (i + 1/2) dx``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
DEFAULT_SEED = 1308

# stream identifiers (arbitrary distinct constants)
S_NOISE_H, S_NOISE_RHO, S_NOISE_P, S_QUADRANT = 1, 2, 3, 4
S_PATCH_SIZE, S_PATCH_CENTRE = 5, 6
S_RIEMANN = 7


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _base(seed: int, stream: int) -> np.uint64:
    key = np.uint64((int(seed) & 0xFFFFFFFF) | ((int(stream) & 0xFFFFFFFF) << 32))
    return _mix(np.array([key], dtype=np.uint64))[0]


def uniform(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1) for the given draw indices."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _base(seed, stream) + (idx + np.uint64(1)) * GOLDEN
    return (_mix(z) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _centres(n: int, lo: float, hi: float, first: int = 0, count: int | None = None):
    """Centres of cells first .. first + count - 1 of n cells on [lo, hi], and
    the cell width."""
    d = (hi - lo) / n
    count = n - first if count is None else count
    return lo + (np.arange(first, first + count) + 0.5) * d, d


def _window(mx: int, my: int, window):
    """(i0, j0, nx, ny) of a window of an mx x my grid (the whole grid for
    None), checked to lie inside it."""
    if window is None:
        return 0, 0, mx, my
    i0, j0, nx, ny = (int(v) for v in window)
    if not (0 <= i0 and 0 <= j0 and nx > 0 and ny > 0 and i0 + nx <= mx and j0 + ny <= my):
        raise ValueError(f"window {window} does not lie inside {mx} x {my} cells")
    return i0, j0, nx, ny


def _cell_index(mx: int, i0: int, j0: int, nx: int, ny: int) -> np.ndarray:
    """Row-major global indices j * mx + i of the window's cells, shape (ny, nx)."""
    j = np.arange(j0, j0 + ny, dtype=np.uint64)[:, None]
    i = np.arange(i0, i0 + nx, dtype=np.uint64)[None, :]
    return j * np.uint64(mx) + i


@dataclass
class Grid:
    """An initial state on a uniform grid."""
    q: np.ndarray          # (meqn, my, mx) float64
    dx: float
    dy: float
    x_lo: float
    y_lo: float


def acoustics_pulse(mx: int = 128, my: int = 128, window=None) -> Grid:
    """Gaussian pressure pulse p = exp(-80 r^2) at (0.5, 0.5) on [0,1]^2, u = v = 0.

    ``window`` (i0, j0, nx, ny), here and in the generators below, returns
    only those cells of the mx x my grid, equal to the same slice of the
    whole grid (x_lo, y_lo then locate the window's first cell)."""
    i0, j0, nx, ny = _window(mx, my, window)
    x, dx = _centres(mx, 0.0, 1.0, i0, nx)
    y, dy = _centres(my, 0.0, 1.0, j0, ny)
    X, Y = np.meshgrid(x, y)
    q = np.zeros((3, ny, nx))
    q[0] = np.exp(-80.0 * ((X - 0.5) ** 2 + (Y - 0.5) ** 2))
    return Grid(q, dx, dy, i0 * dx, j0 * dy)


def advection_pulse(mx: int = 4096, my: int = 4096, window=None) -> Grid:
    """Scalar Gaussian q = exp(-80 r^2) at (0.5, 0.5) on [0,1]^2 plus a unit
    background, for constant-velocity advection on a periodic domain."""
    i0, j0, nx, ny = _window(mx, my, window)
    x, dx = _centres(mx, 0.0, 1.0, i0, nx)
    y, dy = _centres(my, 0.0, 1.0, j0, ny)
    X, Y = np.meshgrid(x, y)
    q = (1.0 + np.exp(-80.0 * ((X - 0.5) ** 2 + (Y - 0.5) ** 2)))[None]
    return Grid(q, dx, dy, i0 * dx, j0 * dy)


def acoustics_layered(mx: int = 4096, my: int = 4096, seed: int = DEFAULT_SEED,
                      window=None) -> Grid:
    """Pressure pulse in a layered medium on [0,1]^2 for variable-coefficient
    acoustics: planes (p, u, v, rho, c).  p = exp(-80 r^2) at (0.5, 0.3),
    u = v = 0; density 1 below y = 0.5 and 3 above, times 1 + U(-0.05, 0.05)
    per cell; sound speed 1 + x, times 1 + U(-0.05, 0.05) per cell."""
    i0, j0, nx, ny = _window(mx, my, window)
    x, dx = _centres(mx, 0.0, 1.0, i0, nx)
    y, dy = _centres(my, 0.0, 1.0, j0, ny)
    X, Y = np.meshgrid(x, y)
    idx = _cell_index(mx, i0, j0, nx, ny)
    q = np.zeros((5, ny, nx))
    q[0] = np.exp(-80.0 * ((X - 0.5) ** 2 + (Y - 0.3) ** 2))
    q[3] = np.where(Y < 0.5, 1.0, 3.0) * (1.0 + 0.05 * (2.0 * uniform(seed, 21, idx) - 1.0))
    q[4] = (1.0 + X) * (1.0 + 0.05 * (2.0 * uniform(seed, 22, idx) - 1.0))
    return Grid(q, dx, dy, i0 * dx, j0 * dy)


def swe_dambreak(mx: int = 4096, my: int = 4096, seed: int = DEFAULT_SEED,
                 noise: float = 1e-3, window=None) -> Grid:
    """Radial dam break on [-1,1]^2: h = 2 for r < 0.5 else 1, plus U(-noise, noise)."""
    i0, j0, nx, ny = _window(mx, my, window)
    x, dx = _centres(mx, -1.0, 1.0, i0, nx)
    y, dy = _centres(my, -1.0, 1.0, j0, ny)
    q = np.zeros((3, ny, nx))
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    h = np.where(r2 < 0.25, 2.0, 1.0)
    if noise:
        h = h + noise * (2.0 * uniform(seed, S_NOISE_H, _cell_index(mx, i0, j0, nx, ny)) - 1.0)
    q[0] = h
    return Grid(q, dx, dy, -1.0 + i0 * dx, -1.0 + j0 * dy)


def euler_quadrants(mx: int = 4096, my: int = 4096, seed: int = DEFAULT_SEED,
                    noise: float = 1e-3, gamma: float = 1.4, window=None) -> Grid:
    """Four-quadrant Riemann data on [0,1]^2.

    Each quadrant (split at x = y = 0.5) draws rho, p ~ U[0.1, 2] and
    u, v ~ U[-1, 1]; every cell then gets U(-noise, noise) added to rho and p.
    The conserved energy is E = p/(gamma-1) + rho (u^2 + v^2)/2.
    """
    i0, j0, nx, ny = _window(mx, my, window)
    x, dx = _centres(mx, 0.0, 1.0, i0, nx)
    y, dy = _centres(my, 0.0, 1.0, j0, ny)
    d = uniform(seed, S_QUADRANT, np.arange(16, dtype=np.uint64)).reshape(4, 4)
    rho_q = 0.1 + 1.9 * d[:, 0]
    p_q = 0.1 + 1.9 * d[:, 1]
    u_q = -1.0 + 2.0 * d[:, 2]
    v_q = -1.0 + 2.0 * d[:, 3]
    quad = (x[None, :] >= 0.5).astype(np.int64) + 2 * (y[:, None] >= 0.5).astype(np.int64)
    rho, p, u, v = rho_q[quad], p_q[quad], u_q[quad], v_q[quad]
    if noise:
        k = _cell_index(mx, i0, j0, nx, ny)
        rho = rho + noise * (2.0 * uniform(seed, S_NOISE_RHO, k) - 1.0)
        p = p + noise * (2.0 * uniform(seed, S_NOISE_P, k) - 1.0)
    q = np.zeros((4, ny, nx))
    q[0] = rho
    q[1] = rho * u
    q[2] = rho * v
    q[3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return Grid(q, dx, dy, i0 * dx, j0 * dy)


@dataclass
class Patch:
    nx: int
    ny: int
    grid: Grid


def patch_sizes(npatch: int = 2000, seed: int = DEFAULT_SEED, lo: int = 16, hi: int = 256):
    """Per-side patch sizes, log-uniform in [lo, hi], rounded to integers."""
    u = uniform(seed, S_PATCH_SIZE, np.arange(2 * npatch, dtype=np.uint64)).reshape(npatch, 2)
    n = np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return n[:, 0], n[:, 1]


def swe_patches(npatch: int = 2000, seed: int = DEFAULT_SEED, h_cell: float = 1.0 / 128.0,
                with_state: bool = True, only=None):
    """Uneven shallow-water patches with a Gaussian hump h = 1 + 0.5 exp(-50 r^2).

    Patch k covers [0, nx h_cell] x [0, ny h_cell]; the hump centre is drawn
    uniformly inside it.  Momentum is zero.  ``only`` (indices into the
    npatch patches) returns just those patches, in that order, each as in
    the whole set.
    """
    nxs, nys = patch_sizes(npatch, seed)
    c = uniform(seed, S_PATCH_CENTRE, np.arange(2 * npatch, dtype=np.uint64)).reshape(npatch, 2)
    out = []
    for k in (range(npatch) if only is None else only):
        nx, ny = int(nxs[k]), int(nys[k])
        if not with_state:
            out.append(Patch(nx, ny, None))
            continue
        x, _ = _centres(nx, 0.0, nx * h_cell)
        y, _ = _centres(ny, 0.0, ny * h_cell)
        xc, yc = c[k, 0] * nx * h_cell, c[k, 1] * ny * h_cell
        q = np.zeros((3, ny, nx))
        q[0] = 1.0 + 0.5 * np.exp(-50.0 * ((x[None, :] - xc) ** 2 + (y[:, None] - yc) ** 2))
        out.append(Patch(nx, ny, Grid(q, h_cell, h_cell, 0.0, 0.0)))
    return out


def riemann_states(n: int, seed: int = DEFAULT_SEED, offset: int = 0):
    """Independent 1D Euler interfaces: rho log-uniform in [0.01, 10], p log-uniform
    in [0.01, 100], u uniform in [-5, 5], left and right drawn independently.

    Returns (rho_l, u_l, p_l, rho_r, u_r, p_r) as float64 arrays.  ``offset``
    selects a disjoint block of draws (e.g. a training set apart from a test set).
    """
    k = (np.arange(n, dtype=np.uint64) + np.uint64(offset)) * np.uint64(6)
    d = [uniform(seed, S_RIEMANN, k + np.uint64(j)) for j in range(6)]
    lr = math.log(0.01), math.log(10.0)
    lp = math.log(0.01), math.log(100.0)
    rho_l = np.exp(lr[0] + d[0] * (lr[1] - lr[0]))
    p_l = np.exp(lp[0] + d[1] * (lp[1] - lp[0]))
    u_l = -5.0 + 10.0 * d[2]
    rho_r = np.exp(lr[0] + d[3] * (lr[1] - lr[0]))
    p_r = np.exp(lp[0] + d[4] * (lp[1] - lp[0]))
    u_r = -5.0 + 10.0 * d[5]
    return rho_l, u_l, p_l, rho_r, u_r, p_r
