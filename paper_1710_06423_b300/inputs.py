"""Seeded synthetic inputs for the SAC-family MHD step: initial states only.

This module is shared by the CUDA path's callers (tests, bench) and by the
oracle's callers; it holds none of the method's arithmetic (no fluxes,
derivatives, diffusion or time stepping), only the initial conditions the
paper's test problems define and a counter-based noise generator.

All states are conserved variables on a cell-centred grid, shape
``(6, ny, nx)``, fields ``(rho, m_x, m_y, e, B_x, B_y)``, float64, with
``e = p/(gamma-1) + rho|v|^2/2 + |B|^2/2`` (units with mu0 = 1, as the
section 2 pressure definitions imply).  With a zero background the
perturbation variables are the full variables.

Workloads (paper section 5):
  * Orszag-Tang vortex (section 5.1): [0,1]^2 periodic, gamma = 5/3,
    rho = 25/(36 pi), p = 5/(12 pi), v = (-sin 2 pi y, sin 2 pi x),
    B = B0 (-sin 2 pi y, sin 4 pi x), B0 = 1/sqrt(4 pi).  The paper prints the
    vortex with the signs and the x/y roles of some terms garbled and without
    rho, p, B0 (it only says they are constants); the standard form above is
    the reading used.
  * Orszag-Tang family: the same vortex with B0 scaled by U[0.5, 1.5],
    gamma in {1.4, 5/3} and a phase shift in each sine term, all seeded.
  * Brio-Wu shock tube (section 5.2): 800 cells on [0,1], gamma = 2,
    B_x = 0.75; left rho = 1, p = 1, B_y = 1; right rho = 0.125, p = 0.1,
    B_y = -1; at rest; discontinuity at x = 0.5.
  * linear sound and Alfven waves (smooth convergence workloads).
"""
from __future__ import annotations

import math

import numpy as np

NF = 6
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 output for state ``seed + (counter + 1) * golden`` (Steele et al. 2014)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, stream: int, n: int) -> np.ndarray:
    """n values U[-1, 1) from splitmix64, counter = stream * 2^40 + index."""
    c = np.arange(n, dtype=np.uint64) + np.uint64(stream) * np.uint64(1 << 40)
    u = (splitmix64(c, seed) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def cell_centres(n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    d = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * d


def conserved(rho, vx, vy, p, bx, by, gamma) -> np.ndarray:
    """Stack primitive fields into the conserved state (6, ny, nx)."""
    e = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy) + 0.5 * (bx * bx + by * by)
    return np.ascontiguousarray(np.stack([rho, rho * vx, rho * vy, e, bx, by]).astype(np.float64))


def orszag_tang(n: int, ny: int | None = None, *, b0: float = 1.0 / math.sqrt(4.0 * math.pi),
                gamma: float = 5.0 / 3.0, phases=(0.0, 0.0, 0.0, 0.0),
                noise: float = 0.0, seed: int = 20171018) -> np.ndarray:
    """Orszag-Tang vortex on an n x ny periodic grid over [0,1]^2.

    ``noise`` > 0 multiplies rho and p by (1 + noise * xi) with xi ~ U[-1,1]
    drawn per cell from splitmix64 (streams 0 and 1 of ``seed``).
    """
    ny = n if ny is None else ny
    x = cell_centres(n)[None, :]
    y = cell_centres(ny)[:, None]
    tp = 2.0 * math.pi
    p1, p2, p3, p4 = phases
    rho = np.full((ny, n), 25.0 / (36.0 * math.pi))
    p = np.full((ny, n), 5.0 / (12.0 * math.pi))
    if noise > 0.0:
        rho = rho * (1.0 + noise * uniform_pm1(seed, 0, n * ny).reshape(ny, n))
        p = p * (1.0 + noise * uniform_pm1(seed, 1, n * ny).reshape(ny, n))
    vx = -np.sin(tp * y + p1) * np.ones((1, n))
    vy = np.sin(tp * x + p2) * np.ones((ny, 1))
    bx = -b0 * np.sin(tp * y + p3) * np.ones((1, n))
    by = b0 * np.sin(2.0 * tp * x + p4) * np.ones((ny, 1))
    return conserved(rho, vx, vy, p, bx, by, gamma)


def ot_family_params(seed: int, index: int):
    """Seeded (b0, gamma, phases) of member ``index`` of the Orszag-Tang family."""
    u = uniform_pm1(seed, 16 + index, 6)          # six U[-1,1) draws
    b0 = (1.0 + 0.5 * u[0]) / math.sqrt(4.0 * math.pi)   # B0 * U[0.5, 1.5]
    gamma = 1.4 if u[1] < 0.0 else 5.0 / 3.0
    phases = tuple(float(math.pi * (1.0 + v)) for v in u[2:6])   # U[0, 2 pi)
    return b0, gamma, phases


def batch_sizes(seed: int, count: int, choices=(256, 512, 1000, 2044)) -> list[int]:
    """Seeded grid sizes for a batch of independent runs."""
    u = uniform_pm1(seed, 99, count)
    idx = np.minimum(((u + 1.0) * 0.5 * len(choices)).astype(np.int64), len(choices) - 1)
    return [int(choices[i]) for i in idx]


def brio_wu(nx: int = 800, ny: int = 1, gamma: float = 2.0) -> np.ndarray:
    """Brio-Wu shock tube along x (uniform along y)."""
    x = cell_centres(nx)[None, :] * np.ones((ny, 1))
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    by = np.where(left, 1.0, -1.0)
    bx = np.full_like(x, 0.75)
    z = np.zeros_like(x)
    return conserved(rho, z, z, p, bx, by, gamma)


def sound_wave(nx: int, ny: int = 1, amp: float = 1e-6, gamma: float = 5.0 / 3.0,
               direction: str = "x") -> np.ndarray:
    """Right-going linear sound wave of one wavelength, rho0 = 1, c_s = 1."""
    n = nx if direction == "x" else ny
    s = np.sin(2.0 * math.pi * cell_centres(n))
    s = s[None, :] * np.ones((ny, 1)) if direction == "x" else s[:, None] * np.ones((1, nx))
    rho = 1.0 + amp * s
    p = 1.0 / gamma + amp * s
    v = amp * s
    z = np.zeros((ny, nx))
    if direction == "x":
        return conserved(rho, v, z, p, z, z, gamma)
    return conserved(rho, z, v, p, z, z, gamma)


def alfven_wave(nx: int, ny: int = 1, amp: float = 1e-6, gamma: float = 5.0 / 3.0) -> np.ndarray:
    """Right-going linear Alfven wave along x: rho = 1, B_x = 1, dv_y = -dB_y."""
    s = np.sin(2.0 * math.pi * cell_centres(nx))[None, :] * np.ones((ny, 1))
    one = np.ones((ny, nx))
    z = np.zeros((ny, nx))
    return conserved(one, z, amp * s, one, one, -amp * s, gamma)


def stratified_background(nx: int, ny: int, *, g: float, scale_height: float, bx: float = 0.0,
                          rho0: float = 1.0, gamma: float = 5.0 / 3.0) -> np.ndarray:
    """Isothermal magnetohydrostatic background on [0,1]^2 under gravity (0, -g):
    rho_b = rho0 exp(-y/H), p_b = rho_b g H (dp_b/dy = -rho_b g), a uniform
    horizontal field B_b = (bx, 0) (no magnetic force).  Returns the four
    background fields (rho_b, e_b, B_bx, B_by), shape (4, ny, nx)."""
    y = cell_centres(ny)[:, None] * np.ones((1, nx))
    rho = rho0 * np.exp(-y / scale_height)
    p = rho * g * scale_height
    e = p / (gamma - 1.0) + 0.5 * bx * bx
    return np.ascontiguousarray(np.stack([rho, e, bx * np.ones_like(y), np.zeros_like(y)]).astype(np.float64))


def gaussian_blob(nx: int, ny: int, *, amp: float, centre=(0.5, 0.5), width: float = 0.1) -> np.ndarray:
    """amp exp(-r^2 / width^2) about `centre` on the cell centres of [0,1]^2, shape (ny, nx)."""
    x = cell_centres(nx)[None, :]
    y = cell_centres(ny)[:, None]
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2
    return np.ascontiguousarray(amp * np.exp(-r2 / (width * width)))


def ot_3d(nx: int, ny: int, nz: int, *, gamma: float = 5.0 / 3.0, b0: float = 1.0 / math.sqrt(4.0 * math.pi),
          tilt: float = 0.2, compress: float = 0.0) -> np.ndarray:
    """A three-dimensional variant of the Orszag-Tang vortex on [0,1]^3: the 2D
    vortex plus z-dependent velocity and field components of relative size
    `tilt` (smooth, periodic, divergence-free B).  `compress` adds the
    compressive flow compress * (sin 2 pi x, 0, cos 2 pi z), so that the shock
    indicator max(0, -div v) is non-zero from the first step.  Eight conserved
    fields (rho, m_x, m_y, m_z, e, B_x, B_y, B_z), shape (8, nz, ny, nx)."""
    x = cell_centres(nx)[None, None, :]
    y = cell_centres(ny)[None, :, None]
    z = cell_centres(nz)[:, None, None]
    tp = 2.0 * math.pi
    one = np.ones((nz, ny, nx))
    rho = 25.0 / (36.0 * math.pi) * one
    p = 5.0 / (12.0 * math.pi) * one
    vx = -np.sin(tp * y) + tilt * np.sin(tp * z) * one
    vy = np.sin(tp * x) + tilt * np.cos(tp * z) * one
    vz = tilt * np.sin(tp * (x + y)) * one
    vx = vx + compress * np.sin(tp * x)
    vz = vz + compress * np.cos(tp * z)
    bx = b0 * (-np.sin(tp * y) + tilt * np.cos(tp * z)) * one
    by = b0 * (np.sin(2 * tp * x) + tilt * np.sin(tp * z)) * one
    bz = b0 * tilt * np.cos(tp * (x - y)) * one
    e = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz)
    return np.ascontiguousarray(np.stack([rho, rho * vx, rho * vy, rho * vz, e, bx, by, bz]).astype(np.float64))
