"""Shared helpers of the GPU parity tests: build matching oracle / CUDA runs."""
import math

import numpy as np

# FP64: the CUDA path follows the oracle's operation order without FMA
# contraction; 1e-12 of each field's max norm leaves room for nothing but a
# different libm/sqrt rounding, which IEEE fixes anyway.
TOL_FP64 = 1e-12
# FP32: perturbation arithmetic in single precision; relative L1 error per field
TOL_FP32_L1 = 1e-5


def problem_kwargs(nx, ny, **kw):
    d = dict(nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=5 / 3, courant=0.3,
             bc_x=0, bc_y=0, hyperdiffusion=1, c2=(0.02, 0.1, 0.1, 0.02, 0.02, 0.02), c_shk=0.5)
    d.update(kw)
    return d


def oracle_problem(oracle, kw):
    return oracle.Problem(**{k: kw[k] for k in ("nx", "ny", "x0", "x1", "y0", "y1", "gamma", "courant",
                                                "bc_x", "bc_y", "hyperdiffusion", "c2", "c_shk")})


def solver(kw, precision, has_background=0):
    from paper_1710_06423_b300.sac import Solver
    return Solver(**kw, precision=precision, has_background=has_background)


def maxrel(a, b):
    """Per-field max |a-b| / max |b| (b the oracle)."""
    num = np.abs(a - b).reshape(a.shape[0], -1).max(axis=1)
    den = np.maximum(np.abs(b).reshape(b.shape[0], -1).max(axis=1), 1e-300)
    return num / den


def l1rel(a, b):
    num = np.abs(a - b).reshape(a.shape[0], -1).sum(axis=1)
    den = np.maximum(np.abs(b).reshape(b.shape[0], -1).sum(axis=1), 1e-300)
    return num / den


def smooth_background(ny, nx, seed=3):
    """A smooth positive background (rho_b, e_b, B_bx, B_by) for split-form cases."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    a = rng.uniform(0.5, 1.5, 8)
    rb = 0.4 + 0.1 * np.sin(2 * math.pi * (X + a[0])) * np.cos(2 * math.pi * (Y + a[1]))
    eb = 1.2 + 0.2 * np.cos(2 * math.pi * (X + a[2]))
    bbx = 0.2 * np.sin(2 * math.pi * (Y + a[3]))
    bby = 0.15 * np.cos(2 * math.pi * (X + a[4]))
    return np.ascontiguousarray(np.stack([rb, eb, bbx, bby]))
