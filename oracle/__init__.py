"""FP64 CPU oracle of the SAC-family 2D ideal-MHD step (arXiv 1710.06423, section 2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library: the arithmetic lives in
``sac_oracle.c`` (plain C, FP64, no FMA contraction) and in ``cnn.py`` (numpy
FP64); this module only marshals numpy arrays through ctypes.

Every function here is a thin call of the C routine of the same role; the
docstrings of ``sac_oracle.c`` give the equations and the paper passages.

Parity status: every function of the MHD oracle is pinned by tests in
``tests/test_oracle_*.py`` (closed forms, invariants, convergence order); the
Brio-Wu shock-tube profile itself has no printed values in the paper (its
figure is missing), so beyond those invariants the Brio-Wu numbers are
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sac_oracle.c")
_LIB = os.path.join(_HERE, "libsac_oracle.so")

BC_PERIODIC, BC_FIXED, BC_OUTFLOW = 0, 1, 2
NF, NB = 6, 4

#: default hyper-diffusion coefficients (rho, mx, my, e, bx, by) and shock coefficient
DEFAULT_C2 = (0.02, 0.1, 0.1, 0.02, 0.02, 0.02)
DEFAULT_CSHK = 0.5


def build(force: bool = False) -> str:
    """Compile ``sac_oracle.c`` into ``libsac_oracle.so`` (gcc, -ffp-contract=off, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("gamma", ctypes.c_double), ("courant", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("hyperdiffusion", ctypes.c_int),
        ("c2", ctypes.c_double * NF),
        ("c_shk", ctypes.c_double),
        ("nthreads", ctypes.c_int),
        ("grav", ctypes.c_double * 2),
        ("hd_single_face", ctypes.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_make_held.argtypes = [P, dp, dp]
        lib.orc_ext_size.argtypes = [P]
        lib.orc_ext_size.restype = ctypes.c_size_t
        lib.orc_rhs.argtypes = [P, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_cmax.argtypes = [P, dp, dp, dp, dp]
        lib.orc_divb.argtypes = [P, dp, dp, dp, ctypes.POINTER(ctypes.c_ubyte)]
        lib.orc_cfl_dt.argtypes = [P, ctypes.c_double, ctypes.c_double]
        lib.orc_cfl_dt.restype = ctypes.c_double
        lib.orc_rk4_step.argtypes = [P, dp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.orc_run.argtypes = [P, dp, dp, dp, dp, ctypes.c_double, ctypes.c_long, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_long)]
        lib.orc_run.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Problem:
    """Grid and method parameters of one run (cell-centred grid on [x0,x1]x[y0,y1])."""
    nx: int
    ny: int
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    gamma: float = 5.0 / 3.0
    courant: float = 0.3
    bc_x: int = BC_PERIODIC
    bc_y: int = BC_PERIODIC
    hyperdiffusion: int = 1
    c2: tuple = DEFAULT_C2
    c_shk: float = DEFAULT_CSHK
    nthreads: int = field(default_factory=lambda: int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1)))
    gravity: tuple = (0.0, 0.0)   # (g_x, g_y): sources rt g in momentum, m.g in energy (section 2)
    hd_single_face: int = 0       # 1: hyper-diffusion ratio from the face itself (no max over 3 faces)

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny

    def _c(self) -> _Params:
        p = _Params()
        p.nx, p.ny = self.nx, self.ny
        p.dx, p.dy = self.dx, self.dy
        p.gamma, p.courant = self.gamma, self.courant
        p.bc_x, p.bc_y = self.bc_x, self.bc_y
        p.hyperdiffusion = self.hyperdiffusion
        for i, v in enumerate(self.c2):
            p.c2[i] = v
        p.c_shk = self.c_shk
        p.nthreads = self.nthreads
        p.grav[0], p.grav[1] = float(self.gravity[0]), float(self.gravity[1])
        p.hd_single_face = int(self.hd_single_face)
        return p


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _state(w, pr: Problem, nf: int):
    a = np.ascontiguousarray(w, dtype=np.float64)
    if a.shape != (nf, pr.ny, pr.nx):
        raise ValueError(f"expected shape {(nf, pr.ny, pr.nx)}, got {a.shape}")
    return a


def make_held(pr: Problem, w0) -> np.ndarray:
    """Ghost values held by fixed boundaries, taken from the starting state w0."""
    lib = _load()
    p = pr._c()
    w0 = _state(w0, pr, NF)
    held = np.zeros(NF * lib.orc_ext_size(ctypes.byref(p)))
    lib.orc_make_held(ctypes.byref(p), _dp(w0), _dp(held))
    return held


def rhs(pr: Problem, w, bg=None, held=None, cmax=(0.0, 0.0)) -> np.ndarray:
    """k = f(w): the semi-discrete right-hand side of all six conserved fields."""
    lib = _load()
    p = pr._c()
    w = _state(w, pr, NF)
    bg = None if bg is None else _state(bg, pr, NB)
    if held is None and (pr.bc_x == BC_FIXED or pr.bc_y == BC_FIXED):
        held = make_held(pr, w)
    k = np.zeros_like(w)
    lib.orc_rhs(ctypes.byref(p), _dp(w), _dp(bg), _dp(held), float(cmax[0]), float(cmax[1]), _dp(k))
    return k


def cmax(pr: Problem, w, bg=None) -> tuple[float, float]:
    """Maximum signal speed |v_d| + c_fast over the interior, per direction."""
    lib = _load()
    p = pr._c()
    w = _state(w, pr, NF)
    bg = None if bg is None else _state(bg, pr, NB)
    cx, cy = ctypes.c_double(), ctypes.c_double()
    lib.orc_cmax(ctypes.byref(p), _dp(w), _dp(bg), ctypes.byref(cx), ctypes.byref(cy))
    return cx.value, cy.value


def div_b(pr: Problem, w, bg=None) -> tuple[np.ndarray, np.ndarray]:
    """Discrete div B of the total field per interior cell, fourth-order
    central differences; returns (div [ny][nx], mask [ny][nx] of the cells
    whose stencil exists: non-periodic sides leave out two cells)."""
    lib = _load()
    p = pr._c()
    w = _state(w, pr, NF)
    bg = None if bg is None else _state(bg, pr, NB)
    div = np.zeros((pr.ny, pr.nx))
    mask = np.zeros((pr.ny, pr.nx), dtype=np.uint8)
    lib.orc_divb(ctypes.byref(p), _dp(w), _dp(bg), _dp(div),
                 mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return div, mask.astype(bool)


def cfl_dt(pr: Problem, cx: float, cy: float) -> float:
    """dt = C min(dx/cmax_x, dy/cmax_y)."""
    lib = _load()
    p = pr._c()
    return lib.orc_cfl_dt(ctypes.byref(p), cx, cy)


def rk4_step(pr: Problem, w, dt: float, bg=None, held=None, cmax_xy=None) -> np.ndarray:
    """One classical RK4 step of size dt; returns the new state (input untouched)."""
    lib = _load()
    p = pr._c()
    w = _state(w, pr, NF).copy()
    bg = None if bg is None else _state(bg, pr, NB)
    if held is None and (pr.bc_x == BC_FIXED or pr.bc_y == BC_FIXED):
        held = make_held(pr, w)
    if cmax_xy is None:
        cmax_xy = cmax(pr, w, bg)
    lib.orc_rk4_step(ctypes.byref(p), _dp(w), _dp(bg), _dp(held), float(dt),
                     float(cmax_xy[0]), float(cmax_xy[1]))
    return w


def run(pr: Problem, w, t0: float = 0.0, t_end: float = float("inf"), max_steps: int = -1,
        bg=None, held=None, fixed_dt: float = 0.0):
    """Advance with CFL steps until t_end (clipped last step) or max_steps.

    Returns (w, t, steps).  Raises FloatingPointError if the state turned non-finite.
    """
    lib = _load()
    p = pr._c()
    w = _state(w, pr, NF).copy()
    bg = None if bg is None else _state(bg, pr, NB)
    if held is None and (pr.bc_x == BC_FIXED or pr.bc_y == BC_FIXED):
        held = make_held(pr, w)
    t = ctypes.c_double(t0)
    steps = ctypes.c_long(0)
    rc = lib.orc_run(ctypes.byref(p), _dp(w), _dp(bg), _dp(held), ctypes.byref(t), float(t_end),
                     int(max_steps), float(fixed_dt), ctypes.byref(steps))
    if rc != 0:
        raise FloatingPointError(f"oracle run stopped: non-finite step after {steps.value} steps")
    return w, t.value, steps.value


# ---- 3D form (eight fields rho, m_x, m_y, m_z, e, B_x, B_y, B_z; periodic) -----
_SRC3 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sac_oracle3d.c")
_LIB3 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsac_oracle3d.so")
NF3 = 8
DEFAULT_C2_3D = (0.02, 0.1, 0.1, 0.1, 0.02, 0.02, 0.02, 0.02)


def build3(force: bool = False) -> str:
    """Compile ``sac_oracle3d.c`` into ``libsac_oracle3d.so`` (same flags as the 2D oracle)."""
    if force or not os.path.exists(_LIB3) or os.path.getmtime(_LIB3) < os.path.getmtime(_SRC3):
        tmp = _LIB3 + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                        "-fPIC", "-shared", "-o", tmp, _SRC3, "-lm"], check=True)
        os.replace(tmp, _LIB3)
    return _LIB3


class _Params3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("courant", ctypes.c_double),
        ("hyperdiffusion", ctypes.c_int),
        ("c2", ctypes.c_double * NF3),
        ("c_shk", ctypes.c_double),
        ("nthreads", ctypes.c_int),
    ]


_lib3 = None


def _load3():
    global _lib3
    if _lib3 is None:
        lib = ctypes.CDLL(build3())
        P = ctypes.POINTER(_Params3)
        dp = ctypes.POINTER(ctypes.c_double)
        d = ctypes.c_double
        lib.orc3_rhs.argtypes = [P, dp, d, d, d, dp]
        lib.orc3_cmax.argtypes = [P, dp, dp, dp, dp]
        lib.orc3_divb.argtypes = [P, dp, dp]
        lib.orc3_cfl_dt.argtypes = [P, d, d, d]
        lib.orc3_cfl_dt.restype = d
        lib.orc3_rk4_step.argtypes = [P, dp, d, d, d, d]
        lib.orc3_run.argtypes = [P, dp, dp, ctypes.c_long, d, ctypes.POINTER(ctypes.c_long)]
        lib.orc3_run.restype = ctypes.c_int
        _lib3 = lib
    return _lib3


@dataclass
class Problem3:
    """Periodic 3D grid on [x0,x1] x [y0,y1] x [z0,z1] (cell-centred)."""
    nx: int
    ny: int
    nz: int
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    z0: float = 0.0
    z1: float = 1.0
    gamma: float = 5.0 / 3.0
    courant: float = 0.3
    hyperdiffusion: int = 1
    c2: tuple = DEFAULT_C2_3D
    c_shk: float = DEFAULT_CSHK
    nthreads: int = field(default_factory=lambda: int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1)))

    def _c(self) -> _Params3:
        p = _Params3()
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        p.dx, p.dy, p.dz = (self.x1 - self.x0) / self.nx, (self.y1 - self.y0) / self.ny, (self.z1 - self.z0) / self.nz
        p.gamma, p.courant = self.gamma, self.courant
        p.hyperdiffusion = self.hyperdiffusion
        for i, v in enumerate(self.c2):
            p.c2[i] = v
        p.c_shk = self.c_shk
        p.nthreads = self.nthreads
        return p


def _state3(w, pr: Problem3):
    a = np.ascontiguousarray(w, dtype=np.float64)
    if a.shape != (NF3, pr.nz, pr.ny, pr.nx):
        raise ValueError(f"state must be ({NF3}, {pr.nz}, {pr.ny}, {pr.nx}), got {a.shape}")
    return a


def rhs3(pr: Problem3, w, cmax=(0.0, 0.0, 0.0)) -> np.ndarray:
    lib = _load3()
    w = _state3(w, pr)
    k = np.empty_like(w)
    lib.orc3_rhs(ctypes.byref(pr._c()), _dp(w), cmax[0], cmax[1], cmax[2], _dp(k))
    return k


def cmax3(pr: Problem3, w) -> tuple[float, float, float]:
    lib = _load3()
    w = _state3(w, pr)
    c = [ctypes.c_double() for _ in range(3)]
    lib.orc3_cmax(ctypes.byref(pr._c()), _dp(w), *[ctypes.byref(x) for x in c])
    return tuple(x.value for x in c)


def div_b3(pr: Problem3, w) -> np.ndarray:
    """Discrete div B per cell [nz][ny][nx] (fourth-order central differences, periodic box)."""
    lib = _load3()
    w = _state3(w, pr)
    div = np.zeros((pr.nz, pr.ny, pr.nx))
    lib.orc3_divb(ctypes.byref(pr._c()), _dp(w), _dp(div))
    return div


def cfl_dt3(pr: Problem3, cx: float, cy: float, cz: float) -> float:
    return _load3().orc3_cfl_dt(ctypes.byref(pr._c()), cx, cy, cz)


def rk4_step3(pr: Problem3, w, dt: float, cmax_xyz) -> np.ndarray:
    """One classical RK4 step of length dt with the given signal speeds (the
    hyper-diffusion coefficients use them); returns the new state."""
    lib = _load3()
    w = _state3(w, pr).copy()
    lib.orc3_rk4_step(ctypes.byref(pr._c()), _dp(w), float(dt), *(float(c) for c in cmax_xyz))
    return w


def run3(pr: Problem3, w, max_steps: int, fixed_dt: float = 0.0, t0: float = 0.0):
    """max_steps CFL steps (or fixed_dt > 0); returns (w, t, steps)."""
    lib = _load3()
    w = _state3(w, pr).copy()
    t = ctypes.c_double(t0)
    steps = ctypes.c_long(0)
    rc = lib.orc3_run(ctypes.byref(pr._c()), _dp(w), ctypes.byref(t), max_steps, fixed_dt, ctypes.byref(steps))
    if rc != 0:
        raise FloatingPointError(f"oracle 3D run turned non-finite after {steps.value} steps")
    return w, t.value, steps.value
