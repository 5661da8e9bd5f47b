"""A block of the decomposed grid computed by the FP64 oracle on the CPU (test
infrastructure): the same interface as paper_1710_06423_b300.decomp.CudaDomain,
so the decomposition's exchange order, neighbour arithmetic and signal-speed
reduction can run on gloo ranks without a GPU.

A stage is the oracle's right-hand side of the block, whose split sides are
fixed and take their ghost values from the exchanged strips (the oracle's
"held" ghosts), followed by the classical RK4 combination in the oracle's own
order: U1 = U0 + dt/2 k1, U2 = U0 + dt/2 k2, U3 = U0 + dt k3,
U = U0 + dt/6 (((k1 + 2 k2) + 2 k3) + k4).  Ghosts of an unsplit periodic
direction are wrapped after every stage, as the GPU's ghost-frame kernel does.
"""
import numpy as np
import torch

G = 3


class OracleDomain:
    def __init__(self, oracle, grid, rank, **kw):
        from paper_1710_06423_b300.decomp import BOTTOM, LEFT, RIGHT, TOP
        self.o, self.grid, self.rank = oracle, grid, rank
        self.block = b = grid.block(rank)
        bc_x, bc_y = grid.local_bc(kw.pop("bc_x", 0), kw.pop("bc_y", 0))
        # the block takes the grid's own cell size bit for bit (the block's
        # extent over its cell count can differ from it in the last bit)
        class BlockProblem(oracle.Problem):
            dx = 1.0 / grid.nx
            dy = 1.0 / grid.ny
        self.pr = BlockProblem(nx=b.nx, ny=b.ny, bc_x=bc_x, bc_y=bc_y, nthreads=1, **kw)
        self.E = np.zeros((6, b.ny + 2 * G, b.nx + 2 * G))
        self.sides = (LEFT, RIGHT, BOTTOM, TOP)
        self.cx = self.cy = 0.0
        self.last = 0
        self._recv = {}

    # interior view of the ghost-extended latest output
    def _int(self):
        return self.E[:, G:-G, G:-G]

    def set_state(self, w_block, bg=None, t=0.0):
        self.E[:] = 0.0
        self._int()[:] = w_block
        self._wrap_unsplit()
        self.U0 = np.array(w_block, dtype=np.float64)
        self.cx, self.cy = self.o.cmax(self.pr, self.U0)
        self.last = 0

    def get_state(self):
        return self._int().copy(), 0.0

    def _wrap_unsplit(self):
        """Ghosts of unsplit periodic directions from the wrapped interior; a
        ghost outside a split (fixed) side is left to the exchange."""
        nx, ny = self.block.nx, self.block.ny
        px_split, py_split = self.grid.px > 1, self.grid.py > 1
        for gj in range(-G, ny + G):
            for gi in range(-G, nx + G):
                ox, oy = gi < 0 or gi >= nx, gj < 0 or gj >= ny
                if not (ox or oy) or (ox and px_split) or (oy and py_split):
                    continue
                self.E[:, gj + G, gi + G] = self.E[:, gj % ny + G, gi % nx + G]

    def stage(self, k):
        w_in = self._int().copy()
        kk = self.o.rhs(self.pr, w_in, held=self.E.reshape(-1).copy(), cmax=(self.cx, self.cy))
        if k == 1:
            self.dt = self.o.cfl_dt(self.pr, self.cx, self.cy)
            self.k1 = kk
            out = self.U0 + (0.5 * self.dt) * kk
        elif k == 2:
            self.k2 = kk
            out = self.U0 + (0.5 * self.dt) * kk
        elif k == 3:
            self.k3 = kk
            out = self.U0 + self.dt * kk
        else:
            out = self.U0 + (self.dt / 6.0) * (((self.k1 + 2.0 * self.k2) + 2.0 * self.k3) + kk)
            self.U0 = out.copy()
            self.cx, self.cy = self.o.cmax(self.pr, out)
        self._int()[:] = out
        self._wrap_unsplit()
        self.last = k

    def _strip(self, side, unpack):
        """Slices of E: the 3 interior cells next to `side` (pack) or the 3
        ghost cells beyond it (unpack); x strips over the extended height, y
        strips over the extended width (E index = cell index + 3)."""
        nx, ny = self.block.nx, self.block.ny
        n = nx if side < 2 else ny
        if side in (0, 2):
            lo = 0 if unpack else G                     # cells -3..-1  |  0..2
        else:
            lo = n + G if unpack else n                 # cells n..n+2  |  n-3..n-1
        sl = slice(lo, lo + G)
        if side < 2:
            return (slice(None), slice(0, ny + 2 * G), sl)
        return (slice(None), sl, slice(0, nx + 2 * G))

    def pack(self, side):
        return torch.from_numpy(np.ascontiguousarray(self.E[self._strip(side, False)]).reshape(-1))

    def strip_buffer(self, side):
        if side not in self._recv:
            self._recv[side] = torch.zeros(self.pack(side).numel(), dtype=torch.float64)
        return self._recv[side]

    def unpack(self, side, strip):
        sl = self._strip(side, True)
        shape = self.E[sl].shape
        self.E[sl] = strip.numpy().reshape(shape)

    def cmax_keys(self):
        return torch.from_numpy(np.array([self.cx, self.cy], dtype=np.float64).view(np.int64).copy())

    def set_cmax_keys(self, keys):
        self.cx, self.cy = (float(v) for v in keys.numpy().astype(np.int64).view(np.float64))
