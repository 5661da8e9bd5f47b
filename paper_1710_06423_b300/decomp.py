"""Block decomposition of one grid over several sub-domains (the paper's
section 3: equal blocks, a halo exchange before every RK stage, and section 2's
maximum wave speed taken over the whole domain).

The paper moves its halos GPU -> host -> MPI -> host -> GPU.  Here a
sub-domain's strips stay in device memory: ``sac_halo_pack`` writes the 3-cell
strip next to a side into a device buffer, a transport moves it (in-process
device copies for sub-domains that share a process, ``torch.distributed``
point-to-point messages, NCCL on GPUs or gloo on CPUs, across processes), and
``sac_halo_unpack`` writes it into the neighbour's ghost cells.  The running
signal-speed maxima (two 64-bit keys per sub-domain) are reduced with a
maximum, so every sub-domain takes the same CFL step and hyper-diffusion
scale as the undivided grid: the decomposed run equals the single-grid run
bit for bit.

Only the exchange order and the neighbour arithmetic live here; every stage,
pack and unpack runs in the library's kernels (``Solver.stage`` and
``Solver.halo_*``).  A sub-domain is any object with the methods of
``CudaDomain``: ``stage(k)``, ``pack(side)``, ``unpack(side, strip)``,
``strip_buffer(side)``, ``cmax_keys()`` and ``set_cmax_keys(keys)``.

Split directions must be periodic on the whole grid (as in the paper's
Orszag-Tang runs); an unsplit direction keeps its own boundary kind.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .sac import BC_FIXED, BC_PERIODIC, NF, Solver

LEFT, RIGHT, BOTTOM, TOP = 0, 1, 2, 3
OPPOSITE = {LEFT: RIGHT, RIGHT: LEFT, BOTTOM: TOP, TOP: BOTTOM}
HALO = 3    # cells each stage reads beyond its own (the stencil reach, section 2)


ALIGN = 4  # block origins are multiples of the stage kernel's 4-cell sweep segment


def split(n: int, parts: int, align: int = ALIGN) -> list[tuple[int, int]]:
    """(start, count) of `parts` nearly equal pieces of n cells whose inner
    boundaries are multiples of `align` (the nearest multiple of align to
    k n / parts).

    The FP32 stage kernel sweeps each row and column in 4-cell segments, and a
    cell's last-place rounding can depend on its position inside its segment
    (measured: one cell in ~6400 differs by one unit in the last place when the
    grid is shifted by a cell count that is not a multiple of 4).  Aligning every
    block to the segment length keeps each cell where the undivided grid has
    it, so the decomposed run stays bit-for-bit the single-grid run."""
    bounds = [0] + [int(round(k * n / parts / align)) * align for k in range(1, parts)] + [n]
    return [(bounds[k], bounds[k + 1] - bounds[k]) for k in range(parts)]


@dataclass(frozen=True)
class Block:
    rank: int
    cx: int
    cy: int
    x0: int
    nx: int
    y0: int
    ny: int


class ProcessGrid:
    """px x py blocks of an nx x ny grid; rank = cy * px + cx (x fastest)."""

    def __init__(self, nx: int, ny: int, px: int, py: int):
        if px < 1 or py < 1:
            raise ValueError("px and py must be >= 1")
        self.nx, self.ny, self.px, self.py = nx, ny, px, py
        self.xs, self.ys = split(nx, px), split(ny, py)
        if (px > 1 and min(c for _, c in self.xs) < HALO) or (py > 1 and min(c for _, c in self.ys) < HALO):
            raise ValueError(f"every block needs at least {HALO} cells across a split direction")

    @property
    def size(self) -> int:
        return self.px * self.py

    def block(self, rank: int) -> Block:
        cx, cy = rank % self.px, rank // self.px
        (x0, nx), (y0, ny) = self.xs[cx], self.ys[cy]
        return Block(rank, cx, cy, x0, nx, y0, ny)

    def neighbor(self, rank: int, side: int) -> int:
        """The rank across `side` (periodic wrap of the process grid)."""
        cx, cy = rank % self.px, rank // self.px
        if side == LEFT:
            cx = (cx - 1) % self.px
        elif side == RIGHT:
            cx = (cx + 1) % self.px
        elif side == BOTTOM:
            cy = (cy - 1) % self.py
        else:
            cy = (cy + 1) % self.py
        return cy * self.px + cx

    def phases(self) -> list[tuple[int, int]]:
        """The exchange phases, x before y: x strips span the ghost-extended
        height and y strips the ghost-extended width, so the y phase carries
        the corner cells the x phase has just filled."""
        out = []
        if self.px > 1:
            out.append((LEFT, RIGHT))
        if self.py > 1:
            out.append((BOTTOM, TOP))
        return out

    def local_bc(self, bc_x: int, bc_y: int) -> tuple[int, int]:
        """Boundary kinds of a block: split sides are fixed (their ghosts come
        from the exchange), unsplit ones keep the grid's own kind."""
        if self.px > 1 and bc_x != BC_PERIODIC:
            raise ValueError("a split direction must be periodic")
        if self.py > 1 and bc_y != BC_PERIODIC:
            raise ValueError("a split direction must be periodic")
        return (BC_FIXED if self.px > 1 else bc_x), (BC_FIXED if self.py > 1 else bc_y)

    def scatter(self, w: np.ndarray, rank: int) -> np.ndarray:
        b = self.block(rank)
        return np.ascontiguousarray(w[:, b.y0:b.y0 + b.ny, b.x0:b.x0 + b.nx])

    def gather(self, parts: dict[int, np.ndarray]) -> np.ndarray:
        first = next(iter(parts.values()))
        out = np.empty((first.shape[0], self.ny, self.nx), dtype=first.dtype)
        for r, a in parts.items():
            b = self.block(r)
            out[:, b.y0:b.y0 + b.ny, b.x0:b.x0 + b.nx] = a
        return out


class CudaDomain:
    """One block on the GPU: a library context of the block's size whose split
    sides are fixed, with preallocated device strips."""

    def __init__(self, grid: ProcessGrid, rank: int, **params):
        import torch
        self.grid, self.rank = grid, rank
        self.block = grid.block(rank)
        bc_x, bc_y = grid.local_bc(params.pop("bc_x", BC_PERIODIC), params.pop("bc_y", BC_PERIODIC))
        x0, x1 = params.pop("x0", 0.0), params.pop("x1", 1.0)
        y0, y1 = params.pop("y0", 0.0), params.pop("y1", 1.0)
        dx, dy = (x1 - x0) / grid.nx, (y1 - y0) / grid.ny
        b = self.block
        self.solver = Solver(nx=b.nx, ny=b.ny, x0=x0 + b.x0 * dx, x1=x0 + (b.x0 + b.nx) * dx,
                             y0=y0 + b.y0 * dy, y1=y0 + (b.y0 + b.ny) * dy, bc_x=bc_x, bc_y=bc_y, **params)
        # the grid's own cell size, bit for bit (the block's extent over its cell
        # count can differ from it in the last bit)
        self.solver.set_cell_size(dx, dy)
        self.dtype = torch.float32 if self.solver.fp32 else torch.float64
        dev = torch.device("cuda", self.solver.params.device)
        self._send = {s: torch.empty(self.solver.halo_size(s), dtype=self.dtype, device=dev)
                      for side_pair in grid.phases() for s in side_pair}
        self._recv = {s: torch.empty_like(t) for s, t in self._send.items()}
        self._keys = torch.zeros(2, dtype=torch.int64, device=dev)

    def set_state(self, w_block, bg=None, t: float = 0.0):
        self.solver.set_state(w_block, bg, t)

    def get_state(self):
        return self.solver.get_state()

    def stage(self, k: int):
        self.solver.stage(k)

    def pack(self, side: int):
        self.solver.halo_pack(side, self._send[side])
        return self._send[side]

    def strip_buffer(self, side: int):
        return self._recv[side]

    def unpack(self, side: int, strip):
        self.solver.halo_unpack(side, strip)

    def cmax_keys(self):
        self.solver.get_cmax_bits(self._keys)
        return self._keys

    def set_cmax_keys(self, keys):
        self.solver.set_cmax_bits(keys)

    def close(self):
        self.solver.close()


# ---- in-process driver: every block in this process ---------------------------------
def exchange_local(grid: ProcessGrid, domains: dict):
    """Halo exchange among blocks that share a process (device copies)."""
    for sides in grid.phases():
        packed = {(r, s): d.pack(s) for r, d in domains.items() for s in sides}
        for r, d in domains.items():
            for s in sides:
                # the strip the neighbour across s packed toward this block
                d.unpack(s, packed[(grid.neighbor(r, s), OPPOSITE[s])])


def reduce_cmax_local(domains: dict):
    """Maximum of every block's signal-speed keys, given back to all."""
    import torch
    keys = [d.cmax_keys() for d in domains.values()]
    m = keys[0].clone()
    for k in keys[1:]:
        m = torch.maximum(m, k)
    for d in domains.values():
        d.set_cmax_keys(m)


def start_local(grid: ProcessGrid, domains: dict):
    """After every block's set_state: ghosts of the initial state and the
    global signal speeds of it."""
    exchange_local(grid, domains)
    reduce_cmax_local(domains)


def step_local(grid: ProcessGrid, domains: dict, nsteps: int = 1):
    """nsteps RK4 steps of all blocks held by this process."""
    for _ in range(nsteps):
        for k in (1, 2, 3, 4):
            for d in domains.values():
                d.stage(k)
            exchange_local(grid, domains)
        reduce_cmax_local(domains)


# ---- one block per process (torch.distributed: NCCL on GPUs, gloo on CPUs) --------
def exchange_dist(grid: ProcessGrid, domain, rank: int, dist, group=None):
    """Halo exchange of this process's block with its neighbours.

    Message order: each rank sends its strips toward (LEFT, RIGHT) [or
    (BOTTOM, TOP)] in that order and receives into its (RIGHT, LEFT) [(TOP,
    BOTTOM)] ghosts in that order, so that with two blocks along a direction,
    where both neighbours are the same rank, the i-th message between the pair
    matches the i-th receive (NCCL matches point-to-point messages in order;
    gloo also gets the sender's side as the tag)."""
    for sides in grid.phases():
        ops, recvs = [], []
        for s in sides:
            ops.append(dist.P2POp(dist.isend, domain.pack(s), grid.neighbor(rank, s), group, tag=s))
        for s in reversed(sides):
            buf = domain.strip_buffer(s)
            # the neighbour across s sent its strip toward OPPOSITE[s]
            ops.append(dist.P2POp(dist.irecv, buf, grid.neighbor(rank, s), group, tag=OPPOSITE[s]))
            recvs.append((s, buf))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for s, buf in recvs:
            domain.unpack(s, buf)


def reduce_cmax_dist(domain, dist, group=None):
    keys = domain.cmax_keys()
    dist.all_reduce(keys, op=dist.ReduceOp.MAX, group=group)
    domain.set_cmax_keys(keys)


def start_dist(grid: ProcessGrid, domain, rank: int, dist, group=None):
    exchange_dist(grid, domain, rank, dist, group)
    reduce_cmax_dist(domain, dist, group)


def step_dist(grid: ProcessGrid, domain, rank: int, dist, nsteps: int = 1, group=None):
    """nsteps RK4 steps of this process's block (every rank calls it)."""
    for _ in range(nsteps):
        for k in (1, 2, 3, 4):
            domain.stage(k)
            exchange_dist(grid, domain, rank, dist, group)
        reduce_cmax_dist(domain, dist, group)
