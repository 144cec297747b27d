"""One 2D grid split across GPUs: bands of rows with ghost rows, and the halo exchange.

Streaming moves every population exactly one cell per time step (section 3,
Eq. 3-stencil-d2q5, lambda = dx/dt), so the scheme is a nearest-neighbour iteration: after
k steps a cell depends only on the cells at most k rows away.  Each rank (one process per
GPU) holds one band of rows [y0, y1) of the global grid plus H ghost rows on every side that
borders another band.  Between exchanges the band's own handle advances at most H steps
with an open (OUTFLOW) rule on those sides: the rule's values spoil the ghost rows one row
per step and never reach the band's own rows, which evolve exactly as in the undivided grid
(the same cell updates on the same values, so bit for bit).  The exchange then copies each
neighbour's outermost H rows of its own band into the ghost rows (all populations: the
ghost cells are recomputed, not just pulled from), and the next H steps can run.

Sides of the global grid keep their rules; with periodic y sides the bands form a ring.
The exchange is the only step with communication: two messages per cut and direction of
H x nx x 13 values, sent with torch.distributed point-to-point operations (NCCL between
GPUs, gloo for host tests); the diagnostics add one all-reduce of four numbers.  Every
compute step runs in the library's kernels (lbm_sw_get_rows / lbm_sw_set_rows copy the
rows; lbm_sw_diagnostics_rows reduces the band without its ghost rows).

``LocalStrips`` drives several bands in one process (sequential steps, direct copies): the
same arithmetic on one GPU, for tests.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lbm_sw

PERIODIC, OUTFLOW = lbm_sw.PERIODIC, lbm_sw.OUTFLOW
YM, YP = lbm_sw.YM, lbm_sw.YP


def band_rows(ny: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [y0, y1) of band `rank` of `world` bands: sizes differ by at most one row."""
    if not 0 <= rank < world or world < 1:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(ny, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


@dataclass
class BandLayout:
    """Where band `rank` sits: its rows [y0, y1) of the global grid, ghost rows below (lo)
    and above (hi) in its local grid, its neighbours (None at a side of the global grid), and
    the local boundary kinds (OUTFLOW on sides that border another band)."""

    rank: int
    world: int
    y0: int
    y1: int
    lo: int
    hi: int
    down: int | None
    up: int | None
    bc: tuple

    @property
    def rows(self) -> int:
        return self.y1 - self.y0

    @property
    def local_ny(self) -> int:
        return self.lo + self.rows + self.hi


def layout(ny: int, world: int, rank: int, halo: int, bc) -> BandLayout:
    bc = tuple(int(b) for b in bc)
    if len(bc) != 4:
        raise ValueError("bc: four sides")
    periodic_y = bc[YM] == PERIODIC
    y0, y1 = band_rows(ny, world, rank)
    if world == 1:
        return BandLayout(rank, world, y0, y1, 0, 0, None, None, bc)
    down = (rank - 1) % world if (rank > 0 or periodic_y) else None
    up = (rank + 1) % world if (rank < world - 1 or periodic_y) else None
    if y1 - y0 < halo:
        raise ValueError(f"band {rank} has {y1 - y0} rows, fewer than the {halo} ghost rows it sends")
    lo, hi = (halo if down is not None else 0), (halo if up is not None else 0)
    local = list(bc)
    local[YM] = OUTFLOW if down is not None else bc[YM]
    local[YP] = OUTFLOW if up is not None else bc[YP]
    return BandLayout(rank, world, y0, y1, lo, hi, down, up, tuple(local))


class Band:
    """One band: its layout and the handle that advances it (an lbm_sw.Simulation of
    nx x local_ny cells, or any object with the same methods)."""

    def __init__(self, nx: int, ny: int, rank: int, world: int, *, halo: int = 6, bc=(PERIODIC,) * 4,
                 stepper=None, **sim_kwargs):
        if halo < 1:
            raise ValueError("halo must be >= 1")
        self.nx, self.ny, self.halo = int(nx), int(ny), int(halo)
        self.L = layout(self.ny, world, rank, self.halo, bc)
        if stepper is None:
            if self.L.lo or self.L.hi:
                sim_kwargs.setdefault("temporal_steps", min(self.halo, 8) if self.halo >= 2 else 0)
            stepper = lbm_sw.Simulation(self.nx, self.L.local_ny, bc=self.L.bc, **sim_kwargs)
        self.sim = stepper
        if self.sim.nx != self.nx or self.sim.ny != self.L.local_ny:
            raise ValueError("stepper size does not match the band")
        spl = getattr(self.sim.info(), "steps_per_launch", 1) if hasattr(self.sim, "info") else 1
        if (self.L.lo or self.L.hi) and spl > self.halo:
            raise ValueError(f"the handle fuses {spl} steps per launch, more than the {self.halo} ghost rows")

    # -- state
    def local_rows(self) -> np.ndarray:
        """Global row index of every local row (ghost rows wrap around a periodic y)."""
        return np.arange(self.L.y0 - self.L.lo, self.L.y1 + self.L.hi) % self.ny

    def set_state(self, h, hu, hv):
        """Equilibrium state of the global fields (FP64 [ny][nx], numpy) on the band and its
        ghost rows."""
        r = self.local_rows()
        self.sim.set_state(*(np.ascontiguousarray(np.asarray(x)[r]) for x in (h, hu, hv)))

    def moments(self):
        """(h, hu, hv) of the band's own rows (FP64 [rows][nx])."""
        h, hu, hv = self.sim.moments()
        s = slice(self.L.lo, self.L.lo + self.L.rows)
        return h[s], hu[s], hv[s]

    def local_diagnostics(self):
        """(sum h, sum hu, sum hv, min h, status) over the band's own rows."""
        return self.sim.diagnostics_rows(self.L.lo, self.L.rows, False)

    # -- halo rows: (first local row, count) of what goes down / up and where it lands
    def send_down(self):
        return self.L.lo, self.halo

    def send_up(self):
        return self.L.lo + self.L.rows - self.halo, self.halo

    def recv_down(self):
        return 0, self.L.lo

    def recv_up(self):
        return self.L.lo + self.L.rows, self.L.hi


def _chunks(n: int, halo: int):
    while n > 0:
        m = min(n, halo)
        yield m
        n -= m


class DistributedStrips:
    """This process's band of a grid split over the ranks of a torch.distributed group.
    Rows travel as tensors on `device` (the GPU of this rank for NCCL, the host for gloo)."""

    def __init__(self, band: Band, *, device=None, group=None):
        import torch
        import torch.distributed as dist

        self.torch, self.dist = torch, dist
        self.band, self.group = band, group
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
                else torch.device("cpu")
        self.device = torch.device(device)
        tdtype = torch.float64 if band.sim.dtype == np.float64 else torch.float32
        shape = (band.sim.q, band.halo, band.nx)
        self.buf = {k: torch.empty(shape, dtype=tdtype, device=self.device)
                    for k in ("send_up", "send_down", "recv_up", "recv_down")}

    def step(self, n: int):
        """n time steps of the whole grid: at most `halo` steps between exchanges."""
        if self.band.L.world == 1:
            self.band.sim.step(n)
            return
        for m in _chunks(int(n), self.band.halo):
            self.band.sim.step(m)
            self.exchange()

    def exchange(self):
        b, L, dist = self.band, self.band.L, self.dist
        if L.down is None and L.up is None:
            return
        ops = []
        # upward messages first (my top rows to `up`, the rows of `down` into my lower ghost
        # rows), then downward: every rank posts the same order, so two messages between the
        # same two ranks (a ring of two) match in order
        if L.up is not None:
            b.sim.get_rows_into(*b.send_up(), self.buf["send_up"])
        if L.down is not None:
            b.sim.get_rows_into(*b.send_down(), self.buf["send_down"])
        if L.up is not None:
            ops.append(dist.P2POp(dist.isend, self.buf["send_up"], L.up, self.group, tag=1))
        if L.down is not None:
            ops.append(dist.P2POp(dist.irecv, self.buf["recv_down"], L.down, self.group, tag=1))
        if L.down is not None:
            ops.append(dist.P2POp(dist.isend, self.buf["send_down"], L.down, self.group, tag=2))
        if L.up is not None:
            ops.append(dist.P2POp(dist.irecv, self.buf["recv_up"], L.up, self.group, tag=2))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        if L.down is not None:
            b.sim.set_rows(*b.recv_down(), self.buf["recv_down"])
        if L.up is not None:
            b.sim.set_rows(*b.recv_up(), self.buf["recv_up"])

    def diagnostics(self):
        """(sum h, sum hu, sum hv, min h) of the whole grid and the number of ranks that saw an
        unstable cell: one all-reduce of the totals and one of the minimum."""
        torch, dist = self.torch, self.dist
        s0, s1, s2, mn, st = self.band.local_diagnostics()
        sums = torch.tensor([s0, s1, s2, 1.0 if st != lbm_sw.OK else 0.0], dtype=torch.float64, device=self.device)
        mins = torch.tensor([mn], dtype=torch.float64, device=self.device)
        if self.band.L.world > 1:
            dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=self.group)
            dist.all_reduce(mins, op=dist.ReduceOp.MIN, group=self.group)
        v = sums.cpu().tolist()
        return v[0], v[1], v[2], float(mins.cpu().item()), int(v[3])


class LocalStrips:
    """Every band of a split grid in this process, stepped one after the other and
    exchanged by direct copies (no communication library): the decomposition's arithmetic
    on one device."""

    def __init__(self, bands):
        self.bands = list(bands)
        self.halo = self.bands[0].halo
        self._tmp = None

    def _rows(self, b: Band, y0: int, n: int):
        if self._tmp is None or self._tmp.shape[1] != n:
            import torch

            on_gpu = isinstance(b.sim, lbm_sw.Simulation)
            tdtype = torch.float64 if b.sim.dtype == np.float64 else torch.float32
            self._tmp = torch.empty((b.sim.q, n, b.nx), dtype=tdtype, device="cuda" if on_gpu else "cpu")
        b.sim.get_rows_into(y0, n, self._tmp)
        return self._tmp

    def step(self, n: int):
        for m in _chunks(int(n), self.halo):
            for b in self.bands:
                b.sim.step(m)
            self.exchange()

    def exchange(self):
        # gather every band's outgoing rows first (the copies below overwrite ghost rows only)
        out = []
        for b in self.bands:
            L = b.L
            out.append((self._rows(b, *b.send_up()).clone() if L.up is not None else None,
                        self._rows(b, *b.send_down()).clone() if L.down is not None else None))
        for b in self.bands:
            L = b.L
            if L.down is not None:
                b.sim.set_rows(*b.recv_down(), out[L.down][0])
            if L.up is not None:
                b.sim.set_rows(*b.recv_up(), out[L.up][1])


def partition_instances(cells, world: int) -> list[list[int]]:
    """The instances of a batch (independent grids, cells[i] cells each) split over `world`
    ranks with no exchange between them: largest first, each to the rank with the least work
    so far (ties to the lower rank), so no rank carries more than the mean plus one instance.
    Returns the sorted instance indices of every rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += int(cells[i])
    return [sorted(p) for p in parts]
