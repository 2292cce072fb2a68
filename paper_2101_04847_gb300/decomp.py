"""Domain decomposition of one grid along x over several solvers (an extension of
the paper's runs, which keep a grid on one GPU).

The grid's columns are cut into consecutive sub-grids, one solver each, created with
the sub-grid's place in the whole grid (``x_offset``, ``nx_total``: the initial
interface follows the whole grid).  Each time step every sub-grid advances alone
(the block-staged or decoupled kernels, which read the two columns beside the grid
from ghost columns), then the ghost columns are refilled from the neighbours: a
sub-grid's left ghosts are its left neighbour's last two columns, its right ghosts
its right neighbour's first two (``lbm_halo_pack`` / ``lbm_halo_unpack``).  The
split run equals the whole-grid run bit for bit.

Two drivers share the exchange pattern:
  * ``LocalSplit``: every sub-grid in this process, on one device; the edge columns
    go from buffer to buffer on the device.
  * ``DistSplit``: one sub-grid per rank of ``torch.distributed`` (launched one
    process per GPU); NCCL carries device buffers, gloo goes through host memory.
This module only moves buffers: every step of the method runs in the CUDA kernels.
"""
from __future__ import annotations

import contextlib
from typing import Callable


def split_columns(nx: int, parts: int) -> list[tuple[int, int]]:
    """Column ranges [x0, x1) of `parts` sub-grids of nearly equal width (each at
    least two columns wide, so that its edge columns exist)."""
    if parts < 1 or nx < 2 * parts:
        raise ValueError(f"cannot split {nx} columns into {parts} sub-grids of two columns or more")
    edges = [round(k * nx / parts) for k in range(parts + 1)]
    return [(edges[k], edges[k + 1]) for k in range(parts)]


def neighbours(rank: int, world: int) -> tuple[int, int]:
    """Left and right neighbour of sub-grid `rank` (periodic in x)."""
    return (rank - 1) % world, (rank + 1) % world


def _new_stream():
    import torch

    return torch.cuda.Stream()


def _on(stream):
    """Run the enclosed torch work on `stream` (None: as it is)."""
    if stream is None:
        return contextlib.nullcontext()
    import torch

    return torch.cuda.stream(stream)


class SolverPart:
    """One sub-grid solved by the CUDA library, with device buffers for its two edges
    (sent) and two ghosts (received)."""

    def __init__(self, params: dict, x0: int, x1: int, nx_total: int, kernel: str = "staged", stream=None):
        import torch

        from paper_2101_04847_gb300 import lbm

        if kernel not in ("staged", "decoupled"):
            raise ValueError("a split grid needs a kernel that reads ghost columns: 'staged' or 'decoupled'")
        d = dict(params)
        d.update(nx=x1 - x0, x_offset=x0, nx_total=nx_total, kernel=kernel)
        # the solver's kernels and the buffer copies of the exchange run on one stream
        with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
            self.solver = lbm.Solver(lbm.default_params(**d))
        n = self.solver.halo_bytes()
        self.send = [torch.empty(n, dtype=torch.uint8, device="cuda") for _ in range(2)]
        self.recv = [torch.empty(n, dtype=torch.uint8, device="cuda") for _ in range(2)]

    def step(self):
        self.solver.step(1)

    def pack(self):
        for side in (0, 1):
            self.solver.halo_pack(side, self.send[side].data_ptr())

    def unpack(self):
        for side in (0, 1):
            self.solver.halo_unpack(side, self.recv[side].data_ptr())

    def close(self):
        self.solver.close()


class LocalSplit:
    """All sub-grids of a split grid in this process, on the current device."""

    def __init__(self, params: dict, parts: int, kernel: str = "staged",
                 make_part: Callable[..., object] | None = None):
        nx = params["nx"]
        self.stream = _new_stream() if make_part is None else None
        make = make_part or (lambda x0, x1: SolverPart(params, x0, x1, nx, kernel, self.stream))
        self.cols = split_columns(nx, parts)
        self.parts = [make(x0, x1) for x0, x1 in self.cols]
        self.exchange()

    def exchange(self):
        with _on(self.stream):
            for q in self.parts:
                q.pack()
            n = len(self.parts)
            for k, q in enumerate(self.parts):
                left, right = self.parts[(k - 1) % n], self.parts[(k + 1) % n]
                q.recv[0].copy_(left.send[1])
                q.recv[1].copy_(right.send[0])
                q.unpack()

    def step(self, n: int = 1):
        for _ in range(n):
            for q in self.parts:
                q.step()
            self.exchange()

    def close(self):
        for q in self.parts:
            q.close()


class DistSplit:
    """One sub-grid per rank of the default torch.distributed group.  Device buffers
    travel by NCCL point-to-point operations; with another backend (gloo) they go
    through host memory."""

    def __init__(self, params: dict, kernel: str = "staged", make_part: Callable[..., object] | None = None):
        import torch.distributed as dist

        self.dist = dist
        self.world = dist.get_world_size()
        self.rank = dist.get_rank()
        nx = params["nx"]
        self.cols = split_columns(nx, self.world)
        x0, x1 = self.cols[self.rank]
        self.stream = _new_stream() if make_part is None else None
        self.part = make_part(x0, x1) if make_part else SolverPart(params, x0, x1, nx, kernel, self.stream)
        self.device_transport = dist.get_backend() == "nccl"
        self.exchange()

    def exchange(self):
        with _on(self.stream):
            self._exchange()

    def _exchange(self):
        import torch

        dist, q = self.dist, self.part
        q.pack()
        left, right = neighbours(self.rank, self.world)
        if self.world == 1:
            q.recv[0].copy_(q.send[1])
            q.recv[1].copy_(q.send[0])
        elif self.device_transport:
            ops = [dist.P2POp(dist.isend, q.send[0], left), dist.P2POp(dist.irecv, q.recv[1], right),
                   dist.P2POp(dist.isend, q.send[1], right), dist.P2POp(dist.irecv, q.recv[0], left)]
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        else:
            send = [b.cpu() for b in q.send]          # waits for the packs on the current stream
            recv = [torch.empty_like(b) for b in send]
            # tags tell the two messages apart when both neighbours are the same rank
            reqs = [dist.isend(send[0], left, tag=0), dist.irecv(recv[1], right, tag=0),
                    dist.isend(send[1], right, tag=1), dist.irecv(recv[0], left, tag=1)]
            for r in reqs:
                r.wait()
            for side in (0, 1):
                q.recv[side].copy_(recv[side])
        q.unpack()

    def step(self, n: int = 1):
        for _ in range(n):
            self.part.step()
            self.exchange()

    def close(self):
        self.part.close()
