"""Domain decomposition along x on CPU (no GPU): the split oracle against the whole
grid, on one process and on two gloo ranks, and the product's exchange pattern
(paper_2101_04847_gb300.decomp) driving oracle-stepped sub-grids on two gloo ranks.
Each must equal the whole-grid oracle bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import lbm_oracle as O
from oracle import split_oracle as S

PARAMS = dict(nx=40, ny=32, G=1.4, g=1e-4, seed=4, amp=3.0, crop_rows=4, G_wall_A=0.1)
STEPS = 12


def whole(p, steps=STEPS):
    return O.step(O.initial_populations(p), p, steps)


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("wall_mode", [0, 1])
def test_split_oracle_equals_the_whole_grid(parts, wall_mode):
    p = O.Params(**PARAMS, wall_mode=wall_mode)
    f = O.initial_populations(p)
    got = S.step_split([f[..., a:b] for a, b in S.split_columns(p.nx, parts)], p, STEPS)
    assert np.array_equal(np.concatenate(got, axis=-1), whole(p))


class OraclePart:
    """A sub-grid stepped by the split oracle behind the part interface the product's
    exchange drives: send[0] / send[1] take its first / last two columns, recv[0] /
    recv[1] are written into its left / right ghost columns."""

    def __init__(self, f, p, x0, x1):
        self.p = p
        self.own = f[..., x0:x1].copy()
        shape = self.own[..., :2].shape
        self.send = [torch.zeros(shape, dtype=torch.float64) for _ in range(2)]
        self.recv = [torch.zeros(shape, dtype=torch.float64) for _ in range(2)]

    def pack(self):
        self.send[0].copy_(torch.from_numpy(self.own[..., :2].copy()))
        self.send[1].copy_(torch.from_numpy(self.own[..., -2:].copy()))

    def unpack(self):
        self.left, self.right = self.recv[0].numpy().copy(), self.recv[1].numpy().copy()

    def step(self):
        self.own = S.step_widened(S.widen(self.own, self.left, self.right), self.p)

    def close(self):
        pass


def test_local_exchange_pattern_with_oracle_parts():
    from paper_2101_04847_gb300 import decomp

    p = O.Params(**PARAMS)
    f = O.initial_populations(p)
    run = decomp.LocalSplit(dict(nx=p.nx), 3, make_part=lambda x0, x1: OraclePart(f, p, x0, x1))
    run.step(STEPS)
    assert np.array_equal(np.concatenate([q.own for q in run.parts], axis=-1), whole(p))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, queue, use_product):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = O.Params(**PARAMS)
    f = O.initial_populations(p)
    if use_product:
        from paper_2101_04847_gb300 import decomp

        run = decomp.DistSplit(dict(nx=p.nx), make_part=lambda x0, x1: OraclePart(f, p, x0, x1))
        run.step(STEPS)
        own = run.part.own
    else:
        # the split oracle's own exchange over gloo: edges to the neighbours, ghosts back
        x0, x1 = S.split_columns(p.nx, world)[rank]
        own = f[..., x0:x1].copy()
        left, right = (rank - 1) % world, (rank + 1) % world
        for _ in range(STEPS):
            send = [torch.from_numpy(own[..., :2].copy()), torch.from_numpy(own[..., -2:].copy())]
            recv = [torch.empty_like(send[0]), torch.empty_like(send[1])]
            reqs = [dist.isend(send[0], left, tag=0), dist.irecv(recv[1], right, tag=0),
                    dist.isend(send[1], right, tag=1), dist.irecv(recv[0], left, tag=1)]
            for r in reqs:
                r.wait()
            own = S.step_widened(S.widen(own, recv[0].numpy(), recv[1].numpy()), p)
    queue.put((rank, own))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("use_product", [False, True])
def test_two_gloo_ranks_equal_the_whole_grid(use_product):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, use_product)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    got = np.concatenate([o for _, o in out], axis=-1)
    assert np.array_equal(got, whole(O.Params(**PARAMS)))


def test_a_five_row_band_steps_its_centre_row_exactly():
    # the full-size parity test steps only the band of rows y - 2 .. y + 2 around a
    # sampled row y (cut to the grid at the walls): the band's own edges act as walls,
    # which changes its outer rows but not row y
    p = O.Params(**PARAMS)
    f = whole(p)
    full = O.step(f, p, 1)
    for y in (0, 1, 2, 15, 16, p.ny - 2, p.ny - 1):
        lo = max(0, y - 2)
        band = f[:, :, lo:min(p.ny, y + 3)]
        got = O.step(band, p.with_(ny=band.shape[2]), 1)[:, :, y - lo]
        assert np.array_equal(got, full[:, :, y]), y
    # a band of three rows is too narrow: the centre row then differs
    y = 16
    narrow = O.step(f[:, :, y - 1:y + 2], p.with_(ny=3), 1)[:, :, 1]
    assert not np.array_equal(narrow, full[:, :, y])
