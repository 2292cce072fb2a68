"""Domain decomposition along x on the GPU: a grid split into sub-grids, one solver
each, with the edge columns exchanged after every step (lbm_halo_pack /
lbm_halo_unpack), equals the whole-grid solver bit for bit.  All sub-grids in one
process (device copies), and one sub-grid per process on two gloo ranks sharing the
GPU (host transport; the kernels of the two processes never wait for each other)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2101_04847_gb300 import decomp, lbm
from tests import inputs

pytestmark = pytest.mark.gpu

BASE = inputs.params(inputs.C0, nx=300, ny=72, crop_rows=4, g=1e-4, amp=4.0, seed=5)
STEPS = 30


def whole_run(d, kernel, steps=STEPS):
    with lbm.Solver(kernel=kernel, **d) as s:
        f0 = s.populations()
        s.step(steps)
        return f0, s.populations()


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("kernel,storage", [("staged", "f32"), ("decoupled", "f32"), ("staged", "f16"),
                                            ("decoupled", "bf16")])
def test_local_split_equals_the_whole_grid(gpu, parts, kernel, storage):
    d = dict(BASE, storage=storage, wall_mode=1 if storage == "bf16" else 0)
    f0, want = whole_run(d, kernel)
    run = decomp.LocalSplit(d, parts, kernel=kernel)
    try:
        start = np.concatenate([q.solver.populations() for q in run.parts], axis=-1)
        run.step(STEPS)
        got = np.concatenate([q.solver.populations() for q in run.parts], axis=-1)
    finally:
        run.close()
    assert np.array_equal(start, f0)        # the sub-grids start from the whole grid's state
    assert np.array_equal(got, want)


def test_split_needs_a_ghost_reading_kernel(gpu):
    with pytest.raises(ValueError):
        decomp.LocalSplit(BASE, 2, kernel="fused")


def test_halo_calls_reject_a_bad_side(gpu):
    import ctypes as C

    import torch

    with lbm.Solver(**BASE) as s:
        buf = torch.empty(s.halo_bytes(), dtype=torch.uint8, device="cuda")
        assert s.halo_bytes() == 36 * BASE["ny"] * 4
        assert s.lib.lbm_halo_pack(s._h, 2, C.c_void_p(buf.data_ptr())) == lbm.LBM_EINVAL
        assert s.lib.lbm_halo_unpack(s._h, -1, C.c_void_p(buf.data_ptr())) == lbm.LBM_EINVAL


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, queue):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    run = decomp.DistSplit(BASE, kernel="staged")
    run.step(STEPS)
    queue.put((rank, run.part.solver.populations()))
    dist.barrier()
    run.close()
    dist.destroy_process_group()


def test_two_ranks_on_one_gpu_equal_the_whole_grid(gpu):
    _, want = whole_run(BASE, "staged")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert np.array_equal(np.concatenate([o for _, o in out], axis=-1), want)
