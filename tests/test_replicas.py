"""The N > 1 benchmark path on CPU: two gloo ranks, each advancing its own
independent realisation (replicas, no collective on the data path), with the
time taken as the maximum over ranks."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, queue):
    import bench
    from oracle import lbm_oracle as O

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed = bench.replica_seed(rank)
    p = O.Params(nx=32, ny=48, seed=seed, crop_rows=5)
    f = O.step(O.initial_populations(p), p, 5)
    mass = float(O.densities(f)[0].sum())
    fake_elapsed = [1.0 + rank, 10.0 - rank]
    mx = bench.max_over_ranks(fake_elapsed)
    queue.put((rank, seed, mass, mx, O.interface_height(p)[:4].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, mx0, y0a), (r1, s1, m1, mx1, y0b) = out
    assert (s0, s1) == (1, 2)                       # distinct seeds: independent realisations
    assert y0a != y0b                               # different interface perturbations
    assert mx0 == mx1 == [2.0, 10.0]                # max over ranks, element-wise
    assert np.isclose(m0, m1, rtol=1e-6)            # same parameters, nearly the same total mass
