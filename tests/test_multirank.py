"""The multi-GPU path of bench.py on two CPU ranks (gloo): weak-scaling
workloads per rank and the max-over-ranks timing reduction.  The data path
has no collective (systems are independent), so this is all there is to
exchange between ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        class A:
            seed, systems = 11, 6
        ens = bench.rank_workload(A, rank)
        elapsed = 100.0 + 50.0 * rank                     # rank 1 is the slow one
        worst = bench.max_over_ranks(elapsed, dist, "cpu")
        value = bench.job_throughput(world, A.systems, 1000, 5, worst)
        out[rank] = (ens.n_systems, float(ens.pos[0, 1, 0]), worst, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_and_max_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
            assert p.exitcode == 0
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 6                            # same per-rank size (weak scaling)
    assert r0[1] != r1[1]                                 # different systems per rank
    assert r0[2] == r1[2] == 150.0                        # both ranks see the slowest time
    assert r0[3] == pytest.approx(2 * 6 * 1000 * 5 / 0.150)


def test_single_process_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
