"""Multi-rank host logic of bench.py on CPU: two gloo ranks on 127.0.0.1 agree on
the max-over-ranks time and the whole-job throughput (weak scaling: every rank
evaluates its own full batch, nothing is exchanged but the time)."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = 1.5 + rank  # seconds this rank measured
    mx = bench.reduce_max(local, world, "cpu")
    out[rank] = (mx, bench.throughput(64, world, 10, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_and_throughput():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    mx, value = out[0]
    assert mx == 2.5
    assert abs(value - 64 * 2 * 10 / 2.5) < 1e-12


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.25, 1) == 3.25
    assert bench.throughput(64, 1, 100, 0.5) == 64 * 100 / 0.5
