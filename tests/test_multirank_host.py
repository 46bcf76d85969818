"""The multi-rank bookkeeping of bench.py (slowest-rank time, whole-job
throughput) on two gloo ranks on the CPU. The path shards by independent
products, so ranks exchange nothing but this reduction and the barrier."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 40.0][rank]
    dist.barrier()
    got = bench.reduce_max(ms, world)
    out[rank] = got
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 40.0
    # whole-job throughput: both ranks' products over the slowest time
    products = 144 * 2
    assert products / (out[0] / 1e3) == pytest.approx(7200.0)


def test_reduce_max_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
