"""Multi-rank host logic of the benchmark on CPU with two gloo ranks: each
rank builds its own events (whole events per rank, no data-path exchange) and
the step time is the maximum over ranks."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, torch.device("cpu"))
    b = bench.make_inputs("c0", rank)
    out[rank] = (t, float(b.x.sum()), b.n_seeds)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_events_and_take_max_time():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 2.5
    assert out[0][1] != out[1][1]  # different events per rank
    assert out[0][2] > 0 and out[1][2] > 0


def test_single_process_max_is_identity():
    import torch
    import bench
    assert bench.max_over_ranks(3.25, torch.device("cpu")) == 3.25
    assert np.isfinite(bench.fp32_peak_tflops())
