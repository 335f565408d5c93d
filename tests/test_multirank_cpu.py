"""Multi-rank host logic of the benchmark on CPU with two gloo ranks: each
rank builds its own events (whole events per rank, no data-path exchange),
the step time is the maximum over ranks, and the one exchange of the path --
the sum over ranks of the alignment gradient and the chi2 of the fit -- equals
the single-process sum."""
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
    assert abs(bench.fp32_peak_tflops(152) - 80.54784) < 1e-9  # 152 SMs x 128 lanes x 2 x 2.07 GHz


def _fit_case(rank):
    """Rank `rank`'s events: a small fit-only batch (true hit lists), its
    oracle chi2 sum and alignment gradient."""
    import oracle
    from synth import make_batch
    from synth.events import true_hit_lists
    b = make_batch("c3", tracks=60, seed=1003 + rank)
    lists, n = true_hit_lists(b, 0, b.det.n_layers)
    lists, n = lists[b.seed_sim], n[b.seed_sim]
    x, y, z, lay = b.event_hits(0)
    tot, ga, gh, gs, each = oracle.fit_grad(b.det, b.params, b.cov, lists, n, x, y, z, lay, b.align)
    return tot, ga


def _exchange_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    tot, ga = _fit_case(rank)
    g, c = bench.sum_alignment_over_ranks(ga, tot, torch.device("cpu"))
    out[rank] = (g.tolist(), c)
    dist.destroy_process_group()


def test_alignment_gradient_sum_over_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_exchange_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    ref = [_fit_case(r) for r in range(world)]
    g_ref = ref[0][1] + ref[1][1]
    c_ref = ref[0][0] + ref[1][0]
    for r in range(world):
        g, c = np.array(out[r][0]), out[r][1]
        assert g.shape == (17, 2)
        assert np.allclose(g, g_ref, rtol=1e-12, atol=0) and abs(c - c_ref) <= 1e-12 * c_ref
    assert not np.allclose(ref[0][1], ref[1][1])  # the ranks contributed different events
