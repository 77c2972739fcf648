"""The N > 1 bench path on CPU (gloo, world size 2): every rank gets the
slowest rank's time, the whole-job value counts all ranks' units, and the
reference arm prints on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    v = bench.weak_scaling_value(world, 8, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * 8 / 15.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.weak_scaling_value(1, 8, 2.0) == 4.0


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import argparse

    import bench
    bench.run_reference(argparse.Namespace(steps=1, warmup=0), 1, 2)
    assert capsys.readouterr().out == ""
