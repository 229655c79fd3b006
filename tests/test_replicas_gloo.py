"""Multi-process host logic on CPU (gloo, world size 2): the replica
aggregation of bench.py (units of all ranks / slowest rank's time) and
detection of a rank that dies before the collective. No GPU."""
import datetime
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _agg_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=30))
    rate, t_ms = bench.aggregate_rate(100.0 * (rank + 1), 32, world, dist, device="cpu")
    out.put((rank, rate, t_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_agg_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, t_ms in got:
        assert t_ms == pytest.approx(200.0)        # max over ranks
        assert rate == pytest.approx(2 * 32 / 0.2)  # all ranks' units / that time


def _fail_worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(3)                   # dies between steps, before the next collective
    import torch
    try:
        t = torch.ones(1)
        dist.all_reduce(t)
        out.put((rank, "no error"))
    except Exception as e:            # the survivor learns of it on the host
        out.put((rank, "detected: %s" % type(e).__name__))
    out.close()
    out.join_thread()                 # flush the queue before the hard exit
    os._exit(0)


def test_dead_rank_is_detected_on_host():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_fail_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    rank, msg = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
    assert rank == 0 and msg.startswith("detected"), msg
    assert ps[1].exitcode == 3 and ps[0].exitcode == 0
