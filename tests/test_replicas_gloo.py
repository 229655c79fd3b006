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


# ---- root-range partitioning of one query (Sec. 6.3.1's first stage) ----

def test_root_slices_partition_the_vertex_ids():
    from paper_2106_14038_b300 import replicas
    for n in (0, 1, 5, 31, 32, 33, 1000, 1 << 20):
        for k in (1, 2, 3, 7, 64):
            sl = replicas.root_slices(n, k)
            assert len(sl) == k
            assert sl[0][0] == 0 and sl[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
            sizes = [hi - lo for lo, hi in sl]
            assert max(sizes) - min(sizes) <= 1 and sum(sizes) == n
    with pytest.raises(ValueError):
        replicas.root_slices(10, 0)


def test_merge_rows_is_the_sorted_union():
    import numpy as np
    from paper_2106_14038_b300 import replicas
    rng = np.random.default_rng(3)
    rows = np.unique(rng.integers(0, 50, size=(400, 3)).astype(np.int32), axis=0)
    root = 1
    parts = [rows[(rows[:, root] >= lo) & (rows[:, root] < hi)]
             for lo, hi in replicas.root_slices(50, 4)]
    rng.shuffle(parts)                                   # any arrival order
    parts = [p[rng.permutation(len(p))] for p in parts]  # unsorted parts
    assert np.array_equal(replicas.merge_rows(parts), rows)
    assert replicas.merge_rows([], n_vars=3).shape == (0, 3)
    assert len(replicas.merge_rows(parts, sort=False)) == len(rows)


def _root_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    import rdfgen
    from paper_2106_14038_b300 import replicas
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=60))
    nv, npred = 60, 3
    s, p, o = rdfgen.random_graph(5, nv, npred, 700)
    ix = oracle.Index(s, p, o, nv, npred)
    pats = np.array([[-1, 1, -2], [-2, 2, -3], [-3, 1, -1]], np.int64)
    whole = ix.eval(pats)
    root = 1
    lo, hi = replicas.root_slices(nv, world)[rank]
    mine = whole[(whole[:, root] >= lo) & (whole[:, root] < hi)]   # this rank's answers
    got = replicas.gather_rows(mine, dist, n_vars=whole.shape[1])
    out.put((rank, bool(np.array_equal(got, whole)), len(mine), len(whole)))
    dist.barrier()
    dist.destroy_process_group()


def test_root_partition_gather_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_root_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _, _ in got)
    assert sum(n for _, _, n, _ in got) == got[0][3] > 0   # the ranges partition the answers
