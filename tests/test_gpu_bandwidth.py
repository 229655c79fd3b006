"""The bandwidth-bound family end to end: the constant-free cycles of
rdfgen/<workload>_bandwidth.txt, each starting with a triple scan over
every label, evaluated one at a time, as one batch (shared scans) and
through the server, row for row against the oracle; on the scale-26 graph
(1.07e9 triples, the bandwidth configuration itself) and on the scale-22
copy (the same shapes, binding trees of about the same size). The oracle's
index needs about 40 GB of host memory at scale 26 beside the 13 GB of
triples; without it that case is skipped, saying so."""
import os

import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _host_gb():
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 2**20
    return 0.0


HOST_GB = {"rmat22": 8.0, "rmat26": 60.0}


@pytest.fixture(scope="module", params=["rmat22", "rmat26"])
def family(request):
    name = request.param
    need = HOST_GB[name]
    if _host_gb() < need:
        pytest.skip("host memory: %.0f GB available, the %s oracle needs about %.0f GB"
                    % (_host_gb(), name, need))
    w = rdfgen.WORKLOADS[name]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    del s, p, o
    qs = rdfgen.bandwidth_workload(w)
    threads = os.cpu_count() or 1
    want = [ix.eval(q.patterns, threads=threads) for q in qs]
    del ix
    yield w, g, qs, want
    g.close()


def test_bandwidth_workload_one_at_a_time(family):
    w, g, qs, want = family
    for q, wnt in zip(qs, want):
        assert q.bound >= len(wnt) >= 1
        assert np.array_equal(g.query(q.patterns), wnt), q.shape


def test_bandwidth_workload_batched_and_served(family):
    w, g, qs, want = family
    plans = [g.plan(q.patterns) for q in qs]
    for frontier in (1, 2):
        b = g.eval_batch(plans, config=gs.BatchConfig(frontier=frontier))
        for i in range(len(qs)):
            assert np.array_equal(b.fetch(i), want[i]), (frontier, qs[i].shape)
        n_scans, n_plans = b.scans()
        assert n_plans == len(qs) and n_scans < len(qs)
        b.close()
    srv = gs.Server(g)
    try:
        tickets = srv.submit_many(plans)
        for t, wnt in zip(tickets, want):
            while not srv.poll(t)[0]:
                pass
            assert np.array_equal(srv.fetch(t), wnt)
    finally:
        srv.stop()


def test_bandwidth_workload_root_ranges(family):
    """Root-range partitioning at full size: three queries (3-cycle, 4-cycle,
    3-cycle with a leaf), each evaluated over 3 ranges of the root ids; the
    parts hold only their roots and together give the whole answer."""
    from paper_2106_14038_b300 import replicas
    w, g, qs, want = family
    for i in (0, 1, 2):
        plan = g.plan(qs[i].patterns)
        root = plan.root_var
        parts = []
        for lo, hi in replicas.root_slices(g.n_vertices, 3):
            r = g.eval(plan, roots=(lo, hi))
            try:
                rows = r.fetch(sort=True)
            finally:
                r.close()
            if len(rows):
                assert rows[:, root].min() >= lo and rows[:, root].max() < hi
            parts.append(rows)
        assert np.array_equal(replicas.merge_rows(parts, n_vars=want[i].shape[1]), want[i]), qs[i].shape
