"""Root-range partitioning (the first-stage partition of Sec. 6.3.1) on one
GPU: a query evaluated once per range of a partition of the vertex ids must
give, concatenated, exactly the whole answer set (each row once), every
part holding only rows whose root binding lies in its range; and the whole
equals the oracle's answers."""
import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen
from paper_2106_14038_b300 import replicas

pytestmark = pytest.mark.gpu


def _check_slices(g, ix, pats, flags, parts_list=(1, 2, 5, 64)):
    plan = g.plan(pats, flags)
    root = plan.root_var
    want = ix.eval(pats, threads=4)
    whole = g.query(pats, sort=True, flags=flags)
    assert np.array_equal(whole, want), (pats, flags)
    for k in parts_list:
        got = []
        for lo, hi in replicas.root_slices(g.n_vertices, k):
            r = g.eval(plan, roots=(lo, hi))
            try:
                rows = r.fetch(sort=True)
            finally:
                r.close()
            assert rows.shape[1] == want.shape[1]
            if len(rows):
                assert rows[:, root].min() >= lo and rows[:, root].max() < hi, (pats, k, lo, hi)
            assert np.array_equal(rows, want[(want[:, root] >= lo) & (want[:, root] < hi)])
            got.append(rows)
        merged = replicas.merge_rows(got, n_vars=want.shape[1])
        assert np.array_equal(merged, want), (pats, flags, k)
    return want


@pytest.mark.parametrize("block", range(3))
def test_root_slices_random_tiny_cases(block):
    # tiny random graphs and BGPs (constants, loops, repeated variables)
    for seed in range(block * 50, block * 50 + 50):
        nv = 3 + seed % 6
        npred = 1 + seed % 3
        s, p, o = rdfgen.random_graph(seed, nv, npred, 4 + seed % 23)
        g = gs.Graph(s, p, o, nv, npred)
        ix = oracle.Index(s, p, o, nv, npred)
        q = rdfgen.random_bgp(seed + 7, nv, npred)
        for flags in (gs.PLAN_DEGREE, gs.PLAN_DIRECTION, gs.PLAN_LISTS):
            _check_slices(g, ix, q, flags, parts_list=(1, 2, 3, nv + 2))
        g.close()


def test_root_slices_rmat14_workload_and_shapes():
    """Scan-rooted (constant-free) shapes, whose root level is compacted from
    a candidate vector, and constant-rooted ones, whose root level is
    expanded from a constant's row, across slices that cut words of the
    candidate vector at odd offsets (64 ranges of 256 of the 16,384 vertices
    and 7 ranges of 2,340 or 2,341)."""
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    qs = [q.patterns for q in rdfgen.queries(w, sm)][:12]
    shapes = [rdfgen.star(3), rdfgen.chain(3), rdfgen.cycle(3), rdfgen.cycle(4),
              rdfgen.snowflake([1, 2])]
    for i, sh in enumerate(shapes):
        qs.append(sm.sample(sh, 55, i, 2e5).patterns)
    sm.close()
    for pat in qs:
        for flags in (gs.PLAN_DEGREE, gs.PLAN_LISTS):
            rows = _check_slices(g, ix, pat, flags, parts_list=(1, 7, 64))
            assert len(rows) >= 1
    g.close()


def test_root_range_edge_cases():
    n_v, n_p = 40, 3
    s, p, o = rdfgen.random_graph(17, n_v, n_p, 500)
    s = np.concatenate([s, np.array([5, 6], np.uint32)])
    p = np.concatenate([p, np.array([1, 2], np.uint32)])
    o = np.concatenate([o, np.array([5, 6], np.uint32)])
    g = gs.Graph(s, p, o, n_v, n_p)
    ix = oracle.Index(s, p, o, n_v, n_p)
    pats = np.array([[-1, 1, -2], [-2, 2, -3]], np.int64)
    want = ix.eval(pats, threads=2)
    assert len(want) > 0
    plan = g.plan(pats)

    def rows(lo, hi):
        r = g.eval(plan, roots=(lo, hi))
        try:
            return r.fetch(sort=True)
        finally:
            r.close()

    assert len(rows(0, 0)) == 0                     # empty range
    assert len(rows(7, 7)) == 0
    assert len(rows(n_v, n_v + 100)) == 0           # past the last vertex
    assert np.array_equal(rows(0, 0xFFFFFFFF), want)   # the whole id space
    # self-loop roots and a root bound only by constants
    for pat in ([[-1, 1, -1], [-1, 2, -2]], [[3, 1, -1], [-1, 2, 4]], [[-1, 1, -2], [-3, 2, -4]]):
        _check_slices(g, ix, np.array(pat, np.int64), gs.PLAN_DEGREE, parts_list=(1, 3, 40))
    with pytest.raises(gs.GsError, match="GS_EINVAL"):
        g.eval(plan, roots=(5, 4))
    paths_plan = g.plan(pats, gs.PLAN_PATHS)
    with pytest.raises(gs.GsError, match="GS_EINVAL"):
        g.eval(paths_plan, roots=(0, 10))
    g.close()
