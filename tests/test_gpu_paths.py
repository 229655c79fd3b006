"""Per-path binding trees (Sec. 7.1) reconciled by local and global
tree-pruning (Sec. 8.1, 8.2) and joined: plans made with GS_PLAN_PATHS must
give exactly the oracle's answers, under both planners (the direction-driven
one has several roots on cyclic and disconnected queries, which is where
global pruning acts)."""
import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = pytest.mark.gpu

PATHS = gs.PLAN_PATHS


def _same(g, ix, pats, flags):
    got = g.query(pats, sort=True, flags=flags)
    want = ix.eval(pats, threads=4)
    assert got.shape == want.shape, (pats, flags, got.shape, want.shape)
    assert np.array_equal(got, want), (pats, flags)
    return want


@pytest.mark.parametrize("block", range(4))
def test_paths_random_tiny_cases(block):
    # the oracle is pinned to exhaustive enumeration on exactly these cases
    for seed in range(block * 60, block * 60 + 60):
        nv = 3 + seed % 5
        npred = 1 + seed % 3
        s, p, o = rdfgen.random_graph(seed, nv, npred, 4 + seed % 23)
        g = gs.Graph(s, p, o, nv, npred)
        ix = oracle.Index(s, p, o, nv, npred)
        q = rdfgen.random_bgp(seed + 7, nv, npred)
        _same(g, ix, q, PATHS)
        _same(g, ix, q, PATHS | gs.PLAN_DIRECTION)
        g.close()


def test_paths_rmat14_workload_and_shapes():
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    qs = [q.patterns for q in rdfgen.queries(w, sm)]
    shapes = [rdfgen.star(3), rdfgen.chain(3), rdfgen.cycle(3), rdfgen.cycle(4),
              rdfgen.snowflake([1, 2]), rdfgen.snowflake([2, 2])]
    for i, sh in enumerate(shapes * 2):
        qs.append(sm.sample(sh, 55, i, 2e5).patterns)
    sm.close()
    for pat in qs:
        for flags in (PATHS, PATHS | gs.PLAN_DIRECTION):
            rows = _same(g, ix, pat, flags)
            assert len(rows) >= 1
    g.close()


def test_paths_edge_cases():
    """A disconnected query (a product of components), a variable bound only
    by constants, a self-loop, parallel edges between one pair, and a
    query with no answer."""
    n_v, n_p = 40, 3
    s, p, o = rdfgen.random_graph(17, n_v, n_p, 500)
    s = np.concatenate([s, np.array([5, 6], np.uint32)])
    p = np.concatenate([p, np.array([1, 2], np.uint32)])
    o = np.concatenate([o, np.array([5, 6], np.uint32)])
    g = gs.Graph(s, p, o, n_v, n_p)
    ix = oracle.Index(s, p, o, n_v, n_p)
    cases = [
        [[-1, 1, -2], [-3, 2, -4]],                  # two components
        [[3, 1, -1], [-1, 2, 4]],                    # bound only by constants
        [[-1, 1, -1], [-1, 2, -2]],                  # self-loop
        [[-1, 1, -2], [-1, 2, -2], [-2, 3, -3]],     # parallel edges
        [[-1, 1, -2], [-2, 1, -1], [-1, 1, -1], [-2, 2, -2], [-2, 3, -3], [-3, 3, -2]],
    ]
    for pat in cases:
        for flags in (PATHS, PATHS | gs.PLAN_DIRECTION):
            _same(g, ix, np.array(pat, np.int64), flags)
    g.close()


def test_paths_trees_are_reported():
    """gs_result_tree reports one binding tree per path in this mode."""
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    plan = g.plan([[-1, 1, -2], [-1, 2, -3], [-1, 3, -4]], PATHS)   # a 3-leaf star: 3 paths
    r = g.eval(plan)
    assert len(r.tree()) == len(plan.paths()) == 3
    assert all(x > 0 for x in r.tree())
    r.close()
    g.close()
