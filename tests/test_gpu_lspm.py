"""Per-query light-weight sparse matrices (Sec. 6.2), reduced on the device
from the resident store: Example 6.3's arrays, the reduced orientations
against the oracle's triples restricted to the kept predicates, and answers
evaluated on the reduced store against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = pytest.mark.gpu


def test_example_6_3_arrays(golden):
    """Ex. 6.3: drop the predicate no query uses (FriendOf), then the empty
    rows. The fixture's triples carry predicates 1..3; triples of a fourth
    predicate stand in for FriendOf (the figure's own ones are not in the
    text), one of them on the row the example eliminates."""
    gd = {k: [int(x) for x in v.split()] for k, v in golden("ex63_csr.txt")}
    rows = [i for i in range(8) if gd["Mr"][i + 1] - gd["Mr"][i] == 1]
    s, p, o = [], [], []
    for r, i in enumerate(rows):
        for k in range(gd["Pr"][r], gd["Pr"][r + 1]):
            s.append(i); p.append(gd["Val"][k]); o.append(gd["Col"][k])
    dropped = [i for i in range(8) if i not in rows]
    assert dropped == [3]
    for a, b in [(3, 6), (0, 7), (5, 2)]:              # the stand-in FriendOf triples
        s.append(a); p.append(4); o.append(b)
    g = gs.Graph(np.array(s), np.array(p), np.array(o), 8, 4)
    L = gs.Lspm(g, row_preds=[1, 2, 3], col_preds=[])
    m, ptr, val, col = L.export()
    assert m.tolist() == gd["Mr"]
    assert ptr.tolist() == gd["Pr"]
    for r in range(len(rows)):
        want = sorted(zip(gd["Val"][gd["Pr"][r]:gd["Pr"][r + 1]], gd["Col"][gd["Pr"][r]:gd["Pr"][r + 1]]))
        got = list(zip(val[ptr[r]:ptr[r + 1]].tolist(), col[ptr[r]:ptr[r + 1]].tolist()))
        assert got == want             # sorted by (label, column) inside the row
    assert L.info() == (7, 11)
    assert L.info(by_column=True) == (0, 0)
    L.close()
    g.close()


def _reduced_from_oracle(ix, n, preds, by_column):
    """Mr/Pr/Val/Idx of the orientation restricted to preds, from the
    oracle's sorted triples."""
    ts, tp, to = ix.triples(by_object=by_column)
    keep = np.isin(tp, np.array(sorted(preds), np.uint32))
    rows, other = (to, ts) if by_column else (ts, to)
    rows, lab, other = rows[keep], tp[keep], other[keep]
    cnt = np.bincount(rows.astype(np.int64), minlength=n)
    m = np.concatenate([[0], np.cumsum(cnt > 0)])
    ptr = np.concatenate([[0], np.cumsum(cnt[cnt > 0])])
    return m, ptr, lab, other


@pytest.mark.parametrize("seed", [3, 4])
def test_reduced_orientations_equal_the_oracle(seed):
    n_v, n_p = 2000, 12
    s, p, o = rdfgen.random_graph(seed, n_v, n_p, 30000)
    s = np.concatenate([s, np.full(5000, 17, np.uint32)])        # a hub row and column
    o = np.concatenate([o, np.full(5000, 17, np.uint32)])
    p = np.concatenate([p, (np.arange(5000) % n_p + 1).astype(np.uint32)])
    g = gs.Graph(s, p, o, n_v, n_p)
    ix = oracle.Index(s, p, o, n_v, n_p)
    rp, cp = [2, 5, 7, 12], [1, 5, 9]
    L = gs.Lspm(g, row_preds=rp, col_preds=cp)
    for by_col, preds in ((False, rp), (True, cp)):
        got = L.export(by_column=by_col)
        want = _reduced_from_oracle(ix, n_v, preds, by_col)
        for a, b in zip(got, want):
            assert np.array_equal(np.asarray(a, np.int64), np.asarray(b, np.int64))
    L.close()
    g.close()


@pytest.fixture(params=["auto", "grid"])
def exec_path(request, monkeypatch):
    monkeypatch.setenv("GS_EXEC", request.param)
    return request.param


def test_answers_on_the_lspm_equal_the_oracle(exec_path):
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    qs = [q.patterns for q in rdfgen.queries(w, sm)]
    a = 0
    while len(qs) < 14:                                   # constant-free cycles too
        q = sm.embed(rdfgen.cycle(3 + len(qs) % 2), 91, a, with_bound=False)
        a += 1
        if q is not None:
            qs.append(q.patterns)
    sm.close()
    for flags in (gs.PLAN_DEGREE, gs.PLAN_DEGREE | gs.PLAN_LISTS):
        for pat in qs:
            plan = g.plan(pat, flags)
            L = gs.Lspm.for_plan(g, plan)
            kept, nnz = L.info()
            assert nnz <= g.n_triples
            r = L.eval(plan)
            assert np.array_equal(r.fetch(), ix.eval(pat)), pat.tolist()
            r.close()
            L.close()
    g.close()


def test_eval_rejects_a_plan_outside_the_lspm():
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    L = gs.Lspm(g, row_preds=[1], col_preds=[1])
    with pytest.raises(gs.GsError) as e:
        L.eval(g.plan([[-1, 2, -2]]))
    assert e.value.status == 1
    L.close()
    g.close()
