"""Triple scans shared across the constant-free plans of a batch (Sec. 5's
grouping applied across queries): one pass over the labels serves every
plan whose predicates fit its slots, and each plan then expands from the
candidate vectors that pass wrote for it. Answers must equal the oracle's
in both frontier forms (candidate bitmaps, or lists with predicate lookups
in label-sorted rows), shared or not, and a batch of plans must run fewer
scans (three kernel launches each) than plans."""
import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = pytest.mark.gpu


def _cycles(s, p, o, nv, npred, n, seed, sizes=(3, 4)):
    """Constant-free cycles sampled from embeddings (each has an answer)."""
    sm = rdfgen.Sampler(s, p, o, nv, npred)
    out, a = [], 0
    while len(out) < n:
        q = sm.embed(rdfgen.cycle(sizes[len(out) % len(sizes)]), seed, a, with_bound=False)
        a += 1
        if q is not None:
            out.append(q.patterns)
    sm.close()
    return out


@pytest.fixture(scope="module")
def rmat14():
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    pats = _cycles(s, p, o, w.n_vertices, w.n_preds, 10, 77)
    want = [ix.eval(q) for q in pats]
    return g, pats, want


@pytest.mark.parametrize("share,frontier", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_batch_of_constant_free_plans_equals_oracle(rmat14, share, frontier):
    g, pats, want = rmat14
    cfg = gs.BatchConfig(scan_share=share, frontier=frontier)
    plans = [g.plan(q) for q in pats]
    b = g.eval_batch(plans, config=cfg)
    for i in range(len(pats)):
        assert np.array_equal(b.fetch(i), want[i]), (share, frontier, i)
    n_scans, n_plans = b.scans()
    assert n_plans == len(pats)
    if share == 1:
        assert n_scans == 1           # 16 predicates fit one pass
    else:
        assert n_scans == len(pats)
    b.close()


def test_shared_scan_saves_three_launches_per_plan(rmat14):
    g, pats, want = rmat14
    plans = [g.plan(q) for q in pats]
    launches = {}
    for share in (1, 2):
        b = g.eval_batch(plans, config=gs.BatchConfig(scan_share=share))
        b.rows()
        launches[share] = b.stats()[1]
        b.close()
    assert launches[2] - launches[1] == 3 * (len(pats) - 1)


def test_list_form_plans_alone_equal_oracle(rmat14, monkeypatch):
    g, pats, want = rmat14
    for path in ("auto", "grid"):
        monkeypatch.setenv("GS_EXEC", path)
        for q, wnt in zip(pats, want):
            assert np.array_equal(g.query(q, flags=gs.PLAN_LISTS), wnt)


def test_wide_passes_beyond_16_predicates_per_direction():
    """Cycles over a 64-predicate graph. In the bitmap form every variable's
    predicates enter the scan: the union needs 32-bit masks and more than
    one pass. In the list form only the roots' predicates do (one out- and
    one in-predicate per 3-cycle), so one pass serves all 24."""
    n_v, n_p = 3000, 64
    s, p, o = rdfgen.random_graph(21, n_v, n_p, 60000)
    g = gs.Graph(s, p, o, n_v, n_p)
    ix = oracle.Index(s, p, o, n_v, n_p)
    pats = _cycles(s, p, o, n_v, n_p, 24, 5, sizes=(3,))
    preds = {int(x) for q in pats for x in q[:, 1]}
    assert len(preds) > 32
    for frontier in (1, 2):
        b = g.eval_batch([g.plan(q) for q in pats], config=gs.BatchConfig(frontier=frontier))
        for i, q in enumerate(pats):
            assert np.array_equal(b.fetch(i), ix.eval(q)), (frontier, i)
        n_scans, n_plans = b.scans()
        assert n_plans == len(pats)
        assert (2 <= n_scans < len(pats)) if frontier == 1 else n_scans == 1
        b.close()
        # the same plans three times over: a repeat adds no predicate to the
        # pass that holds its first occurrence, so it costs no further pass
        rep = pats * 3
        b = g.eval_batch([g.plan(q) for q in rep], config=gs.BatchConfig(frontier=frontier))
        for i, q in enumerate(rep):
            assert np.array_equal(b.fetch(i), ix.eval(q)), (frontier, i)
        assert b.scans() == (n_scans, len(rep))
        b.close()
    g.close()


def test_stalled_shared_scan_fails_every_plan_of_its_pass(rmat14, monkeypatch):
    g, pats, want = rmat14
    monkeypatch.setenv("GS_SCAN_STALL_CYCLES", "0")
    b = g.eval_batch([g.plan(q) for q in pats])
    with pytest.raises(gs.GsError) as e:
        b.rows()
    assert e.value.status == 5
    b.close()
    monkeypatch.delenv("GS_SCAN_STALL_CYCLES")
    b = g.eval_batch([g.plan(q) for q in pats])
    for i in range(len(pats)):
        assert np.array_equal(b.fetch(i), want[i])
    b.close()
