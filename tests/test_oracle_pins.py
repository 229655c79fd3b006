"""Pins of the oracle to things other than itself: exhaustive enumeration on
tiny graphs, closed-form counts, the paper's worked examples and invariants
of the BGP semantics (Sec. 2.2.3). CPU only."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import rdfgen


def brute_force(s, p, o, n_vertices, n_preds, patterns):
    """All assignments of the variables, kept when every pattern's triple
    is in the graph. Exhaustive: n_vertices ** n_vars candidates."""
    adj = np.zeros((n_preds + 1, n_vertices, n_vertices), bool)
    adj[p, s, o] = True
    k = int(max(-x for t in patterns for x in (t[0], t[2]) if x < 0))
    cand = np.indices((n_vertices,) * k).reshape(k, -1).T
    ok = np.ones(len(cand), bool)
    for ts, tp, to in patterns:
        sv = cand[:, -ts - 1] if ts < 0 else np.full(len(cand), ts)
        ov = cand[:, -to - 1] if to < 0 else np.full(len(cand), to)
        ok &= adj[tp, sv, ov]
    rows = cand[ok].astype(np.int32)
    if len(rows):
        rows = rows[np.lexsort(rows.T[::-1])]
    return rows.reshape(-1, k)


@pytest.mark.parametrize("block", range(8))
def test_oracle_equals_brute_force(block):
    for seed in range(block * 100, block * 100 + 100):
        nv = 3 + seed % 5
        npred = 1 + seed % 3
        s, p, o = rdfgen.random_graph(seed, nv, npred, 4 + seed % 23)
        ix = oracle.Index(s, p, o, nv, npred)
        q = rdfgen.random_bgp(seed + 7, nv, npred)
        want = brute_force(s, p, o, nv, npred, q)
        got = ix.eval(q, threads=1 + seed % 3)
        assert got.shape == want.shape, (seed, q.tolist())
        assert np.array_equal(got, want), (seed, q.tolist())


def _dedup(s, p, o):
    t = np.unique(np.stack([s, p, o], 1).astype(np.int64), axis=0)
    return t[:, 0], t[:, 1], t[:, 2]


def _adj(s, o, mask, n):
    m = sp.csr_matrix((np.ones(int(mask.sum()), np.int64), (s[mask], o[mask])), shape=(n, n))
    m.sum_duplicates()
    m.data[:] = 1
    return m


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_star_count_closed_form(seed):
    # centre x with out-edges p1..pk and one in-edge q: |R| = sum_i prod deg
    w = rdfgen.Workload("t", 10, 6000, 5, 1.0, 77 + seed, 0, 0, 0)
    s, p, o = rdfgen.graph(w)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    ds, dp, do = _dedup(s, p, o)
    outs, inn = [1, 2, 2 + seed % 3], 3
    pats = [(-1, q, -(j + 2)) for j, q in enumerate(outs)] + [(-(len(outs) + 2), inn, -1)]
    cnt = np.ones(w.n_vertices, np.float64)
    for q in outs:
        cnt *= np.bincount(ds[dp == q], minlength=w.n_vertices)
    cnt *= np.bincount(do[dp == inn], minlength=w.n_vertices)
    assert len(ix.eval(pats, threads=4)) == int(cnt.sum())


@pytest.mark.parametrize("seed", [1, 2])
def test_chain_count_closed_form(seed):
    # x0 -p1-> x1 -p2-> x2 -p3-> x3: |R| = 1^T A1 A2 A3 1
    w = rdfgen.Workload("t", 10, 6000, 4, 1.0, 91 + seed, 0, 0, 0)
    s, p, o = rdfgen.graph(w)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    ds, dp, do = _dedup(s, p, o)
    preds = [1, 2, 1 + seed]
    pats = [(-(j + 1), q, -(j + 2)) for j, q in enumerate(preds)]
    v = np.ones(w.n_vertices, np.int64)
    for q in reversed(preds):
        v = _adj(ds, do, dp == q, w.n_vertices) @ v
    assert len(ix.eval(pats, threads=2)) == int(v.sum())


@pytest.mark.parametrize("seed", [1, 2])
def test_cycle_count_closed_form(seed):
    # x -p1-> y -p2-> z -p3-> x: |R| = trace(A1 A2 A3) (homomorphisms, loops included)
    w = rdfgen.Workload("t", 9, 5000, 3, 1.0, 55 + seed, 0, 0, 0)
    s, p, o = rdfgen.graph(w)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    ds, dp, do = _dedup(s, p, o)
    a = [_adj(ds, do, dp == q, w.n_vertices) for q in (1, 2, 1 + seed)]
    tr = int((a[0] @ a[1] @ a[2]).diagonal().sum())
    pats = [(-1, 1, -2), (-2, 2, -3), (-3, 1 + seed, -1)]
    assert len(ix.eval(pats)) == tr


def test_single_predicate_triangle_is_trace_a_cubed():
    w = rdfgen.Workload("t", 8, 3000, 1, 1.0, 5, 0, 0, 0)
    s, p, o = rdfgen.graph(w)
    ds, dp, do = _dedup(s, p, o)
    a = _adj(ds, do, dp == 1, w.n_vertices).toarray()
    ix = oracle.Index(s, p, o, w.n_vertices, 1)
    got = len(ix.eval([(-1, 1, -2), (-2, 1, -3), (-3, 1, -1)]))
    assert got == int(np.trace(a @ a @ a))


def _eq1(golden):
    g = dict(golden("eq1_algebra.txt"))
    m = np.array(g["matrix"].split(), int).reshape(3, 3)
    s, o = np.nonzero(m)
    return g, s.astype(np.uint32), m[s, o].astype(np.uint32), o.astype(np.uint32)


def test_eq6_eq7_presence(golden):
    g, s, p, o = _eq1(golden)
    ix = oracle.Index(s, p, o, 3, 9)
    for tag, d in (("eq6", 0), ("eq7", 1)):
        f = g[tag].split()
        pred = int(f[0].split("=")[1])
        want = np.array(f[2:], np.uint8)
        assert np.array_equal(ix.presence(d, pred), want), tag


def test_eq9_label_positions(golden):
    g, s, p, o = _eq1(golden)
    ix = oracle.Index(s, p, o, 3, 9)
    f = g["eq9"].split()
    pred = int(f[0].split("=")[1])
    rows = ix.eval([(-1, pred, -2)])
    assert rows.tolist() == [[int(f[1]), int(f[2])]]


def test_eq10_eq11_grouped_step1(golden):
    # Eq. 17 is the AND of presence vectors; Eq. 10/11 fix AND / OR of vectors
    g, s, p, o = _eq1(golden)
    for tag, op in (("eq10", np.logical_and), ("eq11", np.logical_or)):
        f = g[tag].replace("&", " ").replace("|", " ").replace("=", " ").split()
        x, y, z = (np.array(f[i:i + 3], int) for i in (0, 3, 6))
        assert np.array_equal(op(x, y).astype(int), z)
    ix = oracle.Index(s, p, o, 3, 9)
    # rows holding both a and b (Eq. 17 on Eq. 1) = the conjunctive query result
    v = ix.presence(0, 1) & ix.presence(0, 2)
    rows = ix.eval([(-1, 1, -2), (-1, 2, -3)])
    assert sorted(set(rows[:, 0].tolist())) == np.nonzero(v)[0].tolist()


def test_eq2_eq3_selection(golden):
    g, s, p, o = _eq1(golden)
    ix = oracle.Index(s, p, o, 3, 9)
    ts, tp, to = ix.triples()
    m = np.zeros((3, 3), int)
    m[ts, to] = tp
    f = g["eq2"].split()
    keep = [int(x) for x in f[0].split("=")[1].split(",")]
    sel = np.zeros_like(m)
    sel[keep] = m[keep]
    assert sel.reshape(-1).tolist() == [int(x) for x in f[1:]]
    f = g["eq3"].split()
    keep = [int(x) for x in f[0].split("=")[1].split(",")]
    sel = np.zeros_like(m)
    sel[:, keep] = m[:, keep]
    assert sel.reshape(-1).tolist() == [int(x) for x in f[1:]]


def _ex63(golden):
    g = {k: [int(x) for x in v.split()] for k, v in golden("ex63_csr.txt")}
    mr, pr, val, col = g["Mr"], g["Pr"], g["Val"], g["Col"]
    rows = [i for i in range(len(mr) - 1) if mr[i + 1] - mr[i] == 1]
    s, p, o = [], [], []
    for r, i in enumerate(rows):
        for k in range(pr[r], pr[r + 1]):
            s.append(i); p.append(val[k]); o.append(col[k])
    return g, np.array(s, np.uint32), np.array(p, np.uint32), np.array(o, np.uint32)


def test_ex63_row_wise_matrix(golden):
    g, s, p, o = _ex63(golden)
    assert len(s) == 11
    ix = oracle.Index(s, p, o, 8, 3)
    ts, tp, to = ix.triples()
    ptr, col, lab = oracle.csr_arrays(ts, tp, to, 8)
    nonempty = np.diff(ptr) > 0
    mr = np.concatenate([[0], np.cumsum(nonempty)])
    assert mr.tolist() == g["Mr"]
    pr = np.concatenate([[0], np.cumsum(np.diff(ptr)[nonempty])])
    assert pr.tolist() == g["Pr"]
    # within a row the paper's order is free; compare row contents as multisets
    for r, i in enumerate(np.nonzero(nonempty)[0]):
        want = sorted(zip(g["Val"][g["Pr"][r]:g["Pr"][r + 1]], g["Col"][g["Pr"][r]:g["Pr"][r + 1]]))
        got = sorted(zip(lab[ptr[i]:ptr[i + 1]].tolist(), col[ptr[i]:ptr[i + 1]].tolist()))
        assert got == want


def test_duplicates_removed_and_rows_distinct():
    s = np.array([0, 0, 0, 1, 1], np.uint32)
    p = np.array([1, 1, 2, 1, 1], np.uint32)
    o = np.array([1, 1, 1, 0, 0], np.uint32)
    ix = oracle.Index(s, p, o, 2, 2)
    assert len(ix) == 3
    assert ix.eval([(-1, 1, -2)]).tolist() == [[0, 1], [1, 0]]
    # two predicates between the same pair are two triples (one nonzero each)
    assert ix.eval([(-1, 1, -2), (-1, 2, -2)]).tolist() == [[0, 1]]


def test_self_loop_and_repeated_variable():
    s = np.array([0, 1, 2], np.uint32)
    p = np.array([1, 1, 1], np.uint32)
    o = np.array([0, 2, 2], np.uint32)
    ix = oracle.Index(s, p, o, 3, 1)
    assert ix.eval([(-1, 1, -1)]).tolist() == [[0], [2]]
    assert ix.eval([(-1, 1, -2), (-2, 1, -2)]).tolist() == [[0, 0], [1, 2], [2, 2]]


def test_invalid_queries_rejected():
    ix = oracle.Index(np.array([0], np.uint32), np.array([1], np.uint32), np.array([1], np.uint32), 2, 1)
    for q in ([(0, 1, 1)], [(-1, 2, -2)], [(-1, 0, -2)], [(-1, 1, -3)], [(5, 1, -1)]):
        with pytest.raises(ValueError):
            ix.eval(q)


@pytest.mark.parametrize("seed", range(6))
def test_invariants(seed):
    w = rdfgen.Workload("t", 9, 3000, 4, 1.0, 300 + seed, 0, 0, 0)
    s, p, o = rdfgen.graph(w)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    T = set(zip(*(x.tolist() for x in _dedup(s, p, o))))
    rng = np.random.default_rng(seed)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    for sh in (rdfgen.chain(2), rdfgen.cycle(3), rdfgen.star(3)):
        q = sm.embed(sh, 9 + seed, 0, with_bound=False)
        if q is None:
            continue
        pats = q.patterns
        base = ix.eval(pats)
        # the embedding that produced the query is one of the answers
        emb = tuple(int(q.embedding[v]) for v in range(sh.n_v))
        assert emb in set(map(tuple, base.tolist()))
        # every row satisfies every pattern (checked against the triple set)
        for row in base[:2000]:
            for ts, tp, to in pats:
                a = row[-ts - 1] if ts < 0 else ts
                b = row[-to - 1] if to < 0 else to
                assert (a, tp, b) in T
        # pattern order does not matter
        perm = rng.permutation(len(pats))
        assert np.array_equal(ix.eval(pats[perm]), base)
        # renaming variables permutes the columns
        k = base.shape[1]
        ren = rng.permutation(k)
        p2 = pats.copy()
        for c in (0, 2):
            m = p2[:, c] < 0
            p2[m, c] = -ren[-p2[m, c] - 1] - 1
        r2 = ix.eval(p2)
        back = r2[:, ren]
        back = back[np.lexsort(back.T[::-1])]
        assert np.array_equal(back, base)
        # adding a pattern never adds answers
        extra = np.array([[pats[0][0], 1 + seed % w.n_preds, pats[-1][2]]], np.int64)
        sub = ix.eval(np.concatenate([pats, extra]))
        assert set(map(tuple, sub.tolist())) <= set(map(tuple, base.tolist()))


@pytest.mark.parametrize("seed", range(4))
def test_count_mode_equals_row_count(seed):
    """The count mode walks the same join without storing rows: its count is
    the number of rows eval returns, on any thread count; a step limit below
    the join's work is reported as incomplete with a lower bound."""
    s, p, o = rdfgen.random_graph(seed + 40, 40, 3, 400)
    ix = oracle.Index(s, p, o, 40, 3)
    for q in range(30):
        pat = rdfgen.random_bgp(seed * 1000 + q, 40, 3, max_vars=4, max_patterns=4)
        rows = ix.eval(pat)
        for t in (1, 3):
            n, steps, done = ix.count(pat, threads=t)
            assert done and n == len(rows)
        n, steps, done = ix.count(pat)
        if steps > 4:
            m, _, done2 = ix.count(pat, max_steps=2)
            assert not done2 and m <= n


def test_index_sorted_copies_are_sorted_and_deduplicated():
    """The bucket-sorted copies hold the set of triples, each in its order."""
    s, p, o = rdfgen.random_graph(9, 300, 5, 20000)
    ix = oracle.Index(s, p, o, 300, 5)
    want = sorted(set(zip(s.tolist(), p.tolist(), o.tolist())))
    ts, tp, to = ix.triples()
    assert list(zip(ts.tolist(), tp.tolist(), to.tolist())) == want
    bs, bp, bo = ix.triples(by_object=True)
    assert list(zip(bo.tolist(), bp.tolist(), bs.tolist())) == sorted((c, b, a) for a, b, c in want)
