"""Server admission by estimated intermediate-result bytes. A query whose
estimate does not fit the remaining budget waits; later queries that fit
pass it; every answer equals the same query run alone and the oracle."""
import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = pytest.mark.gpu

MiB = 1 << 20


def _embedded(sm, shape, n, seed):
    out, a = [], 0
    while len(out) < n:
        q = sm.embed(shape, seed, a, with_bound=False)
        a += 1
        if q is not None:
            out.append(q.patterns)
    return out


def test_large_query_waits_and_smaller_ones_pass_it(monkeypatch):
    import time
    # every grid-path query starts with a 256 MiB workspace, so the estimate
    # of a constant-free query (which runs on the grid path) is about that
    monkeypatch.setenv("GS_ARENA_BYTES", str(256 * MiB))
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    big = _embedded(sm, rdfgen.cycle(3), 2, 31)                  # X, then L
    star = rdfgen.star(2)
    star.const = [1]                                             # one leaf constant
    small = _embedded(sm, star, 8, 32)                           # S1..S8 (batch kernel)
    sm.close()
    X, L = g.plan(big[0]), g.plan(big[1])
    S = [g.plan(q) for q in small]
    budget = 420 * MiB        # X + all S fit; X + L do not; L alone does
    srv = gs.Server(g, n_streams=2, max_batch=72, max_wait_us=2_000_000, memory_budget=budget)
    try:
        _run_and_check(srv, g, ix, X, L, S, big, small, budget)
    finally:
        srv.stop()
        g.close()


def _run_and_check(srv, g, ix, X, L, S, big, small, budget):
    import time
    tx = srv.submit(X)
    tl, *ts = srv.submit_many([L] + S)
    tickets = [tx, tl] + ts
    t0 = time.time()
    while not all(srv.poll(t)[0] for t in tickets):
        assert time.time() - t0 < 60
        time.sleep(0.001)
    seq = {t: srv.ticket(t)[0] for t in tickets}
    est = {t: srv.ticket(t)[1] for t in tickets}
    assert est[tl] >= 256 * MiB and all(est[t] < 32 * MiB for t in ts)
    assert all(seq[tl] > seq[t] for t in ts), seq          # the S plans passed L
    passed, _ = srv.admission()
    assert passed >= 1
    completed, batches, peak = srv.stats()
    assert completed == len(tickets) and peak <= budget
    for t, pl, pat in zip(tickets, [X, L] + S, big + small):
        got = srv.fetch(t)
        assert np.array_equal(got, ix.eval(pat))
        assert np.array_equal(got, g.query(pat))


def test_plan_estimates_scale_with_the_query():
    """A constant-free star over the most frequent predicate is estimated far
    larger than the same star seeded by a constant; the estimate covers the
    control block at least."""
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    free_star = g.plan([[-1, 1, -2], [-1, 1, -3]])
    c = int(s[np.flatnonzero(p == 1)[0]])
    seeded = g.plan([[c, 1, -1], [-1, 1, -2]])
    bf, rf = g.estimate(free_star)
    bs, rs = g.estimate(seeded)
    assert bf > bs > 0 and rf > rs > 0
    g.close()
