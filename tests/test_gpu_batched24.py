"""The batched configuration at full size: the 4,096 queries of
tests/golden/rmat24_batched.txt on the scale-24 graph (268M triples) in one
batch. Each query's answer count must equal the exact count the oracle
gave when the file was written (make_rmat24_batched.py, oracle count
mode), and a sample of the queries must give the oracle's rows exactly."""
import os

import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

STORED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rmat24_batched.txt")


@pytest.fixture(scope="module")
def rmat24():
    if not os.path.exists(STORED):
        pytest.skip("tests/golden/rmat24_batched.txt is not written")
    w = rdfgen.WORKLOADS["rmat24"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    qs = rdfgen.load_queries(STORED)
    yield w, (s, p, o), g, qs
    g.close()


def test_batched_counts_equal_the_oracle_counts(rmat24):
    w, _, g, qs = rmat24
    assert len(qs) >= 3000
    plans = [g.plan(q.patterns) for q in qs]
    b = g.eval_batch(plans)
    try:
        rows = np.asarray(b.rows(), np.int64)
        want = np.array([int(q.bound) for q in qs], np.int64)
        bad = np.nonzero(rows != want)[0]
        assert len(bad) == 0, [(int(i), qs[i].shape, int(rows[i]), int(want[i])) for i in bad[:10]]
        assert (rows >= 1).all()
    finally:
        b.close()


def test_batched_rows_equal_the_oracle_on_a_sample(rmat24):
    w, (s, p, o), g, qs = rmat24
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    pick = [i for i, q in enumerate(qs) if q.bound <= 2e5][::32][:96]
    assert len(pick) >= 64
    plans = [g.plan(qs[i].patterns) for i in pick]
    b = g.eval_batch(plans)
    try:
        for k, i in enumerate(pick):
            want = ix.eval(qs[i].patterns, threads=os.cpu_count() or 1)
            assert np.array_equal(b.fetch(k), want), (i, qs[i].shape)
    finally:
        b.close()
