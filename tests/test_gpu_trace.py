"""Tracing: with Graph.set_trace(True) a grid-path evaluation records CUDA
events between its phases (setup + triple scan, each level, enumeration).
The phases must number the levels + 2, be non-negative, add up to the
evaluation's device time, and leave the answers unchanged."""
import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = pytest.mark.gpu


def test_phases_of_grid_path_evaluations(monkeypatch):
    monkeypatch.setenv("GS_EXEC", "grid")
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    qs = [q.patterns for q in rdfgen.queries(w, sm)]
    sm.close()
    try:
        plan = g.plan(qs[0])
        r = g.eval(plan)
        r.info()
        with pytest.raises(gs.GsError, match="GS_ENOTIMPL"):   # tracing off
            r.phases()
        r.close()
        g.set_trace(True)
        for pat in qs:
            plan = g.plan(pat)
            r = g.eval(plan)
            try:
                assert np.array_equal(r.fetch(sort=True), ix.eval(pat))
                ph = r.phases()
                tree = r.tree()
                assert len(ph) == len(tree) + 2
                assert min(ph) >= 0.0
                total = r.time_ms()
                assert sum(ph) == pytest.approx(total, rel=0.05, abs=0.02)
            finally:
                r.close()
        g.set_trace(False)
        r = g.eval(g.plan(qs[1]))
        r.info()
        with pytest.raises(gs.GsError, match="GS_ENOTIMPL"):
            r.phases()
        r.close()
    finally:
        g.close()
