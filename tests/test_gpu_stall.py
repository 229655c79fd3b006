"""A bounded device wait that runs out is reported as GS_ETIMEOUT and leaves
the context usable. GS_SCAN_STALL_CYCLES=0 makes every warp of the triple
scan give up its first wait for its bulk copies at once. Each warp still
waits, with the long limit, for the copies it has in flight before it
exits, so nothing is left running on the device. The status must reach the
caller from the query path (gs_result_info), from gs_scan_candidates and
from gs_scan_candidates_noalloc (gs_scan_status). The next calls, with the
default limit, must equal the oracle again."""
import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = pytest.mark.gpu

ETIMEOUT = 5


def _bits(words, n):
    w = np.asarray(words.cpu().numpy(), np.int64) & 0xffffffff
    return ((w[:, None] >> np.arange(32)) & 1).astype(np.uint8).reshape(-1)[:n]


def test_stalled_scan_is_reported_then_the_next_calls_are_exact(monkeypatch):
    import torch
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    # constant-free 3-cycle: its plan starts with a full triple scan
    cyc = np.array([[-1, 1, -2], [-2, 2, -3], [-3, 1, -1]], np.int64)
    want_rows = ix.eval(cyc)
    want_bits = ix.presence(0, 1) & ix.presence(1, 2)
    words = (w.n_vertices + 31) // 32
    out = torch.empty(words, dtype=torch.int32, device="cuda")

    monkeypatch.setenv("GS_SCAN_STALL_CYCLES", "0")
    r = g.eval(g.plan(cyc))
    with pytest.raises(gs.GsError) as e:
        r.info()
    assert e.value.status == ETIMEOUT
    r.close()
    g.scan([1, 2], [0, 1], out=out)
    with pytest.raises(gs.GsError) as e:
        g.scan_status()
    assert e.value.status == ETIMEOUT
    g.scan_status()                      # the report was cleared
    g.scan_noalloc([1, 2], [0, 1], out)
    with pytest.raises(gs.GsError) as e:
        g.scan_status()
    assert e.value.status == ETIMEOUT

    monkeypatch.delenv("GS_SCAN_STALL_CYCLES")
    got = g.query(cyc)
    assert np.array_equal(got, want_rows)
    for call in (lambda: g.scan([1, 2], [0, 1], out=out),
                 lambda: g.scan_noalloc([1, 2], [0, 1], out)):
        out.fill_(-1)
        call()
        g.scan_status()
        assert np.array_equal(_bits(out, w.n_vertices), want_bits)
    g.close()
