"""CUDA path against the oracle, element by element, through the C ABI.

Every comparison is exact (integer ids): the store's arrays, the candidate
vectors of the triple scan (Eq. 17 / Eq. 21) and the sorted answer rows."""
import os

import numpy as np
import pytest

import oracle
import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = pytest.mark.gpu


@pytest.fixture(params=["auto", "grid"])
def exec_path(request, monkeypatch):
    """auto: single-block kernel for plans without a full scan (escalating
    to the grid path when a level is large); grid: always the grid path."""
    monkeypatch.setenv("GS_EXEC", request.param)
    return request.param


def _graph(s, p, o, nv, npred):
    return gs.Graph(s, p, o, nv, npred), oracle.Index(s, p, o, nv, npred)


def _bits_to_bool(words, n):
    w = np.asarray(words.cpu().numpy(), np.int64) & 0xffffffff
    b = ((w[:, None] >> np.arange(32)) & 1).astype(bool).reshape(-1)
    return b[:n]


@pytest.fixture(scope="module")
def rmat14():
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    g, ix = _graph(s, p, o, w.n_vertices, w.n_preds)
    return w, (s, p, o), g, ix


def test_store_matches_oracle(rmat14):
    w, _, g, ix = rmat14
    assert g.n_triples == len(ix)
    for by_col in (0, 1):
        ts, tp, to = ix.triples(by_object=bool(by_col))
        rows, other = (to, ts) if by_col else (ts, to)
        ptr, idx, lab = oracle.csr_arrays(rows, tp, other, w.n_vertices)
        gp, gi, gl = g.export(by_column=bool(by_col))
        assert np.array_equal(gp.astype(np.int64), ptr)
        assert np.array_equal(gi, idx)
        assert np.array_equal(gl, lab)


def test_store_example_6_3(golden):
    g = {k: [int(x) for x in v.split()] for k, v in golden("ex63_csr.txt")}
    rows = [i for i in range(8) if g["Mr"][i + 1] - g["Mr"][i] == 1]
    s, p, o = [], [], []
    for r, i in enumerate(rows):
        for k in range(g["Pr"][r], g["Pr"][r + 1]):
            s.append(i); p.append(g["Val"][k]); o.append(g["Col"][k])
    G = gs.Graph(np.array(s), np.array(p), np.array(o), 8, 3)
    ptr, idx, lab = G.export()
    nonempty = np.diff(ptr.astype(np.int64)) > 0
    assert np.concatenate([[0], np.cumsum(nonempty)]).tolist() == g["Mr"]
    assert np.concatenate([[0], np.cumsum(np.diff(ptr.astype(np.int64))[nonempty])]).tolist() == g["Pr"]
    for r, i in enumerate(np.nonzero(nonempty)[0]):
        want = sorted(zip(g["Val"][g["Pr"][r]:g["Pr"][r + 1]], g["Col"][g["Pr"][r]:g["Pr"][r + 1]]))
        got = list(zip(lab[ptr[i]:ptr[i + 1]].tolist(), idx[ptr[i]:ptr[i + 1]].tolist()))
        assert got == want      # sorted by (label, column) inside the row


def test_store_rejects_bad_triples():
    s = np.array([0, 5], np.uint32)
    p = np.array([1, 1], np.uint32)
    o = np.array([1, 1], np.uint32)
    with pytest.raises(gs.GsError) as e:
        gs.Graph(s, p, o, 4, 2)
    assert e.value.status == 1
    with pytest.raises(gs.GsError):
        gs.Graph(s[:1], np.array([3], np.uint32), o[:1], 4, 2)


def test_store_device_input_and_duplicates():
    import torch
    s = torch.tensor([0, 0, 1, 1, 1, 2], dtype=torch.int32, device="cuda")
    p = torch.tensor([1, 1, 2, 1, 2, 1], dtype=torch.int32, device="cuda")
    o = torch.tensor([1, 1, 2, 0, 2, 2], dtype=torch.int32, device="cuda")
    g = gs.Graph(s, p, o, 3, 2)
    assert g.n_triples == 4
    ptr, idx, lab = g.export()
    assert ptr.tolist() == [0, 1, 3, 4]
    assert list(zip(lab.tolist(), idx.tolist())) == [(1, 1), (1, 0), (2, 2), (1, 2)]


def _scan_cases(npred, rng, n_cases):
    for _ in range(n_cases):
        m = int(rng.integers(1, 5))
        preds = rng.integers(1, npred + 1, m)
        dirs = rng.integers(0, 2, m)
        yield preds, dirs


def test_scan_matches_oracle(rmat14):
    w, _, g, ix = rmat14
    rng = np.random.default_rng(3)
    pres = {}
    for preds, dirs in _scan_cases(w.n_preds, rng, 40):
        want = np.ones(w.n_vertices, bool)
        for q, d in zip(preds, dirs):
            key = (int(d), int(q))
            if key not in pres:
                pres[key] = ix.presence(int(d), int(q)).astype(bool)
            want &= pres[key]
        got = _bits_to_bool(g.scan(preds, dirs), w.n_vertices)
        assert np.array_equal(got, want), (preds, dirs)


def test_scan_heavy_rows_and_ragged_tail():
    # vertex 7 has 9000 out- and 7000 in-edges (several scan chunks), and N is
    # not a multiple of 32 so the last word is partial
    rng = np.random.default_rng(5)
    n_v, n_p = 1000, 6
    s = np.concatenate([np.full(9000, 7), rng.integers(0, n_v, 7000), rng.integers(0, n_v, 20000)])
    o = np.concatenate([rng.integers(0, n_v, 9000), np.full(7000, 7), rng.integers(0, n_v, 20000)])
    p = np.concatenate([np.full(9000, 3), rng.integers(1, n_p + 1, 7000), rng.integers(1, n_p + 1, 20000)])
    p[5000] = 6
    g, ix = _graph(s, p, o, n_v, n_p)
    for preds, dirs in _scan_cases(n_p, rng, 30):
        want = np.ones(n_v, bool)
        for q, d in zip(preds, dirs):
            want &= ix.presence(int(d), int(q)).astype(bool)
        got = _bits_to_bool(g.scan(preds, dirs), n_v)
        assert np.array_equal(got, want), (preds, dirs)
    assert _bits_to_bool(g.scan([3, 6], [0, 0]), n_v)[7]


@pytest.mark.parametrize("shape", ["hubs", "sparse"])
def test_scan_rows_crossing_work_items(shape):
    # the scan cuts each orientation into work items of about 8.4K units
    # (labels + row ends): "hubs" has a 60,000-entry row and a 50,000-entry
    # column that cross many items, with the column on the last vertex;
    # "sparse" is mostly empty rows, so items hold thousands of rows
    rng = np.random.default_rng(17)
    if shape == "hubs":
        n_v, n_p = 70001, 5
        s = np.concatenate([np.full(60000, 5), rng.integers(0, n_v, 50000), rng.integers(0, n_v, 20000)])
        o = np.concatenate([rng.integers(0, n_v, 60000), np.full(50000, n_v - 1), rng.integers(0, n_v, 20000)])
        p = np.concatenate([1 + np.arange(60000) % 4, rng.integers(1, n_p + 1, 50000),
                            rng.integers(1, n_p + 1, 20000)])
        p[60000 + 777] = 5                       # one rare label inside the hub column
    else:
        n_v, n_p = 300001, 4
        s, o = rng.integers(0, n_v, 500), rng.integers(0, n_v, 500)
        p = rng.integers(1, n_p + 1, 500)
    g, ix = _graph(s, p, o, n_v, n_p)
    cases = list(_scan_cases(n_p, rng, 25)) + [([1, 2, 3, 4], [0, 0, 0, 0])]
    if shape == "hubs":
        cases.append(([5], [1]))
    for preds, dirs in cases:
        want = np.ones(n_v, bool)
        for q, d in zip(preds, dirs):
            want &= ix.presence(int(d), int(q)).astype(bool)
        got = _bits_to_bool(g.scan(preds, dirs), n_v)
        assert np.array_equal(got, want), (shape, preds, dirs)


@pytest.mark.parametrize("n_p", [3000, 60000])
def test_scan_many_predicates(n_p):
    # large predicate ids: the one-hot table no longer fits beside the full
    # warp count (16-bit table with fewer warps, or the byte table)
    rng = np.random.default_rng(n_p)
    n_v = 5000
    s = rng.integers(0, n_v, 60000)
    o = rng.integers(0, n_v, 60000)
    p = rng.integers(1, n_p + 1, 60000)
    p[:20000] = rng.integers(n_p - 5, n_p + 1, 20000)     # frequent high ids
    g, ix = _graph(s, p, o, n_v, n_p)
    for preds, dirs in [([n_p, n_p - 1], [0, 1]), ([1, n_p - 3, n_p - 4], [1, 0, 0])]:
        want = np.ones(n_v, bool)
        for q, d in zip(preds, dirs):
            want &= ix.presence(int(d), int(q)).astype(bool)
        got = _bits_to_bool(g.scan(preds, dirs), n_v)
        assert np.array_equal(got, want), (n_p, preds, dirs)


def _same(g, ix, pats, flags=0):
    got = g.query(pats, sort=True, flags=flags)
    want = ix.eval(pats, threads=4)
    assert got.shape == want.shape, (pats, got.shape, want.shape)
    assert np.array_equal(got, want), pats
    return want


@pytest.mark.parametrize("block", range(4))
def test_eval_random_tiny_cases(block, exec_path):
    # the oracle is pinned to exhaustive enumeration on exactly these cases
    for seed in range(block * 60, block * 60 + 60):
        nv = 3 + seed % 5
        npred = 1 + seed % 3
        s, p, o = rdfgen.random_graph(seed, nv, npred, 4 + seed % 23)
        g, ix = _graph(s, p, o, nv, npred)
        q = rdfgen.random_bgp(seed + 7, nv, npred)
        _same(g, ix, q)
        _same(g, ix, q, flags=gs.PLAN_DIRECTION)


def test_eval_rmat14_workload(rmat14, exec_path):
    w, (s, p, o), g, ix = rmat14
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    for q in rdfgen.queries(w, sm):
        rows = _same(g, ix, q.patterns)
        assert len(rows) >= 1     # the embedding that produced the query matches


def test_eval_mid_size_random_shapes(exec_path):
    w = rdfgen.Workload("t", 12, 40000, 8, 1.0, 4242, 0, 0, 0)
    s, p, o = rdfgen.graph(w)
    g, ix = _graph(s, p, o, w.n_vertices, w.n_preds)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    shapes = [rdfgen.star(2), rdfgen.star(4), rdfgen.chain(2), rdfgen.chain(4), rdfgen.cycle(3),
              rdfgen.cycle(4), rdfgen.cycle(5), rdfgen.snowflake([1, 2]), rdfgen.snowflake([2, 2])]
    n = 0
    for i, sh in enumerate(shapes * 3):
        q = sm.sample(sh, 77, i, 3e5)
        _same(g, ix, q.patterns)
        _same(g, ix, q.patterns, flags=gs.PLAN_DIRECTION)
        n += 1
    assert n == 27


def test_eval_edge_cases(rmat14, exec_path):
    w, (s, p, o), g, ix = rmat14
    t0 = (int(s[0]), int(p[0]), int(o[0]))
    # exactly one row: an (s, p) pair with a single object
    ts, tp, to = ix.triples()
    key = ts.astype(np.int64) * 1000 + tp
    u, first, cnt = np.unique(key, return_index=True, return_counts=True)
    one = first[np.nonzero(cnt == 1)[0][0]]
    assert len(_same(g, ix, [(int(ts[one]), int(tp[one]), -1)])) == 1
    # constant-only pattern that holds / fails, next to a variable pattern
    _same(g, ix, [(t0[0], t0[1], t0[2]), (-1, 1, -2)])
    miss = (t0[0], t0[1], (t0[2] + 1) % w.n_vertices)
    _same(g, ix, [miss, (-1, 1, -2)])
    # empty: a predicate no vertex has twice in a row through a loop
    _same(g, ix, [(-1, w.n_preds, -1), (-1, w.n_preds, -2), (-2, w.n_preds, -1)])
    # self-loops and repeated patterns
    _same(g, ix, [(-1, 1, -1)])
    _same(g, ix, [(-1, 1, -2), (-1, 1, -2), (-2, 2, -2)])
    # disconnected: a cross product of two components
    _same(g, ix, [(-1, 5, t0[2]), (-2, 6, t0[2] ^ 1)])
    _same(g, ix, [(-1, 9, -2), (-3, 16, -3)])
    # two edges between the same pair of variables, both directions
    _same(g, ix, [(-1, 1, -2), (-2, 2, -1), (-1, 3, -2)])
    # every variable order of one chain gives the same rows
    pats = np.array([(-1, 1, -2), (-2, 2, -3), (-3, 3, -4)], np.int64)
    base = _same(g, ix, pats)
    for perm in ([2, 1, 0], [1, 2, 0]):
        assert np.array_equal(g.query(pats[perm]), base)


def test_fetch_unsorted_is_a_permutation_and_overflow(rmat14):
    w, _, g, ix = rmat14
    pats = [(-1, 2, -2), (-2, 3, -3)]
    r = g.eval(pats)
    n, k = r.info()
    assert n > 10
    rows = r.fetch(sort=False)
    srt = rows[np.lexsort(rows.T[::-1])]
    assert np.array_equal(srt, ix.eval(pats))
    small = np.empty((n - 1, k), np.int32)
    with pytest.raises(gs.GsError) as e:
        r.fetch(out=small)
    assert e.value.status == 4
    import torch
    dev = torch.empty((n, k), dtype=torch.int32, device="cuda")
    r.fetch(sort=True, out=dev)
    assert np.array_equal(dev.cpu().numpy(), srt)
    assert r.time_ms() > 0
    r.close()


def test_workspace_retry(rmat14, monkeypatch, exec_path):
    # a tiny first workspace forces the overflow -> grow -> re-run path
    w, _, g, ix = rmat14
    monkeypatch.setenv("GS_ARENA_BYTES", "65536")
    for pats in ([(-1, 1, -2), (-2, 1, -3)], [(-1, 2, -2), (-1, 3, -3), (-1, 4, -4)],
                 [(-2, 8, -1), (-3, 1, -2), (-3, 5, -1)]):
        _same(g, ix, pats)


def test_hub_graph_expansion(exec_path):
    # one hub with 120,000 out-edges (past 10^5): load-balanced expansion over
    # a huge range; through the constant it also exceeds the single-block
    # budget (escalation)
    rng = np.random.default_rng(9)
    n_v = 130000
    s = np.concatenate([np.zeros(120000, np.int64), rng.integers(0, n_v, 60000)])
    o = np.concatenate([np.arange(1, 120001), rng.integers(0, n_v, 60000)])
    p = np.concatenate([np.ones(120000, np.int64), rng.integers(1, 4, 60000)])
    g, ix = _graph(s, p, o, n_v, 3)
    _same(g, ix, [(0, 1, -1), (-1, 2, -2)])
    _same(g, ix, [(0, 1, -1)])
    _same(g, ix, [(0, 1, -1), (-1, 2, -2), (-2, 3, -3)])
    _same(g, ix, [(-1, 1, -2), (-2, 2, -3)])
    _same(g, ix, [(-1, 1, -2), (-1, 1, -3), (-2, 3, -3)])


def test_batch_equals_oracle(rmat14, monkeypatch):
    # one persistent launch over many queries of every shape, including
    # constant-free ones (grid path) and ones that outgrow one CTA
    w, (s, p, o), g, ix = rmat14
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    pats = [q.patterns for q in rdfgen.queries(w, sm)]
    rng = np.random.default_rng(4)
    for i in range(40):
        sh = [rdfgen.star(2), rdfgen.chain(2), rdfgen.cycle(3), rdfgen.snowflake([1, 1])][i % 4]
        sh.const = [int(rng.integers(0, sh.n_v))]
        q = sm.sample(sh, 99, i, 1e5)
        pats.append(q.patterns)
    pats.append(np.array([(-1, 1, -2)], np.int64))        # large: grid path
    b = g.eval_batch(pats)
    rows = b.rows()
    ms, launches, esc = b.stats()
    assert launches >= 1
    for i, pt in enumerate(pats):
        want = ix.eval(pt, threads=4)
        assert int(rows[i]) == len(want), i
        assert np.array_equal(b.fetch(i), want), i
    b.close()


def _batch_pats(w, s, p, o, seed):
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    pats = [q.patterns for q in rdfgen.queries(w, sm)]
    rng = np.random.default_rng(seed)
    for i in range(24):
        sh = [rdfgen.star(2), rdfgen.chain(2), rdfgen.cycle(3), rdfgen.snowflake([1, 1])][i % 4]
        sh.const = [int(rng.integers(0, sh.n_v))]
        pats.append(sm.sample(sh, 99, 100 + i, 1e5).patterns)
    pats.append(np.array([(-1, 1, -2)], np.int64))        # constant-free: grid path
    return pats


@pytest.mark.parametrize("cfg", [dict(blocks_per_sm=1, cand_budget=16, row_budget=16),
                                 dict(row_budget=1 << 20, grid_streams=1),
                                 dict(blocks_per_sm=2, grid_streams=16, cand_budget=1 << 12)])
def test_batch_configs_equal_oracle(rmat14, cfg):
    # tiny budgets hand most queries to the grid path (run on side streams);
    # every configuration gives the oracle's answers
    w, (s, p, o), g, ix = rmat14
    pats = _batch_pats(w, s, p, o, 8)
    b = g.eval_batch(pats, config=gs.BatchConfig(**cfg))
    rows = b.rows()
    _, _, esc = b.stats()
    if cfg.get("row_budget") == 16:
        assert esc > 0
    for i, pt in enumerate(pats):
        want = ix.eval(pt, threads=4)
        assert int(rows[i]) == len(want), (cfg, i)
        assert np.array_equal(b.fetch(i), want), (cfg, i)
    b.close()


def test_batch_autotune_picks_a_working_config(rmat14):
    w, (s, p, o), g, ix = rmat14
    pats = _batch_pats(w, s, p, o, 9)
    cfg, ms = g.autotune_batch(pats)
    assert ms > 0 and cfg.blocks_per_sm >= 1 and cfg.cand_budget > 0 and cfg.row_budget > 0
    b = g.eval_batch(pats, config=cfg)
    for i, pt in enumerate(pats):
        assert np.array_equal(b.fetch(i), ix.eval(pt, threads=4)), i
    b.close()


def test_batch_small_pool_hands_back(rmat14, monkeypatch):
    # a pool too small for most answers: those queries go to the grid path
    w, (s, p, o), g, ix = rmat14
    monkeypatch.setenv("GS_BATCH_POOL_BYTES", "4096")
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    pats = [q.patterns for q in rdfgen.queries(w, sm)]
    b = g.eval_batch(pats)
    for i, pt in enumerate(pats):
        assert np.array_equal(b.fetch(i), ix.eval(pt, threads=4)), i
    assert b.stats()[2] >= 1
    b.close()


def test_torch_allocator_hook(rmat14):
    w, (s, p, o), _, ix = rmat14
    alloc = gs.TorchAllocator()
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds, allocator=alloc)
    assert alloc.calls > 0
    pats = [(-1, 2, -2), (-2, 3, -3)]
    assert np.array_equal(g.query(pats), ix.eval(pats))
    g.close()
    assert not alloc.live        # everything handed back


@pytest.mark.parametrize("fail_after", [1, 3, 6, 12])
def test_allocation_failure_is_a_status(rmat14, fail_after):
    # the hook refuses memory part-way through the store build: the call
    # returns GS_ENOMEM, frees what it took, and the context stays usable
    w, (s, p, o), g_ok, ix = rmat14
    alloc = gs.TorchAllocator(fail_after=fail_after)
    with pytest.raises(gs.GsError) as e:
        gs.Graph(s, p, o, w.n_vertices, w.n_preds, allocator=alloc)
    assert e.value.status == 2
    assert not alloc.live
    pats = [(-1, 2, -2)]
    assert np.array_equal(g_ok.query(pats), ix.eval(pats))


def test_handed_back_queries_resume_on_the_grid_path(rmat14, monkeypatch):
    # constant-seeded queries past the single-block budgets: at a level
    # (more than 1,024 candidates below a small seed level) or at the
    # enumeration (more than 4,096 rows). The grid path continues from the
    # levels the block finished, in its workspace; the answers equal the
    # oracle's and the all-grid evaluation's
    w, (s, p, o), g, ix = rmat14
    s64, p64, o64 = (np.asarray(x, np.int64) for x in (s, p, o))
    top = np.bincount(p64).argmax()
    out_deg = np.bincount(s64, minlength=w.n_vertices)
    # seeds: a constant whose top-predicate row is small, so that level 0 fits
    seeds = [int(v) for v in np.flatnonzero((out_deg >= 20) & (out_deg <= 200))[:40]]
    pats = []
    for c in seeds:
        pred = int(np.bincount(p64[s64 == c]).argmax())
        # ?0 is a level (two patterns); ?1 a level below it; ?2 a leaf
        pats.append([(c, pred, -1), (-1, int(top), -2), (-2, int(top), -3), (-3, int(top), -1)])
        pats.append([(c, pred, -1), (-1, int(top), -2), (-2, int(top), -3)])
    def run(pt):
        r = g.eval(pt)
        r.info()
        nl = r.stats()[1]
        rows = r.fetch()
        r.close()
        return rows, nl

    resumed = 0
    for pt in pats[:24]:
        want = ix.eval(pt, threads=4)
        monkeypatch.setenv("GS_EXEC", "auto")
        got, nl = run(pt)
        monkeypatch.setenv("GS_EXEC", "grid")
        full, nl_full = run(pt)
        assert np.array_equal(got, want), pt
        assert np.array_equal(full, want), pt
        resumed += int(1 < nl < nl_full)   # fewer launches: levels were kept
    assert resumed >= 1


def test_allocator_alignment_is_checked(rmat14):
    # a hook whose blocks start 16 bytes past a 256-byte boundary: the first
    # such block goes straight back to the hook and the build fails as out
    # of memory, with nothing left allocated
    import torch
    w, (s, p, o), g_ok, ix = rmat14
    live = {}

    def _alloc(nbytes, stream, ctx):
        base = torch.cuda.caching_allocator_alloc(int(nbytes) + 256, 0, stream)
        live[base + 16] = base
        return base + 16

    def _free(ptr, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(live.pop(ptr))

    alloc = gs.TorchAllocator()
    alloc._cb_alloc = gs._ALLOC_FN(_alloc)
    alloc._cb_free = gs._FREE_FN(_free)
    alloc.struct = gs._Allocator(alloc._cb_alloc, alloc._cb_free, None)
    with pytest.raises(gs.GsError) as e:
        gs.Graph(s, p, o, w.n_vertices, w.n_preds, allocator=alloc)
    assert e.value.status == 2
    assert not live
    pats = [(-1, 2, -2)]
    assert np.array_equal(g_ok.query(pats), ix.eval(pats))


def test_server_answers_equal_alone(rmat14):
    # continuous batching: the same queries submitted together, interleaved
    # and repeated; every answer equals the query evaluated alone (and the
    # oracle), and admitted memory never exceeds the budget
    import time
    w, (s, p, o), g, ix = rmat14
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    pats = [q.patterns for q in rdfgen.queries(w, sm)]
    rng = np.random.default_rng(8)
    for i in range(24):
        sh = [rdfgen.star(2), rdfgen.chain(3), rdfgen.cycle(3), rdfgen.snowflake([1, 1])][i % 4]
        sh.const = [int(rng.integers(0, sh.n_v))]
        pats.append(sm.sample(sh, 123, i, 1e5).patterns)
    alone = [g.query(pt) for pt in pats]
    budget = 3 << 30
    srv = gs.Server(g, max_batch=8, n_streams=3, memory_budget=budget)
    plans = [g.plan(pt) for pt in pats]
    order = list(range(len(pats))) * 2
    rng.shuffle(order)
    tickets = []
    for j, qi in enumerate(order):
        tickets.append((qi, srv.submit(plans[qi])))
        if j % 5 == 0:
            time.sleep(0.001)     # arrivals while earlier batches run
    for qi, t in tickets:
        t0 = time.time()
        while not srv.poll(t)[0]:
            assert time.time() - t0 < 60
            time.sleep(0.0005)
        got = srv.fetch(t)
        assert np.array_equal(got, alone[qi]), qi
        assert np.array_equal(got, ix.eval(pats[qi], threads=4)), qi
        srv.release(t)
    done, batches, peak = srv.stats()
    assert done == len(order) and batches >= 2
    assert peak <= budget
    srv.stop()


def test_server_replay_completes_every_arrival(rmat14):
    # native Poisson replay: every query finishes, latencies are positive and
    # completions come after arrivals
    w, (s, p, o), g, ix = rmat14
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    plans = [g.plan(q.patterns) for q in rdfgen.queries(w, sm)]
    rng = np.random.default_rng(11)
    sched = np.cumsum(rng.exponential(1.0 / 5000.0, 300))
    srv = gs.Server(g, max_batch=64)
    lat, done = srv.replay(plans, sched, timeout_s=60)
    completed, batches, _ = srv.stats()
    srv.stop()
    assert completed == 300 and batches >= 1
    assert (lat > 0).all() and (done >= sched).all()


@pytest.mark.slow
def test_scan_full_size_rmat26():
    # the bandwidth workload's graph (scale 26, 2^30 draws, 1.07e9 distinct
    # triples, 256 predicates): every word of two grouped scans equals the
    # AND of presence vectors computed on the host from the raw triples
    w = rdfgen.WORKLOADS["rmat26"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    N = w.n_vertices
    pres = {}

    def presence(d, q):
        if (d, q) not in pres:
            f = np.zeros(N, bool)
            f[(o if d else s)[p == q]] = True
            pres[(d, q)] = f
        return pres[(d, q)]

    for preds, dirs in [([1, 2, 3, 1, 2], [0, 0, 0, 1, 1]), ([4, 200, 7], [1, 0, 1])]:
        want = np.ones(N, bool)
        for q, d in zip(preds, dirs):
            want &= presence(d, q)
        got = g.scan(preds, dirs).cpu().numpy().view(np.uint32)
        want_words = np.packbits(want, bitorder="little").view(np.uint32)
        assert np.array_equal(got, want_words), (preds, dirs)
    g.close()


@pytest.mark.slow
def test_batched_workload_rmat24_sample_equals_oracle():
    # the batched workload's graph (scale 24, 2^28 draws, 128 predicates) and
    # 96 of its queries in one batch under the autotuned configuration: every
    # answer equals the oracle's sorted rows
    import time
    w = rdfgen.WORKLOADS["rmat24"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    qs = rdfgen.batched_queries(w, sm, 96)
    sm.close()
    pats = [q.patterns for q in qs]
    cfg, _ = g.autotune_batch(pats[:32])
    b = g.eval_batch(pats, config=cfg)
    rows = b.rows()
    t0 = time.time()
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    print("oracle index %.1f s" % (time.time() - t0))
    for i, pt in enumerate(pats):
        want = ix.eval(pt, threads=os.cpu_count() or 1)
        assert int(rows[i]) == len(want), i
        assert np.array_equal(b.fetch(i), want), i
    b.close()
    g.close()


@pytest.mark.slow
def test_plain_and_batched_rmat22_workload_equal_oracle():
    # the bench's workload at full size (scale 22, 66.9M triples, its 32
    # queries, 20.4M answer rows): one at a time and as one autotuned batch,
    # every row equal to the oracle's sorted rows
    w = rdfgen.WORKLOADS["rmat22"]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    pats = [q.patterns for q in rdfgen.queries(w, sm)]
    sm.close()
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    cfg, _ = g.autotune_batch(pats)
    b = g.eval_batch(pats, config=cfg)
    for i, pt in enumerate(pats):
        want = ix.eval(pt, threads=os.cpu_count() or 1)
        assert np.array_equal(g.query(pt), want), i
        assert np.array_equal(b.fetch(i), want), i
    b.close()
    g.close()


def test_invariance_under_pattern_order_renaming_and_planner(rmat14):
    # the answer set does not depend on the order of the patterns, the names
    # of the variables (columns follow the renaming) or the planner and
    # evaluation mode; every row satisfies every pattern
    w, (s, p, o), g, ix = rmat14
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    pats = [q.patterns for q in rdfgen.queries(w, sm)]
    for i, sh in enumerate([rdfgen.cycle(4), rdfgen.snowflake([2, 1]), rdfgen.chain(4)]):
        pats.append(sm.sample(sh, 123, i, 2e5).patterns)
    sm.close()
    triples = set(zip(s.tolist(), p.tolist(), o.tolist()))
    rng = np.random.default_rng(31)
    for pt in pats:
        pt = np.asarray(pt, np.int64)
        base = g.query(pt)
        k = base.shape[1]
        for row in base[:200]:   # every row satisfies every pattern
            for a, pr, b in pt:
                sa = row[-a - 1] if a < 0 else a
                sb = row[-b - 1] if b < 0 else b
                assert (int(sa), int(pr), int(sb)) in triples
        for _ in range(2):
            perm = rng.permutation(k)                  # variable j -> perm[j]
            q = pt[rng.permutation(len(pt))].copy()
            for c in (0, 2):
                m = q[:, c] < 0
                q[m, c] = -(perm[-q[m, c] - 1] + 1)
            got = g.query(q)
            back = got[:, perm]                        # column perm[j] holds variable j
            order = np.lexsort(back.T[::-1])
            assert np.array_equal(back[order], base), pt
        for flags in (gs.PLAN_DIRECTION, gs.PLAN_LISTS, gs.PLAN_PATHS):
            assert np.array_equal(g.query(pt, flags=flags), base), (pt, flags)
