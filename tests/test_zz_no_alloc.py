"""gs_scan_candidates_noalloc against gs_scan_candidates: same bits, on two
calls in a row, with no device allocation on its call path. The file name
sorts last so it also runs after every other GPU test has used the device."""
import numpy as np
import pytest

import paper_2106_14038_b300 as gs
import rdfgen

pytestmark = pytest.mark.gpu


def _cases(npred, seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        m = int(rng.integers(1, 5))
        out.append((rng.integers(1, npred + 1, m), rng.integers(0, 2, m)))
    return out


def _heavy_graph():
    # vertex 7 holds 9000 out- and 7000 in-edges (heavy rows and columns);
    # N = 1000 leaves a partial last word
    rng = np.random.default_rng(5)
    n_v, n_p = 1000, 6
    s = np.concatenate([np.full(9000, 7), rng.integers(0, n_v, 7000), rng.integers(0, n_v, 20000)])
    o = np.concatenate([rng.integers(0, n_v, 9000), np.full(7000, 7), rng.integers(0, n_v, 20000)])
    p = np.concatenate([np.full(9000, 3), rng.integers(1, n_p + 1, 7000),
                        rng.integers(1, n_p + 1, 20000)])
    return (s, p, o), n_v, n_p


def _oracle_bits(ix, pr, dr, n):
    """The Eq. 17 / Eq. 21 selection from the oracle's Eq. 4 / Eq. 5 vectors."""
    want = np.ones(n, np.uint8)
    for q, d in zip(pr, dr):
        want &= ix.presence(int(d), int(q))
    return want


def _bits(words, n):
    w = np.asarray(words.cpu().numpy(), np.int64) & 0xffffffff
    return ((w[:, None] >> np.arange(32)) & 1).astype(np.uint8).reshape(-1)[:n]


def test_noalloc_matches_scan_on_consecutive_calls():
    import torch
    import oracle
    w = rdfgen.WORKLOADS["rmat14"]
    s, p, o = rdfgen.graph(w)
    alloc = gs.TorchAllocator()
    big = gs.Graph(s, p, o, w.n_vertices, w.n_preds, allocator=alloc)
    (hs, hp, ho), hn, hpn = _heavy_graph()
    small = gs.Graph(hs, hp, ho, hn, hpn, allocator=alloc)
    stream = torch.cuda.Stream()
    pairs = [(big, c) for c in _cases(w.n_preds, 11, 6)] + [(small, c) for c in _cases(hpn, 12, 6)]
    want = [g.scan(pr, dr, stream=stream) for g, (pr, dr) in pairs]
    outs = [torch.full(((g.n_vertices + 31) // 32,), -1, dtype=torch.int32, device="cuda")
            for g, _ in pairs]
    import gc
    gc.collect()                 # earlier tests' garbage is freed before the baseline
    torch.cuda.synchronize()
    calls, live = alloc.calls, dict(alloc.live)
    # cumulative count of the caching allocator's allocations: frees of
    # unrelated tensors do not move it, any allocation does
    made = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    # back to back on one stream, alternating graphs so each call starts on
    # the previous call's leftovers in the static workspace
    for (g, (pr, dr)), out in zip(pairs, outs):
        g.scan_noalloc(pr, dr, out, stream=stream)
    for (g, (pr, dr)), out in zip(pairs[::-1], outs[::-1]):
        g.scan_noalloc(pr, dr, out, stream=stream)
    torch.cuda.synchronize()
    assert alloc.calls == calls and alloc.live == live
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == made
    for (g, (pr, dr)), a, b in zip(pairs, want, outs):
        assert torch.equal(a, b), (g.n_vertices, pr, dr)
    big.scan_status()
    small.scan_status()
    # the first cases also against the oracle (not only the allocating call)
    ix_big = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    ix_small = oracle.Index(hs, hp, ho, hn, hpn)
    for (g, (pr, dr)), b in list(zip(pairs, outs))[:3] + list(zip(pairs, outs))[6:9]:
        ix = ix_big if g is big else ix_small
        assert np.array_equal(_bits(b, g.n_vertices), _oracle_bits(ix, pr, dr, g.n_vertices))
    big.close()
    small.close()


def test_noalloc_rejects_a_graph_beyond_the_static_workspace():
    import torch
    limit = gs.load_library().gs_noalloc_scratch_bytes()
    assert limit == 48 << 20
    n_v = limit // 4 + 1                    # 4 (N + 256) bytes alone exceed the area
    s = np.array([0, 1, n_v - 1], np.uint32)
    p = np.array([1, 2, 1], np.uint32)
    o = np.array([1, 2, 0], np.uint32)
    g = gs.Graph(s, p, o, n_v, 2)
    out = torch.zeros((n_v + 31) // 32, dtype=torch.int32, device="cuda")
    with pytest.raises(gs.GsError) as e:
        g.scan_noalloc([1], [0], out)
    assert e.value.status == 1 and "static area" in str(e.value)
    got = g.scan([1], [0])               # the allocating entry point still serves it
    assert int(got[0].item()) & 0x3 == 0x1 and (int(got[-1].item()) >> ((n_v - 1) % 32)) & 1
    g.close()
