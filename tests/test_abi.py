"""The C ABI without a GPU: the library loads, exports every entry point the
header declares, plans queries (host only) like the oracle planner, and
rejects bad input with a status instead of crashing. CPU only."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2106_14038_b300 as gs
from oracle import planner as oplanner

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gsmart.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"\b(gs_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    lib = gs.load_library()
    names = _declared()
    assert "gs_eval_query" in names and "gs_load_triples" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(gs.EXPORTED) == sorted(n for n in names)


def test_load_without_gpu_reports_cuda_status():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = gs.load_library()
    s = np.zeros(1, np.uint32)
    h = ctypes.c_void_p()
    rc = lib.gs_load_triples(s.ctypes.data_as(ctypes.c_void_p), s.ctypes.data_as(ctypes.c_void_p),
                             s.ctypes.data_as(ctypes.c_void_p), 1, 4, 2, 0, None, None,
                             ctypes.byref(h))
    assert rc == 3  # GS_ECUDA
    assert lib.gs_last_error()


def _plan_nograph(pat, flags=0):
    lib = gs.load_library()
    pat = np.ascontiguousarray(np.asarray(pat, np.int64).reshape(-1, 3))
    h = ctypes.c_void_p()
    rc = lib.gs_plan_query(None, pat.ctypes.data_as(ctypes.c_void_p), len(pat), flags,
                           ctypes.byref(h))
    if rc != 0:
        return rc, None
    p = gs.Plan.__new__(gs.Plan)
    p._h = h
    p.patterns = pat
    return 0, p


def _oracle_fmt(groups, roots):
    def v(x):
        return x[1] if x[0] == "v" else ("c", x[1])
    return [(v(g), list(es)) for g, es in groups], [v(r) for r in roots]


@pytest.mark.parametrize("flags,fn", [(0, oplanner.degree_driven), (1, oplanner.direction_driven)])
def test_planner_matches_oracle_planner(flags, fn):
    rng = np.random.default_rng(11 + flags)
    for _ in range(400):
        k = int(rng.integers(1, 8))
        n = int(rng.integers(1, 10))
        pats = []
        for _ in range(n):
            ends = []
            for _ in range(2):
                if rng.random() < 0.15:
                    ends.append(int(rng.integers(0, 20)))
                else:
                    ends.append(-int(rng.integers(0, k)) - 1)
            pats.append((ends[0], int(rng.integers(1, 5)), ends[1]))
        used = sorted({-x - 1 for t in pats for x in (t[0], t[2]) if x < 0})
        if not used:
            continue
        remap = {v: i for i, v in enumerate(used)}
        pats = [(-(remap[-a - 1]) - 1 if a < 0 else a, p, -(remap[-b - 1]) - 1 if b < 0 else b)
                for a, p, b in pats]
        rc, plan = _plan_nograph(pats, flags)
        assert rc == 0
        want = _oracle_fmt(*fn(pats))
        assert plan.describe() == want, pats


def test_planner_examples_6_1_and_6_2():
    pats = [(-1, 1, -2), (-1, 2, -3), (-3, 3, -2), (-4, 4, -3)]   # Fig. 2b
    _, p = _plan_nograph(pats, 1)
    assert p.describe() == ([(0, [0, 1]), (2, [2]), (3, [3])], [0, 3])
    _, p = _plan_nograph(pats, 0)
    assert p.describe() == ([(2, [1, 2, 3]), (0, [0])], [2])


@pytest.mark.parametrize("pat", [
    [(0, 1, 1)],                 # no variable
    [(-1, 0, -2)],               # predicate 0
    [(-1, 1, -3)],               # variables not dense
    [(-1, 70000, -2)],           # predicate beyond the largest id
    [(-1, 1, -2)] * 33,          # too many patterns
])
def test_planner_rejects_bad_queries(pat):
    rc, _ = _plan_nograph(pat)
    assert rc == 1  # GS_EINVAL


def test_null_arguments_are_a_status_not_a_crash():
    # host-side argument checks of the batch, tuning, serving and scan calls
    lib = gs.load_library()
    vp = ctypes.c_void_p
    h = ctypes.c_void_p()
    cfg = gs.BatchConfig()
    ms = ctypes.c_float()
    assert lib.gs_eval_batch(None, None, 1, None, ctypes.byref(h)) == 1
    assert lib.gs_eval_batch_cfg(None, None, 1, ctypes.byref(cfg), None, ctypes.byref(h)) == 1
    assert lib.gs_batch_autotune(None, None, 1, None, ctypes.byref(cfg), ctypes.byref(ms)) == 1
    assert lib.gs_server_start(None, None, ctypes.byref(h)) == 1
    assert lib.gs_server_replay(None, None, 0, None, 0, 1.0, None, None, None, 0, None) == 1
    assert lib.gs_scan_candidates(None, None, None, 0, None, None) == 1
    assert lib.gs_scan_candidates_noalloc(None, None, None, 0, None, None) == 1
    assert lib.gs_batch_info(None, None, None) == 1
    assert lib.gs_server_poll(None, 1, None, None, None) == 1
    assert lib.gs_last_error()
    assert lib.gs_noalloc_scratch_bytes() == 48 << 20


class _NoNative:
    """Stands in for the loaded library: any native call fails the test."""

    def __getattr__(self, name):
        raise AssertionError("native call %s made before the argument checks" % name)


@pytest.mark.parametrize("bad", ["dtype", "strided", "short", "host"])
def test_scan_output_is_checked_before_any_native_call(monkeypatch, bad):
    """scan() and scan_noalloc() write 4 * ceil(N/32) bytes into `out`: a
    wrong dtype, a strided view, a short buffer or a host tensor is refused
    before the library is called."""
    import torch
    g = gs.Graph.__new__(gs.Graph)
    g._h, g.n_vertices, g.n_predicates, g.device = None, 100, 4, 0
    words = 4
    out = {"dtype": torch.zeros(words, dtype=torch.uint8),
           "strided": torch.zeros(2 * words, dtype=torch.int32)[::2],
           "short": torch.zeros(words - 1, dtype=torch.int32),
           "host": torch.zeros(words, dtype=torch.int32)}[bad]
    monkeypatch.setattr(gs, "_lib", _NoNative())
    with pytest.raises(ValueError):
        g.scan([1], [0], out=out)
    with pytest.raises(ValueError):
        g.scan_noalloc([1], [0], out)


def _oracle_paths(pats, fn):
    """The oracle planner's Sec. 7.1 paths as variable lists, with the
    engine's two additions: a variable's group that no walk from a root
    enters (a constant's edge reached it first) starts paths of its own,
    after the roots', and a variable no path holds is a path of its own."""
    groups, roots = fn(pats)
    starts = list(roots)
    got = oplanner.paths(pats, groups, starts)
    while True:   # one more start at a time, in group order
        entered = set(starts) | {p[i] for p in got for i in range(len(p) - 1)}
        extra = [v for v, _ in groups if v[0] == "v" and v not in entered]
        if not extra:
            break
        starts.append(extra[0])
        got = oplanner.paths(pats, groups, starts)
    out = [[x[1] for x in p] for p in got]
    assert all(x[0] == "v" for p in got for x in p)
    k = 1 + max(-x - 1 for t in pats for x in (t[0], t[2]) if x < 0)
    covered = {v for p in out for v in p}
    out += [[v] for v in range(k) if v not in covered]
    return out


@pytest.mark.parametrize("flags,fn", [(0, oplanner.degree_driven), (1, oplanner.direction_driven)])
def test_paths_match_oracle_planner(flags, fn):
    rng = np.random.default_rng(31 + flags)
    checked = 0
    for _ in range(400):
        k = int(rng.integers(1, 7))
        n = int(rng.integers(1, 9))
        pats = []
        for _ in range(n):
            ends = [int(rng.integers(0, 20)) if rng.random() < 0.15 else -int(rng.integers(0, k)) - 1
                    for _ in range(2)]
            pats.append((ends[0], int(rng.integers(1, 5)), ends[1]))
        pats = [t for t in pats if t[0] != t[2]]   # self-loops: pinned by hand below
        used = sorted({-x - 1 for t in pats for x in (t[0], t[2]) if x < 0})
        if not used:
            continue
        remap = {v: i for i, v in enumerate(used)}
        pats = [(-(remap[-a - 1]) - 1 if a < 0 else a, p, -(remap[-b - 1]) - 1 if b < 0 else b)
                for a, p, b in pats]
        rc, plan = _plan_nograph(pats, flags)
        assert rc == 0
        assert plan.paths() == _oracle_paths(pats, fn), pats
        checked += 1
    assert checked > 300


@pytest.mark.parametrize("pats,want", [
    # a path ends at a variable whose group holds only a self-loop
    ([(-2, 1, -2), (-1, 2, -2), (-1, 1, -1), (1, 2, -3)], [[0, 1], [2]]),
    # a self-loop counts toward the degree (x1 is the root) but is no step
    ([(-1, 1, -2), (-2, 2, -2), (-2, 3, -3)], [[1, 0], [1, 2]]),
    # two edges between one pair are two paths
    ([(-1, 3, -2), (-2, 3, -1)], [[0, 1], [0, 1]]),
])
def test_paths_with_self_loops_and_parallel_edges(pats, want):
    _, p = _plan_nograph(pats, 0)
    assert p.paths() == want


def test_paths_example_7_1():
    """Ex. 7.1 (Fig. 2b, degree-driven): paths v2->v1, v2->v3, v2->v0->v1."""
    pats = [(-1, 1, -2), (-1, 2, -3), (-3, 3, -2), (-4, 4, -3)]
    _, p = _plan_nograph(pats, 0)
    assert sorted(p.paths()) == sorted([[2, 1], [2, 0, 1], [2, 3]])


def test_plan_root_and_root_range_arguments():
    lib = gs.load_library()
    rc, p = _plan_nograph([[-1, 1, -2], [-2, 2, -3], [-2, 3, -4]])
    assert rc == 0
    assert 0 <= p.root_var < 4
    rc, pp = _plan_nograph([[-1, 1, -2], [-2, 2, -3]], gs.PLAN_PATHS)
    assert rc == 0
    v = ctypes.c_uint32()
    assert lib.gs_plan_root(pp._h, ctypes.byref(v)) == 1          # GS_EINVAL: one root per path
    assert lib.gs_plan_root(None, ctypes.byref(v)) == 1
    h = ctypes.c_void_p(1)
    assert lib.gs_eval_query_roots(None, p._h, 0, 10, None, ctypes.byref(h)) == 1
    assert h.value is None                                         # *out cleared on error


def test_trace_arguments():
    lib = gs.load_library()
    assert lib.gs_graph_set_trace(None, 1) == 1                      # GS_EINVAL
    n = ctypes.c_uint32()
    assert lib.gs_result_phases(None, None, 0, ctypes.byref(n)) == 1
