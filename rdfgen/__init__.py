"""Seeded synthetic inputs: R-MAT RDF graphs and BGP queries sampled from them.

This package is the only code that the oracle and the CUDA engine both use.
It produces inputs and holds none of the evaluation method (no candidate
scans, no grouped incident-edge evaluation, no binding trees). The draws are
a counter-based SplitMix64 stream (see rdfgen.c); the same (seed, workload)
always yields the same triples and the same queries.

Workloads stand in for the paper's datasets (Sec. 9, Table 1: WatDiv-100M,
YAGO2, LUBM-1B), which are not available here; the four query shapes follow
the paper's query classes (Sec. 9: linear, star, snowflake, complex).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rdfgen.c")
_LIB = os.path.join(_HERE, "librdfgen.so")

RMAT_ABC = (0.57, 0.19, 0.19)  # Graph500 (a, b, c); d = 0.05


def build(force: bool = False) -> str:
    """Compile rdfgen.c into librdfgen.so beside it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, u32, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_void_p)
        lib.rdfgen_draw.restype = u64
        lib.rdfgen_draw.argtypes = [u64, u64, u64]
        lib.rdfgen_perm.restype = u64
        lib.rdfgen_perm.argtypes = [u64, i32, u64]
        lib.rdfgen_rmat.restype = i32
        lib.rdfgen_rmat.argtypes = [i32, u64, u32, dbl, dbl, dbl, dbl, u64, vp, vp, vp]
        lib.rdfgen_adj_build.restype = vp
        lib.rdfgen_adj_build.argtypes = [vp, vp, vp, u64, u32, u32]
        lib.rdfgen_adj_free.restype = None
        lib.rdfgen_adj_free.argtypes = [vp]
        lib.rdfgen_embed.restype = i32
        lib.rdfgen_embed.argtypes = [vp, u32, u32, vp, vp, vp, vp, vp, u64, u64, vp, vp, vp]
        lib.rdfgen_tree_bound.restype = dbl
        lib.rdfgen_tree_bound.argtypes = [vp, u32, vp, vp, vp, vp, vp]
        lib.rdfgen_tree_bound_rooted.restype = dbl
        lib.rdfgen_tree_bound_rooted.argtypes = [vp, u32, vp, vp, vp, vp, vp, u32, u64]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def draw(seed: int, stream: int, ctr: int) -> int:
    """One 64-bit draw of the counter-based stream (seed, stream, ctr)."""
    return int(_L().rdfgen_draw(seed & (2**64 - 1), stream, ctr))


def rmat_triples(scale: int, n_edges: int, n_preds: int, zipf_s: float, seed: int,
                 abc=RMAT_ABC):
    """Draw exactly n_edges R-MAT triples (duplicates kept).

    Returns (s, p, o) as uint32 arrays; vertex ids in [0, 2**scale),
    predicate ids in [1, n_preds]."""
    s = np.empty(n_edges, np.uint32)
    p = np.empty(n_edges, np.uint32)
    o = np.empty(n_edges, np.uint32)
    rc = _L().rdfgen_rmat(scale, n_edges, n_preds, zipf_s, abc[0], abc[1], abc[2], seed,
                          _ptr(s), _ptr(p), _ptr(o))
    if rc != 0:
        raise ValueError("rdfgen_rmat failed (%d)" % rc)
    return s, p, o


# --------------------------------------------------------------------------
# Query shapes: undirected edges over shape vertices, tree edges first in an
# order where the first end is already reached, non-tree edges last.

@dataclass
class Shape:
    name: str
    n_v: int
    edges: list            # [(u, w)]
    n_tree: int            # = n_v - 1
    const: list = field(default_factory=list)     # shape vertices that are constants
    dir_req: dict = field(default_factory=dict)   # edge index -> 1 (u subject) / 2 (u object)
    pred_range: dict = field(default_factory=dict)  # edge index -> (lowest, highest) predicate id


def star(k: int) -> Shape:
    return Shape("star%d" % k, k + 1, [(0, i) for i in range(1, k + 1)], k)


def chain(k: int) -> Shape:
    return Shape("chain%d" % k, k + 1, [(i, i + 1) for i in range(k)], k)


def cycle(k: int) -> Shape:
    e = [(i, i + 1) for i in range(k - 1)] + [(k - 1, 0)]
    return Shape("cycle%d" % k, k, e, k - 1)


def snowflake(branches) -> Shape:
    """Centre 0 with one arm per entry of `branches`; arm i has branches[i] leaves."""
    edges, nxt, arms = [], 1, []
    for _ in branches:
        edges.append((0, nxt)); arms.append(nxt); nxt += 1
    for a, nl in zip(arms, branches):
        for _ in range(nl):
            edges.append((a, nxt)); nxt += 1
    return Shape("snowflake%d" % nxt, nxt, edges, nxt - 1)


def cycle_leaf(k: int) -> Shape:
    """A k-cycle 0-1-..-(k-1)-0 with one pendant vertex k on vertex 0: the
    tree edges (the path and the pendant edge) first, the closing edge last."""
    e = [(i, i + 1) for i in range(k - 1)] + [(0, k), (k - 1, 0)]
    return Shape("cycle%d+leaf" % k, k + 1, e, k)


@dataclass
class Query:
    patterns: np.ndarray   # (n, 3) int64: s, p, o; variable k is -(k+1)
    n_vars: int
    shape: str
    bound: float           # matches of the spanning tree (upper bound on the result)
    embedding: np.ndarray  # graph vertex of every shape vertex (one known match)
    u_subject: np.ndarray = None   # per shape edge: 1 when its first end is the subject


class Sampler:
    """Embeds query shapes into one graph (keeps the adjacency it needs)."""

    def __init__(self, s, p, o, n_vertices: int, n_preds: int):
        self._keep = (np.ascontiguousarray(s, np.uint32), np.ascontiguousarray(p, np.uint32),
                      np.ascontiguousarray(o, np.uint32))
        self.n_vertices, self.n_preds = n_vertices, n_preds
        self._h = _L().rdfgen_adj_build(_ptr(self._keep[0]), _ptr(self._keep[1]),
                                        _ptr(self._keep[2]), len(self._keep[0]),
                                        n_vertices, n_preds)
        if not self._h:
            raise MemoryError("rdfgen_adj_build failed")

    def close(self):
        if self._h:
            _L().rdfgen_adj_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def embed(self, shape: Shape, seed: int, attempt: int, with_bound: bool = True,
              work_cap: int = 0):
        """One seeded embedding of shape (None if the walk fails). With
        work_cap > 0 and a constant in the shape, the bound is counted from
        the first constant through the vertices actually reached, and is inf
        when that visits more than work_cap adjacency entries."""
        se = np.array(shape.edges, np.uint32).reshape(-1)
        isc = np.zeros(shape.n_v, np.uint8)
        isc[list(shape.const)] = 1
        dreq = np.zeros(len(shape.edges), np.uint8)
        for e, d in shape.dir_req.items():
            dreq[e] = d
        pat = np.zeros((len(shape.edges), 3), np.int64)
        mapped = np.zeros(shape.n_v, np.uint32)
        usub = np.zeros(len(shape.edges), np.uint8)
        plo = phi = None
        if shape.pred_range:
            plo = np.ones(len(shape.edges), np.uint32)
            phi = np.full(len(shape.edges), self.n_preds, np.uint32)
            for e, (lo, hi) in shape.pred_range.items():
                plo[e], phi[e] = lo, hi
        rc = _L().rdfgen_embed(self._h, shape.n_v, len(shape.edges), _ptr(se), _ptr(isc),
                               _ptr(dreq), None if plo is None else _ptr(plo),
                               None if phi is None else _ptr(phi), seed, attempt, _ptr(pat),
                               _ptr(mapped), _ptr(usub))
        if rc != 0:
            return None
        if not with_bound:
            return Query(pat, shape.n_v - len(shape.const), shape.name, float("nan"), mapped,
                         usub)
        bound = float("nan")
        if with_bound and work_cap > 0 and shape.const:
            bound = _L().rdfgen_tree_bound_rooted(self._h, shape.n_v, _ptr(se), _ptr(isc),
                                                  _ptr(mapped), _ptr(pat), _ptr(usub),
                                                  int(shape.const[0]), int(work_cap))
            if bound < 0:
                bound = float("inf")
        elif with_bound:
            bound = _L().rdfgen_tree_bound(self._h, shape.n_v, _ptr(se), _ptr(isc), _ptr(mapped),
                                           _ptr(pat), _ptr(usub))
        return Query(pat, shape.n_v - len(shape.const), shape.name, bound, mapped, usub)

    def tree_bound(self, shape: Shape, q: Query) -> float:
        """Match count of the shape's spanning tree (its first n_v - 1 edges)
        under q's predicates and directions: an upper bound on q's answers."""
        se = np.array(shape.edges, np.uint32).reshape(-1)
        isc = np.zeros(shape.n_v, np.uint8)
        isc[list(shape.const)] = 1
        return float(_L().rdfgen_tree_bound(self._h, shape.n_v, _ptr(se), _ptr(isc),
                                            _ptr(q.embedding), _ptr(q.patterns),
                                            _ptr(q.u_subject)))

    def sample(self, shape: Shape, seed: int, qid: int, cap: float, tries: int = 3,
               escalate: bool = True, work_cap: int = 0):
        """First embedding of `shape` whose spanning-tree bound is <= cap.

        After `tries` rejected attempts one more shape vertex (drawn from the
        stream) becomes a constant, and so on while variables remain."""
        import copy
        sh = copy.deepcopy(shape)
        a = 0
        while True:
            rejected, raw = 0, 0
            while rejected < tries and raw < 64 * tries:
                q = self.embed(sh, seed, qid * 100003 + a, work_cap=work_cap)
                a += 1
                raw += 1
                if q is None:
                    continue
                if q.bound <= cap:
                    return q
                rejected += 1
            free = [v for v in range(sh.n_v) if v not in sh.const]
            if not escalate or len(free) <= 1:
                raise RuntimeError("no embedding of %s within cap %g" % (shape.name, cap))
            pick = free[draw(seed, 7, qid * 64 + len(sh.const)) % len(free)]
            sh.const = sorted(sh.const + [pick])


# --------------------------------------------------------------------------
# Workloads. Seeds: graph = 1000 + k, queries = 2000 + k for workload k.

@dataclass
class Workload:
    name: str
    scale: int
    n_edges: int
    n_preds: int
    zipf_s: float
    graph_seed: int
    query_seed: int
    n_queries: int
    cap: float             # reject queries whose spanning-tree bound exceeds this

    @property
    def n_vertices(self) -> int:
        return 1 << self.scale


WORKLOADS = {
    # scale-14 R-MAT, 131,072 draws, 16 predicates Zipf(1.0); 8 queries
    "rmat14": Workload("rmat14", 14, 131072, 16, 1.0, 1001, 2001, 8, 2e6),
    # scale-22 R-MAT, 2^26 draws (~64M triples), 64 predicates Zipf(1.0); 32 queries
    "rmat22": Workload("rmat22", 22, 1 << 26, 64, 1.0, 1002, 2002, 32, 2e7),
    # scale-26 R-MAT, 2^30 draws (~1.0B triples), 256 predicates Zipf(1.1); 16 queries
    "rmat26": Workload("rmat26", 26, 1 << 30, 256, 1.1, 1003, 2003, 16, 1e8),
    # scale-24 R-MAT, 2^28 draws (~256M triples), 128 predicates Zipf(1.0)
    "rmat24": Workload("rmat24", 24, 1 << 28, 128, 1.0, 1004, 2004, 4096, 1e6),
}


def graph(w: Workload):
    return rmat_triples(w.scale, w.n_edges, w.n_preds, w.zipf_s, w.graph_seed)


def _shapes_rmat14():
    s = star(3)
    s.const = [3]          # one leaf is a constant object: (centre, p, c)
    s.dir_req = {2: 1}
    return [s, s, chain(3), chain(3), cycle(3), cycle(3), snowflake([2, 1]), snowflake([2, 1])]


def _shapes_mixed(w: Workload):
    """Star / chain / cycle / snowflake with 3..8 query vertices and 0..2
    constants, one shape class per query in turn."""
    out = []
    for q in range(w.n_queries):
        r = draw(w.query_seed, 5, q)
        n_v = 3 + (r % 6)                         # 3..8 shape vertices
        kind = q % 4
        if kind == 0:
            sh = star(n_v - 1)
        elif kind == 1:
            sh = chain(n_v - 1)
        elif kind == 2:
            sh = cycle(n_v)
        else:
            n_v = max(n_v, 4)
            rest = n_v - 3                        # centre + 2 arms, rest are leaves
            a = (r >> 8) % (rest + 1)
            sh = snowflake([a, rest - a])
        n_const = (r >> 16) % 3                   # 0, 1 or 2
        n_const = min(n_const, sh.n_v - 2)
        verts = list(range(sh.n_v))
        picks = []
        for j in range(n_const):
            idx = draw(w.query_seed, 6, q * 8 + j) % len(verts)
            picks.append(verts.pop(idx))
        sh.const = sorted(picks)
        out.append(sh)
    return out


def _shapes_batched(w: Workload, n: int):
    """2..10 shape vertices, shape classes uniform, 1..2 constants (so the
    bound can be counted from a constant), and a target match count t drawn
    log-uniformly from [1, 10^6]; returns (shape, t) pairs."""
    out = []
    for q in range(n):
        r = draw(w.query_seed, 30, q)
        kind = r % 4
        n_v = 2 + (r >> 4) % 9                      # 2..10
        if kind == 0 or n_v == 2:
            sh = star(n_v - 1)
        elif kind == 1:
            sh = chain(n_v - 1)
        elif kind == 2:
            sh = cycle(n_v)
        else:
            n_v = max(n_v, 4)
            rest = n_v - 3
            a = (r >> 12) % (rest + 1)
            sh = snowflake([a, rest - a])
        n_const = 1 + (r >> 20) % 2
        n_const = min(n_const, sh.n_v - 1)
        verts = list(range(sh.n_v))
        picks = []
        for j in range(n_const):
            idx = draw(w.query_seed, 31, q * 8 + j) % len(verts)
            picks.append(verts.pop(idx))
        sh.const = sorted(picks)
        t = 10.0 ** (6.0 * (draw(w.query_seed, 32, q) % 1000003) / 1000003.0)
        out.append((sh, t))
    return out


def batched_queries(w: Workload, sampler: Sampler, n: int | None = None,
                    work_cap: int = 5_000_000, threads: int | None = None):
    """The batched workload's queries: each shape's first embedding whose
    spanning-tree bound (counted from its first constant) is at most its
    target; more constants after three rejections, and a ten times larger
    target when every vertex but one is constant."""
    import concurrent.futures as cf
    import os
    pairs = _shapes_batched(w, w.n_queries if n is None else n)

    def one(q):   # a pure function of (seed, q): thread order does not matter
        sh, cap = pairs[q]
        while True:   # no embedding within the target: the next larger decade
            try:
                return sampler.sample(sh, w.query_seed, q, cap, work_cap=work_cap)
            except RuntimeError:
                if cap > 1e7:
                    raise
                cap *= 10.0

    with cf.ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        return list(ex.map(one, range(len(pairs))))


def bandwidth_root(shape: Shape) -> int:
    """The vertex the degree-driven traversal (Sec. 6.1.2) starts from in a
    constant-free query: the most incident edges, ties to the lowest index
    (shape vertex k is variable k here)."""
    deg = [0] * shape.n_v
    for u, v in shape.edges:
        deg[u] += 1
        deg[v] += 1
    return max(range(shape.n_v), key=lambda v: (deg[v], -v))


def rare_cycle(k: int, pendant: bool = False) -> Shape:
    """A k-cycle on vertices 0..k-1 laid out for the bandwidth workload: the
    tree is the path 0, k-1, k-2, .., 1 (its edges take rare predicates),
    the closing edge (1, 0) is the non-tree edge (it takes one of the most
    frequent predicates). With pendant, vertex k hangs on vertex 0 by one
    more rare edge."""
    e = [(0, k - 1)] + [(i, i - 1) for i in range(k - 1, 1, -1)]
    if pendant:
        e.append((0, k))
    e.append((1, 0))
    return Shape("cycle%d%s" % (k, "+leaf" if pendant else ""), k + (1 if pendant else 0), e,
                 k - 1 + (1 if pendant else 0))


def _shapes_bandwidth(w: Workload, n: int):
    """Constant-free cycles, in turn: 3-cycle, 4-cycle, 3-cycle with a
    pendant edge on the root, 4-cycle. The root (vertex 0, where
    the degree-driven traversal starts) is evaluated first with all its
    edges together (Sec. 5): its closing edge takes one of the 8 most
    frequent predicates, so expanding it from the root's candidates reads
    long ranges of a frequent predicate; every other edge takes a predicate
    from the rarer half (ids above P/2), so the answer stays small."""
    top = (1, 8)
    tail = (w.n_preds // 2 + 1, w.n_preds)
    out = []
    for q in range(n):
        kind = q % 4
        sh = rare_cycle(3 if kind in (0, 2) else 4, pendant=kind == 2)
        for e in range(len(sh.edges)):
            sh.pred_range[e] = top if e == len(sh.edges) - 1 else tail
        assert bandwidth_root(sh) == 0
        out.append(sh)
    return out


def bandwidth_queries(w: Workload, sampler: Sampler, n: int | None = None,
                      cap: float | None = None, attempts: int = 2000):
    """The bandwidth-bound workload: for shape q (see _shapes_bandwidth),
    its first seeded embedding whose spanning-tree bound is at most cap.
    The tree holds every edge but the frequent closing one, so the bound
    (the match count of the rare path) caps the exact answer count. Every
    query has at least its embedding as an answer. Bounds depend only on
    the predicates and directions and are cached on them."""
    cap = w.cap if cap is None else cap
    shapes = _shapes_bandwidth(w, w.n_queries if n is None else n)
    cache = {}
    out = []
    for qi, sh in enumerate(shapes):
        got = None
        for a in range(attempts):
            q = sampler.embed(sh, w.query_seed, qi * 100003 + a, with_bound=False)
            if q is None:
                continue
            key = (tuple(q.patterns[:-1, 1].tolist()), tuple(q.u_subject[:-1].tolist()))
            if key not in cache:
                cache[key] = sampler.tree_bound(sh, q)
            q.bound = cache[key]
            if q.bound <= cap:
                got = q
                break
        if got is None:
            raise RuntimeError("no embedding of %s within bound %g in %d attempts"
                               % (sh.name, cap, attempts))
        out.append(got)
    return out


def save_queries(path: str, qs, header: str = ""):
    """Write queries as text: per query one line 'shape bound n s p o ...'."""
    with open(path, "w") as f:
        for line in header.splitlines():
            f.write("# %s\n" % line)
        for q in qs:
            # %.17g keeps an exact count (any integer below 2^53) exact
            f.write("%s %.17g %d %s\n" % (q.shape, q.bound, len(q.patterns),
                                         " ".join(str(int(x)) for x in q.patterns.reshape(-1))))


def load_queries(path: str):
    """Queries written by save_queries (embedding unknown: all zero)."""
    out = []
    with open(path) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            t = line.split()
            n = int(t[2])
            pat = np.array([int(x) for x in t[3:3 + 3 * n]], np.int64).reshape(n, 3)
            k = int(-pat[:, [0, 2]][pat[:, [0, 2]] < 0].min())
            out.append(Query(pat, k, t[0], float(t[1]), np.zeros(0, np.uint32)))
    return out


BANDWIDTH_QUERIES = 16


def bandwidth_file(name: str = "rmat26") -> str:
    """Where make_bandwidth_queries.py stores the family for a workload."""
    return os.path.join(_HERE, "%s_bandwidth.txt" % name)


BANDWIDTH_FILE = bandwidth_file("rmat26")


def bandwidth_workload(w: Workload | None = None):
    """The bandwidth-bound family's queries on w's graph (default: the
    scale-26 workload) as written by make_bandwidth_queries.py (the
    selection of bandwidth_queries, stored so that a run needs no
    sampler)."""
    w = w or WORKLOADS["rmat26"]
    path = bandwidth_file(w.name)
    qs = load_queries(path)
    if len(qs) != BANDWIDTH_QUERIES:
        raise ValueError("%s holds %d queries, the family %d" % (path, len(qs), BANDWIDTH_QUERIES))
    return qs


def queries(w: Workload, sampler: Sampler, n: int | None = None):
    """The workload's query list (deterministic)."""
    shapes = _shapes_rmat14() if w.name == "rmat14" else _shapes_mixed(w)
    if n is not None:
        shapes = shapes[:n]
    return [sampler.sample(sh, w.query_seed, q, w.cap) for q, sh in enumerate(shapes)]


# --------------------------------------------------------------------------
# Small random cases for exhaustive checks (numpy's seeded generator).

def random_graph(seed: int, n_vertices: int, n_preds: int, n_triples: int):
    """Uniform random triples with self-loops and repeated (s, o) pairs under
    several predicates; exact duplicates kept (consumers deduplicate)."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n_vertices, n_triples).astype(np.uint32)
    o = rng.integers(0, n_vertices, n_triples).astype(np.uint32)
    p = rng.integers(1, n_preds + 1, n_triples).astype(np.uint32)
    return s, p, o


def random_bgp(seed: int, n_vertices: int, n_preds: int, max_vars: int = 4,
               max_patterns: int = 4, p_const: float = 0.15):
    """Random BGP over dense variable ids (every variable used), with
    constants, repeated variables and self-loop patterns allowed."""
    rng = np.random.default_rng(seed)
    while True:
        k = int(rng.integers(1, max_vars + 1))
        n = int(rng.integers(1, max_patterns + 1))
        pats = []
        for _ in range(n):
            ends = []
            for _ in range(2):
                if rng.random() < p_const:
                    ends.append(int(rng.integers(0, n_vertices)))
                else:
                    ends.append(-int(rng.integers(0, k)) - 1)
            pats.append((ends[0], int(rng.integers(1, n_preds + 1)), ends[1]))
        used = sorted({-x - 1 for t in pats for x in (t[0], t[2]) if x < 0})
        if not used:
            continue
        remap = {v: i for i, v in enumerate(used)}
        pats = [tuple(-remap[-x - 1] - 1 if x < 0 else x for x in (t[0],)) + (t[1],) +
                tuple(-remap[-x - 1] - 1 if x < 0 else x for x in (t[2],)) for t in pats]
        return np.array(pats, np.int64)
