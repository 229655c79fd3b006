"""ORACLE — test infrastructure only.

The two traversal planners of Sec. 6.1, step by step in the paper's order,
plus the binding-tree paths of Sec. 7.1. The engine has its own planner
(C++); tests compare the two and pin this one to Examples 6.1, 6.2 and 7.1.

Query graph: one vertex per distinct variable and per distinct constant,
one directed edge per triple pattern (Sec. 2.2.1). Vertex keys are
('v', k) for variable k and ('c', id) for a constant vertex id; edges are
pattern indices.

Readings where the text is silent (listed with the other readings of the
paper in the design notes):
  * the root is added to W (the visited set) when it is chosen;
  * only vertices newly added to W are pushed;
  * remaining ties after the paper's criteria go to the lower vertex key
    (variables before constants, then by index): for the root choice the
    lower key wins; for pushes, the lower key is pushed last so it is
    popped first;
  * a popped vertex with no unevaluated edge yields no group;
  * the stray "set i = i + 1" in step 4 is ignored;
  * with constants, when no unvisited vertex adjacent to a constant is left,
    the root is chosen by the rule without constants (the constant variant
    of step 2 does not cover this case).
"""
from __future__ import annotations


def _vkey(x):
    return ("v", -int(x) - 1) if int(x) < 0 else ("c", int(x))


def _order_key(v):
    return (0 if v[0] == "v" else 1, v[1])


class QueryGraph:
    def __init__(self, patterns):
        self.edges = []   # (subject vertex, object vertex)
        self.vertices = []
        seen = set()
        for s, _p, o in patterns:
            a, b = _vkey(s), _vkey(o)
            self.edges.append((a, b))
            for v in (a, b):
                if v not in seen:
                    seen.add(v)
                    self.vertices.append(v)
        self.vertices.sort(key=_order_key)

    def out_edges(self, v, F):
        return [i for i, (a, b) in enumerate(self.edges) if a == v and i not in F]

    def in_edges(self, v, F):
        return [i for i, (a, b) in enumerate(self.edges) if b == v and i not in F]

    def inc_edges(self, v, F):
        return [i for i, (a, b) in enumerate(self.edges) if (a == v or b == v) and i not in F]


def degree_driven(patterns):
    """Sec. 6.1.2 (with its constant variant). Returns (groups, roots):
    groups = [(vertex, [edge indices])] in evaluation order."""
    G = QueryGraph(patterns)
    S, W, F, groups, roots = [], set(), set(), [], []
    consts = [v for v in G.vertices if v[0] == "c"]
    if consts:                                     # constant variant of steps 1-2
        for c in consts:
            W.add(c)
        for c in consts:
            es = G.inc_edges(c, F)
            if es:
                groups.append((c, es))
                F.update(es)
    while len(F) < len(G.edges):                   # step 5 loop
        cand = [v for v in G.vertices if v not in W]
        if consts:
            adj = [v for v in cand if any(
                (a in consts and b == v) or (b in consts and a == v) for a, b in G.edges)]
            if adj:
                cand = adj
        root = max(cand, key=lambda v: (len(G.inc_edges(v, F)), len(G.out_edges(v, F)),
                                        _low_first(v)))
        roots.append(root)
        W.add(root)
        S.append(root)
        while S:                                   # steps 3-4
            v = S.pop()
            es = G.inc_edges(v, F)
            if not es:
                continue
            groups.append((v, es))
            F.update(es)
            new = []
            for i in es:
                a, b = G.edges[i]
                w = b if a == v else a
                if w not in W and w not in new:
                    new.append(w)
            for w in new:
                W.add(w)
            new.sort(key=lambda w: (len(G.inc_edges(w, F)), len(G.out_edges(w, F)),
                                    _low_first(w)))
            S.extend(new)
    return groups, roots


def _low_first(v):
    """Tie key: larger for a lower vertex key, so max() picks the lower key
    and an ascending sort pushes the lower key last (popped first)."""
    k = _order_key(v)
    return (-k[0], -k[1])


def direction_driven(patterns):
    """Sec. 6.1.1 (with its cyclic variant). Queries with constants use the
    degree-driven traversal, as the paper prescribes."""
    G = QueryGraph(patterns)
    if any(v[0] == "c" for v in G.vertices):
        return degree_driven(patterns)
    S, W, F, groups, roots = [], set(), set(), [], []
    while len(F) < len(G.edges):
        cand = [v for v in G.vertices if v not in W]
        noin = [v for v in cand if not G.in_edges(v, F)]
        pool = noin if noin else cand              # cyclic variant
        root = max(pool, key=lambda v: (len(G.out_edges(v, F)), _low_first(v)))
        roots.append(root)
        W.add(root)
        S.append(root)
        while S:
            v = S.pop()
            es = G.out_edges(v, F)
            if not es:
                continue
            groups.append((v, es))
            F.update(es)
            new = []
            for i in es:
                w = G.edges[i][1]
                if w not in W and w not in new:
                    new.append(w)
            for w in new:
                W.add(w)
            new.sort(key=lambda w: (len(G.out_edges(w, F)), _low_first(w)))
            S.extend(new)
    return groups, roots


def paths(patterns, groups, roots):
    """Binding-tree paths of Sec. 7.1: from each root, follow each edge of a
    group to its other end; continue into that end's group when this edge
    is the one that first reached it, else the path ends there."""
    G = QueryGraph(patterns)
    gmap = {v: es for v, es in groups}
    reached_by = {}
    for v, es in groups:
        for i in es:
            a, b = G.edges[i]
            w = b if a == v else a
            if w not in reached_by and w not in roots and w[0] == "v":
                reached_by[w] = i
    out = []

    def walk(v, prefix):
        for i in gmap.get(v, []):
            a, b = G.edges[i]
            w = b if a == v else a
            if w in gmap and reached_by.get(w) == i:
                walk(w, prefix + [w])
            else:
                out.append(prefix + [w])

    for r in roots:
        walk(r, [r])
    return out
