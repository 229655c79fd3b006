"""The traversal planners of Sec. 6.1 (oracle side) against the paper's
worked examples on the query graph of Fig. 2b. CPU only."""
import numpy as np

from oracle import planner


def _fig2b(golden):
    g = dict(golden("fig2b_planner.txt"))
    names = {}
    pats = []
    for k, e in enumerate(g["edges"].split()):
        a, b = e.split(">")
        for v in (a, b):
            names.setdefault(v, -(int(v[1:]) + 1))
        pats.append((names[a], k + 1, names[b]))
    return g, np.array(pats, np.int64)


def _fmt(groups, pats):
    out = []
    for v, es in groups:
        out.append("v%d:" % v[1] + ",".join(
            "v%d>v%d" % (-pats[i][0] - 1, -pats[i][2] - 1) for i in es))
    return " | ".join(out)


def _expect(line):
    plan, _, roots = line.partition(";")
    return plan.strip(), roots.replace("roots", "").split()


def test_example_6_1_direction_driven(golden):
    g, pats = _fig2b(golden)
    plan, roots = _expect(g["direction"])
    groups, rts = planner.direction_driven(pats)
    assert _fmt(groups, pats) == plan
    assert ["v%d" % r[1] for r in rts] == roots


def test_example_6_2_degree_driven(golden):
    g, pats = _fig2b(golden)
    plan, roots = _expect(g["degree"])
    groups, rts = planner.degree_driven(pats)
    assert _fmt(groups, pats) == plan
    assert ["v%d" % r[1] for r in rts] == roots


def test_example_7_1_paths(golden):
    g, pats = _fig2b(golden)
    groups, rts = planner.degree_driven(pats)
    got = {"-".join("v%d" % v[1] for v in path) for path in planner.paths(pats, groups, rts)}
    want = {p.strip() for p in g["paths"].split(";")}
    assert got == want


def test_every_edge_evaluated_once():
    rng = np.random.default_rng(0)
    for _ in range(300):
        k = int(rng.integers(2, 7))
        n = int(rng.integers(1, 9))
        pats = []
        for _ in range(n):
            a = -int(rng.integers(0, k)) - 1 if rng.random() > 0.15 else int(rng.integers(0, 50))
            b = -int(rng.integers(0, k)) - 1 if rng.random() > 0.15 else int(rng.integers(0, 50))
            pats.append((a, 1, b))
        for fn in (planner.degree_driven, planner.direction_driven):
            groups, roots = fn(pats)
            seen = [i for _, es in groups for i in es]
            assert sorted(seen) == list(range(n))
