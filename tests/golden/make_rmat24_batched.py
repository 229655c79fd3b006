"""Writes rmat24_batched.txt: the batched workload's 4,096 queries on the
scale-24 graph with their exact answer counts.

Query q has the shape and constants rdfgen gives it (2..10 shape vertices,
star / chain / cycle / snowflake, 1..2 constants) and a target count t drawn
log-uniformly from [1, 10^6]. Its seeded embeddings are tried in order; the
first whose exact answer count (the oracle's count mode) lies in [t/2, 2t]
is kept, else, after 24 tries, the one whose count is nearest t on a log
scale. A count may take the oracle at most 10^5 + 50 t join steps (a count
in [t/2, 2t] needs far fewer); tries past that are not used, and a query
none of whose tries finishes is left out (the header says how many). Every
query kept has at least its embedding as an answer.

    python tests/golden/make_rmat24_batched.py
"""
import concurrent.futures as cf
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import rdfgen  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "rmat24_batched.txt")
TRIES = 24


def max_steps(t: float) -> int:
    return int(1e5 + 50 * t)


def main():
    w = rdfgen.WORKLOADS["rmat24"]
    t0 = time.time()
    s, p, o = rdfgen.graph(w)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    ix = oracle.Index(s, p, o, w.n_vertices, w.n_preds)
    pairs = rdfgen._shapes_batched(w, w.n_queries)

    def one(q):
        sh, t = pairs[q]
        best, best_d = None, None
        for a in range(TRIES):
            emb = sm.embed(sh, w.query_seed, q * 100003 + a, with_bound=False)
            if emb is None:
                continue
            n, _, done = ix.count(emb.patterns, threads=1, max_steps=max_steps(t))
            if not done:
                continue
            d = abs(math.log(max(n, 1)) - math.log(t))
            if best is None or d < best_d:
                best, best_d = (emb, n), d
            if t / 2 <= n <= 2 * t:
                break
        if best is None:
            return None
        emb, n = best
        emb.bound = float(n)          # the exact count
        return emb, t

    got = []
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        for i, r in enumerate(ex.map(one, range(len(pairs)))):
            got.append(r)
            if (i + 1) % 256 == 0:
                print("%d of %d queries in %.0f s" % (i + 1, len(pairs), time.time() - t0), flush=True)
    dropped = sum(1 for g in got if g is None)
    got = [g for g in got if g is not None]
    qs = [e for e, _ in got]
    inside = sum(1 for e, t in got if t / 2 <= e.bound <= 2 * t)
    header = ("Batched workload: %d queries on R-MAT scale %d, 2^%d draws, %d predicates "
              "Zipf(%g), graph seed %d, query seed %d.\n"
              "Written by tests/golden/make_rmat24_batched.py in %.0f s: per query the first "
              "embedding whose exact answer count (oracle count mode) lies in [t/2, 2t], t "
              "log-uniform in [1, 1e6]; %d of %d within, the others nearest t; %d left out "
              "(no try counted within 1e5 + 50 t join steps).\n"
              "Per line: shape, exact answer count, patterns, then s p o per pattern "
              "(variable k is -(k+1))."
              % (len(qs), w.scale, w.n_edges.bit_length() - 1, w.n_preds, w.zipf_s, w.graph_seed,
                 w.query_seed, time.time() - t0, inside, len(qs), dropped))
    rdfgen.save_queries(OUT, qs, header)
    print("wrote %s (%d of %d within [t/2, 2t])" % (OUT, inside, len(qs)))


if __name__ == "__main__":
    main()
