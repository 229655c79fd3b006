"""Writes <workload>_bandwidth.txt: the bandwidth-bound family's 16 queries
on a workload's graph (rdfgen.bandwidth_queries with the workload's seeds),
so that benchmarks and tests load them without building the sampler's
adjacency (about 40 GB of host memory at scale 26).

    python -m rdfgen.make_bandwidth_queries              # rmat26, its answer cap
    python -m rdfgen.make_bandwidth_queries rmat22 1e9   # the scale-22 copy

The scale-26 file is the bandwidth configuration's query set. The scale-22
one holds the same shapes with a rare-path bound of at most 1e9 (the tail
predicates of the 64-predicate graph are less rare), so that its binding
trees are about as large as at scale 26 on a graph ncu can replay.
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import rdfgen  # noqa: E402


def main(argv):
    name = argv[1] if len(argv) > 1 else "rmat26"
    w = rdfgen.WORKLOADS[name]
    cap = float(argv[2]) if len(argv) > 2 else w.cap
    t0 = time.time()
    s, p, o = rdfgen.graph(w)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    qs = rdfgen.bandwidth_queries(w, sm, n=rdfgen.BANDWIDTH_QUERIES, cap=cap)
    sm.close()
    header = ("Bandwidth-bound workload: %d constant-free cycles on R-MAT scale %d, 2^%d draws, "
              "%d predicates Zipf(%g), graph seed %d, query seed %d.\n"
              "Written by rdfgen/make_bandwidth_queries.py (rdfgen.bandwidth_queries, answer "
              "cap %g by the rare-path bound) in %.0f s.\n"
              "Per line: shape, rare-path bound, patterns, then s p o per pattern "
              "(variable k is -(k+1))."
              % (len(qs), w.scale, w.n_edges.bit_length() - 1, w.n_preds, w.zipf_s, w.graph_seed,
                 w.query_seed, cap, time.time() - t0))
    out = rdfgen.bandwidth_file(name)
    rdfgen.save_queries(out, qs, header)
    print("wrote %s" % out)


if __name__ == "__main__":
    main(sys.argv)
