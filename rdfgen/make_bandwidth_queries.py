"""Writes rmat26_bandwidth.txt: the bandwidth-bound workload's queries on the
scale-26 graph (rdfgen.bandwidth_queries with the workload's seeds and its
answer cap), so that benchmarks and tests load them without building the
sampler's adjacency (about 40 GB of host memory at this size).

    python -m rdfgen.make_bandwidth_queries
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import rdfgen  # noqa: E402


def main():
    w = rdfgen.WORKLOADS["rmat26"]
    t0 = time.time()
    s, p, o = rdfgen.graph(w)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    qs = rdfgen.bandwidth_queries(w, sm)
    sm.close()
    header = ("Bandwidth-bound workload: %d constant-free cycles on R-MAT scale %d, 2^%d draws, "
              "%d predicates Zipf(%g), graph seed %d, query seed %d.\n"
              "Written by rdfgen/make_bandwidth_queries.py (rdfgen.bandwidth_queries, answer "
              "cap %g by the rare-path bound) in %.0f s.\n"
              "Per line: shape, rare-path bound, patterns, then s p o per pattern "
              "(variable k is -(k+1))."
              % (len(qs), w.scale, w.n_edges.bit_length() - 1, w.n_preds, w.zipf_s, w.graph_seed,
                 w.query_seed, w.cap, time.time() - t0))
    rdfgen.save_queries(rdfgen.BANDWIDTH_FILE, qs, header)
    print("wrote %s" % rdfgen.BANDWIDTH_FILE)


if __name__ == "__main__":
    main()
