"""The seeded input generator (rdfgen) on its own, CPU only: determinism,
and the two counts of a query's spanning-tree matches (the dense one and
the one walked from a constant) agree. The tree count is checked against
the oracle's answer count where the shape is a tree."""
import numpy as np
import pytest

import oracle
import rdfgen


@pytest.fixture(scope="module")
def small():
    s, p, o = rdfgen.rmat_triples(10, 6000, 6, 1.0, 77)
    return s, p, o, rdfgen.Sampler(s, p, o, 1 << 10, 6), oracle.Index(s, p, o, 1 << 10, 6)


def test_rmat_is_deterministic():
    a = rdfgen.rmat_triples(8, 1000, 4, 1.0, 5)
    b = rdfgen.rmat_triples(8, 1000, 4, 1.0, 5)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert a[1].min() >= 1 and a[1].max() <= 4 and a[0].max() < 256


@pytest.mark.parametrize("q", range(24))
def test_rooted_bound_equals_dense_bound(small, q):
    s, p, o, sm, _ = small
    sh = [rdfgen.star(3), rdfgen.chain(3), rdfgen.snowflake([1, 1]), rdfgen.chain(2)][q % 4]
    sh.const = [q % sh.n_v]
    a = sm.embed(sh, 9, q)
    if a is None:
        pytest.skip("walk failed")
    b = sm.embed(sh, 9, q, work_cap=10 ** 9)
    assert np.array_equal(a.patterns, b.patterns)
    assert a.bound == b.bound


@pytest.mark.parametrize("q", range(12))
def test_tree_bound_is_the_answer_count_of_tree_shapes(small, q):
    # for a tree-shaped query on deduplicated triples the spanning-tree count
    # is the exact answer count (homomorphisms)
    s, p, o, _, ix = small
    trip = np.unique(np.stack([s, p, o], 1), axis=0)
    ds, dp, do = (np.ascontiguousarray(trip[:, i]) for i in range(3))
    sm = rdfgen.Sampler(ds, dp, do, 1 << 10, 6)
    sh = [rdfgen.star(2), rdfgen.chain(3)][q % 2]
    sh.const = [q % sh.n_v]
    qq = sm.embed(sh, 4, q, work_cap=10 ** 9)
    if qq is None:
        pytest.skip("walk failed")
    assert qq.bound == len(ix.eval(qq.patterns))


def test_batched_sampling_is_deterministic_across_threads(small):
    s, p, o, sm, _ = small
    import dataclasses
    w = dataclasses.replace(rdfgen.WORKLOADS["rmat24"], n_queries=30)
    a = rdfgen.batched_queries(w, sm, threads=1)
    b = rdfgen.batched_queries(w, sm, threads=4)
    assert all(np.array_equal(x.patterns, y.patterns) for x, y in zip(a, b))
