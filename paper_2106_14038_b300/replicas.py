"""Root-range partitioning of one query over replicas (Sec. 6.3.1).

The paper's first-stage partition splits the work of a query by its root
bindings: every answer has exactly one binding of the root variable (the
plan's first level), so ranges of root vertex ids that partition [0, N)
partition the answers too. Each replica holds the whole graph, evaluates
the query for its own range (gs_eval_query_roots), and the only exchange is
the final gather of the answer rows, merged on the host.

Host logic only: the slices, the merge and the gather over an initialized
torch.distributed process group (gloo or NCCL; rows travel as Python
objects, so any backend that gathers objects works).
"""
from __future__ import annotations

import numpy as np


def root_slices(n_vertices: int, parts: int):
    """[(lo, hi)] * parts: consecutive ranges of vertex ids, sizes differing
    by at most one, covering [0, n_vertices) exactly."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    n = int(n_vertices)
    q, r = divmod(n, parts)
    out, lo = [], 0
    for k in range(parts):
        hi = lo + q + (1 if k < r else 0)
        out.append((lo, hi))
        lo = hi
    return out


def sort_rows(rows: np.ndarray) -> np.ndarray:
    """Rows in ascending lexicographic order (column 0 first)."""
    rows = np.asarray(rows)
    if rows.ndim != 2 or rows.shape[0] < 2 or rows.shape[1] == 0:
        return rows
    order = np.lexsort(rows.T[::-1])
    return rows[order]


def merge_rows(parts, n_vars: int | None = None, sort: bool = True) -> np.ndarray:
    """The answers of all ranges: their rows concatenated (range order), or
    in lexicographic order when sort. Parts are int32 (rows, n_vars) arrays;
    n_vars is needed only when every part is empty and none has a shape."""
    parts = [np.asarray(p, np.int32) for p in parts]
    if n_vars is None:
        n_vars = next((p.shape[1] for p in parts if p.ndim == 2), 0)
    parts = [p.reshape(-1, n_vars) for p in parts]
    rows = np.concatenate(parts, axis=0) if parts else np.zeros((0, n_vars), np.int32)
    return sort_rows(rows) if sort else rows


def eval_slice(graph, plan, rank: int, world: int, sort: bool = True, stream=None) -> np.ndarray:
    """This rank's answers: plan evaluated on graph for root range `rank` of
    `world` equal ranges."""
    lo, hi = root_slices(graph.n_vertices, world)[rank]
    r = graph.eval(plan, stream=stream, roots=(lo, hi))
    try:
        return r.fetch(sort=sort)
    finally:
        r.close()


def gather_rows(local_rows: np.ndarray, dist, n_vars: int, sort: bool = True, group=None):
    """Every rank's rows gathered to all ranks and merged (the one exchange
    of a root-partitioned query). dist is torch.distributed, initialized."""
    world = dist.get_world_size(group)
    got = [None] * world
    dist.all_gather_object(got, np.asarray(local_rows, np.int32), group=group)
    return merge_rows(got, n_vars=n_vars, sort=sort)
