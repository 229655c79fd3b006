"""B300 engine for SPARQL basic graph patterns by grouped incident-edge
evaluation over a sparse RDF matrix (gSmart, arXiv 2106.14038).

Thin ctypes binding over libgsmart.so (include/gsmart.h): argument
marshalling only; every step of the evaluation runs in the library's CUDA
kernels. PyTorch supplies CUDA streams and device tensors. There is no CPU
fallback: without the built library, or without a GPU, calls raise.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

import numpy as np

from ._build import LIB, build

__all__ = ["Graph", "Plan", "Result", "Batch", "Server", "GsError", "TorchAllocator", "load_library", "PLAN_DEGREE",
           "PLAN_DIRECTION", "PLAN_LISTS", "PLAN_PATHS", "BatchConfig", "Lspm", "build"]

PLAN_DEGREE = 0
PLAN_DIRECTION = 1
PLAN_LISTS = 2         # option bit: the list frontier form
PLAN_PATHS = 4         # option bit: per-path binding trees with tree-pruning
_STATUS = {0: "GS_OK", 1: "GS_EINVAL", 2: "GS_ENOMEM", 3: "GS_ECUDA", 4: "GS_EOVERFLOW",
           5: "GS_ETIMEOUT", 6: "GS_ENOTIMPL"}

EXPORTED = ["gs_load_triples", "gs_graph_info", "gs_graph_export", "gs_plan_query",
            "gs_plan_describe", "gs_eval_query", "gs_result_info", "gs_fetch_bindings",
            "gs_result_stats", "gs_scan_candidates", "gs_free_graph", "gs_free_plan",
            "gs_free_result", "gs_last_error", "gs_eval_batch", "gs_batch_info",
            "gs_batch_fetch", "gs_batch_stats", "gs_free_batch", "gs_batch_poll",
            "gs_server_start", "gs_server_submit", "gs_server_poll", "gs_server_fetch",
            "gs_server_release", "gs_server_stats", "gs_server_stop",
            "gs_scan_candidates_noalloc", "gs_noalloc_scratch_bytes", "gs_eval_batch_cfg",
            "gs_batch_autotune", "gs_server_replay", "gs_scan_status", "gs_batch_scans",
            "gs_plan_estimate", "gs_server_ticket", "gs_server_admission",
            "gs_server_submit_many", "gs_lspm_build", "gs_lspm_for_plan", "gs_lspm_info",
            "gs_lspm_export", "gs_eval_query_lspm", "gs_free_lspm", "gs_server_work",
            "gs_result_tree", "gs_plan_paths", "gs_eval_query_roots", "gs_plan_root",
            "gs_graph_set_trace", "gs_result_phases"]


class GsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class BatchConfig(ctypes.Structure):
    """gs_batch_config: tunables of a batched evaluation (0 = default)."""
    _fields_ = [("blocks_per_sm", ctypes.c_uint32), ("grid_streams", ctypes.c_uint32),
                ("cand_budget", ctypes.c_uint64), ("row_budget", ctypes.c_uint64),
                ("pool_bytes", ctypes.c_uint64), ("scan_share", ctypes.c_uint32),
                ("frontier", ctypes.c_uint32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator
    (passed through the C ABI's gs_allocator hook). `fail_after` makes the
    n-th and later allocations fail (returns NULL), for failure tests."""

    def __init__(self, device: int = 0, fail_after: int | None = None):
        import torch
        self._torch = torch
        self.device = device
        self.fail_after = fail_after
        self.calls = 0
        self.live = {}

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.fail_after is not None and self.calls >= self.fail_after:
                return None
            try:
                ptr = self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream)
            except Exception:
                return None
            self.live[ptr] = nbytes
            return ptr

        def _free(ptr, stream, ctx):
            if ptr:
                self.live.pop(ptr, None)
                self._torch.cuda.caching_allocator_delete(ptr)

        self._cb_alloc = _ALLOC_FN(_alloc)
        self._cb_free = _FREE_FN(_free)
        self.struct = _Allocator(self._cb_alloc, self._cb_free, None)


_lib = None
_live_servers = weakref.WeakSet()   # stopped before their graph is freed, and at exit
_live_lspm = weakref.WeakSet()      # freed before their graph


def _stop_servers(graph=None):
    for srv in list(_live_servers):
        if graph is None or srv._graph is graph:
            srv.stop()


atexit.register(_stop_servers)


def load_library(path: str | None = None):
    """Load libgsmart.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise ImportError("libgsmart.so is not built; run paper_2106_14038_b300.build() "
                          "(nvcc for sm_103a)")
    lib = ctypes.CDLL(path)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "gs_load_triples": [vp, vp, vp, u64, u32, u32, i32, vp, vp, P(vp)],
        "gs_graph_info": [vp, P(u64), P(u32), P(u32)],
        "gs_graph_export": [vp, i32, vp, vp, vp, i32, vp],
        "gs_plan_query": [vp, vp, u32, u32, P(vp)],
        "gs_plan_describe": [vp, vp, u32, P(u32)],
        "gs_plan_paths": [vp, vp, u32, P(u32)],
        "gs_eval_query": [vp, vp, vp, P(vp)],
        "gs_eval_query_roots": [vp, vp, u32, u32, vp, P(vp)],
        "gs_plan_root": [vp, P(u32)],
        "gs_graph_set_trace": [vp, i32],
        "gs_result_phases": [vp, vp, u32, P(u32)],
        "gs_result_info": [vp, P(u64), P(u32)],
        "gs_fetch_bindings": [vp, vp, u64, i32, i32],
        "gs_result_stats": [vp, P(ctypes.c_float), P(u32)],
        "gs_result_tree": [vp, vp, u32, P(u32)],
        "gs_scan_candidates": [vp, vp, vp, u32, vp, vp],
        "gs_scan_candidates_noalloc": [vp, vp, vp, u32, vp, vp],
        "gs_scan_status": [vp, vp],
        "gs_eval_batch": [vp, vp, u32, vp, P(vp)],
        "gs_eval_batch_cfg": [vp, vp, u32, vp, vp, P(vp)],
        "gs_batch_autotune": [vp, vp, u32, vp, vp, P(ctypes.c_float)],
        "gs_server_replay": [vp, vp, u32, vp, u64, ctypes.c_double, vp, vp, vp, u64, P(u64)],
        "gs_server_work": [vp, P(u64), P(u64), P(u64)],
        "gs_batch_info": [vp, vp, P(u64)],
        "gs_batch_fetch": [vp, u32, vp, u64, i32, i32],
        "gs_batch_stats": [vp, P(ctypes.c_float), P(u32), P(u32)],
        "gs_batch_poll": [vp, P(i32)],
        "gs_batch_scans": [vp, P(u32), P(u32)],
        "gs_plan_estimate": [vp, vp, P(u64), P(ctypes.c_double)],
        "gs_server_start": [vp, vp, P(vp)],
        "gs_server_submit": [vp, vp, P(u64)],
        "gs_server_poll": [vp, u64, P(i32), P(u64), P(ctypes.c_double)],
        "gs_server_fetch": [vp, u64, vp, u64, i32, i32],
        "gs_server_release": [vp, u64],
        "gs_server_stats": [vp, P(u64), P(u64), P(u64)],
        "gs_server_ticket": [vp, u64, P(u64), P(u64)],
        "gs_server_submit_many": [vp, vp, u32, vp],
        "gs_lspm_build": [vp, vp, u32, vp, u32, vp, P(vp)],
        "gs_lspm_for_plan": [vp, vp, vp, P(vp)],
        "gs_lspm_info": [vp, i32, P(u64), P(u64)],
        "gs_lspm_export": [vp, i32, vp, vp, vp, vp, i32, vp],
        "gs_eval_query_lspm": [vp, vp, vp, vp, P(vp)],
        "gs_server_admission": [vp, P(u64), P(u64)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = i32
    for name in ("gs_free_graph", "gs_free_plan", "gs_free_result", "gs_free_batch",
                 "gs_server_stop", "gs_free_lspm"):
        f = getattr(lib, name)
        f.argtypes = [vp]
        f.restype = None
    lib.gs_noalloc_scratch_bytes.argtypes = []
    lib.gs_noalloc_scratch_bytes.restype = ctypes.c_size_t
    lib.gs_last_error.argtypes = []
    lib.gs_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise GsError(rc, _lib.gs_last_error().decode(errors="replace"))


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _host_u32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.uint32)


class Graph:
    """The RDF matrix resident on the device (CSR + CSC with labels)."""

    def __init__(self, s, p, o, n_vertices: int, n_predicates: int, stream=None,
                 allocator: "TorchAllocator | None" = None):
        lib = load_library()
        import torch
        self._keep = None
        self._allocator = allocator      # callbacks must outlive the graph
        self.device = torch.cuda.current_device()
        on_dev = hasattr(s, "is_cuda") and s.is_cuda
        if on_dev:
            import torch
            s, p, o = (x.to(torch.int32).contiguous() for x in (s, p, o))
            ptrs = [ctypes.c_void_p(x.data_ptr()) for x in (s, p, o)]
            n = s.numel()
            self._keep = (s, p, o)
        else:
            s, p, o = _host_u32(s), _host_u32(p), _host_u32(o)
            ptrs = [x.ctypes.data_as(ctypes.c_void_p) for x in (s, p, o)]
            n = len(s)
            self._keep = (s, p, o)
        h = ctypes.c_void_p()
        aptr = ctypes.byref(allocator.struct) if allocator is not None else None
        _check(lib.gs_load_triples(*ptrs, n, n_vertices, n_predicates, int(on_dev), aptr,
                                   _stream_handle(stream), ctypes.byref(h)))
        self._keep = None
        self._h = h
        self.n_vertices, self.n_predicates = int(n_vertices), int(n_predicates)
        m = ctypes.c_uint64()
        _check(lib.gs_graph_info(h, ctypes.byref(m), None, None))
        self.n_triples = int(m.value)

    def close(self):
        if getattr(self, "_h", None):
            _stop_servers(self)          # a running server uses the graph
            for l in list(_live_lspm):   # so does a reduced matrix
                if l._graph is self:
                    l.close()
            _lib.gs_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self, by_column: bool = False, stream=None):
        """(ptr, idx, lab) numpy arrays of the row-wise (or column-wise) copy."""
        ptr = np.empty(self.n_vertices + 1, np.uint32)
        idx = np.empty(max(self.n_triples, 1), np.uint32)
        lab = np.empty(max(self.n_triples, 1), np.uint32)
        _check(_lib.gs_graph_export(self._h, int(by_column), ptr.ctypes.data_as(ctypes.c_void_p),
                                    idx.ctypes.data_as(ctypes.c_void_p),
                                    lab.ctypes.data_as(ctypes.c_void_p), 0, _stream_handle(stream)))
        return ptr, idx[:self.n_triples], lab[:self.n_triples]

    def set_trace(self, on: bool = True):
        """Record per-phase CUDA events in later grid-path evaluations
        (Result.phases)."""
        _check(_lib.gs_graph_set_trace(self._h, int(bool(on))))

    def plan(self, patterns, flags: int = PLAN_DEGREE) -> "Plan":
        return Plan(self, patterns, flags)

    def eval(self, plan_or_patterns, stream=None, roots=None) -> "Result":
        """Evaluate a plan; with roots=(lo, hi) only the answers whose root
        binding (column plan.root_var) lies in [lo, hi)."""
        plan = plan_or_patterns if isinstance(plan_or_patterns, Plan) else self.plan(plan_or_patterns)
        h = ctypes.c_void_p()
        if roots is None:
            _check(_lib.gs_eval_query(self._h, plan._h, _stream_handle(stream), ctypes.byref(h)))
        else:
            lo, hi = (int(x) for x in roots)
            _check(_lib.gs_eval_query_roots(self._h, plan._h, lo, hi, _stream_handle(stream),
                                            ctypes.byref(h)))
        return Result(h, plan)

    def query(self, patterns, sort: bool = True, flags: int = PLAN_DEGREE, stream=None):
        """Answer rows (numpy int32, n_rows x n_vars) of a BGP."""
        r = self.eval(self.plan(patterns, flags), stream)
        try:
            return r.fetch(sort=sort)
        finally:
            r.close()

    def eval_batch(self, plans, stream=None, config: "BatchConfig | None" = None) -> "Batch":
        """Evaluate many plans (or pattern arrays) in one persistent launch,
        under `config` (a BatchConfig; None: defaults)."""
        plans = [p if isinstance(p, Plan) else self.plan(p) for p in plans]
        arr = (ctypes.c_void_p * max(1, len(plans)))(*[p._h.value for p in plans])
        h = ctypes.c_void_p()
        if config is None:
            _check(_lib.gs_eval_batch(self._h, arr, len(plans), _stream_handle(stream),
                                      ctypes.byref(h)))
        else:
            _check(_lib.gs_eval_batch_cfg(self._h, arr, len(plans), ctypes.byref(config),
                                          _stream_handle(stream), ctypes.byref(h)))
        return Batch(h, plans)

    def autotune_batch(self, plans, stream=None):
        """The batch configuration the native autotuner picks for these plans
        (a sample of the workload) and its wall time in ms."""
        plans = [p if isinstance(p, Plan) else self.plan(p) for p in plans]
        arr = (ctypes.c_void_p * max(1, len(plans)))(*[p._h.value for p in plans])
        cfg = BatchConfig()
        ms = ctypes.c_float()
        _check(_lib.gs_batch_autotune(self._h, arr, len(plans), _stream_handle(stream),
                                      ctypes.byref(cfg), ctypes.byref(ms)))
        return cfg, float(ms.value)

    def _check_bits_out(self, out):
        """The candidate-bit buffer must be a contiguous int32 CUDA tensor of
        at least ceil(N/32) words on the graph's device (the kernel writes
        4 * ceil(N/32) bytes into it)."""
        import torch
        words = (self.n_vertices + 31) // 32
        if not isinstance(out, torch.Tensor):
            raise ValueError("out must be a torch tensor")
        if out.dtype != torch.int32:
            raise ValueError("out must be int32, not %s" % out.dtype)
        if not out.is_contiguous():
            raise ValueError("out must be contiguous")
        if out.numel() < words:
            raise ValueError("out holds %d words, the vector needs %d" % (out.numel(), words))
        if not out.is_cuda or out.device.index != self.device:
            raise ValueError("out must be on cuda:%d, the graph's device" % self.device)

    def scan(self, preds, dirs, out=None, stream=None):
        """Eq. 17 / Eq. 21 on its own: a torch int32 tensor of ceil(N/32)
        words, bit x set when row x holds every preds[i] with dirs[i] == 0
        and column x every preds[i] with dirs[i] == 1. A stalled scan is
        reported by scan_status()."""
        import torch
        words = (self.n_vertices + 31) // 32
        if out is None:
            out = torch.empty(words, dtype=torch.int32, device="cuda:%d" % self.device)
        self._check_bits_out(out)
        pr = _host_u32(preds)
        dr = np.ascontiguousarray(np.asarray(dirs), dtype=np.uint8)
        _check(_lib.gs_scan_candidates(self._h, pr.ctypes.data_as(ctypes.c_void_p),
                                       dr.ctypes.data_as(ctypes.c_void_p), len(pr),
                                       ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def scan_noalloc(self, preds, dirs, out, stream=None):
        """scan() with the workspace in the library's static device array:
        the call allocates nothing, so `out` (int32, ceil(N/32) words on the
        graph's device) is required. Calls overlapping in time on one device
        race on that array."""
        self._check_bits_out(out)
        pr = _host_u32(preds)
        dr = np.ascontiguousarray(np.asarray(dirs), dtype=np.uint8)
        _check(_lib.gs_scan_candidates_noalloc(self._h, pr.ctypes.data_as(ctypes.c_void_p),
                                               dr.ctypes.data_as(ctypes.c_void_p), len(pr),
                                               ctypes.c_void_p(out.data_ptr()),
                                               _stream_handle(stream)))
        return out


    def estimate(self, plan):
        """(estimated device bytes, estimated answer rows) of evaluating plan."""
        b, r = ctypes.c_uint64(), ctypes.c_double()
        _check(_lib.gs_plan_estimate(self._h, plan._h, ctypes.byref(b), ctypes.byref(r)))
        return int(b.value), float(r.value)

    def scan_status(self, stream=None):
        """Synchronize the stream; raise GsError (GS_ETIMEOUT) when a bounded
        wait of a scan()/scan_noalloc() call on this graph ran out since the
        last check (that scan's bits are incomplete)."""
        _check(_lib.gs_scan_status(self._h, _stream_handle(stream)))


class Lspm:
    """Per-query light-weight sparse matrix (Sec. 6.2) reduced on the device
    from a graph: Lspm(graph, row_preds, col_preds) or Lspm.for_plan(plan)."""

    def __init__(self, graph: Graph, row_preds=(), col_preds=(), stream=None, _plan=None):
        h = ctypes.c_void_p()
        if _plan is not None:
            _check(_lib.gs_lspm_for_plan(graph._h, _plan._h, _stream_handle(stream), ctypes.byref(h)))
        else:
            r, c = _host_u32(list(row_preds)), _host_u32(list(col_preds))
            _check(_lib.gs_lspm_build(graph._h, r.ctypes.data_as(ctypes.c_void_p), len(r),
                                      c.ctypes.data_as(ctypes.c_void_p), len(c),
                                      _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self._graph = graph
        _live_lspm.add(self)

    @classmethod
    def for_plan(cls, graph: Graph, plan: "Plan", stream=None) -> "Lspm":
        return cls(graph, stream=stream, _plan=plan)

    def info(self, by_column: bool = False):
        """(rows or columns kept, entries kept)."""
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.gs_lspm_info(self._h, int(by_column), ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def export(self, by_column: bool = False, stream=None):
        """(M, P, Val, Idx) numpy arrays: Mr/Pr/Val/Col (or Mc/Pc/Val/Row)."""
        kept, nnz = self.info(by_column)
        m = np.empty(self._graph.n_vertices + 1, np.uint32)
        ptr = np.empty(kept + 1, np.uint32)
        val = np.empty(max(nnz, 1), np.uint32)
        idx = np.empty(max(nnz, 1), np.uint32)
        _check(_lib.gs_lspm_export(self._h, int(by_column), m.ctypes.data_as(ctypes.c_void_p),
                                   ptr.ctypes.data_as(ctypes.c_void_p),
                                   val.ctypes.data_as(ctypes.c_void_p),
                                   idx.ctypes.data_as(ctypes.c_void_p), 0, _stream_handle(stream)))
        return m, ptr, val[:nnz], idx[:nnz]

    def eval(self, plan: "Plan", stream=None) -> "Result":
        h = ctypes.c_void_p()
        _check(_lib.gs_eval_query_lspm(self._graph._h, self._h, plan._h, _stream_handle(stream),
                                       ctypes.byref(h)))
        return Result(h, plan)

    def close(self):
        if getattr(self, "_h", None):
            _lib.gs_free_lspm(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    def __init__(self, graph: Graph, patterns, flags: int = PLAN_DEGREE):
        load_library()
        pat = patterns
        if not (isinstance(pat, np.ndarray) and pat.dtype == np.int64 and pat.ndim == 2
                and pat.flags.c_contiguous):
            pat = np.ascontiguousarray(np.asarray(patterns, dtype=np.int64).reshape(-1, 3))
        h = ctypes.c_void_p()
        _check(_lib.gs_plan_query(graph._h, pat.ctypes.data, len(pat), flags, ctypes.byref(h)))
        self._h = h
        self.patterns = pat
        self._n_vars = None

    @property
    def n_vars(self) -> int:
        """Number of variables (answer columns)."""
        if self._n_vars is None:
            ends = self.patterns[:, [0, 2]]
            self._n_vars = int(-ends[ends < 0].min()) if (ends < 0).any() else 0
        return self._n_vars

    @property
    def root_var(self) -> int:
        """The root variable (answer column) that root ranges partition."""
        v = ctypes.c_uint32()
        _check(_lib.gs_plan_root(self._h, ctypes.byref(v)))
        return int(v.value)

    def describe(self):
        """(groups, roots): groups = [(vertex, [edge indices])]; a vertex is a
        variable index k >= 0 or ('c', id) for a constant."""
        n = ctypes.c_uint32()
        _lib.gs_plan_describe(self._h, None, 0, ctypes.byref(n))
        buf = np.zeros(n.value, np.int32)
        _check(_lib.gs_plan_describe(self._h, buf.ctypes.data_as(ctypes.c_void_p), n.value,
                                     ctypes.byref(n)))
        w = buf.tolist()

        def vert(x):
            return x if x >= 0 else ("c", -x - 1)

        i = 0
        ng = w[i]; i += 1
        groups = []
        for _ in range(ng):
            v, ne = w[i], w[i + 1]
            groups.append((vert(v), w[i + 2:i + 2 + ne]))
            i += 2 + ne
        nr = w[i]; i += 1
        roots = [vert(x) for x in w[i:i + nr]]
        return groups, roots

    def paths(self):
        """Binding-tree paths (Sec. 7.1): lists of variable indices."""
        n = ctypes.c_uint32()
        _lib.gs_plan_paths(self._h, None, 0, ctypes.byref(n))
        buf = np.zeros(max(1, n.value), np.int32)
        _check(_lib.gs_plan_paths(self._h, buf.ctypes.data_as(ctypes.c_void_p), n.value,
                                  ctypes.byref(n)))
        w = buf[:n.value].tolist()
        out, i = [], 1
        for _ in range(w[0]):
            out.append(w[i + 1:i + 1 + w[i]])
            i += 1 + w[i]
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.gs_free_plan(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    def __init__(self, h, plans):
        self._h = h
        self._plans = plans       # the plans must outlive the batch

    def rows(self):
        """Answer row count of every query (numpy uint64)."""
        n = len(self._plans)
        out = np.zeros(max(1, n), np.uint64)
        tot = ctypes.c_uint64()
        _check(_lib.gs_batch_info(self._h, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(tot)))
        return out[:n]

    def fetch(self, q: int, sort: bool = True):
        n = int(self.rows()[q])
        k = self._plans[q].n_vars
        out = np.empty((n, k), np.int32)
        _check(_lib.gs_batch_fetch(self._h, q, out.ctypes.data_as(ctypes.c_void_p), n, 0, int(sort)))
        return out

    def scans(self):
        """(triple scans run, plans they served)."""
        a, b = ctypes.c_uint32(), ctypes.c_uint32()
        _check(_lib.gs_batch_scans(self._h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def stats(self):
        """(device milliseconds, kernels launched, queries sent to the grid path)."""
        ms = ctypes.c_float()
        nl = ctypes.c_uint32()
        ne = ctypes.c_uint32()
        _check(_lib.gs_batch_stats(self._h, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(ne)))
        return float(ms.value), int(nl.value), int(ne.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.gs_free_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("n_streams", ctypes.c_uint32),
                ("memory_budget", ctypes.c_uint64), ("max_wait_us", ctypes.c_uint32),
                ("pool_bytes_per_query", ctypes.c_uint64), ("batch", BatchConfig)]


class Server:
    """Continuous-batching server over a resident graph (gs_server_*)."""

    def __init__(self, graph: Graph, max_batch: int = 0, n_streams: int = 0,
                 memory_budget: int = 0, max_wait_us: int = 0, pool_bytes_per_query: int = 0,
                 batch: "BatchConfig | None" = None):
        cfg = _ServerConfig(max_batch, n_streams, memory_budget, max_wait_us, pool_bytes_per_query,
                            batch if batch is not None else BatchConfig())
        h = ctypes.c_void_p()
        _check(_lib.gs_server_start(graph._h, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._graph = graph
        self._plans = {}
        _live_servers.add(self)

    def submit(self, plan: "Plan") -> int:
        t = ctypes.c_uint64()
        _check(_lib.gs_server_submit(self._h, plan._h, ctypes.byref(t)))
        self._plans[t.value] = plan
        return int(t.value)

    def submit_many(self, plans):
        """Queue several plans at once (the worker sees all or none)."""
        arr = (ctypes.c_void_p * max(1, len(plans)))(*[p._h.value for p in plans])
        out = np.zeros(max(1, len(plans)), np.uint64)
        _check(_lib.gs_server_submit_many(self._h, arr, len(plans), out.ctypes.data_as(ctypes.c_void_p)))
        for t, p in zip(out[:len(plans)].tolist(), plans):
            self._plans[int(t)] = p
        return [int(t) for t in out[:len(plans)]]

    def poll(self, ticket: int):
        """(done, rows, latency_us)."""
        d = ctypes.c_int()
        n = ctypes.c_uint64()
        lat = ctypes.c_double()
        _check(_lib.gs_server_poll(self._h, ticket, ctypes.byref(d), ctypes.byref(n),
                                   ctypes.byref(lat)))
        return bool(d.value), int(n.value), float(lat.value)

    def fetch(self, ticket: int, sort: bool = True):
        done, n, _ = self.poll(ticket)
        if not done:
            raise RuntimeError("ticket %d is not finished" % ticket)
        k = self._plans[ticket].n_vars
        out = np.empty((n, k), np.int32)
        _check(_lib.gs_server_fetch(self._h, ticket, out.ctypes.data_as(ctypes.c_void_p), n, 0,
                                    int(sort)))
        return out

    def release(self, ticket: int):
        _check(_lib.gs_server_release(self._h, ticket))
        self._plans.pop(ticket, None)

    def ticket(self, ticket: int):
        """(sequence number of the batch that took it, estimated device bytes)."""
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.gs_server_ticket(self._h, ticket, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def admission(self):
        """(admissions that passed an older waiting query, bytes in flight)."""
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.gs_server_admission(self._h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def stats(self):
        """(completed queries, batches launched, peak admitted device bytes)."""
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.gs_server_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return int(a.value), int(b.value), int(c.value)

    def replay(self, plans, arrival_s, timeout_s: float = 120.0, fetch_into=None):
        """Native load replay: query i is plans[i % len(plans)], submitted at
        arrival_s[i] seconds; returns (latency_us, done_s) arrays. With
        fetch_into (a host int32 array, e.g. pinned torch memory as numpy)
        every answer is copied there before release; then returns
        (latency_us, done_s, fetched_bytes)."""
        arr = (ctypes.c_void_p * max(1, len(plans)))(*[p._h.value for p in plans])
        at = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(len(at))
        done = np.zeros(len(at))
        fb = ctypes.c_uint64()
        buf, cap = None, 0
        if fetch_into is not None:
            k = max(p.n_vars for p in plans)
            buf, cap = fetch_into.ctypes.data_as(ctypes.c_void_p), fetch_into.size // max(k, 1)
        _check(_lib.gs_server_replay(self._h, arr, len(plans), at.ctypes.data_as(ctypes.c_void_p),
                                     len(at), float(timeout_s), lat.ctypes.data_as(ctypes.c_void_p),
                                     done.ctypes.data_as(ctypes.c_void_p), buf, cap,
                                     ctypes.byref(fb)))
        if fetch_into is not None:
            return lat, done, int(fb.value)
        return lat, done

    def work(self):
        """(kernel launches, triple scans, plans those scans served) of the
        completed batches."""
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.gs_server_work(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return int(a.value), int(b.value), int(c.value)

    def stop(self):
        if getattr(self, "_h", None):
            _lib.gs_server_stop(self._h)
            self._h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


class Result:
    def __init__(self, h, plan: Plan):
        self._h = h
        self._plan = plan

    def info(self):
        n = ctypes.c_uint64()
        k = ctypes.c_uint32()
        _check(_lib.gs_result_info(self._h, ctypes.byref(n), ctypes.byref(k)))
        return int(n.value), int(k.value)

    def stats(self):
        """(device milliseconds of the last evaluation, kernels it launched)."""
        ms = ctypes.c_float()
        n = ctypes.c_uint32()
        _check(_lib.gs_result_stats(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return float(ms.value), int(n.value)

    def tree(self):
        """Nodes per level of the binding tree (grid-path evaluations)."""
        buf = np.zeros(32, np.uint64)
        n = ctypes.c_uint32()
        _check(_lib.gs_result_tree(self._h, buf.ctypes.data_as(ctypes.c_void_p), 32, ctypes.byref(n)))
        return buf[:n.value].tolist()

    def phases(self):
        """Device ms of the traced phases: [setup + triple scan, level 0,
        ..., level L-1, enumeration] (needs Graph.set_trace(True) before
        the evaluation, and the grid path)."""
        buf = np.zeros(40, np.float32)
        n = ctypes.c_uint32()
        _check(_lib.gs_result_phases(self._h, buf.ctypes.data_as(ctypes.c_void_p), 40, ctypes.byref(n)))
        return buf[:n.value].tolist()

    def time_ms(self) -> float:
        return self.stats()[0]

    def fetch(self, sort: bool = True, out=None):
        """Answer rows. out: None (a new numpy array), a numpy int32 array,
        or a torch CUDA int32 tensor (device-to-device copy)."""
        n, k = self.info()
        if out is None:
            out = np.empty((n, k), np.int32)
        on_dev = hasattr(out, "is_cuda") and out.is_cuda
        if on_dev:
            ptr = ctypes.c_void_p(out.data_ptr())
            cap = out.numel() // max(k, 1)
        else:
            ptr = out.ctypes.data_as(ctypes.c_void_p)
            cap = out.size // max(k, 1)
        _check(_lib.gs_fetch_bindings(self._h, ptr, cap, int(on_dev), int(sort)))
        return out if on_dev else out[:n]

    def close(self):
        if getattr(self, "_h", None):
            _lib.gs_free_result(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
