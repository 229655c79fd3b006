"""ORACLE — test infrastructure only.

Plain CPU reference for what the engine computes: BGP answers by the
definition (a conjunction of triple patterns, Sec. 2.2.3), the predicate
selection vectors of Eq. 4 / Eq. 5, the sorted triple lists behind the CSR
and CSC RDF matrices (Sec. 6.2), and the two traversal planners of Sec. 6.1
(planner.py). Only the tests, the smoke entry point and the benchmark's CPU
baseline leg may import this package. It shares no code with the engine.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bgp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile bgp_oracle.c into liboracle.so beside it (plain C, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        lib.orc_index_build.restype = vp
        lib.orc_index_build.argtypes = [vp, vp, vp, u64, u32, u32]
        lib.orc_index_free.restype = None
        lib.orc_index_free.argtypes = [vp]
        lib.orc_index_size.restype = u64
        lib.orc_index_size.argtypes = [vp]
        lib.orc_index_triples.restype = None
        lib.orc_index_triples.argtypes = [vp, i32, vp, vp, vp]
        lib.orc_presence.restype = None
        lib.orc_presence.argtypes = [vp, i32, u32, vp]
        lib.orc_eval.restype = i32
        lib.orc_eval.argtypes = [vp, vp, u32, i32, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)),
                                 ctypes.POINTER(u64), ctypes.POINTER(u32)]
        lib.orc_free.restype = None
        lib.orc_free.argtypes = [vp]
        lib.orc_count.restype = i32
        lib.orc_count.argtypes = [vp, vp, u32, i32, u64, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Index:
    """Deduplicated triples in (s,p,o), (o,p,s) and (p,s,o) order."""

    def __init__(self, s, p, o, n_vertices: int, n_preds: int):
        s = np.ascontiguousarray(s, np.uint32)
        p = np.ascontiguousarray(p, np.uint32)
        o = np.ascontiguousarray(o, np.uint32)
        self.n_vertices, self.n_preds = int(n_vertices), int(n_preds)
        self._h = _L().orc_index_build(_ptr(s), _ptr(p), _ptr(o), len(s), n_vertices, n_preds)
        if not self._h:
            raise ValueError("oracle index build failed (bad triple or out of memory)")

    def __del__(self):
        try:
            if self._h:
                _L().orc_index_free(self._h)
                self._h = None
        except Exception:
            pass

    def __len__(self):
        return int(_L().orc_index_size(self._h))

    def triples(self, by_object: bool = False):
        """(s, p, o) sorted by (s,p,o), or by (o,p,s) when by_object."""
        n = len(self)
        s, p, o = (np.empty(n, np.uint32) for _ in range(3))
        _L().orc_index_triples(self._h, int(by_object), _ptr(s), _ptr(p), _ptr(o))
        return s, p, o

    def presence(self, direction: int, pred: int) -> np.ndarray:
        """Eq. 4 (direction 0: rows holding pred) or Eq. 5 (direction 1:
        columns holding pred) as a 0/1 uint8 vector of length n_vertices."""
        out = np.empty(self.n_vertices, np.uint8)
        _L().orc_presence(self._h, int(direction), int(pred), _ptr(out))
        return out

    def eval(self, patterns, threads: int = 1) -> np.ndarray:
        """Sorted int32 answer rows (n_rows, n_vars) of a BGP.

        patterns: (n, 3) int64 (s, p, o); s, o >= 0 are constant vertex ids,
        s, o < 0 are variables -(k+1); p is a predicate id."""
        pat = np.ascontiguousarray(np.asarray(patterns, np.int64).reshape(-1, 3))
        rows = ctypes.POINTER(ctypes.c_int32)()
        n = ctypes.c_uint64()
        k = ctypes.c_uint32()
        rc = _L().orc_eval(self._h, _ptr(pat), len(pat), int(threads), ctypes.byref(rows),
                           ctypes.byref(n), ctypes.byref(k))
        if rc == -1:
            raise ValueError("invalid query")
        if rc == -2:
            raise MemoryError("oracle out of memory")
        if rc != 0:
            raise RuntimeError("oracle internal error %d" % rc)
        try:
            nr, nk = int(n.value), int(k.value)
            if nr == 0:
                return np.zeros((0, nk), np.int32)
            buf = np.ctypeslib.as_array(rows, shape=(nr * nk,))
            return buf.copy().reshape(nr, nk)
        finally:
            _L().orc_free(ctypes.cast(rows, ctypes.c_void_p))

    def count(self, patterns, threads: int = 1, max_steps: int = 0):
        """(answer rows, join steps, complete) of a BGP without storing the
        rows; with max_steps > 0 the join gives up after about that many
        steps (complete is then False and rows a lower bound)."""
        pat = np.ascontiguousarray(np.asarray(patterns, np.int64).reshape(-1, 3))
        n = ctypes.c_uint64()
        st = ctypes.c_uint64()
        rc = _L().orc_count(self._h, _ptr(pat), len(pat), int(threads), int(max_steps),
                            ctypes.byref(n), ctypes.byref(st))
        if rc == -1:
            raise ValueError("invalid query")
        if rc == -2:
            raise MemoryError("oracle out of memory")
        if rc not in (0, -4):
            raise RuntimeError("oracle internal error %d" % rc)
        return int(n.value), int(st.value), rc == 0


def csr_arrays(s, p, o, n_rows: int):
    """Row pointers / column / label arrays of the RDF matrix stored by rows,
    from triples already sorted by (s,p,o) (use Index.triples()). For the
    column-wise matrix pass (o, p, s) sorted by (o,p,s)."""
    counts = np.bincount(np.asarray(s, np.int64), minlength=n_rows)
    ptr = np.zeros(n_rows + 1, np.int64)
    np.cumsum(counts, out=ptr[1:])
    return ptr, np.asarray(o, np.uint32), np.asarray(p, np.uint32)
