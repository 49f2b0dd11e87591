"""CPU oracle for exact vertex cover (test infrastructure only).

This package is the plain sequential branch-and-reduce search of Sec. II-B, written in C
(``vc_oracle.c``) and loaded through ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the library in ``paper_2204_10402_gb300`` never imports it,
and the two share no code.

Functions:
  greedy(g)                 -> (size, cover mask)              Sec. II-B, greedy upper bound
  mvc(g)                    -> (size, cover mask, stats)       Sec. II-B, MVC search
  pvc(g, k)                 -> (found, cover mask, stats)      Sec. II-B, PVC search
  reduce_node(g, deg, ...)  -> (deg, S, m, pruned)             Sec. II-B / IV-D reduction rules
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

MVC, PVC = 0, 1
RULE_DEG1, RULE_DEG2TRI, RULE_HIGH, RULE_ALL = 1, 2, 4, 7


class OracleLimit(RuntimeError):
    """The search hit its node limit before finishing."""


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so`` (portable flags, no -march)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Oracle:
    """ctypes view of one compiled copy of ``vc_oracle.c`` (the default build, or a test's copy)."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orc_greedy.restype = ctypes.c_int32
        lib.orc_greedy.argtypes = [ctypes.c_int32, i32p, i32p, i32p]
        lib.orc_mvc.restype = ctypes.c_int32
        lib.orc_mvc.argtypes = [ctypes.c_int32, i32p, i32p, i32p, ctypes.c_int64, i64p]
        lib.orc_pvc.restype = ctypes.c_int32
        lib.orc_pvc.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p, ctypes.c_int64, i64p]
        lib.orc_reduce_node.restype = ctypes.c_int32
        lib.orc_reduce_node.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i64p,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        self.lib = lib

    def greedy(self, g):
        off, adj = _arrays(g)
        cover = np.zeros(max(g.n, 1), dtype=np.int32)
        size = self.lib.orc_greedy(g.n, _p32(off), _p32(adj), _p32(cover))
        return int(size), cover[: g.n].astype(bool)

    def mvc(self, g, max_nodes: int = 0):
        """Minimum cover size, a cover of that size, and stats {nodes, greedy, max_depth}."""
        off, adj = _arrays(g)
        cover = np.zeros(max(g.n, 1), dtype=np.int32)
        stats = np.zeros(3, dtype=np.int64)
        r = self.lib.orc_mvc(g.n, _p32(off), _p32(adj), _p32(cover), int(max_nodes),
                             stats.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        if r == -2:
            raise OracleLimit(f"MVC search exceeded {max_nodes} nodes")
        if r < 0:
            raise MemoryError("oracle allocation failed")
        return int(r), cover[: g.n].astype(bool), {"nodes": int(stats[0]), "greedy": int(stats[1]),
                                                   "max_depth": int(stats[2])}

    def pvc(self, g, k: int, max_nodes: int = 0):
        """Whether a cover of size <= k exists, such a cover (if found), and stats."""
        off, adj = _arrays(g)
        cover = np.zeros(max(g.n, 1), dtype=np.int32)
        stats = np.zeros(3, dtype=np.int64)
        r = self.lib.orc_pvc(g.n, _p32(off), _p32(adj), int(k), _p32(cover), int(max_nodes),
                             stats.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        if r == -2:
            raise OracleLimit(f"PVC search exceeded {max_nodes} nodes")
        if r < 0:
            raise MemoryError("oracle allocation failed")
        return bool(r), cover[: g.n].astype(bool), {"nodes": int(stats[0]), "greedy": int(stats[1]),
                                                    "max_depth": int(stats[2])}

    def reduce_node(self, g, deg, S: int, m: int, mode: int, bound: int, rules: int = RULE_ALL):
        """Reduce one tree node to its fixpoint.  ``deg`` is the degree array (-1 = in S)."""
        off, adj = _arrays(g)
        d = np.array(deg, dtype=np.int32).copy()
        if d.size == 0:
            d = np.zeros(1, dtype=np.int32)
        s = ctypes.c_int32(S)
        mm = ctypes.c_int64(m)
        pruned = self.lib.orc_reduce_node(g.n, _p32(off), _p32(adj), _p32(d), ctypes.byref(s),
                                          ctypes.byref(mm), mode, bound, rules)
        return d[: g.n].copy(), int(s.value), int(mm.value), bool(pruned)


def _default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _arrays(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.int32)
    adj = np.ascontiguousarray(g.neighbors, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)
    return off, adj


def greedy(g):
    return _default().greedy(g)


def mvc(g, max_nodes: int = 0):
    return _default().mvc(g, max_nodes)


def pvc(g, k: int, max_nodes: int = 0):
    return _default().pvc(g, k, max_nodes)


def reduce_node(g, deg, S: int, m: int, mode: int, bound: int, rules: int = RULE_ALL):
    return _default().reduce_node(g, deg, S, m, mode, bound, rules)


def verify_cover(g, cover_mask) -> bool:
    """True iff every edge has an endpoint in the cover (Sec. II-A definition)."""
    u, v = g.edges()
    c = np.asarray(cover_mask, dtype=bool)
    return bool(np.all(c[u] | c[v]))
