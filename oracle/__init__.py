"""FP64 CPU oracle for the Bezier edge build and the graph search.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2411_13507_gb300``) and never imports it.

Pieces:
  tables.py       exact-rational coefficient tables (Lemma 1, Theorem 1, Eq. BezDef)
  plan_oracle.c   plain double loops over pairs, membership, nearest vertex and
                  a binary-heap Dijkstra (Sec. III-A, III-C; Properties 1-2)
  refine.py       FP64 smoothed-barrier + snap-energy loss and its gradient

All functions take plain numpy arrays (or any object with the attributes of a
generated problem: states, T, poly_off, A, b, model.{m,gamma,degree,bounds,
tighten,cost_mode}).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

from . import tables as _tables

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plan_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2 -ffp-contract=off, OpenMP if available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("gamma", ctypes.c_int), ("p", ctypes.c_int),
                ("nT", ctypes.c_int), ("N", ctypes.c_int), ("K", ctypes.c_int),
                ("cost_mode", ctypes.c_int),
                ("states", ctypes.c_void_p), ("poly_off", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("eps", ctypes.c_double),
                ("bounds", ctypes.c_void_p), ("D", ctypes.c_void_p), ("H", ctypes.c_void_p),
                ("C", ctypes.c_void_p)]


def _bind(lib):
    vp, i32 = ctypes.c_void_p, ctypes.c_int
    lib.orc_membership.argtypes = [vp, vp]
    lib.orc_candidate_counts.argtypes = [vp, vp, i32, vp, vp]
    lib.orc_edges_rows.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.orc_nearest.argtypes = [vp, vp]
    lib.orc_nearest.restype = i32
    lib.orc_dijkstra.argtypes = [i32, vp, vp, vp, i32, vp, vp]
    lib.orc_dijkstra.restype = i32
    lib.orc_num_threads.restype = i32
    return lib


def load_variant(path: str):
    """Load another build of plan_oracle.c (tests plant mistakes in a copy)."""
    return _bind(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleProblem:
    """Holds contiguous FP64 copies of one query plus the oracle's own tables."""

    def __init__(self, prob, tables: Optional[dict] = None, lib=None):
        self._lib = lib
        mdl = prob.model
        self.m, self.gamma, self.p = int(mdl.m), int(mdl.gamma), int(mdl.degree)
        self.n = self.m * self.gamma
        self.states = np.ascontiguousarray(prob.states, dtype=np.float64).reshape(-1, self.n)
        self.T = np.ascontiguousarray(prob.T, dtype=np.float64)
        self.poly_off = np.ascontiguousarray(prob.poly_off, dtype=np.int32)
        self.A = np.ascontiguousarray(prob.A, dtype=np.float64).reshape(-1, self.m)
        self.b = np.ascontiguousarray(prob.b, dtype=np.float64)
        self.bounds = np.ascontiguousarray(np.asarray(mdl.bounds, dtype=np.float64))
        self.eps = float(getattr(mdl, "tighten", 0.0))
        self.cost_mode = 1 if getattr(mdl, "cost_mode", "state") == "pos" else 0
        self.N, self.K, self.nT = self.states.shape[0], self.poly_off.shape[0] - 1, self.T.shape[0]
        self.interior = getattr(mdl, "interior", "elevate")
        tb = tables if tables is not None else _tables.tables(self.gamma, self.p, self.T, self.interior)
        self.D = np.ascontiguousarray(tb["D"], dtype=np.float64)
        self.H = np.ascontiguousarray(tb["H"], dtype=np.float64)
        self.C = np.ascontiguousarray(tb["C"], dtype=np.float64)
        self._c = _Problem(self.m, self.gamma, self.p, self.nT, self.N, self.K, self.cost_mode,
                           _ptr(self.states), _ptr(self.poly_off), _ptr(self.A), _ptr(self.b),
                           self.eps, _ptr(self.bounds), _ptr(self.D), _ptr(self.H), _ptr(self.C))
        self._in = None

    @property
    def lib(self):
        return self._lib if self._lib is not None else _load()

    @property
    def cref(self):
        return ctypes.byref(self._c)

    def membership(self) -> np.ndarray:
        if self._in is None:
            out = np.zeros((self.N, self.K), dtype=np.uint8)
            if self.N and self.K:
                self.lib.orc_membership(self.cref, _ptr(out))
            self._in = out
        return self._in

    def candidate_counts(self, rows=None) -> np.ndarray:
        rows = np.arange(self.N, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
        inm = self.membership()
        cnt = np.zeros(rows.shape[0], dtype=np.int64)
        if rows.size:
            self.lib.orc_candidate_counts(self.cref, _ptr(inm), int(rows.size), _ptr(rows), _ptr(cnt))
        return cnt

    def edges(self, rows=None, with_detail: bool = True) -> dict:
        """Every candidate pair of the given rows: i, j, mask, best w, best t (+costs, margins)."""
        rows = np.arange(self.N, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
        inm = self.membership()
        cnt = self.candidate_counts(rows)
        off = np.zeros(rows.shape[0], dtype=np.int64)
        if rows.size:
            off[1:] = np.cumsum(cnt)[:-1]
        P = int(cnt.sum())
        out = {"i": np.zeros(P, np.int32), "j": np.zeros(P, np.int32), "mask": np.zeros(P, np.uint32),
               "w": np.zeros(P, np.float64), "t": np.zeros(P, np.int32)}
        if with_detail:
            for key in ("costs", "rmarg", "fmarg"):
                out[key] = np.zeros((P, self.nT), np.float64)
        if P:
            g = lambda k: _ptr(out[k]) if k in out else None
            self.lib.orc_edges_rows(self.cref, _ptr(inm), int(rows.size), _ptr(rows), _ptr(off),
                                   g("i"), g("j"), g("mask"), g("w"), g("t"), g("costs"), g("rmarg"), g("fmarg"))
        out["counts"] = cnt
        return out

    def csr(self, with_detail: bool = False) -> dict:
        """Feasible-edge CSR over all rows, sorted (i asc, j asc)."""
        e = self.edges(None, with_detail=with_detail)
        keep = e["mask"] != 0
        row_off = np.zeros(self.N + 1, dtype=np.int64)
        np.add.at(row_off, e["i"][keep].astype(np.int64) + 1, 1)
        row_off = np.cumsum(row_off)
        res = {"row_off": row_off, "col": e["j"][keep], "w": e["w"][keep], "t": e["t"][keep],
               "mask": e["mask"][keep], "candidates": int(e["i"].shape[0])}
        if with_detail:
            res["costs"] = e["costs"][keep]
            res["all"] = e
        return res

    def nearest(self, pos) -> int:
        q = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(self.m))
        return int(self.lib.orc_nearest(self.cref, _ptr(q)))


def dijkstra(N: int, row_off, col, w, s: int):
    row_off = np.ascontiguousarray(row_off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    dist = np.zeros(N, dtype=np.float64)
    pred = np.zeros(N, dtype=np.int32)
    if N:
        rc = _load().orc_dijkstra(int(N), _ptr(row_off), _ptr(col), _ptr(w), int(s), _ptr(dist), _ptr(pred))
        if rc != 0:
            raise MemoryError("oracle dijkstra: allocation failed")
    return dist, pred


def walk(pred, s: int, g: int):
    """Path s -> g from a predecessor array, or None if g is unreachable."""
    if s == g:
        return [s]
    path = [g]
    v = g
    for _ in range(len(pred)):
        v = int(pred[v])
        if v < 0:
            return None
        path.append(v)
        if v == s:
            return path[::-1]
    raise RuntimeError("predecessor cycle")


def search(op: OracleProblem, csr: dict, start_pos, goal_pos) -> dict:
    """findPath (Sec. III-C): nearest start/goal vertices, then Dijkstra."""
    s = op.nearest(start_pos)
    g = op.nearest(goal_pos)
    dist, pred = dijkstra(op.N, csr["row_off"], csr["col"], csr["w"], s)
    path = walk(pred, s, g)
    return {"start": s, "goal": g, "path": path, "cost": float(dist[g]) if path is not None else float("inf"),
            "dist": dist, "pred": pred}
