"""Python binding of libplan (ctypes): argument marshalling only.

Every step of the planner runs in the CUDA kernels behind the C ABI declared
in ``include/plan.h``; this module allocates torch tensors for the outputs,
passes raw pointers and the current CUDA stream, and reads statuses.  There is
no CPU fallback: if ``libplan.so`` cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import build as _build

PLAN_OK, PLAN_ERR_INVALID_ARG, PLAN_ERR_UNSUPPORTED, PLAN_ERR_CAPACITY = 0, 1, 2, 3
PLAN_ERR_CUDA, PLAN_ERR_TIMEOUT, PLAN_ERR_NO_PATH, PLAN_ERR_NO_MEMORY = 4, 5, 6, 7
ARITH = {"f64": 0, "f32": 1, "tf32": 2, "bf16": 3}
INPUT = {"f64": 0, "f32": 1}
COST = {"state": 0, "pos": 1}
DET_SLOTS, DET_RECHECK, DET_OUTPUT = 1, 2, 3
DET_CUTLIST = 10

_lib = None


class PlanError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"plan status {status} ({status_string(status)}){': ' + msg if msg else ''}")


class _Model(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("gamma", ctypes.c_int), ("degree", ctypes.c_int),
                ("arith", ctypes.c_int), ("input", ctypes.c_int), ("cost_mode", ctypes.c_int),
                ("bound", ctypes.c_double * 4), ("tighten", ctypes.c_double), ("interior", ctypes.c_int)]


class _Edges(ctypes.Structure):
    _fields_ = [("row_off", ctypes.c_void_p), ("col", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("tidx", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("cap", ctypes.c_int64),
                ("count", ctypes.c_void_p)]


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("detail", ctypes.c_int32), ("memberships", ctypes.c_int64),
                ("slots", ctypes.c_int64), ("candidates", ctypes.c_int64), ("checks", ctypes.c_int64),
                ("reach_pass", ctypes.c_int64), ("feasible", ctypes.c_int64), ("rechecks", ctypes.c_int64),
                ("edges", ctypes.c_int64), ("search_iters", ctypes.c_int64), ("start", ctypes.c_int32),
                ("goal", ctypes.c_int32), ("need_slots", ctypes.c_int64), ("need_rechecks", ctypes.c_int64),
                ("work_reach_rows", ctypes.c_int64), ("work_free_rows", ctypes.c_int64), ("work_costs", ctypes.c_int64),
                ("screened", ctypes.c_int64), ("cut_units", ctypes.c_int64), ("cut_tests", ctypes.c_int64),
                ("cut_box", ctypes.c_int64), ("cut_near", ctypes.c_int64), ("cut_step1", ctypes.c_int64),
                ("cut_step2", ctypes.c_int64), ("cut_games", ctypes.c_int64), ("cut_lp64", ctypes.c_int64),
                ("cut_ties", ctypes.c_int64), ("shard_lo", ctypes.c_int32), ("shard_hi", ctypes.c_int32)]


class _Obstacles(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("off", ctypes.c_void_p), ("max_rows", ctypes.c_int), ("A", ctypes.c_void_p),
                ("b", ctypes.c_void_p)]


class _Query(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("states", ctypes.c_void_p), ("nT", ctypes.c_int),
                ("T", ctypes.POINTER(ctypes.c_double)), ("K", ctypes.c_int), ("poly_off", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("out", _Edges)]


class _SearchQuery(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("states", ctypes.c_void_p), ("edges", _Edges),
                ("start_pos", ctypes.c_double * 4), ("goal_pos", ctypes.c_double * 4),
                ("path", ctypes.c_void_p), ("path_cap", ctypes.c_int), ("path_len", ctypes.c_void_p),
                ("cost", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class _RefineW(ctypes.Structure):
    _fields_ = [("w_snap", ctypes.c_double), ("mu", ctypes.c_double), ("delta", ctypes.c_double)]


class _MpcParams(ctypes.Structure):
    _fields_ = [("horizon", ctypes.c_int), ("dt", ctypes.c_double), ("Q", ctypes.c_void_p), ("F", ctypes.c_void_p),
                ("R", ctypes.c_void_p), ("V", ctypes.c_void_p), ("keepin_rows", ctypes.c_int),
                ("keepin_A", ctypes.c_void_p), ("keepin_b", ctypes.c_void_p)]


PLAN_MPC_OK, PLAN_MPC_INFEASIBLE, PLAN_MPC_ITERATION_LIMIT = 0, 1, 2


EXPORTS = ["plan_create", "plan_destroy", "plan_build_edges", "plan_build_edges_shard", "plan_search", "plan_wait", "plan_model_tables",
           "plan_set_search_limits", "plan_refine", "plan_prepare_batched", "plan_build_edges_batched",
           "plan_set_tile", "plan_autotune", "plan_prepare_search_batched", "plan_search_batched",
           "plan_search_noalloc", "plan_cut_edges", "plan_cut_timing", "plan_search_at", "plan_search_to", "plan_obstacle_planes", "plan_nearest_planes", "plan_mpc_qp",
           "plan_set_accounting", "plan_set_timing", "plan_timing", "plan_measure_lane_rate", "plan_status_string",
           "plan_last_error", "plan_version"]


def lib_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libplan.so (building it first when sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale and _build.is_stale():
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libplan.so not built ({path}); run paper_2411_13507_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    lib.plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Model), vp]
    lib.plan_create.restype = i32
    lib.plan_destroy.argtypes = [vp]
    lib.plan_destroy.restype = None
    lib.plan_build_edges.argtypes = [vp, i32, vp, i32, dp, i32, vp, i32, vp, vp, ctypes.POINTER(_Edges)]
    lib.plan_build_edges.restype = i32
    lib.plan_build_edges_shard.argtypes = [vp, i32, vp, i32, dp, i32, vp, i32, vp, vp, i32, i32, ctypes.POINTER(_Edges)]
    lib.plan_build_edges_shard.restype = i32
    lib.plan_search.argtypes = [vp, i32, vp, ctypes.POINTER(_Edges), dp, dp, vp, i32, vp, vp]
    lib.plan_search.restype = i32
    lib.plan_wait.argtypes = [vp, ctypes.POINTER(_Info)]
    lib.plan_wait.restype = i32
    lib.plan_model_tables.argtypes = [ctypes.POINTER(_Model), i32, dp, dp, dp, dp]
    lib.plan_model_tables.restype = i32
    lib.plan_set_search_limits.argtypes = [vp, i32, i64]
    lib.plan_set_search_limits.restype = i32
    lib.plan_prepare_batched.argtypes = [vp, i32, ctypes.POINTER(_Query), i32]
    lib.plan_prepare_batched.restype = i32
    lib.plan_build_edges_batched.argtypes = [vp]
    lib.plan_build_edges_batched.restype = i32
    lib.plan_prepare_search_batched.argtypes = [vp, i32, ctypes.POINTER(_SearchQuery)]
    lib.plan_prepare_search_batched.restype = i32
    lib.plan_search_batched.argtypes = [vp]
    lib.plan_search_batched.restype = i32
    lib.plan_search_noalloc.argtypes = [i32, i32, i32, i32, i32, vp, ctypes.POINTER(_Edges), dp, dp, vp, i32, vp, vp, vp, vp]
    lib.plan_search_noalloc.restype = i32
    lib.plan_cut_edges.argtypes = [vp, i32, vp, i32, dp, ctypes.POINTER(_Edges), ctypes.POINTER(_Obstacles),
                                   ctypes.POINTER(_Edges)]
    lib.plan_cut_edges.restype = i32
    lib.plan_obstacle_planes.argtypes = [vp, i32, vp, ctypes.POINTER(_Obstacles), vp, vp, vp, vp, vp]
    lib.plan_obstacle_planes.restype = i32
    lib.plan_nearest_planes.argtypes = [vp, i32, vp, ctypes.POINTER(_Obstacles), vp, vp, vp]
    lib.plan_nearest_planes.restype = i32
    lib.plan_mpc_qp.argtypes = [vp, i32, ctypes.POINTER(_MpcParams), vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.plan_mpc_qp.restype = i32
    lib.plan_search_at.argtypes = [vp, i32, vp, ctypes.POINTER(_Edges), vp, vp, i32, vp, vp]
    lib.plan_search_to.argtypes = [vp, i32, vp, ctypes.POINTER(_Edges), vp, i32, vp, i32, vp, vp]
    lib.plan_search_to.restype = i32
    lib.plan_search_at.restype = i32
    lib.plan_cut_timing.argtypes = [vp, dp, dp, ctypes.POINTER(i64), i32]
    lib.plan_cut_timing.restype = i32
    lib.plan_set_tile.argtypes = [vp, i32, i32, i32, i32]
    lib.plan_set_tile.restype = i32
    lib.plan_autotune.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                  ctypes.POINTER(i32), dp]
    lib.plan_autotune.restype = i32
    lib.plan_refine.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32, ctypes.POINTER(_RefineW), vp, vp, vp, vp]
    lib.plan_refine.restype = i32
    lib.plan_set_accounting.argtypes = [vp, i32]
    lib.plan_set_accounting.restype = i32
    lib.plan_set_timing.argtypes = [vp, i32]
    lib.plan_set_timing.restype = i32
    lib.plan_timing.argtypes = [vp, dp, ctypes.POINTER(i64), dp, ctypes.POINTER(i64), ctypes.POINTER(i64), i32]
    lib.plan_timing.restype = i32
    lib.plan_measure_lane_rate.argtypes = [i32, i32, dp, dp]
    lib.plan_measure_lane_rate.restype = i32
    lib.plan_status_string.argtypes = [i32]
    lib.plan_status_string.restype = ctypes.c_char_p
    lib.plan_last_error.argtypes = [vp]
    lib.plan_last_error.restype = ctypes.c_char_p
    lib.plan_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def status_string(s: int) -> str:
    try:
        return load().plan_status_string(int(s)).decode()
    except Exception:
        return "?"


INTERIOR = {"elevate": 0, "minsnap": 1}


def _model(m, gamma, degree, bounds, arith="f64", input="f64", cost_mode="state", tighten=0.0,
           interior="elevate") -> _Model:
    b = (ctypes.c_double * 4)(*([float(x) for x in bounds] + [0.0] * (4 - len(bounds))))
    return _Model(int(m), int(gamma), int(degree), ARITH[arith], INPUT[input], COST[cost_mode], b, float(tighten),
                  INTERIOR[interior])


def model_tables(gamma: int, degree: int, T: Sequence[float], interior: str = "elevate"):
    """The library's FP64 coefficient tables (host only, no GPU): D, H, C."""
    lib = load()
    T = np.ascontiguousarray(np.asarray(T, dtype=np.float64))
    g, p, nT = int(gamma), int(degree), T.shape[0]
    rax = sum(p - k + 1 for k in range(1, g + 1))
    D = np.zeros((nT, p + 1, 2 * g))
    H = np.zeros((nT, rax, 2 * g))
    C = np.zeros((nT, g, p, 2 * g))
    mdl = _model(1, g, p, [1.0] * g, interior=interior)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = lib.plan_model_tables(ctypes.byref(mdl), nT, dp(T), dp(D), dp(H), dp(C))
    if rc != 0:
        raise PlanError(rc)
    return {"D": D, "H": H, "C": C}


def measure_lane_rate(mix: int = 0, iters: int = 1 << 16) -> dict:
    """Sustained lane operations per second on the current device (mix 0: FP32
    add + |.|-max, the reach/free row pattern; 1: FP32 fused multiply-add; 2, 3:
    the same in FP64)."""
    lib = load()
    r, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib.plan_measure_lane_rate(int(mix), int(iters), ctypes.byref(r), ctypes.byref(ms))
    if rc != 0:
        raise PlanError(rc, "plan_measure_lane_rate")
    return {"lane_ops_per_s": r.value, "ms": ms.value}


def search_noalloc(m: int, gamma: int, input: str, w_f64: bool, dp, graph, start_pos, goal_pos, out: dict,
                   stream=None) -> int:
    """plan_search_noalloc through the C ABI: a search that allocates no device
    memory (its scratch is a static device array of the library, N <= 65536).
    ``out`` holds device tensors path, path_len, cost and an int32 status.
    Returns the host status of the call; the device status lands in out["status"]."""
    import torch
    lib = load()
    sp = np.ascontiguousarray(np.asarray(start_pos, dtype=np.float64))
    gp = np.ascontiguousarray(np.asarray(goal_pos, dtype=np.float64))
    st = stream if stream is not None else torch.cuda.current_stream()
    dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return lib.plan_search_noalloc(int(m), int(gamma), INPUT[input], 1 if w_f64 else 0, int(dp.N),
                                   ctypes.c_void_p(dp.states.data_ptr()), ctypes.byref(graph.cstruct()), dptr(sp), dptr(gp),
                                   ctypes.c_void_p(out["path"].data_ptr()), int(out["path"].shape[0]),
                                   ctypes.c_void_p(out["path_len"].data_ptr()), ctypes.c_void_p(out["cost"].data_ptr()),
                                   ctypes.c_void_p(out["status"].data_ptr()), ctypes.c_void_p(st.cuda_stream))


@dataclass
class Graph:
    """Feasible-edge CSR on the device (torch tensors)."""
    N: int
    row_off: "torch.Tensor"
    col: "torch.Tensor"
    w: "torch.Tensor"
    tidx: "torch.Tensor"
    mask: "torch.Tensor"      # int32 storage of uint32 masks
    count: "torch.Tensor"
    cap: int

    def cstruct(self) -> _Edges:
        return _Edges(self.row_off.data_ptr(), self.col.data_ptr(), self.w.data_ptr(), self.tidx.data_ptr(),
                      self.mask.data_ptr(), int(self.cap), self.count.data_ptr())

    @property
    def E(self) -> int:
        return int(self.count.item())

    def to_numpy(self) -> dict:
        E = self.E
        return {"row_off": self.row_off.cpu().numpy().astype(np.int64), "col": self.col[:E].cpu().numpy(),
                "w": self.w[:E].cpu().numpy().astype(np.float64), "t": self.tidx[:E].cpu().numpy().astype(np.int32),
                "mask": self.mask[:E].cpu().numpy().view(np.uint32)}


@dataclass
class DeviceProblem:
    """Inputs of one query resident on the GPU."""
    N: int
    K: int
    max_rows: int
    states: "torch.Tensor"
    poly_off: "torch.Tensor"
    A: "torch.Tensor"
    b: "torch.Tensor"
    T: np.ndarray
    start_pos: np.ndarray
    goal_pos: np.ndarray


@dataclass
class DeviceObstacles:
    """Convex obstacles {z : A z <= b} resident on the GPU."""
    n: int
    max_rows: int
    off: "torch.Tensor"
    A: "torch.Tensor"
    b: "torch.Tensor"

    def cstruct(self) -> _Obstacles:
        return _Obstacles(int(self.n), self.off.data_ptr(), int(self.max_rows), self.A.data_ptr(), self.b.data_ptr())


def obstacles_to_device(obs, input: str = "f64", device=None) -> DeviceObstacles:
    """Upload generated obstacles (synth.Obstacles) to torch device tensors."""
    import torch
    dt = torch.float32 if input == "f32" else torch.float64
    dev = device or torch.device("cuda")
    off = np.asarray(obs.off, dtype=np.int32)
    n = off.shape[0] - 1
    max_rows = int(np.max(np.diff(off))) if n > 0 else 1
    return DeviceObstacles(n=n, max_rows=max(1, max_rows), off=torch.as_tensor(off).to(dev),
                           A=torch.as_tensor(np.ascontiguousarray(obs.A), dtype=dt).reshape(-1).to(dev).contiguous(),
                           b=torch.as_tensor(np.ascontiguousarray(obs.b), dtype=dt).to(dev).contiguous())


def to_device(prob, input: str = "f64", device=None) -> DeviceProblem:
    """Upload a generated problem (numpy arrays) to torch device tensors."""
    import torch
    dt = torch.float32 if input == "f32" else torch.float64
    dev = device or torch.device("cuda")
    off = np.asarray(prob.poly_off, dtype=np.int32)
    K = off.shape[0] - 1
    max_rows = int(np.max(np.diff(off))) if K > 0 else 1
    st = torch.as_tensor(np.ascontiguousarray(prob.states), dtype=dt).to(dev)
    return DeviceProblem(
        N=int(prob.states.shape[0]), K=K, max_rows=max(1, max_rows),
        states=st.contiguous(),
        poly_off=torch.as_tensor(off).to(dev),
        A=torch.as_tensor(np.ascontiguousarray(prob.A), dtype=dt).to(dev).contiguous(),
        b=torch.as_tensor(np.ascontiguousarray(prob.b), dtype=dt).to(dev).contiguous(),
        T=np.ascontiguousarray(np.asarray(prob.T, dtype=np.float64)),
        start_pos=np.asarray(prob.start_pos, dtype=np.float64), goal_pos=np.asarray(prob.goal_pos, dtype=np.float64))


class Planner:
    """One libplan context bound to a CUDA stream."""

    def __init__(self, m: int, gamma: int, degree: int, bounds: Sequence[float], arith: str = "f64",
                 input: str = "f64", cost_mode: str = "state", tighten: float = 0.0, stream=None,
                 interior: str = "elevate"):
        import torch
        self.lib = load()
        self.model = _model(m, gamma, degree, bounds, arith, input, cost_mode, tighten, interior)
        self.arith, self.input = arith, input
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ctypes.c_void_p()
        rc = self.lib.plan_create(ctypes.byref(ctx), ctypes.byref(self.model), ctypes.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise PlanError(rc, "plan_create")
        self.ctx = ctx
        self.last_info: Optional[_Info] = None

    @classmethod
    def for_problem(cls, prob, arith: str = None, input: str = None, **kw) -> "Planner":
        mdl = prob.model
        dt = getattr(prob, "dtype", "f64")
        return cls(mdl.m, mdl.gamma, mdl.degree, mdl.bounds, arith=arith or dt, input=input or dt,
                   cost_mode=mdl.cost_mode, tighten=mdl.tighten, interior=getattr(mdl, "interior", "elevate"), **kw)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.plan_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _err(self, rc, what):
        msg = self.lib.plan_last_error(self.ctx).decode() if self.ctx else ""
        return PlanError(rc, f"{what}: {msg}")

    def alloc_graph(self, N: int, cap: int) -> Graph:
        import torch
        dev = torch.device("cuda")
        wdt = torch.float64 if self.arith == "f64" else torch.float32
        cap = max(int(cap), 1)
        return Graph(N=N, row_off=torch.zeros(N + 1, dtype=torch.int32, device=dev),
                     col=torch.empty(cap, dtype=torch.int32, device=dev), w=torch.empty(cap, dtype=wdt, device=dev),
                     tidx=torch.empty(cap, dtype=torch.uint8, device=dev), mask=torch.empty(cap, dtype=torch.int32, device=dev),
                     count=torch.zeros(1, dtype=torch.int64, device=dev), cap=cap)

    def wait(self) -> int:
        info = _Info()
        rc = self.lib.plan_wait(self.ctx, ctypes.byref(info))
        self.last_info = info
        return rc

    def info(self) -> dict:
        i = self.last_info
        return {f: getattr(i, f) for f, _ in _Info._fields_} if i is not None else {}

    def build_edges_async(self, dp: DeviceProblem, graph: Graph) -> None:
        T = dp.T
        rc = self.lib.plan_build_edges(self.ctx, dp.N, ctypes.c_void_p(dp.states.data_ptr()), int(T.shape[0]),
                                       T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), dp.K,
                                       ctypes.c_void_p(dp.poly_off.data_ptr()), dp.max_rows,
                                       ctypes.c_void_p(dp.A.data_ptr()), ctypes.c_void_p(dp.b.data_ptr()),
                                       ctypes.byref(graph.cstruct()))
        if rc != 0:
            raise self._err(rc, "plan_build_edges")

    def build_edges_shard_async(self, dp: DeviceProblem, graph: Graph, shard: int, nshard: int) -> None:
        T = dp.T
        rc = self.lib.plan_build_edges_shard(self.ctx, dp.N, ctypes.c_void_p(dp.states.data_ptr()), int(T.shape[0]),
                                             T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), dp.K,
                                             ctypes.c_void_p(dp.poly_off.data_ptr()), dp.max_rows,
                                             ctypes.c_void_p(dp.A.data_ptr()), ctypes.c_void_p(dp.b.data_ptr()),
                                             int(shard), int(nshard), ctypes.byref(graph.cstruct()))
        if rc != 0:
            raise self._err(rc, "plan_build_edges_shard")

    def build_edges_shard(self, dp: DeviceProblem, shard: int, nshard: int, graph: Optional[Graph] = None,
                          cap: Optional[int] = None) -> Graph:
        """The rows of one shard of the graph (plan_build_edges_shard), growing scratch/output on CAPACITY."""
        return self.build_edges(dp, graph, cap, shard=(int(shard), int(nshard)))

    def build_edges(self, dp: DeviceProblem, graph: Optional[Graph] = None, cap: Optional[int] = None,
                    shard=None) -> Graph:
        """Build the feasible-edge graph, growing scratch/output and repeating on CAPACITY."""
        if graph is None:
            graph = self.alloc_graph(dp.N, cap if cap is not None else max(1024, 64 * dp.N))
        for _ in range(6):
            if shard is None:
                self.build_edges_async(dp, graph)
            else:
                self.build_edges_shard_async(dp, graph, *shard)
            st = self.wait()
            if st == PLAN_OK:
                return graph
            if st == PLAN_ERR_CAPACITY:
                det = self.last_info.detail
                if det == DET_OUTPUT:
                    graph = self.alloc_graph(dp.N, int(self.last_info.edges * 1.1) + 1024)
                continue
            raise self._err(st, "build_edges")
        raise self._err(PLAN_ERR_CAPACITY, "build_edges: capacity retries exhausted")

    def cut_edges_async(self, dp: DeviceProblem, graph: Graph, obst: DeviceObstacles, out: Graph) -> None:
        T = dp.T
        rc = self.lib.plan_cut_edges(self.ctx, dp.N, ctypes.c_void_p(dp.states.data_ptr()), int(T.shape[0]),
                                     T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(graph.cstruct()),
                                     ctypes.byref(obst.cstruct()), ctypes.byref(out.cstruct()))
        if rc != 0:
            raise self._err(rc, "plan_cut_edges")

    def cut_edges(self, dp: DeviceProblem, graph: Graph, obst: DeviceObstacles, out: Optional[Graph] = None) -> Graph:
        """Keep-out cut of a built graph: a new CSR without the (edge, T) whose
        curves may meet an obstacle (repeats once the game lists have grown)."""
        if out is None:
            out = self.alloc_graph(dp.N, max(1, graph.cap))
        for _ in range(6):
            self.cut_edges_async(dp, graph, obst, out)
            st = self.wait()
            if st == PLAN_OK:
                return out
            if st == PLAN_ERR_CAPACITY and self.last_info.detail == DET_CUTLIST:
                continue
            raise self._err(st, "cut_edges")
        raise self._err(PLAN_ERR_CAPACITY, "cut_edges: capacity retries exhausted")

    def search_async(self, dp: DeviceProblem, graph: Graph, start_pos, goal_pos, out: dict) -> None:
        sp = np.ascontiguousarray(np.asarray(start_pos, dtype=np.float64))
        gp = np.ascontiguousarray(np.asarray(goal_pos, dtype=np.float64))
        rc = self.lib.plan_search(self.ctx, dp.N, ctypes.c_void_p(dp.states.data_ptr()), ctypes.byref(graph.cstruct()),
                                  sp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  gp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.c_void_p(out["path"].data_ptr()), int(out["path"].shape[0]),
                                  ctypes.c_void_p(out["path_len"].data_ptr()), ctypes.c_void_p(out["cost"].data_ptr()))
        if rc != 0:
            raise self._err(rc, "plan_search")

    def obstacle_planes_async(self, points, obst: DeviceObstacles, out: dict) -> None:
        """plan_obstacle_planes into the device tensors of ``out`` (keys closest,
        plane, dist, nearest, nearest_dist; any may be None)."""
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)
        rc = self.lib.plan_obstacle_planes(self.ctx, int(points.shape[0]), ctypes.c_void_p(points.data_ptr()),
                                           ctypes.byref(obst.cstruct()), ptr(out.get("closest")), ptr(out.get("plane")),
                                           ptr(out.get("dist")), ptr(out.get("nearest")), ptr(out.get("nearest_dist")))
        if rc != 0:
            raise self._err(rc, "plan_obstacle_planes")

    def obstacle_planes(self, points, obst: DeviceObstacles, nearest_only: bool = False) -> dict:
        """Closest points, distances, separating planes (all pairs unless
        nearest_only) and the nearest obstacle of every point."""
        import torch
        P, n, m = int(points.shape[0]), int(obst.n), int(self.model.m)
        dev = points.device
        out = {"nearest": torch.empty(P, dtype=torch.int32, device=dev),
               "nearest_dist": torch.empty(P, dtype=torch.float32, device=dev)}
        if not nearest_only:
            out.update({"closest": torch.empty((P, n, m), dtype=torch.float32, device=dev),
                        "plane": torch.empty((P, n, m + 1), dtype=torch.float32, device=dev),
                        "dist": torch.empty((P, n), dtype=torch.float32, device=dev)})
        self.obstacle_planes_async(points, obst, out)
        st = self.wait()
        if st != PLAN_OK:
            raise self._err(st, "obstacle_planes")
        return out

    def nearest_planes_async(self, points, obst: DeviceObstacles, plane, nearest=None, nearest_dist=None) -> None:
        """plan_nearest_planes: per point the plane of its nearest obstacle
        into ``plane`` (float32 [P][m+1])."""
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)
        rc = self.lib.plan_nearest_planes(self.ctx, int(points.shape[0]), ctypes.c_void_p(points.data_ptr()),
                                          ctypes.byref(obst.cstruct()), ptr(plane), ptr(nearest), ptr(nearest_dist))
        if rc != 0:
            raise self._err(rc, "plan_nearest_planes")

    def mpc_params(self, horizon: int, dt: float, Q, F, R, V, keepin_A=None, keepin_b=None):
        """plan_mpc_params with the host arrays kept alive on the returned object."""
        n, m = int(self.model.m * self.model.gamma), int(self.model.m)
        arrs = {k: np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), (sz,)))
                for k, v, sz in (("Q", Q, n), ("F", F, n), ("R", R, m), ("V", V, n))}
        nk = 0
        if keepin_A is not None:
            arrs["KA"] = np.ascontiguousarray(np.asarray(keepin_A, dtype=np.float64).reshape(-1, m))
            arrs["Kb"] = np.ascontiguousarray(np.asarray(keepin_b, dtype=np.float64).reshape(-1))
            nk = int(arrs["KA"].shape[0])
        ptr = lambda a: a.ctypes.data if a is not None else None
        prm = _MpcParams(int(horizon), float(dt), ptr(arrs["Q"]), ptr(arrs["F"]), ptr(arrs["R"]), ptr(arrs["V"]), nk,
                         ptr(arrs.get("KA")), ptr(arrs.get("Kb")))
        prm._keep = arrs
        return prm

    def alloc_mpc(self, B: int, horizon: int) -> dict:
        import torch
        dev = torch.device("cuda")
        n, m = int(self.model.m * self.model.gamma), int(self.model.m)
        return {"x": torch.empty((B, horizon + 1, n), dtype=torch.float64, device=dev),
                "u": torch.empty((B, horizon, m), dtype=torch.float64, device=dev),
                "obj": torch.empty(B, dtype=torch.float64, device=dev),
                "status": torch.empty(B, dtype=torch.int32, device=dev),
                "iters": torch.empty(B, dtype=torch.int32, device=dev),
                "nodes": torch.empty((B, horizon, m), dtype=torch.float64, device=dev)}

    def mpc_qp_async(self, prm, x0, ref, planes, out: dict) -> None:
        """plan_mpc_qp on device tensors: x0 float64 [B][n], ref float64
        [B][H+1][n], planes float32 [B][H][m+1]; results into ``out``."""
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)
        rc = self.lib.plan_mpc_qp(self.ctx, int(x0.shape[0]), ctypes.byref(prm), ptr(x0), ptr(ref), ptr(planes),
                                  ptr(out["x"]), ptr(out["u"]), ptr(out["obj"]), ptr(out["status"]),
                                  ptr(out.get("iters")), ptr(out.get("nodes")))
        if rc != 0:
            raise self._err(rc, "plan_mpc_qp")

    def mpc_refine_async(self, prm, x0, ref, obst: DeviceObstacles, out: dict, sqp_iters: int = 3,
                         planes=None) -> None:
        """The SQP refinement of Sec. III-D: planes of the nearest obstacles at
        the nodes x_0 .. x_{H-1} of the current iterate (the reference first),
        then the QP; sqp_iters rounds.  ``planes`` (float32 [B][H][m+1]) is
        scratch, allocated when None."""
        import torch
        B, H, m = int(x0.shape[0]), int(prm.horizon), int(self.model.m)
        if planes is None:
            planes = torch.empty((B, H, m + 1), dtype=torch.float32, device=x0.device)
        if out.get("nodes") is None:
            out["nodes"] = torch.empty((B, H, m), dtype=torch.float64, device=x0.device)
        nodes = ref[:, :H, :m].contiguous()         # the reference's node positions (input marshalling)
        for _ in range(int(sqp_iters)):
            pts = nodes.float() if self.input == "f32" else nodes
            self.nearest_planes_async(pts.view(B * H, m), obst, planes.view(B * H, m + 1))
            self.mpc_qp_async(prm, x0, ref, planes, out)
            nodes = out["nodes"]                    # positions of the new nodes, written by the QP kernel

    def search_at_async(self, dp: DeviceProblem, graph: Graph, endpoints, out: dict) -> None:
        """plan_search_at: start and goal read from the device tensor
        ``endpoints`` (float64 [2][m]) when the search runs."""
        rc = self.lib.plan_search_at(self.ctx, dp.N, ctypes.c_void_p(dp.states.data_ptr()), ctypes.byref(graph.cstruct()),
                                     ctypes.c_void_p(endpoints.data_ptr()), ctypes.c_void_p(out["path"].data_ptr()),
                                     int(out["path"].shape[0]), ctypes.c_void_p(out["path_len"].data_ptr()),
                                     ctypes.c_void_p(out["cost"].data_ptr()))
        if rc != 0:
            raise self._err(rc, "plan_search_at")

    def search_to_async(self, dp: DeviceProblem, graph: Graph, endpoints, out: dict, warm: bool = True) -> None:
        """plan_search_to: distances to the goal vertex, warm-started from the
        previous call when the goal vertex is the same."""
        rc = self.lib.plan_search_to(self.ctx, dp.N, ctypes.c_void_p(dp.states.data_ptr()), ctypes.byref(graph.cstruct()),
                                     ctypes.c_void_p(endpoints.data_ptr()), 1 if warm else 0,
                                     ctypes.c_void_p(out["path"].data_ptr()), int(out["path"].shape[0]),
                                     ctypes.c_void_p(out["path_len"].data_ptr()), ctypes.c_void_p(out["cost"].data_ptr()))
        if rc != 0:
            raise self._err(rc, "plan_search_to")

    def alloc_search(self, N: int, path_cap: Optional[int] = None) -> dict:
        import torch
        dev = torch.device("cuda")
        return {"path": torch.empty(max(1, path_cap or N), dtype=torch.int32, device=dev),
                "path_len": torch.zeros(1, dtype=torch.int32, device=dev),
                "cost": torch.zeros(1, dtype=torch.float64, device=dev)}

    def search(self, dp: DeviceProblem, graph: Graph, start_pos=None, goal_pos=None) -> dict:
        out = self.alloc_search(dp.N)
        self.search_async(dp, graph, dp.start_pos if start_pos is None else start_pos,
                          dp.goal_pos if goal_pos is None else goal_pos, out)
        st = self.wait()
        info = self.last_info
        res = {"status": st, "start": int(info.start), "goal": int(info.goal), "iters": int(info.search_iters)}
        if st not in (PLAN_OK, PLAN_ERR_NO_PATH):
            raise self._err(st, "search")
        L = int(out["path_len"].item())
        res["path"] = out["path"][:L].cpu().numpy().tolist() if st == PLAN_OK else None
        res["cost"] = float(out["cost"].item())
        return res

    def set_search_limits(self, max_sweeps: int = 0, spin_limit: int = 0):
        rc = self.lib.plan_set_search_limits(self.ctx, int(max_sweeps), int(spin_limit))
        if rc != 0:
            raise self._err(rc, "plan_set_search_limits")

    # ---- batching form -------------------------------------------------
    def prepare_batched(self, dps, graphs) -> None:
        """Host work of a batch (tables, offsets, scratch, descriptor upload)."""
        qs = (_Query * len(dps))()
        self._batch_keep = []
        max_rows = 1
        for q, (dp, g) in enumerate(zip(dps, graphs)):
            T = np.ascontiguousarray(dp.T, dtype=np.float64)
            self._batch_keep.append(T)
            qs[q] = _Query(dp.N, dp.states.data_ptr(), int(T.shape[0]), T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           dp.K, dp.poly_off.data_ptr(), dp.A.data_ptr(), dp.b.data_ptr(), g.cstruct())
            max_rows = max(max_rows, dp.max_rows)
        rc = self.lib.plan_prepare_batched(self.ctx, len(dps), qs, max_rows)
        if rc != 0:
            raise self._err(rc, "plan_prepare_batched")

    def build_batched_async(self) -> None:
        rc = self.lib.plan_build_edges_batched(self.ctx)
        if rc != 0:
            raise self._err(rc, "plan_build_edges_batched")

    def build_batched(self, dps, graphs=None, cap_per_state: int = 64):
        """Edge graphs of many queries in one pass (grows scratch/outputs on CAPACITY)."""
        if graphs is None:
            graphs = [self.alloc_graph(dp.N, max(1024, cap_per_state * dp.N)) for dp in dps]
        for _ in range(8):
            self.prepare_batched(dps, graphs)
            self.build_batched_async()
            st = self.wait()
            if st == PLAN_OK:
                return graphs
            if st == PLAN_ERR_CAPACITY:
                if self.last_info.detail == DET_OUTPUT:
                    graphs = [g if g.E <= g.cap else self.alloc_graph(dp.N, int(g.E * 1.1) + 1024)
                              for dp, g in zip(dps, graphs)]
                continue
            raise self._err(st, "build_batched")
        raise self._err(PLAN_ERR_CAPACITY, "build_batched: capacity retries exhausted")

    def prepare_search_batched(self, dps, graphs, outs) -> None:
        qs = (_SearchQuery * len(dps))()
        for q, (dp, g, o) in enumerate(zip(dps, graphs, outs)):
            sp = (ctypes.c_double * 4)(*([float(x) for x in dp.start_pos] + [0.0] * (4 - len(dp.start_pos))))
            gp = (ctypes.c_double * 4)(*([float(x) for x in dp.goal_pos] + [0.0] * (4 - len(dp.goal_pos))))
            qs[q] = _SearchQuery(dp.N, dp.states.data_ptr(), g.cstruct(), sp, gp, o["path"].data_ptr(),
                                 int(o["path"].shape[0]), o["path_len"].data_ptr(), o["cost"].data_ptr(),
                                 o["status"].data_ptr())
        rc = self.lib.plan_prepare_search_batched(self.ctx, len(dps), qs)
        if rc != 0:
            raise self._err(rc, "plan_prepare_search_batched")

    def search_batched_async(self) -> None:
        rc = self.lib.plan_search_batched(self.ctx)
        if rc != 0:
            raise self._err(rc, "plan_search_batched")

    def alloc_search_batched(self, dps) -> list:
        import torch
        outs = []
        for dp in dps:
            o = self.alloc_search(dp.N)
            o["status"] = torch.zeros(1, dtype=torch.int32, device=o["path"].device)
            outs.append(o)
        return outs

    def search_batched(self, dps, graphs) -> list:
        outs = self.alloc_search_batched(dps)
        self.prepare_search_batched(dps, graphs, outs)
        self.search_batched_async()
        st = self.wait()
        if st != PLAN_OK:
            raise self._err(st, "search_batched")
        res = []
        for o in outs:
            s = int(o["status"].item())
            L = int(o["path_len"].item())
            res.append({"status": s, "path": o["path"][:L].cpu().numpy().tolist() if s == PLAN_OK else None,
                        "cost": float(o["cost"].item())})
        return res

    def set_tile(self, tile: int = 0, ctas_per_sm: int = 0, tchunks: int = 0, pipeline: int = 0) -> None:
        rc = self.lib.plan_set_tile(self.ctx, int(tile), int(ctas_per_sm), int(tchunks), int(pipeline))
        if rc != 0:
            raise self._err(rc, "plan_set_tile")

    def autotune(self, reps: int = 3) -> dict:
        """Time every (tile, CTAs/SM) candidate on the prepared batch; keep the best."""
        t, c, k, pp, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        rc = self.lib.plan_autotune(self.ctx, int(reps), ctypes.byref(t), ctypes.byref(c), ctypes.byref(k),
                                    ctypes.byref(pp), ctypes.byref(ms))
        if rc != 0:
            raise self._err(rc, "plan_autotune")
        return {"tile": t.value, "ctas_per_sm": c.value, "tchunks": k.value, "pipeline": pp.value, "pair_ms": ms.value}

    def refine_async(self, P, T, A, b, nrows, weights=(1.0, 1.0, 0.1), grad_loss=None, loss=None, dP=None, dT=None):
        """Launch the refinement loss (and, with grad_loss, its gradient) on device float tensors."""
        S = int(P.shape[0])
        w = _RefineW(*[float(x) for x in weights])
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        rc = self.lib.plan_refine(self.ctx, S, ptr(P), ptr(T), ptr(A), ptr(b), ptr(nrows), int(A.shape[1]),
                                  ctypes.byref(w), ptr(grad_loss), ptr(loss), ptr(dP), ptr(dT))
        if rc != 0:
            raise self._err(rc, "plan_refine")

    def set_accounting(self, on: bool):
        self.lib.plan_set_accounting(self.ctx, 1 if on else 0)

    def set_timing(self, on: bool):
        self.lib.plan_set_timing(self.ctx, 1 if on else 0)

    def timing(self, reset: bool = True) -> dict:
        pm, sm = ctypes.c_double(), ctypes.c_double()
        pl, sl, tl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rc = self.lib.plan_timing(self.ctx, ctypes.byref(pm), ctypes.byref(pl), ctypes.byref(sm), ctypes.byref(sl),
                                  ctypes.byref(tl), 1 if reset else 0)
        if rc != 0:
            raise self._err(rc, "plan_timing")
        return {"pair_ms": pm.value, "pair_launches": pl.value, "search_ms": sm.value,
                "search_launches": sl.value, "launches": tl.value}

    def cut_timing(self, reset: bool = True) -> dict:
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        rc = self.lib.plan_cut_timing(self.ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n), 1 if reset else 0)
        if rc != 0:
            raise self._err(rc, "plan_cut_timing")
        return {"scan_ms": a.value, "cut_ms": b.value, "cuts": n.value}


class Replanner:
    """The replanning loop of Algorithm 1 (cutGraph and findPath every tick, the
    graph of buildGraph fixed): each tick refreshes the obstacles and the start/goal positions on
    the device from pinned host buffers, cuts the fixed graph against the
    obstacles (plan_cut_edges), searches the cut graph and copies the path
    back -- all replayed from one captured CUDA graph.  The search is the
    goal-rooted plan_search_to warm-started from the previous tick (warm=True,
    the default) or plan_search_at (warm=False).

    The obstacle arrays have a fixed capacity (n_max obstacles, rows_max >= 2m
    rows each); a tick with fewer obstacles fills the other slots with unit
    boxes at -1e12 in every axis, which the certified bounding boxes separate
    from every curve.

    One tick is in flight at a time: the pinned staging buffers feed the
    tick's host-to-device copies, so a tick_async issued before the previous
    tick's result() first waits for that tick and drops its result (status
    and path); result() then reports the newer tick alone."""

    def __init__(self, planner: "Planner", dp: DeviceProblem, graph: Graph, n_max: int, rows_max: int,
                 path_cap: Optional[int] = None, warm: bool = True):
        import torch
        if planner.stream.cuda_stream == 0:
            raise ValueError("the planner needs its own stream (a graph cannot be captured on the default stream)")
        self.pl, self.dp, self.graph = planner, dp, graph
        self.warm = bool(warm)   # goal-rooted search warm-started from the previous tick (else plan_search_at)
        self.m = int(planner.model.m)
        self.n_max, self.rows_max = int(n_max), int(rows_max)
        if self.rows_max < 2 * self.m:
            raise ValueError("rows_max must be at least 2m (the padding boxes)")
        dev = torch.device("cuda")
        R = self.n_max * self.rows_max
        adt = torch.float32 if planner.input == "f32" else torch.float64
        self.h_off = torch.zeros(self.n_max + 1, dtype=torch.int32).pin_memory()
        self.h_A = torch.zeros(R * self.m, dtype=adt).pin_memory()
        self.h_b = torch.zeros(R, dtype=adt).pin_memory()
        self.h_ends = torch.zeros(2 * self.m, dtype=torch.float64).pin_memory()
        self.obst = DeviceObstacles(n=self.n_max, max_rows=self.rows_max,
                                    off=torch.zeros(self.n_max + 1, dtype=torch.int32, device=dev),
                                    A=torch.zeros(R * self.m, dtype=adt, device=dev),
                                    b=torch.zeros(R, dtype=adt, device=dev))
        self.ends = torch.zeros(2 * self.m, dtype=torch.float64, device=dev)
        self.out = planner.alloc_graph(dp.N, graph.cap)
        self.sbuf = planner.alloc_search(dp.N, path_cap)
        self.h_path = torch.zeros(self.sbuf["path"].shape[0], dtype=torch.int32).pin_memory()
        self.h_len = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.h_cost = torch.zeros(1, dtype=torch.float64).pin_memory()
        self.cg = None
        self._inflight = False

    def _stage(self, obstacles, start_pos, goal_pos) -> None:
        if self._inflight:           # the previous tick's copies still read the staging buffers
            self.pl.wait()           # ... and its device status must not mix with the next tick's
            self._inflight = False
        off = np.asarray(obstacles.off, dtype=np.int64)
        n = off.shape[0] - 1
        if n > self.n_max or (n > 0 and int(np.max(np.diff(off))) > self.rows_max):
            raise ValueError("obstacles exceed the replanner's capacity")
        A = np.asarray(obstacles.A, dtype=np.float64).reshape(-1, self.m)
        b = np.asarray(obstacles.b, dtype=np.float64)
        # far unit boxes in the unused slots: -1e12 <= z_a <= -1e12 + 1
        pad = self.n_max - n
        eye = np.concatenate([np.eye(self.m), -np.eye(self.m)])
        bb = np.concatenate([np.full(self.m, -1e12 + 1.0), np.full(self.m, 1e12)])
        A_all = np.concatenate([A, np.tile(eye, (pad, 1))]) if pad else A
        b_all = np.concatenate([b, np.tile(bb, pad)]) if pad else b
        off_all = np.concatenate([off, off[-1] + 2 * self.m * np.arange(1, pad + 1)]) if pad else off
        R = b_all.shape[0]
        self.h_off.numpy()[:] = 0
        self.h_off.numpy()[:off_all.shape[0]] = off_all.astype(np.int32)
        self.h_A.numpy()[:R * self.m] = A_all.reshape(-1)
        self.h_b.numpy()[:R] = b_all
        self.h_ends.numpy()[:self.m] = np.asarray(start_pos, dtype=np.float64)[:self.m]
        self.h_ends.numpy()[self.m:] = np.asarray(goal_pos, dtype=np.float64)[:self.m]

    def _issue(self) -> None:
        o = self.obst
        o.off.copy_(self.h_off, non_blocking=True)
        o.A.copy_(self.h_A, non_blocking=True)
        o.b.copy_(self.h_b, non_blocking=True)
        self.ends.copy_(self.h_ends, non_blocking=True)
        self.pl.cut_edges_async(self.dp, self.graph, o, self.out)
        if self.warm:
            self.pl.search_to_async(self.dp, self.out, self.ends, self.sbuf, warm=True)
        else:
            self.pl.search_at_async(self.dp, self.out, self.ends, self.sbuf)
        self.h_path.copy_(self.sbuf["path"], non_blocking=True)
        self.h_len.copy_(self.sbuf["path_len"], non_blocking=True)
        self.h_cost.copy_(self.sbuf["cost"], non_blocking=True)

    def capture(self, obstacles, start_pos, goal_pos) -> None:
        """Size every scratch with one direct tick, then capture the tick."""
        import torch
        self._stage(obstacles, start_pos, goal_pos)
        with torch.cuda.stream(self.pl.stream):
            for _ in range(3):      # grow the cut's pair list if it must
                self._issue()
                st = self.pl.wait()
                if st != PLAN_ERR_CAPACITY:
                    break
            self.cg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.cg, stream=self.pl.stream):
                self._issue()
        self.pl.wait()

    def tick_async(self, obstacles, start_pos, goal_pos) -> None:
        import torch
        self._stage(obstacles, start_pos, goal_pos)
        with torch.cuda.stream(self.pl.stream):
            self.cg.replay()
        self._inflight = True

    def result(self) -> dict:
        """Waits for the tick; status, path (host list) and cost."""
        st = self.pl.wait()
        self._inflight = False
        L = int(self.h_len.item())
        return {"status": st, "path": self.h_path[:L].tolist() if st == PLAN_OK else None,
                "cost": float(self.h_cost.item()), "edges": int(self.out.count.item()), "info": self.pl.info()}

    def tick(self, obstacles, start_pos, goal_pos) -> dict:
        self.tick_async(obstacles, start_pos, goal_pos)
        r = self.result()
        if r["status"] == PLAN_ERR_CAPACITY and r["info"].get("detail") == DET_CUTLIST:
            # the pair list has grown at plan_wait: capture again and repeat
            self.capture(obstacles, start_pos, goal_pos)
            self.tick_async(obstacles, start_pos, goal_pos)
            r = self.result()
        return r
