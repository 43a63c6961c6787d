"""Host-side checks of libplan that need no GPU: the shared library loads and
exports every entry point declared in include/plan.h, and the library's FP64
coefficient tables (its own route: Hermite recurrences, elevation and
hodograph differences, correctly rounded) equal the oracle's exact-rational
tables bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2411_13507_gb300 import plan as P
from oracle import tables as OT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "plan.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(plan_[a-z_]+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for req in ("plan_create", "plan_build_edges", "plan_cut_edges", "plan_search", "plan_wait", "plan_destroy",
                "plan_search_at", "plan_search_to", "plan_obstacle_planes", "plan_nearest_planes", "plan_mpc_qp"):
        assert req in names


def test_library_exports_every_declared_symbol():
    lib = P.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert b"sm_103a" in lib.plan_version()


@pytest.mark.parametrize("gamma,p,interior", [(2, 3, "elevate"), (2, 5, "elevate"), (3, 5, "elevate"),
                                               (3, 7, "elevate"), (1, 3, "elevate"), (4, 9, "elevate"),
                                               (2, 5, "minsnap"), (3, 7, "minsnap"), (1, 3, "minsnap"),
                                               (2, 7, "minsnap"), (3, 9, "minsnap")])
def test_tables_bitwise_equal_to_oracle(gamma, p, interior):
    rng = np.random.default_rng(gamma * 31 + p)
    Ts = np.concatenate([[0.1, 0.2, 0.5, 1.0, 2.0, 3.0, 1e-3, 37.5], np.exp(rng.uniform(np.log(0.05), np.log(5.0), 24))])
    Ts = np.concatenate([Ts, Ts.astype(np.float32).astype(np.float64)])
    lib = P.model_tables(gamma, p, Ts, interior=interior)
    orc = OT.tables(gamma, p, Ts, interior)
    for key in ("D", "H", "C"):
        a, b = lib[key], orc[key]
        assert a.shape == b.shape, key
        diff = np.nonzero(a.view(np.uint64) != b.view(np.uint64))
        assert diff[0].size == 0, (key, [(a[d], b[d]) for d in zip(*diff)][:5])


def test_model_tables_rejects_bad_input():
    lib = P.load()
    mdl = P._model(1, 2, 5, [1.0, 1.0])
    z = np.zeros(64)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    T = np.array([-1.0])
    assert lib.plan_model_tables(ctypes.byref(mdl), 1, dp(T), dp(z), dp(z), dp(z)) == P.PLAN_ERR_INVALID_ARG
    T = np.array([np.nan])
    assert lib.plan_model_tables(ctypes.byref(mdl), 1, dp(T), dp(z), dp(z), dp(z)) == P.PLAN_ERR_INVALID_ARG
    bad = P._model(1, 3, 4, [1.0] * 3)   # degree below 2*gamma-1
    T = np.array([1.0])
    assert lib.plan_model_tables(ctypes.byref(bad), 1, dp(T), dp(z), dp(z), dp(z)) == P.PLAN_ERR_INVALID_ARG
    big = P._model(1, 2, 11, [1.0] * 2, interior="minsnap")   # beyond the exact minimum-energy solve
    zz = np.zeros(4096)
    assert lib.plan_model_tables(ctypes.byref(big), 1, dp(T), dp(zz), dp(zz), dp(zz)) == P.PLAN_ERR_INVALID_ARG
    odd = P._model(1, 2, 5, [1.0] * 2)
    odd.interior = 7
    assert lib.plan_model_tables(ctypes.byref(odd), 1, dp(T), dp(zz), dp(zz), dp(zz)) == P.PLAN_ERR_INVALID_ARG


def test_status_strings():
    assert P.status_string(0) == "ok"
    assert "capacity" in P.status_string(3)
