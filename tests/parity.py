"""Comparison of a GPU edge graph / search result against the oracle.

Bar (written here, used by every parity test):
  * feasibility masks, edge sets (row offsets, end vertices): bit-exact;
  * edge weights: within 1e-9 relative (FP64 arithmetic) or 1e-5 relative
    (FP32 arithmetic) of the oracle's FP64 value;
  * best-duration index: equal wherever the oracle's best cost is untied, i.e.
    every other feasible duration costs more than (1 + 2 tol) times it;
  * start/goal vertex ids: exact;
  * path node ids: exact, unless the GPU path re-costed with the oracle's own
    weights is within tol of the oracle optimum (a declared tie, reported).
"""
from __future__ import annotations

import numpy as np

# the precision form keeps the cost rows in FP32, so it meets the FP32 bar
TOL = {"f64": 1e-9, "f32": 1e-5, "tf32": 1e-5, "bf16": 1e-5}
PATH_TOL = {"f64": 1e-12, "f32": 1e-5, "tf32": 1e-5, "bf16": 1e-5}


def compare_rows(gpu: dict, orc_edges: dict, rows, nT: int, arith: str) -> dict:
    """gpu: numpy CSR (row_off, col, w, t, mask); orc_edges: oracle.edges(rows) output."""
    tol = TOL[arith]
    stats = {"edges": 0, "tidx_checked": 0, "tidx_tied": 0, "max_rel_w": 0.0}
    keep = orc_edges["mask"] != 0
    oi, oj = orc_edges["i"][keep], orc_edges["j"][keep]
    om, ow, ot = orc_edges["mask"][keep], orc_edges["w"][keep], orc_edges["t"][keep]
    oc = orc_edges["costs"][keep] if "costs" in orc_edges else None
    ro = gpu["row_off"]
    order = np.argsort(oi, kind="stable")       # oracle rows are grouped; keep j order
    oi, oj, om, ow, ot = oi[order], oj[order], om[order], ow[order], ot[order]
    if oc is not None:
        oc = oc[order]
    for i in rows:
        lo_, hi_ = np.searchsorted(oi, i, "left"), np.searchsorted(oi, i, "right")
        sel = slice(lo_, hi_)
        a, b = int(ro[i]), int(ro[i + 1])
        gj = gpu["col"][a:b]
        assert np.array_equal(gj, oj[sel]), f"row {i}: edge set differs ({len(gj)} vs {hi_ - lo_})"
        gm = gpu["mask"][a:b]
        bad = np.nonzero(gm != om[sel])[0]
        assert bad.size == 0, f"row {i}: mask differs at j={gj[bad[:5]]}: gpu {gm[bad[:5]]} oracle {om[sel][bad[:5]]}"
        gw = gpu["w"][a:b].astype(np.float64)
        rel = np.abs(gw - ow[sel]) / np.maximum(np.abs(ow[sel]), 1e-300)
        if rel.size:
            stats["max_rel_w"] = max(stats["max_rel_w"], float(rel.max()))
        assert np.all(rel <= tol), f"row {i}: weight rel err {rel.max():.3e} > {tol}"
        stats["edges"] += hi_ - lo_
        if oc is not None and hi_ > lo_:
            gt = gpu["t"][a:b]
            costs = oc[sel]                                   # [e][nT]
            mk = om[sel].astype(np.int64)
            bits = ((mk[:, None] >> np.arange(nT)[None, :]) & 1).astype(bool)
            best = ot[sel]
            bc = costs[np.arange(costs.shape[0]), best]
            others = np.where(bits, costs, np.inf)
            others[np.arange(costs.shape[0]), best] = np.inf
            untied = np.all(others > (bc * (1 + 2 * tol))[:, None], axis=1)
            stats["tidx_checked"] += int(untied.sum())
            stats["tidx_tied"] += int((~untied).sum())
            bad = np.nonzero(untied & (gt != best))[0]
            assert bad.size == 0, f"row {i}: tidx differs at j={gj[bad[:5]]}: {gt[bad[:5]]} vs {best[bad[:5]]}"
    return stats


def compare_full(gpu: dict, orc_csr: dict, N: int, nT: int, arith: str) -> dict:
    assert np.array_equal(gpu["row_off"], orc_csr["row_off"]), "row offsets differ"
    e = orc_csr["all"] if "all" in orc_csr else None
    if e is None:
        raise ValueError("oracle csr needs with_detail=True")
    return compare_rows(gpu, e, range(N), nT, arith)


def path_cost(path, csr: dict) -> float:
    """Cost of a vertex path under the given CSR's weights (FP64 left-to-right)."""
    c = 0.0
    for u, v in zip(path[:-1], path[1:]):
        a, b = int(csr["row_off"][u]), int(csr["row_off"][u + 1])
        js = csr["col"][a:b]
        k = np.searchsorted(js, v)
        assert k < len(js) and js[k] == v, f"edge {u}->{v} not in the oracle graph"
        c = c + float(csr["w"][a + k])
    return c


def compare_search(gpu: dict, orc: dict, orc_csr: dict, arith: str) -> str:
    assert gpu["start"] == orc["start"] and gpu["goal"] == orc["goal"], (gpu["start"], gpu["goal"], orc["start"], orc["goal"])
    if orc["path"] is None:
        assert gpu["path"] is None
        return "no-path"
    assert gpu["path"] is not None, "GPU found no path"
    tol = PATH_TOL[arith]
    assert abs(gpu["cost"] - orc["cost"]) <= TOL[arith] * max(1.0, orc["cost"]), (gpu["cost"], orc["cost"])
    if list(gpu["path"]) == list(orc["path"]):
        return "equal"
    c = path_cost(gpu["path"], orc_csr)
    assert c <= orc["cost"] * (1 + tol) + 1e-300, f"path differs and is not a tie: {c} vs {orc['cost']}"
    return "tie"
