"""Tile autotuner with an on-disk cache.

The choice (tile side, CTAs per SM) of the pair kernel is made by timing every
candidate on the prepared batch (plan_autotune, in the library) and cached in
a JSON file keyed by (m, gamma, p, arithmetic, SM count, workload class); a
later process with the same key reuses it without timing.
"""
from __future__ import annotations

import json
import os

from . import plan as _plan

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")


def key(planner: "_plan.Planner", workload: str) -> str:
    import torch
    m = planner.model
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return f"m{m.m}-g{m.gamma}-p{m.degree}-{planner.arith}-sm{sms}-{workload}"


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def tune(planner: "_plan.Planner", workload: str, reps: int = 3, path: str = CACHE, force: bool = False) -> dict:
    """Apply the cached choice for this key, or time the candidates and cache the winner.
    The planner must have a prepared batch (prepare_batched / build_batched)."""
    k = key(planner, workload)
    cache = load_cache(path)
    if not force and k in cache:
        c = cache[k]
        planner.set_tile(c["tile"], c["ctas_per_sm"], c.get("tchunks", 0), c.get("pipeline", 0))
        return dict(c, cached=True)
    res = planner.autotune(reps)
    cache[k] = res
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return dict(res, cached=False)
