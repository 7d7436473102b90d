"""Launch-shape autotuning for the cooperative PCG, cached in JSON.

The library times every shape (threads per BSR row x blocks per SM) on the
first linear system of the next step (sim_tuning with autotune_next_step) and
keeps the fastest.  This module remembers the choice per (kernel, GPU,
precision, size bucket) in a JSON file so later runs reuse it.
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_CACHE = os.environ.get(
    "IPCSIM_TUNING_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json"))


def _key(sim, precision):
    try:
        import torch
        gpu = torch.cuda.get_device_name()
    except Exception:
        gpu = "unknown"
    bucket = 1 << max(0, math.ceil(math.log2(max(sim.n_nodes, 1))))
    return f"k_pcg|{gpu}|{'mixed' if precision else 'fp64'}|nodes<={bucket}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def prepare(sim, precision=0, cache_path=DEFAULT_CACHE):
    """Apply a cached shape, or arrange for the next step to autotune.  Returns True on a cache hit."""
    entry = _load(cache_path).get(_key(sim, precision))
    if entry:
        sim.tuning(rowg=entry["rowg"], blocks_per_sm=entry["blocks_per_sm"])
        return True
    sim.tuning(autotune_next_step=True)
    return False


def record(sim, precision=0, cache_path=DEFAULT_CACHE):
    """Store the shape the last autotuning chose; returns it."""
    (rowg, bps), ms = sim.tuning()
    cache = _load(cache_path)
    cache[_key(sim, precision)] = {"rowg": rowg, "blocks_per_sm": bps, "ms": [round(m, 4) for m in ms]}
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return {"rowg": rowg, "blocks_per_sm": bps}
