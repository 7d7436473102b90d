"""Launch-shape autotuning for the cooperative PCG, cached in JSON.

Two ways to choose a shape (threads per BSR row x blocks per SM):
- in the library: every shape timed on the first linear system of the next
  step (sim_tuning with autotune_next_step), the fastest kept;
- over whole steps (tune_on_steps): every shape timed on a set of
  representative steps replayed from saved states, the smallest total kept.
  A shape changes the PCG iteration count as well as the time per iteration
  (the coarse aggregates are runs of CTAs), and the first system of a
  trajectory (often without contact) can favour another shape than the
  contact-rich steps that dominate it.
This module remembers the choice per (kernel, GPU, precision, size bucket) in
a JSON file so later runs reuse it.
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


def cached(sim, precision=0, cache_path=DEFAULT_CACHE):
    """Apply the cached shape if there is one; returns True on a hit."""
    entry = _load(cache_path).get(_key(sim, precision))
    if entry:
        sim.tuning(rowg=entry["rowg"], blocks_per_sm=entry["blocks_per_sm"])
        return True
    return False


ROW_GROUPS = (1, 2, 4, 8)
BLOCKS_PER_SM = (1, 2)


def tune_on_steps(sim, run_step, n):
    """Time every launch shape over the steps run_step(0), ..., run_step(n - 1) (each restores a saved
    state and runs one step, returning its device time in ms) and keep the shape with the smallest total.
    A shape with no co-resident launch is skipped (time -1).  Returns ((rowg, blocks_per_sm), times in
    ms indexed like the library's: 4 * (blocks_per_sm - 1) + index of rowg)."""
    from paper_2609_25653_b300.ipcsim import IpcError
    ms = [-1.0] * 8
    best, best_shape = None, sim.tuning()[0]
    for bi, bps in enumerate(BLOCKS_PER_SM):
        for ri, rowg in enumerate(ROW_GROUPS):
            sim.tuning(rowg=rowg, blocks_per_sm=bps)
            try:
                total = sum(run_step(j) for j in range(n))
            except IpcError:
                continue
            ms[4 * bi + ri] = total
            if best is None or total < best:
                best, best_shape = total, (rowg, bps)
    sim.tuning(rowg=best_shape[0], blocks_per_sm=best_shape[1])
    return best_shape, ms


def record(sim, precision=0, cache_path=DEFAULT_CACHE, ms=None):
    """Store the shape in use (after an autotuning) with the times it was chosen from; returns it."""
    (rowg, bps), lib_ms = sim.tuning()
    ms = lib_ms if ms is None else ms
    cache = _load(cache_path)
    cache[_key(sim, precision)] = {"rowg": rowg, "blocks_per_sm": bps, "ms": [round(m, 4) for m in ms]}
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return {"rowg": rowg, "blocks_per_sm": bps}
