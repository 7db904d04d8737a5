"""Autotuner of the batched form: picks traversal launch parameters by timing
short batched runs on a sample of the workload.

Searched: shared-memory stack depth (8, 16, 32 entries per ray), the refill
threshold of the while-while traversal (a warp takes new rays when fewer than
this many lanes are busy), threads per block and blocks per SM.  The sample
is a few items of the smallest and the largest mesh of the batch; each
candidate is timed twice through rtmc_run_batch and the faster time counts.
The library's own defaults (DEFAULTS) are timed first and kept unless another
candidate is faster by more than MARGIN, so timing noise on a small sample
does not move a run off the defaults for nothing.  Results are cached in a
JSON file keyed by device name, node format and mesh sizes.
"""
from __future__ import annotations

import itertools
import json
import os

from . import rtmc

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rtmc_autotune.json")

# what the library uses when the descriptor leaves the fields at 0
DEFAULTS = {"stack_depth": 16, "fetch_threshold": 28, "block_threads": 64, "blocks_per_sm": 0}
MARGIN = 0.02

SPACE = {
    "stack_depth": (8, 16, 32),
    "fetch_threshold": (12, 20, 28),
    "block_threads": (64, 128),
    "blocks_per_sm": (0, 12),
}


def _key(ctx_name, kinds, n_tris):
    return f"{ctx_name}|{'/'.join(map(str, kinds))}|{min(n_tris)}-{max(n_tris)}"


def tune(ctx: rtmc.Context, mesh_ids, n_tris, energies, thetas, kind=0, seed=1806, n_sample=150_000,
         cache_path: str | None = DEFAULT_CACHE, device_name: str = "gpu", space=None, fp64_retest=False):
    """Return the best run_desc keyword arguments for this batch shape."""
    space = space or SPACE
    key = _key(device_name, [kind], n_tris)
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
            if key in cache:
                return cache[key]["params"]
        except (OSError, ValueError):
            pass
    order = sorted(range(len(mesh_ids)), key=lambda i: n_tris[i])
    sample_ids = [mesh_ids[order[0]], mesh_ids[order[-1]]]
    sample_e = [energies[0], energies[len(energies) // 2], energies[-1]]
    sample_t = [thetas[0], thetas[-1]]
    names = list(space)

    def timed(params):
        desc = rtmc.run_desc(fp64_retest=fp64_retest, **params)
        ms = float("inf")
        for _ in range(2):
            res, _, _ = ctx.run_batch(sample_ids, sample_e, sample_t, n_sample, seed, desc=desc)
            ms = min(ms, res[0]["gpu_ms"])
        return ms

    default_ms = timed(DEFAULTS)
    best, best_ms, trials = dict(DEFAULTS), default_ms, [(default_ms, dict(DEFAULTS))]
    for values in itertools.product(*(space[k] for k in names)):
        params = dict(zip(names, values))
        if params == DEFAULTS:
            continue
        if params["blocks_per_sm"] and params["blocks_per_sm"] * params["block_threads"] > 2048:
            continue
        ms = timed(params)
        trials.append((ms, params))
        if ms < best_ms:
            best, best_ms = params, ms
    if best_ms > default_ms * (1.0 - MARGIN):
        best, best_ms = dict(DEFAULTS), default_ms
    if cache_path:
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            cache = {}
            if os.path.exists(cache_path):
                cache = json.load(open(cache_path))
            cache[key] = {"params": best, "ms": best_ms, "trials": len(trials)}
            json.dump(cache, open(cache_path, "w"), indent=1)
        except (OSError, ValueError):
            pass
    return best
