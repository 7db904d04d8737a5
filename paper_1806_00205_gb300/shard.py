"""Replica sharding of primaries across ranks and the merge of their results.

Primaries are independent (the paper's Section 2.2, last paragraph, and
Section 4: replicas need no communication), so N ranks run disjoint primary-id
ranges of the same work (``primary_offset``) and only the final tallies are
combined.  Integer tallies add exactly; energy moments are summed in rank
order so the merged result does not depend on timing; SEY and its standard
error are recomputed from the merged sums.
"""
from __future__ import annotations

import math

INT_KEYS = ("n_primaries", "rays", "escaped", "absorbed_low", "absorbed_other", "emitters", "emitted",
            "regenerated", "capped", "lost", "wraps", "sum_k", "sum_k2")
FLOAT_KEYS = ("e_sum", "e2_sum")


def primary_offset(rank: int, n_per_rank: int, base: int = 0) -> int:
    """First primary id of `rank` when every rank runs `n_per_rank` primaries."""
    return base + rank * n_per_rank


def merge_results(parts):
    """Combine per-rank result dicts (same item) in the given order."""
    out = {k: sum(int(p[k]) for p in parts) for k in INT_KEYS}
    for k in FLOAT_KEYS:
        acc = 0.0
        for p in parts:
            acc += float(p[k])
        out[k] = acc
    n = out["n_primaries"]
    out["sey"] = out["sum_k"] / n if n else 0.0
    if n > 1:
        var = (out["sum_k2"] / n - out["sey"] ** 2) / (n - 1)
        out["sey_se"] = math.sqrt(var) if var > 0 else 0.0
    else:
        out["sey_se"] = 0.0
    for h in ("hist_e", "hist_a", "hist_z"):
        if all(h in p for p in parts):
            acc = None
            for p in parts:
                acc = list(p[h]) if acc is None else [a + int(b) for a, b in zip(acc, p[h])]
            out[h] = acc
    return out


def gather_merge(result, group=None):
    """Gather every rank's result dict to rank 0 and merge them in rank order.

    Returns the merged dict on rank 0 and None elsewhere (torch.distributed,
    any backend; one object collective at the end of the run)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    parts = [None] * world if rank == 0 else None
    plain = {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in result.items() if k != "records"}
    dist.gather_object(plain, parts, dst=0, group=group)
    return merge_results(parts) if rank == 0 else None


def reduce_timing(ms, counts, device=None, group=None):
    """Whole-job timing of a sharded step: the slowest rank's time and the summed counts.

    Every rank passes its own elapsed time `ms` and its counts (rays, primaries, ...); all
    ranks get back (max ms over ranks, [sum of each count over ranks]).  One all-reduce of
    each kind, on `device` (the rank's GPU under NCCL, the CPU under gloo).  Without an
    initialised process group the inputs come back unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(ms), [float(c) for c in counts]
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    return t.item(), c.tolist()
