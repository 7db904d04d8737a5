"""Helpers for comparing CUDA-path records with oracle records (test-only)."""
import numpy as np

M64 = (1 << 64) - 1
_C1, _C2, _C3 = np.uint64(0x9E3779B97F4A7C15), np.uint64(0xBF58476D1CE4E5B9), np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """splitmix64 finaliser on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + _C1
        z = (z ^ (z >> np.uint64(30))) * _C2
        z = (z ^ (z >> np.uint64(27))) * _C3
        return z ^ (z >> np.uint64(31))


def record_hashes(rec):
    """Per-record hash as documented for rtmc_record_hash (include/rtmc.h)."""
    u32 = lambda a: a.astype(np.int64).astype(np.uint64) & np.uint64(0xFFFFFFFF)
    h = splitmix64(rec["prim"].astype(np.uint64))
    h = splitmix64(h ^ (u32(rec["path"]) | (u32(rec["fate"]) << np.uint64(32))))
    h = splitmix64(h ^ (u32(rec["tri"]) | (u32(rec["k"]) << np.uint64(32))))
    h = splitmix64(h ^ (u32(rec["e_bin"]) | (u32(rec["a_bin"]) << np.uint64(32))))
    h = splitmix64(h ^ u32(rec["wraps"]))
    return h


def primary_hashes(rec, prim_ids):
    """Sum (mod 2^64) of record hashes per primary, in the order of prim_ids."""
    h = record_hashes(rec)
    order = {int(p): i for i, p in enumerate(prim_ids)}
    out = np.zeros(len(prim_ids), dtype=np.uint64)
    idx = np.array([order[int(p)] for p in rec["prim"]], dtype=np.int64)
    with np.errstate(over="ignore"):
        np.add.at(out, idx, h)
    return out


INT_FIELDS = ("gen", "fate", "tri", "k", "e_bin", "a_bin", "wraps")


def compare_records(gpu, orc, length_scale=10.0):
    """Match rays by (prim, path).  Returns a dict of match statistics.

    Hit distances are compared as |t_gpu - t_oracle| / max(t_oracle, length_scale):
    FP32 ray origins carry an absolute error of about one ulp of the cell
    coordinates (~1e-5 nm at 100 nm), so for segments much shorter than the
    mesh resolution (the voxel edge, 10 nm) a plain relative error measures
    that rounding, not the intersection."""
    kg = gpu["prim"].astype(np.uint64) * np.uint64(1 << 32) + gpu["path"].astype(np.uint64)
    ko = orc["prim"].astype(np.uint64) * np.uint64(1 << 32) + orc["path"].astype(np.uint64)
    assert np.unique(kg).size == kg.size, "duplicate GPU ray ids"
    assert np.unique(ko).size == ko.size, "duplicate oracle ray ids"
    common, ig, io = np.intersect1d(kg, ko, return_indices=True)
    g, o = gpu[ig], orc[io]
    same = np.ones(common.size, dtype=bool)
    for f in INT_FIELDS:
        same &= g[f] == o[f]
    # hit distance parity on rays whose events agree and that end on a facet
    hit = same & (o["tri"] >= 0)
    rel = np.abs(g["t"][hit] - o["t"][hit]) / np.maximum(np.abs(o["t"][hit]), length_scale)
    return dict(n_oracle=int(ko.size), n_gpu=int(kg.size), n_common=int(common.size),
                n_same=int(same.sum()), frac_same=float(same.sum()) / max(1, ko.size),
                t_rel_max=float(rel.max()) if rel.size else 0.0,
                t_rel_p9999=float(np.quantile(rel, 0.9999)) if rel.size else 0.0,
                t_rel_p999=float(np.quantile(rel, 0.999)) if rel.size else 0.0,
                mismatch=(g[~same], o[~same]))
