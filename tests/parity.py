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


U32 = 2.0 ** -24           # unit roundoff of FP32
# Daughter energies: the FP32 inverse of the spectrum CDF (or the FP32 Eq. 7 at an
# FP32 incidence angle) against FP64.  Relative error a few roundings, plus an
# absolute part: E = phi (1/s - 1) cancels near E = 0, and Eq. 7's alpha sin(E)
# carries the rounding of E itself (E u of argument) and of the angle near
# normal incidence.
E_REL = 1e-5
E_ABS = 1e-4               # eV
T_REL = 1e-5               # FP32 intersection of one ray against FP64 (the stated hit-distance tolerance)
K_SETUP = 16.0             # FP32 roundings per ray set-up step (see t_error_bound)


def facet_condition(mesh):
    """|e1| |e2| / |e1 x e2| per facet (FP64): how much a rounding of the edge
    vectors turns the FP32 unit normal, relative to the unit roundoff."""
    t = mesh.tri.astype(np.float64)
    e1, e2 = t[:, 1] - t[:, 0], t[:, 2] - t[:, 0]
    cr = np.linalg.norm(np.cross(e1, e2), axis=1)
    with np.errstate(divide="ignore"):
        return np.where(cr > 0, np.linalg.norm(e1, axis=1) * np.linalg.norm(e2, axis=1) / cr, np.inf)


def t_error_bound(orc, mesh):
    """Per-ray bound on |t_gpu - t_oracle| for every oracle record (0 where none applies).

    The CUDA path traces each ray in FP32 from an FP32 set-up; the oracle in
    FP64 from an exact one.  On one and the same ray the FP32 test is within
    T_REL t of FP64 (pinned by the closest-hit tests).  The set-up adds an
    origin error of a few roundings of the cell coordinates (M = the largest
    |coordinate|) and a direction error of a few roundings (times the facet's
    normal conditioning kappa for a daughter, whose direction is built on the
    FP32 normal); over a flight of length L they move the ray by
    u (M + kappa L) per set-up step, and a facet met at incidence cosine c turns a
    sideways offset delta into a distance error of delta / |c|.  A daughter
    starts at its parent's hit point, whose offset is the parent's error over
    the parent's |c|.  Hence, with K_SETUP roundings per step:

        E(r) = M + kappa_p L_r + E(parent) / |c_parent|      (E = M + L_r at generation 0)
        |t_gpu - t_oracle| <= T_REL t_r + K_SETUP u E(r) / |c_r|

    c is -d.n at a facet hit and d_z for an escape through the top plane
    (whose distance is measured along z).  Lost rays get no bound."""
    box = mesh.box
    M = max(box.lx, box.ly, abs(box.z_min), abs(box.z_top))
    kap = facet_condition(mesh)
    key = orc["prim"].astype(np.uint64) * np.uint64(1 << 32) + orc["path"].astype(np.uint64)
    order = np.argsort(key)
    skey = key[order]
    err = np.zeros(orc.size)
    c = np.abs(orc["cos_in"])
    L = orc["flight"]
    gen = orc["gen"]
    for g in range(int(gen.max()) + 1 if orc.size else 0):
        sel = np.flatnonzero(gen == g)
        if g == 0:
            err[sel] = M + L[sel]
            continue
        pkey = orc["prim"][sel].astype(np.uint64) * np.uint64(1 << 32) + (orc["path"][sel] >> 4).astype(np.uint64)
        pos = np.searchsorted(skey, pkey)
        par = order[np.minimum(pos, skey.size - 1)]
        assert np.array_equal(key[par], pkey), "a daughter's parent record is missing"
        kp = kap[orc["tri"][par]]
        with np.errstate(divide="ignore", invalid="ignore"):
            err[sel] = M + kp * L[sel] + err[par] / c[par]
    with np.errstate(divide="ignore", invalid="ignore"):
        bound = T_REL * orc["t"] + K_SETUP * U32 * err / c
    bound[(orc["fate"] == LOST_FATE) | ~np.isfinite(bound)] = 0.0
    return bound


LOST_FATE = 4


def _parents(orc):
    """Index of each record's parent record (-1 for primaries)."""
    key = orc["prim"].astype(np.uint64) * np.uint64(1 << 32) + orc["path"].astype(np.uint64)
    order = np.argsort(key)
    skey = key[order]
    par = np.full(orc.size, -1, dtype=np.int64)
    sel = np.flatnonzero(orc["gen"] > 0)
    pkey = orc["prim"][sel].astype(np.uint64) * np.uint64(1 << 32) + (orc["path"][sel] >> 4).astype(np.uint64)
    pos = np.minimum(np.searchsorted(skey, pkey), max(skey.size - 1, 0))
    par[sel] = order[pos]
    assert np.array_equal(key[par[sel]], pkey), "a daughter's parent record is missing"
    return par


def paper_fit_energy_gain(e_parent, cos_parent):
    """|d E_SEE / d E| of Eq. 7 at the parent's energy E and incidence angle alpha
    (from its FP64 cosine), with a 1e-3 degree allowance on alpha: the factor by
    which a daughter inherits its parent's energy error.  sin(E) takes E in radians,
    so the alpha sin(E) term alone contributes up to 0.148 alpha |cos E|."""
    a = np.degrees(np.arccos(np.clip(cos_parent, -1.0, 1.0))) + 1e-3
    return np.abs(0.195 + 3.2e-4 * e_parent + 3.44e-15 * a ** 7) + 0.148 * a * np.abs(np.cos(e_parent))


def energy_bound(orc, gain=None):
    """Per-ray bound on |E_gpu - E_oracle|: E_REL E + E_ABS for the ray's own sampling,
    plus gain(E_parent, cos_parent) times the parent's bound when the daughter energy
    is a function of the parent's (the paper-fit emission); the table emission draws
    it afresh."""
    b = E_REL * orc["energy"] + E_ABS
    if gain is None or orc.size == 0:
        return b
    par = _parents(orc)
    for g in range(1, int(orc["gen"].max()) + 1):
        sel = np.flatnonzero(orc["gen"] == g)
        p = par[sel]
        b[sel] += gain(orc["energy"][p], orc["cos_in"][p]) * b[p]
    return b


def compare_records(gpu, orc, length_scale=10.0, mesh=None, energy_gain=None):
    """Match rays by (prim, path).  Returns a dict of match statistics.

    Hit distances are compared as |t_gpu - t_oracle| / max(t_oracle, length_scale):
    FP32 ray origins carry an absolute error of about one ulp of the cell
    coordinates (~1e-5 nm at 100 nm), so for segments much shorter than the
    mesh resolution (the voxel edge, 10 nm) a plain relative error measures
    that rounding, not the intersection.  With ``mesh``, every ray whose events
    agree and that ends on a facet or escapes is also held to its own bound
    (t_error_bound): ``t_bound_violations`` counts the rays beyond it and
    ``t_bound_ratio_max`` is the largest |dt| / bound."""
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
    out = dict(n_oracle=int(ko.size), n_gpu=int(kg.size), n_common=int(common.size),
               n_same=int(same.sum()), frac_same=float(same.sum()) / max(1, ko.size),
               t_rel_max=float(rel.max()) if rel.size else 0.0,
               t_rel_p9999=float(np.quantile(rel, 0.9999)) if rel.size else 0.0,
               t_rel_p999=float(np.quantile(rel, 0.999)) if rel.size else 0.0,
               mismatch=(g[~same], o[~same]))
    # escaped-energy moments: rays whose events agree carry the same energy up to
    # the FP32 sampling error; an escape on one side only adds its whole energy
    esc_same = same & (o["fate"] == 0)
    eg, eo = g["energy"][esc_same], o["energy"][esc_same]
    agreed_o = np.zeros(orc.size, dtype=bool)
    agreed_o[io[esc_same]] = True
    agreed_g = np.zeros(gpu.size, dtype=bool)
    agreed_g[ig[esc_same]] = True
    lone_o = orc[(orc["fate"] == 0) & ~agreed_o]["energy"]
    lone_g = gpu[(gpu["fate"] == 0) & ~agreed_g]["energy"]
    de = np.abs(eg - eo)
    eb = energy_bound(orc, energy_gain)[io][esc_same]
    out.update(e_ratio_max=float(np.max(de / eb)) if eo.size else 0.0,
               e_abs_max=float(de.max()) if eo.size else 0.0,
               e_tol=float(np.sum(eb)), e2_tol=float(np.sum(2.0 * eb * (eo + eb))),
               e_lone=float(lone_o.sum() + lone_g.sum()),
               e2_lone=float((lone_o ** 2).sum() + (lone_g ** 2).sum()),
               e_rec_sum_gpu=float(np.sum(gpu[gpu["fate"] == 0]["energy"])),
               e2_rec_sum_gpu=float(np.sum(gpu[gpu["fate"] == 0]["energy"] ** 2)))
    if mesh is not None:
        bound = t_error_bound(orc, mesh)[io]
        chk = same & (bound > 0)
        dt = np.abs(g["t"][chk] - o["t"][chk])
        ratio = dt / bound[chk]
        out.update(n_t_checked=int(chk.sum()), t_bound_violations=int((ratio > 1.0).sum()),
                   t_bound_ratio_max=float(ratio.max()) if ratio.size else 0.0,
                   t_bound_worst=(g[chk][np.argsort(ratio)[-5:]], o[chk][np.argsort(ratio)[-5:]],
                                  np.sort(ratio)[-5:]))
    return out


def check_moments(g, o, st):
    """Escaped-energy moments of a run (the FP64 sums of the tallies) against the oracle's.

    Returns (relative error of sum E, relative error of sum E^2).  The GPU sums
    must equal the sums over its own records (the float-pair accumulation adds
    nothing beyond 1e-9 relative); every ray whose events agree must carry the
    oracle's energy within its own bound b (energy_bound); the totals may then
    differ by the sum of those bounds (for E^2: 2 b (E + b) per ray) plus the
    energies of escapes that only one side has."""
    assert abs(g["e_sum"] - st["e_rec_sum_gpu"]) <= 1e-9 * st["e_rec_sum_gpu"]
    assert abs(g["e2_sum"] - st["e2_rec_sum_gpu"]) <= 1e-9 * st["e2_rec_sum_gpu"]
    assert st["e_ratio_max"] <= 1.0, (st["e_ratio_max"], st["e_abs_max"])
    d1, d2 = abs(g["e_sum"] - o["e_sum"]), abs(g["e2_sum"] - o["e2_sum"])
    assert d1 <= st["e_tol"] + st["e_lone"], (d1, o["e_sum"], st["e_tol"], st["e_lone"])
    assert d2 <= st["e2_tol"] + st["e2_lone"], (d2, o["e2_sum"], st["e2_tol"], st["e2_lone"])
    return d1 / o["e_sum"], d2 / o["e2_sum"]
