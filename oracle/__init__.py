"""ctypes front end of the FP64 CPU oracle (oracle/rtmc_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it to check and time the CUDA path.  The
product path never imports it.  Nothing here does arithmetic of the method;
it marshals arrays into the C oracle and back.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

_lib = None


class OrcBox(C.Structure):
    _fields_ = [("lx", C.c_double), ("ly", C.c_double), ("z_min", C.c_double), ("z_top", C.c_double)]


class OrcPhysics(C.Structure):
    _fields_ = [("delta", C.POINTER(C.c_float)), ("n_e", C.c_int32), ("n_theta", C.c_int32),
                ("e_lo_ev", C.c_double), ("e_hi_ev", C.c_double), ("theta_step_deg", C.c_double),
                ("phi_ev", C.c_double), ("e_cut_ev", C.c_double), ("absorb_min_ev", C.c_double),
                ("regen_min_ev", C.c_double), ("max_generation", C.c_int32), ("k_max", C.c_int32),
                ("model", C.c_int32)]


class OrcRun(C.Structure):
    _fields_ = [("energy_ev", C.c_double), ("theta_deg", C.c_double), ("seed", C.c_uint64),
                ("item", C.c_uint32), ("random_azimuth", C.c_int32), ("n_primaries", C.c_int64),
                ("primary_offset", C.c_uint64), ("prim_ids", C.POINTER(C.c_uint64)),
                ("src_x0", C.c_double), ("src_x1", C.c_double), ("src_y0", C.c_double),
                ("src_y1", C.c_double), ("n_ebins", C.c_int32), ("n_abins", C.c_int32),
                ("hist_e_max_ev", C.c_double), ("max_wraps", C.c_int32), ("n_threads", C.c_int32),
                ("random_polar", C.c_int32), ("n_zbins", C.c_int32)]


class OrcResult(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "n_primaries", "rays", "escaped", "absorbed_low", "absorbed_other", "emitters", "emitted",
        "regenerated", "capped", "lost", "wraps", "sum_k", "sum_k2")] + [
        (n, C.c_double) for n in ("e_sum", "e2_sum", "sey", "sey_se")]


RECORD_DTYPE = np.dtype([("prim", "<u8"), ("path", "<u4"), ("gen", "<i4"), ("fate", "<i4"),
                         ("tri", "<i4"), ("k", "<i4"), ("e_bin", "<i4"), ("a_bin", "<i4"),
                         ("wraps", "<i4"), ("t", "<f8"), ("energy", "<f8"), ("cos_in", "<f8"),
                         ("flight", "<f8")])
assert RECORD_DTYPE.itemsize == 72

ESCAPED, EMITTER, ABSORBED_LOW, ABSORBED_OTHER, LOST = 0, 1, 2, 3, 4


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        fp = np.ctypeslib.ndpointer
        L.orc_run_rtmc.restype = C.c_int
        L.orc_run_rtmc.argtypes = [C.c_void_p, C.c_int64, C.POINTER(OrcBox), C.POINTER(OrcPhysics),
                                   C.POINTER(OrcRun), C.POINTER(OrcResult), C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]
        for name in ("orc_closest_hit",):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64,
                                         C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_closest_hit_mt.restype = None
        L.orc_closest_hit_mt.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64,
                                         C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_trace_ray.restype = C.c_int
        L.orc_trace_ray.argtypes = [C.c_void_p, C.c_int64, C.POINTER(OrcBox), C.c_void_p, C.c_void_p,
                                    C.c_int64, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_int32), C.c_void_p]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_lookup_delta.restype = C.c_double
        L.orc_lookup_delta.argtypes = [C.POINTER(OrcPhysics), C.c_double, C.c_double]
        L.orc_poisson.restype = C.c_int
        L.orc_poisson.argtypes = [C.c_double, C.c_double, C.c_int32, C.POINTER(C.c_int)]
        L.orc_sample_energy.restype = C.c_double
        L.orc_sample_energy.argtypes = [C.POINTER(OrcPhysics), C.c_double]
        for name in ("orc_gamma_fit", "orc_esee_fit"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double, C.c_double]
        L.orc_round_stochastic.restype = C.c_int
        L.orc_round_stochastic.argtypes = [C.c_double, C.c_double, C.c_int32, C.POINTER(C.c_int)]
        L.orc_cosine_dir.restype = None
        L.orc_cosine_dir.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p]
        _lib = L
    return _lib


@dataclasses.dataclass
class Emission:
    """Secondary-emission parameters of one run (defaults: the tiny/paper configs)."""
    phi_ev: float = 4.55
    e_cut_ev: float = 50.0
    absorb_min_ev: float = 10.0
    regen_min_ev: float = float("inf")
    max_generation: int = 1
    k_max: int = 15
    model: int = 0                  # 0: yield table; 1: the paper's fits (Eq. 6, Eq. 7)


MODEL_TABLE, MODEL_PAPER_FIT = 0, 1


def paper_emission(e_c_ev=10.0, max_generation=6):
    """The paper's own emission rules: Eq. 6 yield rounded stochastically, Eq. 7
    energies, the two-daughter split, re-emission above E_c = phi + E_F."""
    return Emission(absorb_min_ev=e_c_ev, regen_min_ev=e_c_ev, max_generation=max_generation,
                    model=MODEL_PAPER_FIT)


def _physics(table, em: Emission):
    delta = np.ascontiguousarray(table.delta, dtype=np.float32)
    ph = OrcPhysics(delta.ctypes.data_as(C.POINTER(C.c_float)), table.n_e, table.n_theta,
                    table.e_lo_ev, table.e_hi_ev, table.theta_step_deg, em.phi_ev, em.e_cut_ev,
                    em.absorb_min_ev, em.regen_min_ev, em.max_generation, em.k_max, em.model)
    return ph, delta


def _box(box):
    return OrcBox(*box.as_tuple())


def run(mesh, table, energy_ev, theta_deg, n_primaries, seed, *, item=0, emission=None,
        primary_offset=0, prim_ids=None, window=None, random_azimuth=False, n_ebins=64,
        n_abins=18, hist_e_max_ev=50.0, max_wraps=1024, n_threads=0, records=False,
        random_polar=False, n_zbins=0):
    """One (energy, angle) RTMC run on the CPU.  Returns a dict of tallies."""
    L = lib()
    em = emission or Emission()
    ph, delta_keep = _physics(table, em)
    tri = np.ascontiguousarray(mesh.tri, dtype=np.float32)
    ids_keep = None
    if prim_ids is not None:
        ids_keep = np.ascontiguousarray(prim_ids, dtype=np.uint64)
        n_primaries = ids_keep.size
    x0, x1, y0, y1 = window if window is not None else (0.0, 0.0, 0.0, 0.0)
    r = OrcRun(float(energy_ev), float(theta_deg), int(seed), int(item), int(bool(random_azimuth)),
               int(n_primaries), int(primary_offset),
               ids_keep.ctypes.data_as(C.POINTER(C.c_uint64)) if ids_keep is not None else None,
               x0, x1, y0, y1, int(n_ebins), int(n_abins), float(hist_e_max_ev), int(max_wraps),
               int(n_threads), int(bool(random_polar)), int(n_zbins))
    out = OrcResult()
    he = np.zeros(n_ebins, dtype=np.int64)
    ha = np.zeros(n_abins, dtype=np.int64)
    hz = np.zeros(max(int(n_zbins), 1), dtype=np.int64)
    rec = None
    nrec = C.c_int64(0)
    if records:
        cap = int(n_primaries) * (1 + em.k_max) ** max(1, em.max_generation) + 16
        cap = min(cap, int(n_primaries) * 64 + 1024)
        rec = np.zeros(cap, dtype=RECORD_DTYPE)
    rc = L.orc_run_rtmc(tri.ctypes.data, tri.shape[0], C.byref(_box(mesh.box)), C.byref(ph),
                        C.byref(r), C.byref(out), he.ctypes.data, ha.ctypes.data, hz.ctypes.data,
                        rec.ctypes.data if rec is not None else None,
                        rec.size if rec is not None else 0, C.byref(nrec))
    if rc != 0:
        raise ValueError(f"orc_run_rtmc failed ({rc})")
    res = {name: getattr(out, name) for name, _ in OrcResult._fields_}
    res["hist_e"] = he
    res["hist_a"] = ha
    if n_zbins:
        res["hist_z"] = hz
    if rec is not None:
        rr = rec[:nrec.value]
        res["records"] = np.sort(rr, order=["prim", "gen", "path"])
    return res


def closest_hit(mesh, o, d, exclude=-1, method="watertight", eps=1e-12):
    L = lib()
    tri = np.ascontiguousarray(mesh.tri, dtype=np.float32)
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    t, j, u, v = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
    if method == "watertight":
        L.orc_closest_hit(tri.ctypes.data, tri.shape[0], o.ctypes.data, d.ctypes.data, int(exclude),
                          C.byref(t), C.byref(j), C.byref(u), C.byref(v))
    else:
        L.orc_closest_hit_mt(tri.ctypes.data, tri.shape[0], o.ctypes.data, d.ctypes.data,
                             int(exclude), float(eps), C.byref(t), C.byref(j), C.byref(u), C.byref(v))
    return t.value, j.value, u.value, v.value


def trace_ray(mesh, o, d, origin_tri=-1, max_wraps=1024):
    L = lib()
    tri = np.ascontiguousarray(mesh.tri, dtype=np.float32)
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    j, t, u, v, w = C.c_int64(), C.c_double(), C.c_double(), C.c_double(), C.c_int32()
    ol = np.zeros(3)
    fate = L.orc_trace_ray(tri.ctypes.data, tri.shape[0], C.byref(_box(mesh.box)), o.ctypes.data,
                           d.ctypes.data, int(origin_tri), int(max_wraps), C.byref(j), C.byref(t),
                           C.byref(u), C.byref(v), C.byref(w), ol.ctypes.data)
    return dict(fate=fate, tri=j.value, t=t.value, u=u.value, v=v.value, wraps=w.value, o_last=ol)


def philox(ctr, key):
    L = lib()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    L.orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def lookup_delta(table, e_ev, alpha_rad, emission=None):
    ph, keep = _physics(table, emission or Emission())
    return lib().orc_lookup_delta(C.byref(ph), float(e_ev), float(alpha_rad))


def poisson(lam, u, k_max=15):
    cap = C.c_int(0)
    k = lib().orc_poisson(float(lam), float(u), int(k_max), C.byref(cap))
    return k, cap.value


class _NoTable:
    delta = np.ones((2, 2), dtype=np.float32)
    n_e = n_theta = 2
    e_lo_ev, e_hi_ev, theta_step_deg = 1.0, 2.0, 1.0


def sample_energy(u, emission=None):
    ph, keep = _physics(_NoTable, emission or Emission())
    return lib().orc_sample_energy(C.byref(ph), float(u))


def cosine_dir(n, u1, u2):
    n = np.ascontiguousarray(n, dtype=np.float64)
    d = np.zeros(3)
    lib().orc_cosine_dir(n.ctypes.data, float(u1), float(u2), d.ctypes.data)
    return d


def gamma_fit(e_ev, alpha_deg):
    return lib().orc_gamma_fit(float(e_ev), float(alpha_deg))


def esee_fit(e_ev, alpha_deg):
    return lib().orc_esee_fit(float(e_ev), float(alpha_deg))


def round_stochastic(gamma, u, k_max=15):
    cap = C.c_int(0)
    k = lib().orc_round_stochastic(float(gamma), float(u), int(k_max), C.byref(cap))
    return k, cap.value
