"""Python binding of librtmc (include/rtmc.h): argument marshalling only.

Every step of the RTMC path runs in the CUDA library; this module converts
numpy arrays / torch tensors into pointers and C structs and back.  Pointers
may be host memory (numpy) or device memory (torch CUDA tensors).  There is
no fallback: if ``librtmc.so`` has not been built, importing fails.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librtmc.so")

OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NOT_LOADED", -5: "NOT_BUILT",
          -6: "CAPACITY", -7: "TIMEOUT", -8: "DEVICE_CHECK"}
BVH_FP32 = 0
BVH_Q8 = 1
BVH_W4 = 2
BVH_Q4 = 3
ESCAPED, EMITTER, ABSORBED_LOW, ABSORBED_OTHER, LOST = 0, 1, 2, 3, 4

EXPORTS = ["rtmc_create", "rtmc_destroy", "rtmc_last_error", "rtmc_load_mesh", "rtmc_unload_mesh",
           "rtmc_load_see_tables",
           "rtmc_build_bvh", "rtmc_run", "rtmc_run_records", "rtmc_trace_rays", "rtmc_philox",
           "rtmc_record_hash", "rtmc_run_noalloc", "rtmc_export_bvh", "rtmc_run_batch",
           "rtmc_probe_bandwidth"]
NOALLOC_MAX_PRIMARIES = 4096
BVH_PLOC = 1 << 16


class RtmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rtmc error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Box(C.Structure):
    _fields_ = [("lx", C.c_double), ("ly", C.c_double), ("z_min", C.c_double), ("z_top", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("n_e", C.c_int32), ("n_theta", C.c_int32), ("e_lo_ev", C.c_double),
                ("e_hi_ev", C.c_double), ("theta_step_deg", C.c_double)]


class EmissionC(C.Structure):
    _fields_ = [("phi_ev", C.c_double), ("e_cut_ev", C.c_double), ("absorb_min_ev", C.c_double),
                ("regen_min_ev", C.c_double), ("max_generation", C.c_int32), ("k_max", C.c_int32),
                ("model", C.c_int32)]


class RunDesc(C.Structure):
    _fields_ = [("n_ebins", C.c_int32), ("n_abins", C.c_int32), ("hist_e_max_ev", C.c_double),
                ("primary_offset", C.c_uint64), ("random_azimuth", C.c_int32), ("max_wraps", C.c_int32),
                ("src_x0", C.c_double), ("src_x1", C.c_double), ("src_y0", C.c_double), ("src_y1", C.c_double),
                ("chunk", C.c_int64), ("block_threads", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("prim_hash", C.c_void_p), ("profile", C.c_int32), ("count_visits", C.c_int32),
                ("traversal", C.c_int32), ("fp64_retest", C.c_int32), ("item_base", C.c_uint32),
                ("no_graph", C.c_int32), ("stack_depth", C.c_int32), ("fetch_threshold", C.c_int32),
                ("random_polar", C.c_int32), ("n_zbins", C.c_int32), ("hist_z", C.c_void_p),
                ("id_order", C.c_int32), ("max_visits", C.c_int32), ("queue_factor", C.c_double)]


class Batch(C.Structure):
    _fields_ = [("mesh_ids", C.POINTER(C.c_int32)), ("n_meshes", C.c_int32),
                ("energies_ev", C.POINTER(C.c_double)), ("n_e", C.c_int32),
                ("theta_deg", C.POINTER(C.c_double)), ("n_theta", C.c_int32),
                ("n_primaries", C.c_int64), ("seed", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "n_primaries", "rays", "escaped", "absorbed_low", "absorbed_other", "emitters", "emitted",
        "regenerated", "capped", "lost", "wraps", "sum_k", "sum_k2")] + [
        (n, C.c_double) for n in ("e_sum", "e2_sum", "sey", "sey_se", "gpu_ms")] + [
        (n, C.c_int64) for n in ("launches", "node_visits", "tri_tests")] + [
        (n, C.c_double) for n in ("ms_generate", "ms_traverse", "ms_shade", "ms_finalize")] + [
        ("traverse_launches", C.c_int64), ("retested", C.c_int64), ("ms_column", C.c_double),
        ("column_rays", C.c_int64), ("queue_retries", C.c_int64)]


class Record(C.Structure):
    _fields_ = [("prim", C.c_uint64), ("path", C.c_uint32), ("gen", C.c_int32), ("fate", C.c_int32),
                ("tri", C.c_int32), ("k", C.c_int32), ("e_bin", C.c_int32), ("a_bin", C.c_int32),
                ("wraps", C.c_int32), ("t", C.c_double), ("energy", C.c_double)]


RECORD_DTYPE = np.dtype([("prim", "<u8"), ("path", "<u4"), ("gen", "<i4"), ("fate", "<i4"),
                         ("tri", "<i4"), ("k", "<i4"), ("e_bin", "<i4"), ("a_bin", "<i4"),
                         ("wraps", "<i4"), ("t", "<f8"), ("energy", "<f8")])
HIT_DTYPE = np.dtype([("t", "<f4"), ("u", "<f4"), ("v", "<f4"), ("tri", "<i4")])
assert C.sizeof(Record) == RECORD_DTYPE.itemsize == 56

_lib = None


def lib():
    """Load librtmc.so; raises ImportError if the CUDA library is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librtmc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.POINTER(C.c_double)
    L.rtmc_create.argtypes = [C.POINTER(vp), i32, vp]
    L.rtmc_destroy.argtypes = [vp]
    L.rtmc_destroy.restype = None
    L.rtmc_last_error.argtypes = [vp]
    L.rtmc_last_error.restype = C.c_char_p
    L.rtmc_load_mesh.argtypes = [vp, vp, i64, C.POINTER(Box), C.POINTER(i32)]
    L.rtmc_unload_mesh.argtypes = [vp, i32]
    L.rtmc_load_see_tables.argtypes = [vp, vp, C.POINTER(Grid), C.POINTER(EmissionC)]
    L.rtmc_build_bvh.argtypes = [vp, i32, i32]
    L.rtmc_run.argtypes = [vp, i32, dp, i32, dp, i32, i64, u64, C.POINTER(RunDesc), C.POINTER(Result), vp, vp]
    L.rtmc_run_records.argtypes = [vp, i32, C.c_double, C.c_double, C.c_uint32, i64, u64, C.POINTER(RunDesc),
                                   C.POINTER(Result), vp, i64, C.POINTER(i64)]
    L.rtmc_trace_rays.argtypes = [vp, i32, vp, vp, vp, i64, vp]
    L.rtmc_run_noalloc.argtypes = [vp, i32, C.c_double, C.c_double, C.c_uint32, i64, u64, C.POINTER(RunDesc),
                                   C.POINTER(Result), vp, vp]
    L.rtmc_philox.argtypes = [vp, vp, i64, u64, vp]
    L.rtmc_export_bvh.argtypes = [vp, i32, i32, vp, i64, C.POINTER(i64)]
    L.rtmc_run_batch.argtypes = [vp, C.POINTER(Batch), C.POINTER(RunDesc), C.POINTER(Result), vp, vp]
    L.rtmc_probe_bandwidth.argtypes = [vp, i64, i32, C.POINTER(C.c_double)]
    L.rtmc_record_hash.argtypes = [C.POINTER(Record)]
    L.rtmc_record_hash.restype = u64
    for name in EXPORTS:
        if name not in ("rtmc_destroy", "rtmc_last_error", "rtmc_record_hash"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(x):
    """Pointer of a numpy array or torch tensor (host or device)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


@dataclasses.dataclass
class Emission:
    phi_ev: float = 4.55
    e_cut_ev: float = 50.0
    absorb_min_ev: float = 10.0
    regen_min_ev: float = float("inf")
    max_generation: int = 1
    k_max: int = 15
    model: int = 0                  # EMISSION_TABLE or EMISSION_PAPER_FIT


EMISSION_TABLE, EMISSION_PAPER_FIT = 0, 1


def paper_emission(e_c_ev=10.0, max_generation=6):
    """The paper's emission rules (Eq. 6 and Eq. 7, stochastic rounding, the
    two-daughter split) with re-emission above E_c = phi + E_F."""
    return Emission(absorb_min_ev=e_c_ev, regen_min_ev=e_c_ev, max_generation=max_generation,
                    model=EMISSION_PAPER_FIT)


def run_desc(n_ebins=64, n_abins=18, hist_e_max_ev=50.0, primary_offset=0, random_azimuth=False,
             max_wraps=1024, window=None, chunk=0, block_threads=0, blocks_per_sm=0, prim_hash=None,
             profile=False, count_visits=False, traversal=0, fp64_retest=False, item_base=0, no_graph=False,
             stack_depth=0, fetch_threshold=0, id_order=False, random_polar=False, n_zbins=0, max_visits=0,
             queue_factor=0.0):
    """Run descriptor.  ``random_polar`` draws each primary's polar angle from
    the cosine law (the item angle is ignored); ``n_zbins`` > 0 adds the
    penetration-depth histogram, returned as ``hist_z`` in each result dict
    (the binding owns that buffer; ``hist_z`` is filled in per call)."""
    x0, x1, y0, y1 = window if window is not None else (0.0, 0.0, 0.0, 0.0)
    return RunDesc(n_ebins=int(n_ebins), n_abins=int(n_abins), hist_e_max_ev=float(hist_e_max_ev),
                   primary_offset=int(primary_offset), random_azimuth=int(bool(random_azimuth)),
                   max_wraps=int(max_wraps), src_x0=x0, src_x1=x1, src_y0=y0, src_y1=y1, chunk=int(chunk),
                   block_threads=int(block_threads), blocks_per_sm=int(blocks_per_sm),
                   prim_hash=prim_hash.data_ptr() if prim_hash is not None else None,
                   profile=int(bool(profile)), count_visits=int(bool(count_visits)), traversal=int(traversal),
                   fp64_retest=int(bool(fp64_retest)), item_base=int(item_base), no_graph=int(bool(no_graph)),
                   stack_depth=int(stack_depth), fetch_threshold=int(fetch_threshold),
                   random_polar=int(bool(random_polar)), n_zbins=int(n_zbins), hist_z=None,
                   id_order=int(bool(id_order)), max_visits=int(max_visits), queue_factor=float(queue_factor))


def _with_hist_z(desc, n_items):
    """A copy of ``desc`` whose hist_z points at a fresh [n_items, n_zbins] array."""
    d = RunDesc.from_buffer_copy(desc)
    hz = np.zeros((n_items, max(d.n_zbins, 0)), dtype=np.uint64)
    d.hist_z = hz.ctypes.data if d.n_zbins > 0 else None
    return d, hz


def result_dict(r: Result):
    return {name: getattr(r, name) for name, _ in Result._fields_}


def _results(out, hz, n_zbins):
    res = [result_dict(r) for r in out]
    if n_zbins > 0:
        for k, r in enumerate(res):
            r["hist_z"] = hz[k]
    return res


class Context:
    """A librtmc context on one CUDA device (owns meshes, tables and scratch)."""

    def __init__(self, device: int = 0, stream=None):
        self._L = lib()
        h = C.c_void_p()
        s = None
        if stream is not None:
            s = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        rc = self._L.rtmc_create(C.byref(h), int(device), s)
        if rc != 0:
            raise RtmcError(rc, "rtmc_create failed (no CUDA device?)")
        self.h = h
        self.n_ebins = 64
        self.n_abins = 18

    def close(self):
        if getattr(self, "h", None):
            self._L.rtmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != 0:
            raise RtmcError(rc, self._L.rtmc_last_error(self.h).decode())

    # ---- C-ABI calls ---------------------------------------------------------
    def load_mesh(self, tri, box) -> int:
        if not hasattr(tri, "data_ptr"):
            tri = np.ascontiguousarray(tri, dtype=np.float32)
        n = int(tri.shape[0])
        mid = C.c_int32()
        b = Box(*box.as_tuple()) if hasattr(box, "as_tuple") else Box(*box)
        self._check(self._L.rtmc_load_mesh(self.h, _ptr(tri), n, C.byref(b), C.byref(mid)))
        return mid.value

    def unload_mesh(self, mesh_id: int):
        self._check(self._L.rtmc_unload_mesh(self.h, int(mesh_id)))

    def load_see_tables(self, table, emission: Emission | None = None):
        em = emission or Emission()
        delta = np.ascontiguousarray(table.delta, dtype=np.float32)
        g = Grid(table.n_e, table.n_theta, table.e_lo_ev, table.e_hi_ev, table.theta_step_deg)
        e = EmissionC(em.phi_ev, em.e_cut_ev, em.absorb_min_ev, em.regen_min_ev, em.max_generation, em.k_max,
                      em.model)
        self._check(self._L.rtmc_load_see_tables(self.h, _ptr(delta), C.byref(g), C.byref(e)))

    def build_bvh(self, mesh_id: int, kind: int = BVH_FP32, leaf: int = 0, ploc: bool = False):
        """Build the mesh's BVH: node format `kind`, leaves of up to `leaf` triangles
        (0: 4), hierarchy by Karras splits or (ploc=True) locally-ordered clustering."""
        self._check(self._L.rtmc_build_bvh(self.h, int(mesh_id),
                                           int(kind) | (int(leaf) << 8) | (BVH_PLOC if ploc else 0)))

    def run(self, mesh_id, energies, thetas, n_primaries, seed, desc: RunDesc | None = None):
        """All (energy, angle) items; returns (results list, hist_e [items, nE], hist_a [items, nA])."""
        e = np.ascontiguousarray(np.atleast_1d(energies), dtype=np.float64)
        t = np.ascontiguousarray(np.atleast_1d(thetas), dtype=np.float64)
        n_items = e.size * t.size
        d, hz = _with_hist_z(desc or run_desc(), n_items)
        out = (Result * n_items)()
        he = np.zeros((n_items, d.n_ebins), dtype=np.uint64)
        ha = np.zeros((n_items, d.n_abins), dtype=np.uint64)
        self._check(self._L.rtmc_run(self.h, int(mesh_id), e.ctypes.data_as(C.POINTER(C.c_double)), e.size,
                                     t.ctypes.data_as(C.POINTER(C.c_double)), t.size, int(n_primaries),
                                     int(seed), C.byref(d), out, _ptr(he), _ptr(ha)))
        return _results(out, hz, d.n_zbins), he, ha

    def run_records(self, mesh_id, energy, theta, n_primaries, seed, item=0, desc=None, rec_cap=None):
        d, hz = _with_hist_z(desc or run_desc(), 1)
        cap = int(rec_cap) if rec_cap else int(n_primaries) * 40 + 1024
        rec = np.zeros(cap, dtype=RECORD_DTYPE)
        res = Result()
        n = C.c_int64()
        self._check(self._L.rtmc_run_records(self.h, int(mesh_id), float(energy), float(theta), int(item),
                                             int(n_primaries), int(seed), C.byref(d), C.byref(res), _ptr(rec),
                                             cap, C.byref(n)))
        out = result_dict(res)
        if d.n_zbins > 0:
            out["hist_z"] = hz[0]
        out["records"] = np.sort(rec[:n.value], order=["prim", "gen", "path"])
        return out

    def run_batch(self, mesh_ids, energies, thetas, n_primaries, seed, desc: RunDesc | None = None):
        """Batched form over meshes x energies x angles; returns (results, hist_e, hist_a)."""
        ids = np.ascontiguousarray(np.atleast_1d(mesh_ids), dtype=np.int32)
        e = np.ascontiguousarray(np.atleast_1d(energies), dtype=np.float64)
        t = np.ascontiguousarray(np.atleast_1d(thetas), dtype=np.float64)
        n_items = ids.size * e.size * t.size
        d, hz = _with_hist_z(desc or run_desc(), n_items)
        b = Batch(ids.ctypes.data_as(C.POINTER(C.c_int32)), ids.size, e.ctypes.data_as(C.POINTER(C.c_double)),
                  e.size, t.ctypes.data_as(C.POINTER(C.c_double)), t.size, int(n_primaries), int(seed))
        out = (Result * n_items)()
        he = np.zeros((n_items, d.n_ebins), dtype=np.uint64)
        ha = np.zeros((n_items, d.n_abins), dtype=np.uint64)
        self._check(self._L.rtmc_run_batch(self.h, C.byref(b), C.byref(d), out, _ptr(he), _ptr(ha)))
        return _results(out, hz, d.n_zbins), he, ha

    def run_noalloc(self, mesh_id, energy, theta, n_primaries, seed, item=0, desc=None):
        """One item through rtmc_run_noalloc (static device scratch, no allocation).

        Returns (result dict, hist_e, hist_a)."""
        d, hz = _with_hist_z(desc or run_desc(), 1)
        res = Result()
        he = np.zeros(d.n_ebins, dtype=np.uint64)
        ha = np.zeros(d.n_abins, dtype=np.uint64)
        self._check(self._L.rtmc_run_noalloc(self.h, int(mesh_id), float(energy), float(theta), int(item),
                                             int(n_primaries), int(seed), C.byref(d), C.byref(res), _ptr(he),
                                             _ptr(ha)))
        return _results([res], hz, d.n_zbins)[0], he, ha

    def trace_rays(self, mesh_id, o, d, skip=None):
        o = np.ascontiguousarray(o, dtype=np.float32)
        d = np.ascontiguousarray(d, dtype=np.float32)
        n = o.shape[0]
        sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int32)
        hits = np.zeros(n, dtype=HIT_DTYPE)
        self._check(self._L.rtmc_trace_rays(self.h, int(mesh_id), _ptr(o), _ptr(d), _ptr(sk), n, _ptr(hits)))
        return hits

    def export_bvh(self, mesh_id, which):
        """Raw bytes of a built BVH array (0 FP32 nodes, 1 Q8 nodes, 2 triangles, 3 4-wide nodes,
        4 quantised 4-wide nodes)."""
        need = C.c_int64()
        self._check(self._L.rtmc_export_bvh(self.h, int(mesh_id), int(which), None, 0, C.byref(need)))
        buf = np.zeros(need.value, dtype=np.uint8)
        self._check(self._L.rtmc_export_bvh(self.h, int(mesh_id), int(which), _ptr(buf), need.value, C.byref(need)))
        return buf

    def probe_bandwidth(self, nbytes, iters=20):
        """Streaming read bandwidth (GB/s) over a buffer of `nbytes`."""
        g = C.c_double()
        self._check(self._L.rtmc_probe_bandwidth(self.h, int(nbytes), int(iters), C.byref(g)))
        return g.value

    def philox(self, ctr, key):
        c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
        out = np.zeros_like(c)
        self._check(self._L.rtmc_philox(self.h, _ptr(c), c.shape[0], int(key), _ptr(out)))
        return out


def record_hash(rec) -> int:
    r = Record(*[rec[n].item() for n in RECORD_DTYPE.names])
    return int(lib().rtmc_record_hash(C.byref(r)))
