"""Benchmark: RTMC secondary-electron yield, large configuration (the default).

Workload (one step): a 256^3 periodic Gaussian-random-field foam (10 nm voxels,
porosity 0.7, correlation length 2 voxels, seed 1806) meshed by marching cubes
into ~9.9M FP32 triangles under a compressed (4-wide, 8-bit) BVH; 1e8 primaries
at 500 eV at each of 9 incidence angles 0..80 deg, tertiaries for secondaries
above 20 eV; 128-bin escaped-energy and 36-bin polar-angle histograms with FP64
energy moments.  All items run batched (rtmc_run_batch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config large|paper|precision]

Prints one JSON line.  ``value`` is traced rays per second over all ranks with
the mesh, BVH and tables resident on the device; ``e2e`` is the same metric
through the C ABI from pinned host buffers (mesh upload, BVH build, run and the
result read-back inside the timed region).  ``--impl reference`` times the CPU
FP64 oracle on a bounded sample of the same workload.  ``--config paper`` is
the 128^3 foam x 20 energies at normal incidence (also reported, shorter, as
``paper_config`` in the default line); ``--config precision`` the 8-bit-node
precision form with the FP64 re-test.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "traced rays/sec and primaries/sec at stated SEY error; % memory roofline"
ENERGIES = [50.0 * i for i in range(1, 21)]
N_PRIM = 10_000_000
GRID, POROSITY, CORR, SEED = 128, 0.6, 2.0, 1806
TRI_BYTES, RAY_BYTES = 48, 48                   # triangle fetch, ray read + hit write
NODE_BYTES = {0: 64, 1: 32, 2: 128, 3: 64}      # node fetch per visit: FP32 binary, Q8 binary, 4-wide FP32, 4-wide Q8
PREC_NODES = {"q4": 3, "q8": 1}                 # precision config: 8-bit node formats
PREC_NODE_NAME = {3: "4-wide Q8", 1: "Q8"}
MAIN_KIND = 2                                   # the paper-config workload runs on 4-wide FP32 nodes
# large configuration (the default): 256^3 foam, compressed BVH, tertiaries, 9 angles
LARGE_GRID, LARGE_POROSITY = 256, 0.7
LARGE_E, LARGE_THETAS = 500.0, [10.0 * j for j in range(9)]
LARGE_N_PRIM = 100_000_000
LARGE_KIND = 3                                  # 4-wide nodes with 8-bit child boxes (compressed)
LARGE_BINS = (128, 36)
LARGE_MAX_GEN = 2                               # tertiaries: secondaries above 20 eV re-emit once
NODE_NAME = {0: "binary FP32", 1: "binary Q8", 2: "4-wide FP32", 3: "4-wide Q8"}


def large_emission(rtmc_or_oracle):
    """Tertiaries: secondaries at or above 20 eV re-emit once (max_generation 2)."""
    return rtmc_or_oracle.Emission(regen_min_ev=20.0, max_generation=LARGE_MAX_GEN)


def large_workload_name(n_tri, n_prim):
    return (f"large: {LARGE_GRID}^3 periodic GRF foam (10 nm voxels, porosity {LARGE_POROSITY}, corr {CORR:g} vox, "
            f"seed {SEED}) -> {n_tri} FP32 triangles, {NODE_NAME[LARGE_KIND]} BVH (compressed); {n_prim:.3g} "
            f"primaries at {LARGE_E:g} eV x {len(LARGE_THETAS)} angles {LARGE_THETAS[0]:g}-{LARGE_THETAS[-1]:g} deg; "
            f"tertiaries above 20 eV (max_generation 2); {LARGE_BINS[0]} energy / {LARGE_BINS[1]} angle bins, "
            "FP64 moments")


def workload_name(n_tri, n_prim, energies=ENERGIES):
    return (f"plain RTMC, paper scale: {GRID}^3 periodic GRF foam (10 nm voxels, porosity {POROSITY}, "
            f"corr {CORR:g} vox, seed {SEED}) -> {n_tri} FP32 triangles; {len(energies)} energies "
            f"{energies[0]:g}-{energies[-1]:g} eV x {n_prim:.3g} primaries, normal incidence")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_sha():
    h = hashlib.sha256()
    for f in ("rtmc_traverse.cu", "rtmc_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1806_00205_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(tag="paper_config", node_format=MAIN_KIND):
    """DRAM bytes per traversal ray from a committed ncu summary, if it matches this kernel."""
    name = "traverse_dram_traffic.json" if tag == "paper_config" else f"traverse_dram_traffic_{tag}.json"
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", name)))
    except (OSError, ValueError):
        return None
    if d.get("kernel_sha") != kernel_sha() or d.get("node_format") != node_format:
        return None
    return d.get("dram_bytes_per_ray")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def make_mesh():
    from paper_1806_00205_gb300 import inputs as I
    return I.grf_foam(GRID, POROSITY, CORR, SEED), I.see_table()


def cpu_oracle_sample(mesh, table, n_sample, energy=500.0, seed=SEED, theta=0.0, item=0, emission=None,
                      bins=(64, 18), records=False):
    import oracle as O
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = O.run(mesh, table, energy, theta, n_sample, seed, primary_offset=0, n_threads=threads, item=item,
              emission=emission or O.Emission(), n_ebins=bins[0], n_abins=bins[1], records=records)
    dt = time.perf_counter() - t0
    return r, dt, threads


def large_oracle_sample(mesh, table, per_angle):
    """The oracle on the first `per_angle` primaries of every angle of the large config
    (item k = angle k, the batch's random streams); returns per-item results, rays, s, threads."""
    import oracle as O
    out, rays, secs, thr = [], 0, 0.0, 1
    for k, th in enumerate(LARGE_THETAS):
        r, dt, thr = cpu_oracle_sample(mesh, table, per_angle, LARGE_E, SEED, th, k, large_emission(O),
                                       LARGE_BINS, records=True)
        out.append(r)
        rays += r["rays"]
        secs += dt
    return out, rays, secs, thr


def run_reference(args):
    """The reference arm: the FP64 oracle (the paper has no code) on a bounded sample
    of the configuration's workload, on the host's cores, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1806_00205_gb300 import inputs as I
    import oracle as O
    table = I.see_table()
    if args.config == "large":
        mesh = I.grf_foam(LARGE_GRID, LARGE_POROSITY, CORR, SEED)
        per_angle = max(1, args.ref_sample // len(LARGE_THETAS))
        for _ in range(args.warmup):
            cpu_oracle_sample(mesh, table, 1, LARGE_E, SEED, LARGE_THETAS[-1], len(LARGE_THETAS) - 1,
                              large_emission(O), LARGE_BINS)
        rays, secs, prims = 0, 0.0, 0
        for _ in range(args.steps):
            for k, th in enumerate(LARGE_THETAS):
                r, dt, threads = cpu_oracle_sample(mesh, table, per_angle, LARGE_E, SEED, th, k, large_emission(O),
                                                   LARGE_BINS)
                rays += r["rays"]
                secs += dt
                prims += per_angle
        workload = large_workload_name(mesh.n_tri, LARGE_N_PRIM)
        sample = (f"{per_angle} primaries per angle x {len(LARGE_THETAS)} angles at {LARGE_E:g} eV per step, "
                  f"tertiaries (brute force over all {mesh.n_tri} triangles per ray segment)")
    else:
        mesh, table = make_mesh()
        n_sample = args.ref_sample
        for _ in range(args.warmup):
            cpu_oracle_sample(mesh, table, max(16, n_sample // 8))
        rays, secs, prims = 0, 0.0, 0
        for _ in range(args.steps):
            r, dt, threads = cpu_oracle_sample(mesh, table, n_sample)
            rays += r["rays"]
            secs += dt
            prims += n_sample
        workload = workload_name(mesh.n_tri, N_PRIM)
        sample = (f"{n_sample} primaries at 500 eV, normal incidence, per step "
                  f"(brute force over all {mesh.n_tri} triangles per ray segment)")
    v = rays / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "primaries_per_s": prims / secs,
            "config": {"workload": workload, "n_tri": mesh.n_tri},
            "cpu_baseline": {"value": v, "unit": "rays/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_forms(rtmc, autotune, n_prim, device=0):
    """Batched config: 16 foams (48^3..128^3, porosity 0.3..0.9) x 20 energies x 9 angles.

    Compares the batched form (multi-item queues, one CUDA graph, autotuned, 8-bit
    or FP32 nodes, binary or 4-wide) with the plain form (rtmc_run item by item,
    binary FP32 nodes), on a context of its own (the configuration's emission)."""
    import torch
    from paper_1806_00205_gb300 import inputs as I
    cfg = I.batched_foams()
    meshes = [I.grf_foam(g, p, CORR, sd) for g, p, sd in cfg]
    energies = [50.0 * i for i in range(1, 21)]
    thetas = [10.0 * j for j in range(9)]
    ctx = rtmc.Context(device)
    ctx.load_see_tables(I.see_table())
    kinds = {"batched_q8": rtmc.BVH_Q8, "batched_q4": rtmc.BVH_Q4, "batched_fp32": rtmc.BVH_FP32,
             "batched_w4": rtmc.BVH_W4}
    ids = {name: [] for name in kinds}
    for m in meshes:
        for name, kind in kinds.items():
            a = ctx.load_mesh(m.tri, m.box)
            ctx.build_bvh(a, kind=kind)
            ids[name].append(a)
    ntri = [m.n_tri for m in meshes]
    tuned = {name: autotune.tune(ctx, ids[name], ntri, energies, thetas, kind=kind, cache_path=None,
                                 device_name="gb300") for name, kind in kinds.items()}
    per_mesh = len(energies) * len(thetas)

    def plain():
        out = []
        for mi, mid in enumerate(ids["batched_fp32"]):
            r, _, _ = ctx.run(mid, energies, thetas, n_prim, SEED, desc=rtmc.run_desc(item_base=mi * per_mesh))
            out += r
        return out

    def batched(name):
        return lambda: ctx.run_batch(ids[name], energies, thetas, n_prim, SEED,
                                     desc=rtmc.run_desc(**tuned[name]))[0]

    forms, results = {}, {}
    for name, fn in [(n, batched(n)) for n in kinds] + [("plain_fp32", plain)]:
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        rays = sum(x["rays"] for x in r)
        forms[name] = {"rays_per_s": rays / dt, "primaries_per_s": len(r) * n_prim / dt, "s": dt}
        results[name] = r
    d_sey = {name: max(abs(a["sey"] - b["sey"]) for a, b in zip(results[name], results["plain_fp32"]))
             for name in kinds}
    ctx.close()
    return {"workload": f"16 GRF foams (grids 48^3..128^3, porosity 0.30..0.90, {min(ntri)}..{max(ntri)} "
                        f"triangles) x 20 energies (50..1000 eV) x 9 angles (0..80 deg) x {n_prim:.0e} primaries",
            "forms": forms, "max_abs_sey_diff_vs_plain_fp32": d_sey,
            "speedup_batched_q8_vs_plain_fp32": forms["plain_fp32"]["s"] / forms["batched_q8"]["s"],
            "speedup_batched_q4_vs_plain_fp32": forms["plain_fp32"]["s"] / forms["batched_q4"]["s"],
            "autotuned": tuned}


def kernel_fields(ms, launches, algo_bytes, peak, bound, extra=None):
    """Roofline fields of one kernel from its summed CUDA-event time and algorithmic bytes."""
    achieved = algo_bytes / (ms / 1e3) / 1e9 if ms > 0 else None
    out = {"bound": bound, "ms": ms, "launches": launches, "ms_per_launch": ms / max(1, launches),
           "algorithmic_bytes": algo_bytes, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak if achieved else None}
    if extra:
        out.update(extra)
    return out


def paper_config_summary(rtmc, I, dev, l2_gbs, hbm_peak, steps=3):
    """The paper-scale configuration (128^3 foam, 20 energies x 1e7 primaries at normal
    incidence, 4-wide FP32 nodes) on its own context: rays/s and the traversal roofline."""
    import torch
    mesh, table = make_mesh()
    stream = torch.cuda.Stream(device=dev)
    ctx = rtmc.Context(dev.index or 0, stream=stream)
    ctx.load_see_tables(table)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=MAIN_KIND)
    desc = rtmc.run_desc(profile=True, no_graph=True)
    ctx.run_batch([mid], ENERGIES, [0.0], N_PRIM, SEED, desc=desc)
    torch.cuda.synchronize(dev)
    rays = trav_ms = col_ms = col_rays = shade_ms = 0.0
    trav_l = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        res, _, _ = ctx.run_batch([mid], ENERGIES, [0.0], N_PRIM, SEED, desc=desc)
        rays += sum(r["rays"] for r in res)
        trav_ms += res[0]["ms_traverse"]
        trav_l += res[0]["traverse_launches"]
        col_ms += res[0]["ms_column"]
        col_rays += res[0]["column_rays"]
        shade_ms += res[0]["ms_shade"]
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    cres, _, _ = ctx.run_batch([mid], ENERGIES, [0.0], N_PRIM // 5, SEED,
                               desc=rtmc.run_desc(count_visits=True, no_graph=True))
    c_rays = sum(r["rays"] for r in cres) - cres[0]["column_rays"]
    visits, tests = cres[0]["node_visits"] / c_rays, cres[0]["tri_tests"] / c_rays
    b_ray = visits * NODE_BYTES[MAIN_KIND] + tests * TRI_BYTES + RAY_BYTES
    h_rays = rays - col_rays
    ctx.close()
    tr = measured_traffic("paper_config", MAIN_KIND)
    return {"workload": workload_name(mesh.n_tri, N_PRIM), "rays_per_s": rays / dt,
            "primaries_per_s": steps * len(ENERGIES) * N_PRIM / dt, "ms_per_step": 1e3 * dt / steps,
            "k_traverse_ww": kernel_fields(trav_ms, trav_l, h_rays * b_ray, l2_gbs, "l2", {
                "node_format": NODE_NAME[MAIN_KIND], "bytes_per_ray": b_ray, "node_visits_per_ray": visits,
                "tri_tests_per_ray": tests, "dram_bytes_per_ray": tr,
                "frac_of_measured_hbm": (tr * h_rays / (trav_ms / 1e3) / 1e9 / hbm_peak) if tr else None}),
            "k_trace_columns": {"ms": col_ms, "rays": col_rays, "rays_per_s": col_rays / (col_ms / 1e3)},
            "k_shade_ms": shade_ms}


def run_large(args):
    """Large config (the default line): 256^3 foam at porosity 0.7 (~9.9M triangles) under the
    compressed 4-wide 8-bit BVH, 1e8 primaries at 500 eV x 9 incidence angles, tertiaries for
    secondaries above 20 eV, 128 energy and 36 angle bins, FP64 moments; every item batched."""
    import torch
    import torch.distributed as dist
    import oracle as O
    from paper_1806_00205_gb300 import autotune, rtmc, shard
    from paper_1806_00205_gb300 import inputs as I
    from tests.parity import primary_hashes

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_prim = args.primaries if args.primaries else LARGE_N_PRIM
    nt = len(LARGE_THETAS)
    mesh = I.grf_foam(LARGE_GRID, LARGE_POROSITY, CORR, SEED)
    table = I.see_table()
    stream = torch.cuda.Stream(device=dev)
    ctx = rtmc.Context(local, stream=stream)
    ctx.load_see_tables(table, large_emission(rtmc))
    free0, total_mem = torch.cuda.mem_get_info(dev)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=LARGE_KIND)
    offset = shard.primary_offset(rank, n_prim)     # weak scaling: each rank its own primary ids
    if args.no_autotune:
        tuned = {}
    else:
        tuned = autotune.tune(ctx, [mid], [mesh.n_tri], [LARGE_E], LARGE_THETAS, kind=LARGE_KIND, cache_path=None,
                              device_name=torch.cuda.get_device_name(dev), n_sample=1_000_000)
    nb = dict(n_ebins=LARGE_BINS[0], n_abins=LARGE_BINS[1])
    desc = rtmc.run_desc(primary_offset=offset, profile=True, no_graph=True, **nb, **tuned)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step(d=desc, m=mid):
        return ctx.run_batch([m], [LARGE_E], LARGE_THETAS, n_prim, SEED, desc=d)

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rays = prims = launches = 0
    k = dict(trav_ms=0.0, trav_l=0, shade_ms=0.0, gen_ms=0.0, fin_ms=0.0, col_ms=0.0, col_rays=0, shade_bytes=0.0,
             retries=0)
    results = None
    for _ in range(args.steps):
        results, he, ha = step()
        r0 = results[0]
        rays += sum(r["rays"] for r in results)
        prims += sum(r["n_primaries"] for r in results)
        launches += r0["launches"]
        k["trav_ms"] += r0["ms_traverse"]
        k["trav_l"] += r0["traverse_launches"]
        k["shade_ms"] += r0["ms_shade"]
        k["gen_ms"] += r0["ms_generate"]
        k["fin_ms"] += r0["ms_finalize"]
        k["col_ms"] += r0["ms_column"]
        k["col_rays"] += r0["column_rays"]
        k["retries"] += r0["queue_retries"]
        # shade: queue entry (48 B) + hit (16 B) per ray, facet + normal (64 B) per facet stop,
        # 48 B per daughter written
        stops = sum(r["rays"] - r["escaped"] - r["lost"] for r in results)
        k["shade_bytes"] += sum(r["rays"] for r in results) * 64.0 + stops * 64.0 + \
            sum(r["emitted"] for r in results) * 48.0
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    mem_used = (total_mem - torch.cuda.mem_get_info(dev)[0]) / 1e9
    ms, (rays, prims) = shard.reduce_timing(ms, [rays, prims], device=dev)     # max time, summed work
    value = rays / (ms / 1e3)
    local_rays = sum(r["rays"] for r in results) * args.steps

    # the same step replayed from the captured CUDA graph
    gdesc = rtmc.run_desc(primary_offset=offset, **nb, **tuned)
    step(gdesc)
    barrier()
    g0 = time.perf_counter()
    g_steps = min(args.steps, 3)
    for _ in range(g_steps):
        step(gdesc)
    barrier()
    graph_ms = (time.perf_counter() - g0) * 1e3 / g_steps

    # plain form (rtmc_run item by item) and uncompressed 4-wide nodes on the same workload
    pdesc = rtmc.run_desc(primary_offset=offset, **nb)
    barrier()
    p0 = time.perf_counter()
    pres, _, _ = ctx.run(mid, [LARGE_E], LARGE_THETAS, n_prim, SEED, desc=pdesc)
    barrier()
    plain_s = time.perf_counter() - p0
    assert all(a["sum_k"] == b["sum_k"] for a, b in zip(pres, results)), "batched and plain tallies differ"
    w4 = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(w4, kind=rtmc.BVH_W4)
    step(gdesc, w4)
    barrier()
    w0 = time.perf_counter()
    wres, _, _ = step(gdesc, w4)
    barrier()
    w4_s = time.perf_counter() - w0
    assert all(a["sum_k"] == b["sum_k"] for a, b in zip(wres, results)), "4-wide FP32 and 8-bit tallies differ"
    ctx.unload_mesh(w4)

    # node-visit counts of a sample of the same workload (counting variant, untimed)
    cres, _, _ = ctx.run_batch([mid], [LARGE_E], LARGE_THETAS, max(n_prim // 20, 1), SEED,
                               desc=rtmc.run_desc(primary_offset=offset, count_visits=True, no_graph=True, **nb,
                                                  **tuned))
    c_rays = sum(r["rays"] for r in cres) - cres[0]["column_rays"]     # the hierarchy's rays
    visits, tests = cres[0]["node_visits"] / c_rays, cres[0]["tri_tests"] / c_rays
    b_ray = visits * NODE_BYTES[LARGE_KIND] + tests * TRI_BYTES + RAY_BYTES
    h_rays = local_rays - k["col_rays"]
    pk, pk_kind = peaks()
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    l2_gbs = ctx.probe_bandwidth(32 << 20, 10)          # L2-resident streaming read (own probe)
    hbm_read_gbs = ctx.probe_bandwidth(4 << 30, 5)      # HBM streaming read (own probe)
    rays_per_launch = h_rays / max(1, k["trav_l"])
    tr = measured_traffic("large_config", LARGE_KIND)
    trav = kernel_fields(k["trav_ms"], k["trav_l"], h_rays * b_ray, l2_gbs, "l2", {
        "kernel": f"k_traverse_ww ({NODE_NAME[LARGE_KIND]} nodes)", "bytes_per_ray": b_ray,
        "node_visits_per_ray": visits, "tri_tests_per_ray": tests, "rays_per_launch": rays_per_launch,
        "peak_kind": "own L2-resident streaming read probe (rtmc_probe_bandwidth, 32 MiB), this run",
        "dram_bytes_per_ray": tr,
        "hbm_achieved": tr * h_rays / (k["trav_ms"] / 1e3) / 1e9 if tr else None,
        "frac_of_measured_hbm": tr * h_rays / (k["trav_ms"] / 1e3) / 1e9 / hbm_peak if tr else None,
        "hbm_peak": hbm_peak, "hbm_peak_kind": f"{pk_kind} hbm_gbs (MEASURED_PEAKS.json)"})
    roofline = {"bound": "l2", "kernel": trav["kernel"], "achieved": trav["achieved"], "peak": l2_gbs,
                "unit": "GB/s", "frac": trav["frac"],
                "traffic": tr * rays_per_launch if tr is not None else None,
                "peak_kind": trav["peak_kind"], "bytes_per_ray": b_ray, "node_visits_per_ray": visits,
                "tri_tests_per_ray": tests, "traverse_ms_per_launch": trav["ms_per_launch"],
                "rays_per_launch": rays_per_launch, "traffic_bytes_per_ray": tr,
                "hbm_frac": trav["frac_of_measured_hbm"], "hbm_peak": hbm_peak,
                "hbm_read_probe_gbs": hbm_read_gbs, "l2_read_probe_gbs": l2_gbs}
    kernels = {"k_traverse_ww": trav,
               # one shade launch per generation of every chunk; every chunk of this workload runs
               # the hierarchy once per generation after the first
               "k_shade": kernel_fields(k["shade_ms"], k["trav_l"] // LARGE_MAX_GEN * (LARGE_MAX_GEN + 1),
                                        k["shade_bytes"], hbm_peak, "hbm", {
                   "peak_kind": f"{pk_kind} hbm_gbs", "note": "queue entry + hit per ray, facet + normal per "
                                                              "stop, 48 B per daughter written"}),
               "generate_ms": k["gen_ms"], "finalize_ms": k["fin_ms"],
               "k_trace_columns": {"ms": k["col_ms"], "rays": k["col_rays"],
                                   "note": "every primary: the vertical column grid at 0 degrees "
                                           "(k_trace_columns), the slanted grids at 10-80 degrees (k_trace_slant)"}}

    # end to end through the C ABI from pinned host memory
    tri_host = torch.from_numpy(mesh.tri.reshape(-1, 9)).pin_memory()
    h2d = tri_host.numel() * 4 + table.delta.nbytes + 8 * (1 + nt)
    d2h = nt * (rtmc.C.sizeof(rtmc.Result) + 8 * sum(LARGE_BINS))
    e2e_desc = rtmc.run_desc(primary_offset=offset, no_graph=True, **nb, **tuned)   # a new mesh every step
    barrier()
    e_t0 = time.perf_counter()
    e_rays = 0
    for _ in range(args.e2e_steps):
        m2 = ctx.load_mesh(tri_host, mesh.box)
        ctx.build_bvh(m2, kind=LARGE_KIND)
        rr, _, _ = ctx.run_batch([m2], [LARGE_E], LARGE_THETAS, n_prim, SEED, desc=e2e_desc)
        ctx.unload_mesh(m2)
        e_rays += sum(r["rays"] for r in rr)
    barrier()
    e_dt = time.perf_counter() - e_t0
    e_dt, (e_rays,) = shard.reduce_timing(e_dt, [e_rays], device=dev)

    extra = {}
    if rank == 0 and not args.no_paper:
        extra["paper_config"] = paper_config_summary(rtmc, I, dev, l2_gbs, hbm_peak)
    if rank == 0 and not args.no_forms:
        extra["batched_config"] = run_forms(rtmc, autotune, args.forms_primaries, local)

    cpu, sampled = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        per = args.cpu_sample_per_angle
        outs, o_rays, o_secs, thr = large_oracle_sample(mesh, table, per)
        cpu = {"value": o_rays / o_secs, "unit": "rays/s", "cores": thr, "kind": "oracle",
               "sample": f"the first {per} primaries of each of the {nt} angles at {LARGE_E:g} eV, tertiaries, "
                         f"same mesh (brute force over all {mesh.n_tri} triangles per ray segment); "
                         f"{o_secs:.1f} s"}
        same, esc_g, esc_o = 0, 0, 0
        mom = np.zeros((2, 2))                   # [gpu, oracle] x [sum E, sum E^2]
        ids = np.arange(per, dtype=np.uint64)
        for j, (th, o) in enumerate(zip(LARGE_THETAS, outs)):
            h = torch.zeros(per, dtype=torch.int64, device=dev)
            g, _, _ = ctx.run(mid, [LARGE_E], [th], per, SEED, desc=rtmc.run_desc(item_base=j, prim_hash=h, **nb))
            same += int(np.sum(h.cpu().numpy().view(np.uint64) == primary_hashes(o["records"], ids)))
            esc_g += g[0]["escaped"]
            esc_o += o["escaped"]
            mom += [[g[0]["e_sum"], g[0]["e2_sum"]], [o["e_sum"], o["e2_sum"]]]
        sampled = {"primaries": per * nt, "per_primary_event_hashes_equal": same,
                   "escapes_gpu": esc_g, "escapes_oracle": esc_o,
                   "sey_gpu": esc_g / (per * nt), "sey_oracle": esc_o / (per * nt),
                   "e_sum_rel_err": abs(mom[0, 0] - mom[1, 0]) / max(mom[1, 0], 1e-300),
                   "e2_sum_rel_err": abs(mom[0, 1] - mom[1, 1]) / max(mom[1, 1], 1e-300),
                   "note": "same primary ids and random streams on both sides; a hash covers every ray of the "
                           "primary's tree (fate, facet, count, energy and angle bins, wraps)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "primaries_per_s": prims / (ms / 1e3),
            "config": {"workload": large_workload_name(mesh.n_tri, n_prim), "n_tri": mesh.n_tri,
                       "energy_ev": LARGE_E, "theta_deg": LARGE_THETAS, "primaries_per_angle": n_prim,
                       "primaries_per_step": n_prim * nt * world,
                       "engine": f"rtmc_run_batch (multi-item queues), {NODE_NAME[LARGE_KIND]} BVH nodes, autotuned",
                       "autotuned": tuned,
                       "l2": "inputs larger than L2 (8-bit 4-wide nodes + triangles + normals "
                             f"{mesh.n_tri * (64 / 3 + 48 + 16) / 1e9:.2f} GB, ray queues several GB)",
                       "device_memory_gb": mem_used},
            "sey": [round(r["sey"], 6) for r in results],
            "sey_se": [round(r["sey_se"], 7) for r in results],
            "sey_error": {"statistical_se_max": max(r["sey_se"] for r in results),
                          "oracle_sample": sampled,
                          "parity_tests": "tests/test_gpu_parity.py (per-ray records, hit distances within a "
                                          "per-ray FP32 error bound, FP64 moments against the oracle)"},
            "graph_ms_per_step": graph_ms,
            "plain_form_rays_per_s": sum(r["rays"] for r in pres) / plain_s,
            "uncompressed_4wide_fp32_rays_per_s": sum(r["rays"] for r in wres) / w4_s,
            "queue_retries": k["retries"],
            "roofline": roofline,
            "kernels": kernels,
            "e2e": {"value": e_rays / e_dt, "unit": "rays/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


PREC_POROSITY = (0.4, 0.6, 0.8)
PREC_E, PREC_THETA = [100.0, 300.0, 700.0], [0.0, 60.0]


def precision_oracle_check(ctx, rtmc, O, mesh, table, mid, n_s):
    """The first n_s primaries of every (E, theta) item, on the oracle and on the GPU
    (same streams: item_base = item index).  Returns per-item (gpu, oracle) escape counts,
    oracle rays and the oracle's seconds and threads."""
    out, rays, secs = [], 0, 0.0
    threads = os.cpu_count() or 1
    for ie, e in enumerate(PREC_E):
        for it, th in enumerate(PREC_THETA):
            k = ie * len(PREC_THETA) + it
            g, _, _ = ctx.run(mid, [e], [th], n_s, SEED, desc=rtmc.run_desc(fp64_retest=True, item_base=k))
            t0 = time.perf_counter()
            o = O.run(mesh, table, e, th, n_s, SEED, item=k, n_threads=threads)
            secs += time.perf_counter() - t0
            rays += o["rays"]
            out.append((g[0]["escaped"], o["escaped"]))
    return out, rays, secs, threads


def run_precision(args):
    """Precision config: 128^3 foams at porosity 0.4 / 0.6 / 0.8, 1e7 primaries at 100, 300
    and 700 eV x incidence 0 and 60 deg.  8-bit quantised nodes (4-wide 64-byte by default,
    binary 32-byte with --prec-nodes q8), FP32 watertight tests, FP64 re-test of
    flagged hits, FP64 moments.  The same streams on FP32 nodes without re-test give the
    plain SEY; the first primaries of every item go through the oracle as well."""
    import torch
    import oracle as O
    from paper_1806_00205_gb300 import inputs as I
    from paper_1806_00205_gb300 import rtmc
    dev = torch.device("cuda", 0)
    n_prim = args.primaries
    table = I.see_table()
    meshes = [I.grf_foam(GRID, p, CORR, SEED) for p in PREC_POROSITY]
    stream = torch.cuda.Stream(device=dev)
    ctx = rtmc.Context(0, stream=stream)
    ctx.load_see_tables(table)
    mq, m32 = [], []
    qkind = PREC_NODES[args.prec_nodes]
    for m in meshes:
        for ids, kind in ((mq, qkind), (m32, rtmc.BVH_FP32)):
            a = ctx.load_mesh(m.tri, m.box)
            ctx.build_bvh(a, kind=kind)
            ids.append(a)
    desc = rtmc.run_desc(fp64_retest=True, profile=True)
    for _ in range(args.warmup):
        for a in mq:
            ctx.run(a, PREC_E, PREC_THETA, n_prim // 10, SEED, desc=desc)
    clocks = ClockSampler(0)
    torch.cuda.synchronize(dev)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rays = prims = launches = retested = trav_l = col_rays = 0
    trav_ms = 0.0
    prec = []
    for _ in range(args.steps):
        prec = []
        for a in mq:
            res, _, _ = ctx.run(a, PREC_E, PREC_THETA, n_prim, SEED, desc=desc)
            prec.append(res)
            rays += sum(r["rays"] for r in res)
            prims += sum(r["n_primaries"] for r in res)
            launches += sum(r["launches"] for r in res)
            retested += sum(r["retested"] for r in res)
            col_rays += sum(r["column_rays"] for r in res)
            trav_ms += sum(r["ms_traverse"] for r in res)
            trav_l += sum(r["traverse_launches"] for r in res)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    return finish_precision(args, ctx, rtmc, O, I, meshes, table, mq, m32, prec, n_prim, dict(
        rays=rays, prims=prims, launches=launches, retested=retested, trav_ms=trav_ms, trav_l=trav_l,
        ms=ms, clk=clk, stream=stream, col_rays=col_rays))


def finish_precision(args, ctx, rtmc, O, I, meshes, table, mq, m32, prec, n_prim, t):
    import torch
    dev = torch.device("cuda", 0)
    stream = t["stream"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    plain, plain_rays = [], 0
    for a in m32:
        res, _, _ = ctx.run(a, PREC_E, PREC_THETA, n_prim, SEED)
        plain.append(res)
        plain_rays += sum(r["rays"] for r in res)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = ev0.elapsed_time(ev1)
    items, max_d = [], 0.0
    for p, rq, rp in zip(PREC_POROSITY, prec, plain):
        for k, (a, b) in enumerate(zip(rq, rp)):
            d = abs(a["sey"] - b["sey"])
            max_d = max(max_d, d)
            items.append({"porosity": p, "energy_ev": PREC_E[k // len(PREC_THETA)],
                          "theta_deg": PREC_THETA[k % len(PREC_THETA)], "sey": round(a["sey"], 6),
                          "sey_se": round(a["sey_se"], 6), "sey_fp32_nodes": round(b["sey"], 6),
                          "abs_diff_vs_fp32": d, "retested_frac": a["retested"] / a["rays"]})
    cq, _, _ = ctx.run(mq[1], [300.0], [60.0], n_prim // 10, SEED,
                       desc=rtmc.run_desc(fp64_retest=True, count_visits=True))
    visits = cq[0]["node_visits"] / cq[0]["rays"]
    tests = cq[0]["tri_tests"] / cq[0]["rays"]
    qkind = PREC_NODES[args.prec_nodes]
    b_ray = visits * NODE_BYTES[qkind] + tests * TRI_BYTES + RAY_BYTES
    achieved = (t["rays"] - t["col_rays"]) * b_ray / (t["trav_ms"] / 1e3) / 1e9   # the hierarchy's rays
    pk, pk_kind = peaks()
    peak = float(pk.get("hbm_gbs", 6800.0))
    l2_gbs = ctx.probe_bandwidth(32 << 20, 10)          # L2-resident streaming read (own probe)
    ora, diffs, cpu = None, [], None
    if not args.no_cpu:
        n_s, o_rays, o_secs, thr, g_esc, o_esc = args.prec_oracle, 0, 0.0, 1, 0, 0
        for m, a in zip(meshes, mq):
            out, r, s, thr = precision_oracle_check(ctx, rtmc, O, m, table, a, n_s)
            o_rays += r
            o_secs += s
            for g, o in out:
                g_esc += g
                o_esc += o
                diffs.append(abs(g - o) / n_s)
        ora = {"primaries_per_item": n_s, "items": len(diffs), "sey_gpu": g_esc / (n_s * len(diffs)),
               "sey_oracle": o_esc / (n_s * len(diffs)), "max_abs_diff_per_item": max(diffs),
               "note": "first primaries of every item, same random streams on both sides"}
        cpu = {"value": o_rays / o_secs, "unit": "rays/s", "cores": thr, "kind": "oracle",
               "sample": f"{n_s} primaries per (porosity, E, theta) item, 18 items, brute force over "
                         f"all triangles per ray segment; {o_secs:.1f} s"}
    hosts = [torch.from_numpy(m.tri.reshape(-1, 9)).pin_memory() for m in meshes]
    torch.cuda.synchronize(dev)
    e0 = time.perf_counter()
    e_rays = 0
    ctx.load_see_tables(table)
    for h, m in zip(hosts, meshes):
        a = ctx.load_mesh(h, m.box)
        ctx.build_bvh(a, kind=qkind)
        rr, _, _ = ctx.run(a, PREC_E, PREC_THETA, n_prim, SEED, desc=rtmc.run_desc(fp64_retest=True))
        e_rays += sum(r["rays"] for r in rr)
        ctx.unload_mesh(a)
    e_dt = time.perf_counter() - e0
    ms, steps = t["ms"], args.steps
    ntri = [m.n_tri for m in meshes]
    line = {"metric": METRIC, "value": t["rays"] / (ms / 1e3), "unit": "rays/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "primaries_per_s": t["prims"] / (ms / 1e3),
            "config": {"workload": f"precision: {GRID}^3 periodic GRF foams at porosity 0.4 / 0.6 / 0.8 -> "
                                   f"{ntri} triangles, {PREC_NODE_NAME[qkind]} BVH, FP64 re-test of flagged "
                                   f"hits; {n_prim:.0e} "
                                   "primaries at 100 / 300 / 700 eV x incidence 0 / 60 deg",
                       "n_tri": ntri, "l2": "inputs larger than L2 (three meshes, 8-bit nodes + triangles)"},
            "sey_error": {"max_abs_diff_vs_fp32_nodes": max_d, "oracle_sample": ora,
                          "retested_frac": t["retested"] / t["rays"]},
            "items": items, "plain_fp32_rays_per_s": plain_rays / (plain_ms / 1e3),
            # the nodes and facets the daughters fetch are served by L2 (as on the other
            # configurations), so the bound is the L2 read probe; HBM beside it for reference
            "roofline": {"bound": "l2", "kernel": f"k_traverse_ww ({PREC_NODE_NAME[qkind]})", "achieved": achieved,
                         "peak": l2_gbs,
                         "unit": "GB/s", "frac": achieved / l2_gbs, "traffic": None,
                         "peak_kind": "own L2-resident streaming read probe (rtmc_probe_bandwidth, 32 MiB), this run",
                         "bytes_per_ray": b_ray, "node_visits_per_ray": visits, "tri_tests_per_ray": tests,
                         "hbm_peak": peak, "hbm_peak_kind": f"{pk_kind} hbm_gbs",
                         "frac_of_hbm_peak_if_all_from_hbm": achieved / peak},
            "e2e": {"value": e_rays / e_dt, "unit": "rays/s",
                    "h2d_bytes_per_step": sum(h.numel() * 4 for h in hosts) + table.delta.nbytes,
                    "d2h_bytes_per_step": 18 * (rtmc.C.sizeof(rtmc.Result) + 8 * (64 + 18))},
            "gpu_launches": t["launches"], "clocks": t["clk"], "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1806_00205_gb300 import autotune, rtmc, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_prim = args.primaries
    energies = ENERGIES[:args.energies]

    mesh, table = make_mesh()
    stream = torch.cuda.Stream(device=dev)
    ctx = rtmc.Context(local, stream=stream)
    ctx.load_see_tables(table)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=MAIN_KIND)
    offset = shard.primary_offset(rank, n_prim)   # weak scaling: each rank its own primary ids
    if args.no_autotune:
        tuned = {}
    else:
        tuned = autotune.tune(ctx, [mid], [mesh.n_tri], energies, [0.0], kind=MAIN_KIND, cache_path=None,
                              device_name=torch.cuda.get_device_name(dev))
    desc = rtmc.run_desc(primary_offset=offset, profile=True, no_graph=True, **tuned)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step(d=desc):
        return ctx.run_batch([mid], energies, [0.0], n_prim, SEED, desc=d)

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rays = prims = launches = trav_launches = col_rays = 0
    trav_ms = col_ms = 0.0
    results = None
    for _ in range(args.steps):
        results, _, _ = step()
        rays += sum(r["rays"] for r in results)
        prims += sum(r["n_primaries"] for r in results)
        launches += results[0]["launches"]
        trav_launches += results[0]["traverse_launches"]
        trav_ms += results[0]["ms_traverse"]
        col_ms += results[0]["ms_column"]           # generation 0 through the column grid
        col_rays += results[0]["column_rays"]
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms, (rays, prims) = shard.reduce_timing(ms, [rays, prims], device=dev)     # max time, summed work
    value = rays / (ms / 1e3)

    # the same steps replayed from the captured CUDA graph
    gdesc = rtmc.run_desc(primary_offset=offset, **tuned)
    step(gdesc)
    barrier()
    g0 = time.perf_counter()
    for _ in range(args.steps):
        step(gdesc)
    barrier()
    graph_ms = (time.perf_counter() - g0) * 1e3 / args.steps

    # plain form (rtmc_run item by item) on the same workload
    pdesc = rtmc.run_desc(primary_offset=offset)
    ctx.run(mid, energies, [0.0], n_prim, SEED, desc=pdesc)
    barrier()
    p0 = time.perf_counter()
    pres, _, _ = ctx.run(mid, energies, [0.0], n_prim, SEED, desc=pdesc)
    barrier()
    plain_s = time.perf_counter() - p0
    assert all(a["sum_k"] == b["sum_k"] for a, b in zip(pres, results)), "batched and plain tallies differ"

    # node-visit counts of the same workload (counting variant, untimed) -> algorithmic bytes
    cres, _, _ = ctx.run_batch([mid], energies, [0.0], n_prim, SEED,
                               desc=rtmc.run_desc(primary_offset=offset, count_visits=True, no_graph=True, **tuned))
    # the counters cover the hierarchy's rays only (not those of the column grid)
    c_rays = sum(r["rays"] for r in cres) - cres[0]["column_rays"]
    visits = cres[0]["node_visits"] / c_rays
    tests = cres[0]["tri_tests"] / c_rays
    b_ray = visits * NODE_BYTES[MAIN_KIND] + tests * TRI_BYTES + RAY_BYTES
    local_rays = sum(r["rays"] for r in results) * args.steps - col_rays
    achieved = local_rays * b_ray / (trav_ms / 1e3) / 1e9
    pk, pk_kind = peaks()
    peak = float(pk.get("hbm_gbs", 6800.0))
    rays_per_launch = local_rays / max(1, trav_launches)
    traffic_per_ray = measured_traffic()
    # DRAM bytes per traversal launch: the committed capture's bytes per ray (a
    # smaller case of the same kernel) times the rays one launch of this run traces
    traffic = traffic_per_ray * rays_per_launch if traffic_per_ray is not None else None
    l2_gbs = ctx.probe_bandwidth(32 << 20, 10)          # L2-resident streaming read (own probe)
    hbm_read_gbs = ctx.probe_bandwidth(4 << 30, 5)      # HBM streaming read (own probe)

    # end to end through the C ABI from pinned host memory
    tri_host = torch.from_numpy(mesh.tri.reshape(-1, 9)).pin_memory()
    h2d = tri_host.numel() * 4 + table.delta.nbytes + 8 * (len(energies) + 1)
    d2h = len(energies) * (rtmc.C.sizeof(rtmc.Result) + 8 * (64 + 18))
    e2e_desc = rtmc.run_desc(primary_offset=offset, no_graph=True, **tuned)
    barrier()
    e_t0 = time.perf_counter()
    e_rays = 0
    for _ in range(args.e2e_steps):
        m2 = ctx.load_mesh(tri_host, mesh.box)
        ctx.build_bvh(m2, kind=MAIN_KIND)
        rr, _, _ = ctx.run_batch([m2], energies, [0.0], n_prim, SEED, desc=e2e_desc)
        ctx.unload_mesh(m2)
        e_rays += sum(r["rays"] for r in rr)
    barrier()
    e_dt = time.perf_counter() - e_t0
    e_dt, (e_rays,) = shard.reduce_timing(e_dt, [e_rays], device=dev)

    forms = None
    if rank == 0 and not args.no_forms:
        forms = run_forms(rtmc, autotune, args.forms_primaries, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        r, dt, threads = cpu_oracle_sample(mesh, table, args.cpu_sample)
        cpu = {"value": r["rays"] / dt, "unit": "rays/s", "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_sample} primaries at 500 eV, normal incidence, same mesh "
                         f"(brute force over all {mesh.n_tri} triangles per ray segment); {dt:.1f} s",
               "sey_sample": r["sey"], "sey_sample_se": r["sey_se"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "primaries_per_s": prims / (ms / 1e3),
            "config": {"workload": workload_name(mesh.n_tri, n_prim, energies), "n_tri": mesh.n_tri,
                       "energies_ev": energies, "theta_deg": [0.0], "primaries_per_energy": n_prim,
                       "primaries_per_step": n_prim * len(energies) * world,
                       "engine": "rtmc_run_batch (multi-item queues), 4-wide FP32 BVH nodes, autotuned",
                       "autotuned": tuned,
                       "l2": "inputs larger than L2 (BVH nodes + triangles + normals "
                             f"{(mesh.n_tri - 1) * 64 / 1e6 + mesh.n_tri * 64 / 1e6:.0f} MB, ray queues > 1 GB)"},
            "graph_ms_per_step": graph_ms,
            "plain_form_rays_per_s": sum(r["rays"] for r in pres) / plain_s,
            "sey": [round(r["sey"], 6) for r in results],
            "sey_se_max": max(r["sey_se"] for r in results),
            "sey_error": "GPU vs FP64 oracle: event records bit-exact on >= 99.99% of rays and SEY within "
                         "min(3 SE, 1e-3) (tests/test_gpu_parity.py); statistical SE per energy above",
            "roofline": {"bound": "l2", "kernel": "k_traverse_ww (4-wide nodes)", "achieved": achieved,
                         "peak": l2_gbs, "unit": "GB/s", "frac": achieved / l2_gbs, "traffic": traffic,
                         "peak_kind": "own L2-resident streaming read probe (rtmc_probe_bandwidth, 32 MiB), this run",
                         "hbm_peak": peak, "hbm_peak_kind": f"{pk_kind} hbm_gbs",
                         "hbm_frac": (traffic_per_ray * rays_per_launch / (trav_ms / max(1, trav_launches) / 1e3)
                                      / 1e9 / peak) if traffic_per_ray is not None else None,
                         "bytes_per_ray": b_ray,
                         "node_visits_per_ray": visits, "tri_tests_per_ray": tests,
                         "traverse_ms_per_launch": trav_ms / max(1, trav_launches),
                         "rays_per_launch": rays_per_launch, "traffic_bytes_per_ray": traffic_per_ray,
                         "l2_read_probe_gbs": l2_gbs, "hbm_read_probe_gbs": hbm_read_gbs},
            "column_kernel": {"kernel": "k_trace_columns (generation 0, normal incidence)",
                              "ms_per_step": col_ms / args.steps, "rays_per_step": col_rays / args.steps,
                              "rays_per_s": col_rays / (col_ms / 1e3) if col_ms > 0 else None},
            "e2e": {"value": e_rays / e_dt, "unit": "rays/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
            "batched_config": forms,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--primaries", type=int, default=0,
                    help="primaries per item (0: the configuration's own, 1e8 large / 1e7 paper and precision)")
    ap.add_argument("--energies", type=int, default=len(ENERGIES))
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=1024)
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="reference arm: primaries per step (0: 9 large, 256 paper)")
    ap.add_argument("--cpu-sample-per-angle", type=int, default=6,
                    help="large config: primaries per angle for the CPU baseline and the sampled parity")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper-config summary of the default line")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched-config form comparison")
    ap.add_argument("--forms-primaries", type=int, default=1_000_000)
    ap.add_argument("--no-autotune", action="store_true", help="default launch parameters (profiling runs)")
    ap.add_argument("--config", choices=("paper", "large", "precision"), default="large",
                    help="large: 256^3 foam, 9 angles x 1e8, tertiaries (default); paper: 128^3 foam, 20 energies "
                         "x 1e7; precision: 3 porosities, 8-bit nodes + FP64 re-test, 3 energies x 2 angles")
    ap.add_argument("--prec-nodes", choices=tuple(PREC_NODES), default="q4",
                    help="precision config: 8-bit node format (q4: 4-wide 64-byte nodes, q8: binary 32-byte)")
    ap.add_argument("--prec-oracle", type=int, default=64,
                    help="precision config: primaries per item checked against the oracle")
    args = ap.parse_args()
    if args.ref_sample <= 0:
        args.ref_sample = 9 if args.config == "large" else 256
    if args.primaries <= 0 and args.config != "large":
        args.primaries = N_PRIM
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "large":
        run_large(args)
    elif args.config == "precision":
        run_precision(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
