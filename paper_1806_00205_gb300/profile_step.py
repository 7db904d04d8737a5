"""One batched RTMC step for a profiler, and summaries of the profiler's CSV output.

Run mode (the command a profiler wraps)::

    python -m paper_1806_00205_gb300.profile_step --grid 192 --primaries 2000000 --angles 0,40,80

builds a periodic GRF foam (the synthetic porous-surface recipe of the inputs module), its
BVH and column grids, runs ``--warmup`` batched steps (``rtmc_run_batch``: every incidence
energy and angle one item, tertiaries for secondaries above ``--regen-min`` eV), then brackets
``--steps`` more with ``cudaProfilerStart`` / ``cudaProfilerStop`` so that ``ncu
--profile-from-start off`` sees only those launches, and prints one JSON line with the
rays traced and the device time of each phase.  With ``--build`` the bracket covers the mesh
upload, the BVH and vertical-grid build and one step instead, whose first use of each
oblique angle builds that angle's slanted grid (no warm-up).

Summary modes (no GPU)::

    python -m paper_1806_00205_gb300.profile_step --launches launches.csv
    python -m paper_1806_00205_gb300.profile_step --traffic dram.csv --step-json step.json

``--launches`` turns an ``ncu --metrics gpu__time_duration.sum --csv`` launch list into a
table of kernels with launches, total time and share; ``--traffic`` turns an ``ncu
--metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum -k
regex:k_traverse_ww --csv`` capture plus the run mode's JSON line into DRAM bytes per
traversal ray (the hierarchy's rays: every ray the column grids do not take).
"""
import argparse
import csv
import hashlib
import io
import json
import os
import re
import sys

PKG = os.path.dirname(os.path.abspath(__file__))


def traverse_sha():
    """Identity of the traversal kernel's sources: a traffic record is valid for this one only."""
    h = hashlib.sha256()
    for f in ("rtmc_traverse.cu", "rtmc_device.cuh"):
        h.update(open(os.path.join(PKG, "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def run_step(a):
    import torch
    from . import inputs as I
    from . import rtmc

    mesh = I.grf_foam(a.grid, a.porosity, 2.0, a.seed)
    ctx = rtmc.Context(0)
    ctx.load_see_tables(I.see_table(), rtmc.Emission(regen_min_ev=a.regen_min, max_generation=a.max_generation))
    thetas = [float(x) for x in a.angles.split(",")]
    energies = [float(x) for x in a.energies.split(",")]
    desc = rtmc.run_desc(n_ebins=128, n_abins=36, no_graph=True, profile=True, chunk=a.chunk)
    cudart = torch.cuda.cudart()
    if a.build:
        # the profiled range: mesh upload, BVH and vertical grid, then one step,
        # whose first use of each oblique angle builds that angle's slanted grid
        torch.cuda.synchronize()
        cudart.cudaProfilerStart()
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=a.kind)

    def step():
        return ctx.run_batch([mid], energies, thetas, a.primaries, a.seed, desc=desc)

    if not a.build:
        for _ in range(a.warmup):
            step()
        torch.cuda.synchronize()
        cudart.cudaProfilerStart()
    out = []
    for _ in range(a.steps):
        res, _, _ = step()
        r0 = res[0]
        rays = sum(r["rays"] for r in res)
        out.append(dict(rays=rays, column_rays=r0["column_rays"], hierarchy_rays=rays - r0["column_rays"],
                        ms_traverse=r0["ms_traverse"], ms_column=r0["ms_column"], ms_shade=r0["ms_shade"],
                        ms_generate=r0["ms_generate"], ms_finalize=r0["ms_finalize"],
                        launches=r0["launches"], traverse_launches=r0["traverse_launches"]))
    torch.cuda.synchronize()
    cudart.cudaProfilerStop()
    print(json.dumps(dict(grid=a.grid, porosity=a.porosity, n_tri=mesh.n_tri, kind=a.kind, energies=energies,
                          angles=thetas, primaries=a.primaries, max_generation=a.max_generation, steps=out,
                          kernel_sha=traverse_sha())),
          flush=True)
    ctx.close()


def read_ncu_csv(path):
    """Rows of an ncu --csv log (leading ==PROF== lines skipped), one dict per metric value."""
    text = open(path).read()
    start = text.find('"ID"')
    if start < 0:
        raise SystemExit(f"{path}: no ncu CSV header")
    return list(csv.DictReader(io.StringIO(text[start:])))


def kernel_label(name):
    """Kernel name without the parameter list and anonymous-namespace prefix."""
    name = name.replace("void ", "").replace("unnamed>::", "").replace("(anonymous namespace)::", "")
    depth = 0
    for i, ch in enumerate(name):
        if ch == "<":
            depth += 1
        elif ch == ">":
            depth -= 1
        elif ch == "(" and depth == 0:
            return name[:i]
    return name


def summarize_launches(path):
    per = {}
    for r in read_ncu_csv(path):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        scale = {"ns": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "nsecond": 1e-6}
        ms = float(r["Metric Value"].replace(",", "")) * scale.get(r["Metric Unit"], 1e-6)
        k = kernel_label(r["Kernel Name"])
        n, t = per.get(k, (0, 0.0))
        per[k] = (n + 1, t + ms)
    total = sum(t for _, t in per.values())
    lines = ["| kernel | launches | total ms | share |", "|---|---|---|---|"]
    for k, (n, t) in sorted(per.items(), key=lambda kv: -kv[1][1]):
        lines.append(f"| `{k}` | {n} | {t:.3f} | {100.0 * t / total:.1f} % |")
    lines.append(f"| all | {sum(n for n, _ in per.values())} | {total:.3f} | 100 % |")
    print("\n".join(lines))


def summarize_traffic(path, step_json, kind):
    launches = {}
    for r in read_ncu_csv(path):
        if not re.search(r"k_traverse_ww", r["Kernel Name"]):
            continue
        d = launches.setdefault(int(r["ID"]), {"kernel": kernel_label(r["Kernel Name"])})
        v = float(r["Metric Value"].replace(",", ""))
        if r["Metric Name"] == "dram__bytes_read.sum":
            d["dram_read_bytes"] = v * {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}[r["Metric Unit"]]
        elif r["Metric Name"] == "dram__bytes_write.sum":
            d["dram_write_bytes"] = v * {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}[r["Metric Unit"]]
        elif r["Metric Name"] == "gpu__time_duration.sum":
            d["ms"] = v * {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0}[r["Metric Unit"]]
    step = None
    for line in open(step_json):
        if line.startswith("{"):
            step = json.loads(line)
    if step is None:
        raise SystemExit(f"{step_json}: no JSON line")
    hier = sum(s["hierarchy_rays"] for s in step["steps"])
    lst = [launches[i] for i in sorted(launches)]
    tot = sum(d.get("dram_read_bytes", 0.0) + d.get("dram_write_bytes", 0.0) for d in lst)
    rec = dict(kernel=lst[0]["kernel"] if lst else None, kernel_sha=step["kernel_sha"], node_format=kind,
               dram_bytes_per_ray=tot / hier if hier else None, hierarchy_rays=hier,
               workload=dict((k, step[k]) for k in ("grid", "porosity", "n_tri", "energies", "angles", "primaries",
                                                    "max_generation")),
               launches=lst)
    print(json.dumps(rec, indent=1))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--grid", type=int, default=192, help="foam voxels per side")
    ap.add_argument("--porosity", type=float, default=0.7)
    ap.add_argument("--kind", type=int, default=3, help="BVH node format (3: 4-wide 8-bit boxes)")
    ap.add_argument("--primaries", type=int, default=2_000_000, help="per item (energy, angle)")
    ap.add_argument("--angles", default="0,40,80", help="incidence angles, degrees")
    ap.add_argument("--energies", default="500", help="primary energies, eV (every energy x angle is one item)")
    ap.add_argument("--regen-min", type=float, default=20.0)
    ap.add_argument("--max-generation", type=int, default=2)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--seed", type=int, default=1806)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--build", action="store_true",
                    help="profile the mesh upload, the BVH and grid builds and one step instead (no warm-up)")
    ap.add_argument("--launches", metavar="CSV", help="summarise an ncu launch list")
    ap.add_argument("--traffic", metavar="CSV", help="DRAM bytes per traversal ray from an ncu capture")
    ap.add_argument("--step-json", metavar="FILE", help="run-mode output belonging to --traffic")
    a = ap.parse_args(argv)
    if a.launches:
        summarize_launches(a.launches)
    elif a.traffic:
        if not a.step_json:
            ap.error("--traffic needs --step-json")
        summarize_traffic(a.traffic, a.step_json, a.kind)
    else:
        run_step(a)


if __name__ == "__main__":
    main(sys.argv[1:])
