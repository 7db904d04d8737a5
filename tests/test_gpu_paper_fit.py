"""Paper-fit emission model on the GPU (Section 2.2: Eq. 6 yield with
stochastic rounding, Eq. 7 secondary energy, two-daughter split, re-emission
above E_c), against the FP64 oracle through the C ABI (needs a GB300)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1806_00205_gb300 import inputs as I
from tests.parity import check_moments, compare_records, paper_fit_energy_gain

pytestmark = pytest.mark.gpu
TABLE = I.see_table()


@pytest.fixture(scope="module")
def pctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_00205_gb300 import rtmc
    c = rtmc.Context(0)
    c.load_see_tables(TABLE, rtmc.paper_emission())
    yield c, rtmc
    c.close()


def _mesh_id(ctx, mesh):
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid)
    return mid


@pytest.mark.parametrize("energy,theta", [(416.0, 0.0), (1500.0, 30.0)])
def test_paper_fit_records_match_oracle(pctx, energy, theta):
    """Whole ray trees (up to 6 generations) record by record on a small foam."""
    ctx, rtmc = pctx
    mesh = I.grf_foam(16, 0.5)
    mid = _mesh_id(ctx, mesh)
    n = 20_000
    g = ctx.run_records(mid, energy, theta, n, seed=23, desc=rtmc.run_desc(n_zbins=32))
    o = O.run(mesh, TABLE, energy, theta, n, seed=23, emission=O.paper_emission(), records=True, n_zbins=32)
    st = compare_records(g["records"], o["records"], mesh=mesh, energy_gain=paper_fit_energy_gain)
    assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
    check_moments(g, o, st)
    assert g["regenerated"] > 0 and g["rays"] == n + g["emitted"]
    assert abs(int(g["rays"]) - int(o["rays"])) <= max(3, 1e-4 * o["rays"])
    assert np.abs(g["hist_z"].astype(np.int64) - o["hist_z"]).sum() <= max(6, int(3e-4 * o["rays"]))


def test_paper_fit_flat_plane_gpu(pctx):
    """E[SEY] = gamma(E, 0) of Eq. 6 on a flat surface, with 4M primaries."""
    ctx, rtmc = pctx
    fp = I.flat_plane(160.0)
    mid = _mesh_id(ctx, fp)
    n = 4_000_000
    res, _, _ = ctx.run(mid, [416.0, 800.0], [0.0], n, 41)
    for r, e in zip(res, (416.0, 800.0)):
        g = O.gamma_fit(e, 0.0)
        f = g - math.floor(g)
        assert r["lost"] == 0 and r["escaped"] == r["emitted"]
        assert abs(r["sey"] - g) < 4.0 * math.sqrt(f * (1 - f) / n), (e, r["sey"], g)


def test_random_incidence_yields_more_at_high_energy(pctx):
    """Section 3.2 on a 4 % solid foam with the paper's physics: random incidence
    yields more than normal incidence at 1 keV, and normal-incidence electrons
    stop deeper at 100 eV."""
    ctx, rtmc = pctx
    mesh = I.grf_foam(32, 0.96)
    mid = _mesh_id(ctx, mesh)
    n = 1_000_000
    r, _, _ = ctx.run(mid, [1000.0], [0.0], n, 9)
    q, _, _ = ctx.run(mid, [1000.0], [0.0], n, 9, desc=rtmc.run_desc(random_polar=True))
    assert q[0]["sey"] - r[0]["sey"] > 4.0 * math.hypot(q[0]["sey_se"], r[0]["sey_se"])
    box, nz = mesh.box, 64
    c = (np.arange(nz) + 0.5) * (box.z_top - box.z_min) / nz
    mean = []
    for polar in (False, True):
        s, _, _ = ctx.run(mid, [100.0], [0.0], n, 9, desc=rtmc.run_desc(random_polar=polar, n_zbins=nz))
        hz = s[0]["hist_z"].astype(np.float64)
        mean.append((hz * c).sum() / hz.sum())
    assert mean[0] > mean[1] + 5.0, mean
