"""Batched form: many (mesh, energy, angle) items in one captured CUDA graph (GB300)."""
import numpy as np
import pytest

from paper_1806_00205_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TABLE = I.see_table()
INT_KEYS = ("rays", "escaped", "absorbed_low", "absorbed_other", "emitters", "emitted", "capped", "lost",
            "wraps", "sum_k", "sum_k2")


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_00205_gb300 import rtmc
    c = rtmc.Context(0)
    c.load_see_tables(TABLE)
    meshes = [I.grf_foam(16, 0.5), I.grf_foam(24, 0.8, seed=3), I.grf_foam(12, 0.35, seed=4),
              I.grf_foam(16, 0.6, seed=5)]
    ids = []
    for k, m in enumerate(meshes):
        mid = c.load_mesh(m.tri, m.box)
        c.build_bvh(mid, kind=(rtmc.BVH_FP32, rtmc.BVH_Q8, rtmc.BVH_W4, rtmc.BVH_Q4)[k])
        ids.append(mid)
    yield c, ids, rtmc
    c.close()


def test_batch_items_equal_plain_runs(setup):
    """Item k of the batch uses the streams of a plain run with item_base = k: identical tallies."""
    ctx, ids, rtmc = setup
    energies, thetas, n = [80.0, 450.0], [0.0, 40.0, 75.0], 30_000
    desc = rtmc.run_desc(chunk=50_000)          # chunks span item boundaries
    res, he, ha = ctx.run_batch(ids, energies, thetas, n, 77, desc=desc)
    per_mesh = len(energies) * len(thetas)
    for mi, mid in enumerate(ids):
        plain, phe, pha = ctx.run(mid, energies, thetas, n, 77, desc=rtmc.run_desc(item_base=mi * per_mesh))
        for j in range(per_mesh):
            b = res[mi * per_mesh + j]
            for k in INT_KEYS:
                assert b[k] == plain[j][k], (mi, j, k, b[k], plain[j][k])
            assert abs(b["e_sum"] - plain[j]["e_sum"]) <= 1e-9 * max(1.0, plain[j]["e_sum"])
            assert np.array_equal(he[mi * per_mesh + j], phe[j]) and np.array_equal(ha[mi * per_mesh + j], pha[j])


def test_batch_random_incidence_depth_profile_equals_plain_runs(setup):
    ctx, ids, rtmc = setup
    energies, thetas, n = [150.0, 900.0], [0.0], 25_000
    desc = rtmc.run_desc(random_polar=True, n_zbins=48, chunk=30_000)
    res, he, _ = ctx.run_batch(ids, energies, thetas, n, 31, desc=desc)
    per_mesh = len(energies) * len(thetas)
    for mi, mid in enumerate(ids):
        plain, phe, _ = ctx.run(mid, energies, thetas, n, 31,
                                desc=rtmc.run_desc(random_polar=True, n_zbins=48, item_base=mi * per_mesh))
        for j in range(per_mesh):
            b = res[mi * per_mesh + j]
            for k in INT_KEYS:
                assert b[k] == plain[j][k], (mi, j, k, b[k], plain[j][k])
            assert np.array_equal(b["hist_z"], plain[j]["hist_z"])
            assert b["hist_z"].sum() == b["emitters"] + b["absorbed_low"] + b["absorbed_other"]
            assert np.array_equal(he[mi * per_mesh + j], phe[j])


def test_batch_fp64_retest_equals_plain_runs(setup):
    """The FP64 re-test decides each ambiguous facet against the best hit of its cell, so a
    ray's result does not depend on the launch: batched items equal plain runs with the
    re-test on, on binary FP32, Q8 and 4-wide meshes, and the batch's re-test count (a
    batch total) is the sum of the plain runs'.  Both send the normal-incidence items'
    primaries through the column grid and every other ray through the hierarchy (the
    count depends on which facets a path tests)."""
    ctx, ids, rtmc = setup
    energies, thetas, n = [120.0, 600.0], [0.0, 70.0], 40_000
    res, he, _ = ctx.run_batch(ids, energies, thetas, n, 13, desc=rtmc.run_desc(fp64_retest=True, chunk=70_000))
    per_mesh = len(energies) * len(thetas)
    total = 0
    for mi, mid in enumerate(ids):
        plain, phe, _ = ctx.run(mid, energies, thetas, n, 13,
                                desc=rtmc.run_desc(fp64_retest=True, item_base=mi * per_mesh))
        total += sum(r["retested"] for r in plain)
        for j in range(per_mesh):
            b = res[mi * per_mesh + j]
            for k in INT_KEYS:
                assert b[k] == plain[j][k], (mi, j, k, b[k], plain[j][k])
            assert np.array_equal(he[mi * per_mesh + j], phe[j])
    assert res[0]["retested"] == total > 0


def test_batch_graph_replay_equals_eager(setup):
    ctx, ids, rtmc = setup
    args = (ids, [100.0, 700.0], [0.0, 60.0], 20_000, 5)
    eager, he0, _ = ctx.run_batch(*args, desc=rtmc.run_desc(no_graph=True))
    first, he1, _ = ctx.run_batch(*args)            # captures the graph
    again, he2, _ = ctx.run_batch(*args)            # replays it
    for a, b, c in zip(eager, first, again):
        for k in INT_KEYS:
            assert a[k] == b[k] == c[k]
    assert np.array_equal(he0, he1) and np.array_equal(he1, he2)
    # a different shape re-captures; results stay consistent with a plain run
    other, _, _ = ctx.run_batch(ids[:1], [300.0], [0.0], 10_000, 5)
    plain, _, _ = ctx.run(ids[0], [300.0], [0.0], 10_000, 5)
    assert other[0]["sum_k"] == plain[0]["sum_k"]


def test_batch_rejects_what_it_cannot_do(setup):
    ctx, ids, rtmc = setup
    with pytest.raises(rtmc.RtmcError):
        ctx.run_batch([12345], [300.0], [0.0], 10, 1)
    with pytest.raises(rtmc.RtmcError):
        ctx.run_batch(ids, [300.0], [95.0], 10, 1)


def test_batch_column_grids_for_fixed_incidence_items(setup):
    """In a batch that mixes angles, every fixed-incidence item's primaries take a column
    grid (vertical or slanted, several directions in one chunk), random azimuths the
    hierarchy; every item keeps the tallies of its plain run."""
    ctx, ids, rtmc = setup
    energies, thetas, n = [200.0, 650.0], [0.0, 30.0, 0.0, 60.0], 12_000
    res, he, _ = ctx.run_batch(ids, energies, thetas, n, 41, desc=rtmc.run_desc(chunk=20_000))
    per_mesh = len(energies) * len(thetas)
    assert res[0]["column_rays"] == len(ids) * per_mesh * n
    ra, _, _ = ctx.run_batch(ids, energies, thetas, n, 41, desc=rtmc.run_desc(chunk=20_000, random_azimuth=True))
    n_vertical = sum(1 for t in thetas if t == 0.0) * len(energies)
    assert ra[0]["column_rays"] == len(ids) * n_vertical * n
    for mi, mid in enumerate(ids):
        plain, phe, _ = ctx.run(mid, energies, thetas, n, 41, desc=rtmc.run_desc(item_base=mi * per_mesh))
        for j in range(per_mesh):
            b = res[mi * per_mesh + j]
            for k in INT_KEYS:
                assert b[k] == plain[j][k], (mi, j, k, b[k], plain[j][k])
            assert np.array_equal(he[mi * per_mesh + j], phe[j])


def test_batch_graph_follows_angles_and_rebuilds(setup):
    """A cached batch graph is recorded again when the angles change the kernels it holds
    (the column grid at normal incidence, the hierarchy otherwise) or a mesh is rebuilt."""
    ctx, ids, rtmc = setup
    mid, n = ids[2], 20_000
    a, _, _ = ctx.run_batch([mid], [300.0], [0.0], n, 9)       # records the vertical column grid
    b, _, _ = ctx.run_batch([mid], [300.0], [35.0], n, 9)      # same shape, oblique: the slanted grid
    pb, _, _ = ctx.run(mid, [300.0], [35.0], n, 9)
    r, _, _ = ctx.run_batch([mid], [300.0], [35.0], n, 9, desc=rtmc.run_desc(random_azimuth=True))
    assert a[0]["column_rays"] == n and b[0]["column_rays"] == n and r[0]["column_rays"] == 0
    for k in INT_KEYS:
        assert b[0][k] == pb[0][k], k
    ctx.build_bvh(mid, kind=rtmc.BVH_W4)                         # new device arrays
    c, _, _ = ctx.run_batch([mid], [300.0], [0.0], n, 9)
    for k in INT_KEYS:
        assert c[0][k] == a[0][k], k


@pytest.mark.parametrize("model", ["tertiaries", "paper_fit"])
def test_batch_deeper_trees_equal_plain_runs(model):
    """Every generation the emission allows runs batched (Section 2.2's ray tree):
    tertiaries above 20 eV (the large config's physics) and the paper's own fits
    with up to 6 generations give each item the tallies of a plain run, on all
    four node formats, with and without the column grid for generation 0."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_00205_gb300 import rtmc
    em = rtmc.Emission(regen_min_ev=20.0, max_generation=2) if model == "tertiaries" else rtmc.paper_emission()
    energies = [500.0, 1500.0] if model == "tertiaries" else [416.0, 2000.0]
    with rtmc.Context(0) as c:
        c.load_see_tables(TABLE, em)
        meshes = [I.grf_foam(16, 0.6, seed=6), I.grf_foam(24, 0.9, seed=7)]
        for kind in (rtmc.BVH_FP32, rtmc.BVH_Q8, rtmc.BVH_W4, rtmc.BVH_Q4):
            ids = []
            for m in meshes:
                mid = c.load_mesh(m.tri, m.box)
                c.build_bvh(mid, kind=kind)
                ids.append(mid)
            for thetas in ([0.0], [0.0, 50.0]):
                n = 15_000
                res, he, ha = c.run_batch(ids, energies, thetas, n, 19, desc=rtmc.run_desc(chunk=40_000))
                per_mesh = len(energies) * len(thetas)
                deep = 0
                for mi, mid in enumerate(ids):
                    plain, phe, pha = c.run(mid, energies, thetas, n, 19,
                                            desc=rtmc.run_desc(item_base=mi * per_mesh))
                    for j in range(per_mesh):
                        b = res[mi * per_mesh + j]
                        for k in INT_KEYS + ("regenerated",):
                            assert b[k] == plain[j][k], (kind, thetas, mi, j, k, b[k], plain[j][k])
                        assert abs(b["e_sum"] - plain[j]["e_sum"]) <= 1e-9 * max(1.0, plain[j]["e_sum"])
                        assert np.array_equal(he[mi * per_mesh + j], phe[j])
                        assert np.array_equal(ha[mi * per_mesh + j], pha[j])
                        deep += b["regenerated"]
                assert deep > 0
            for mid in ids:
                c.unload_mesh(mid)


def test_batch_equals_plain_runs_at_oblique_angles_at_scale(setup):
    """1e6 primaries per angle at nine angles: the batched and the plain path give each
    item identical tallies (both take the incidence direction as the FP64 angle's sine
    and cosine rounded once to FP32, the direction nearest the oracle's)."""
    ctx, ids, rtmc = setup
    thetas = [10.0 * j for j in range(9)]
    res, he, ha = ctx.run_batch([ids[3]], [500.0], thetas, 1_000_000, 1806)
    plain, phe, pha = ctx.run(ids[3], [500.0], thetas, 1_000_000, 1806)
    for j in range(len(thetas)):
        for k in INT_KEYS:
            assert res[j][k] == plain[j][k], (j, k, res[j][k], plain[j][k])
    assert np.array_equal(he, phe) and np.array_equal(ha, pha)
