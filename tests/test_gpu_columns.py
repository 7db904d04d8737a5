"""Column grids: generation 0 at fixed incidence traced through per-pixel facet lists
sorted by top z instead of the hierarchy (GB300) -- vertical lists at normal incidence,
slanted lists (facets projected along the ray direction, with the wraps before each)
at oblique incidence.  Same facet tests and the hierarchy's own wrap replay, so the
same hit records: every tally, histogram and per-primary event hash equals the
hierarchy's."""
import numpy as np
import pytest

from paper_1806_00205_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TABLE = I.see_table()
INT_KEYS = ("rays", "escaped", "absorbed_low", "absorbed_other", "emitters", "emitted", "capped", "lost",
            "wraps", "sum_k", "sum_k2", "retested")


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_00205_gb300 import rtmc
    c = rtmc.Context(0)
    c.load_see_tables(TABLE)
    yield c
    c.close()


def _both(ctx, mid, energy, n, seed, **kw):
    import torch
    from paper_1806_00205_gb300 import rtmc
    hc = torch.zeros(n, dtype=torch.int64, device="cuda")
    hb = torch.zeros(n, dtype=torch.int64, device="cuda")
    col = ctx.run(mid, [energy], [0.0], n, seed, desc=rtmc.run_desc(prim_hash=hc, **kw))
    bvh = ctx.run(mid, [energy], [0.0], n, seed, desc=rtmc.run_desc(prim_hash=hb, traversal=2, **kw))
    return col, bvh, hc, hb


@pytest.mark.parametrize("grid,porosity,kind", [(16, 0.5, 0), (48, 0.3, 1), (48, 0.8, 2), (128, 0.6, 2),
                                                (128, 0.6, 1)])
@pytest.mark.parametrize("retest", [False, True])
def test_column_grid_equals_hierarchy(ctx, grid, porosity, kind, retest):
    import torch
    mesh = I.grf_foam(grid, porosity)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=kind)
    n = 200_000 if grid < 128 else 1_000_000
    for energy in (60.0, 400.0):
        (rc, hec, hac), (rb, heb, hab), hc, hb = _both(ctx, mid, energy, n, 91, fp64_retest=retest)
        a, b = rc[0], rb[0]
        assert a["column_rays"] == n and b["column_rays"] == 0
        for k in INT_KEYS[:-1]:
            assert a[k] == b[k], (energy, k, a[k], b[k])
        # which near-edge facets get an FP64 decision depends on the facets a path
        # tests (the grid and the hierarchy test different sets), not the outcome
        assert (a["retested"] > 0) == (b["retested"] > 0) or not retest
        assert abs(a["e_sum"] - b["e_sum"]) <= 1e-9 * max(1.0, b["e_sum"])
        assert np.array_equal(hec, heb) and np.array_equal(hac, hab)
        assert torch.equal(hc, hb)
    ctx.unload_mesh(mid)


def test_vertical_grid_only_at_normal_incidence(ctx):
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(24, 0.6, seed=5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=rtmc.BVH_W4)
    n = 20_000
    r0, _, _ = ctx.run(mid, [300.0], [0.0, 30.0], n, 3, desc=rtmc.run_desc(fp64_retest=True))
    assert r0[0]["column_rays"] == n and r0[1]["column_rays"] == 0      # no slanted grid with the FP64 re-test
    rp, _, _ = ctx.run(mid, [300.0], [0.0], n, 3, desc=rtmc.run_desc(random_polar=True))
    assert rp[0]["column_rays"] == 0
    ra, _, _ = ctx.run(mid, [300.0], [0.0], n, 3, desc=rtmc.run_desc(random_azimuth=True))
    rb, _, _ = ctx.run(mid, [300.0], [0.0], n, 3, desc=rtmc.run_desc(random_azimuth=True, traversal=2))
    assert ra[0]["column_rays"] == n
    for k in INT_KEYS:
        assert ra[0][k] == rb[0][k], k
    # the batched engine: all items at normal incidence take the grid, with the plain runs' tallies
    res, _, _ = ctx.run_batch([mid], [100.0, 800.0], [0.0], n, 3)
    plain, _, _ = ctx.run(mid, [100.0, 800.0], [0.0], n, 3, desc=rtmc.run_desc(traversal=2))
    assert res[0]["column_rays"] == 2 * n
    for a, b in zip(res, plain):
        for k in INT_KEYS[:-1]:
            assert a[k] == b[k], k
    ctx.unload_mesh(mid)


def test_column_grid_records_match_oracle(ctx):
    """Per-ray records of the tiny config through the column grid against the FP64 oracle."""
    import oracle as O
    from tests.parity import check_moments, compare_records
    mesh = I.grf_foam(16, 0.5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid)
    n = 50_000
    g = ctx.run_records(mid, 300.0, 0.0, n, seed=1806)
    ctx.unload_mesh(mid)
    assert g["column_rays"] == n
    o = O.run(mesh, TABLE, 300.0, 0.0, n, seed=1806, records=True)
    st = compare_records(g["records"], o["records"], mesh=mesh)
    assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
    check_moments(g, o, st)


@pytest.mark.parametrize("model", ["tertiaries", "paper_fit"])
def test_column_grid_under_deeper_trees(model):
    """Generation 0 through the grid feeds trees of several generations (tertiaries above
    20 eV; the paper-fit emission, up to 6 generations): the hierarchy's tallies."""
    import torch
    from paper_1806_00205_gb300 import rtmc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    em = rtmc.Emission(regen_min_ev=20.0, max_generation=2) if model == "tertiaries" else rtmc.paper_emission()
    mesh = I.grf_foam(32, 0.7, seed=11)
    with rtmc.Context(0) as c:
        c.load_see_tables(TABLE, em)
        mid = c.load_mesh(mesh.tri, mesh.box)
        c.build_bvh(mid, kind=rtmc.BVH_W4)
        n = 100_000
        a, ha, _ = c.run(mid, [500.0, 1500.0], [0.0], n, 44)
        b, hb, _ = c.run(mid, [500.0, 1500.0], [0.0], n, 44, desc=rtmc.run_desc(traversal=2))
    for x, y in zip(a, b):
        assert x["column_rays"] == n and x["regenerated"] > 0
        for k in INT_KEYS[:-1] + ("regenerated",):
            assert x[k] == y[k], k
    assert np.array_equal(ha, hb)


def test_column_grid_retries_coarser_for_a_wide_facet(ctx):
    """A facet as wide as the cell spans more pixels than the grid allows at first: the build
    retries with coarser pixels, and the vertical rays still give the hierarchy's tallies."""
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(16, 0.5, seed=9)
    b = mesh.box
    z = b.z_min + 0.25 * (b.z_top - b.z_min) * 0.01
    big = np.array([[0.0, 0.0, z, b.lx, 0.0, z, 0.0, b.ly, z]], dtype=np.float32)   # faces up, under the foam
    tri = np.concatenate([mesh.tri.reshape(-1, 9).astype(np.float32), big])
    mid = ctx.load_mesh(tri, b)
    ctx.build_bvh(mid, kind=rtmc.BVH_W4)
    n = 50_000
    a, ha, _ = ctx.run(mid, [300.0], [0.0], n, 5)
    c, hc, _ = ctx.run(mid, [300.0], [0.0], n, 5, desc=rtmc.run_desc(traversal=2))
    ctx.unload_mesh(mid)
    assert a[0]["column_rays"] == n and c[0]["column_rays"] == 0
    for k in INT_KEYS[:-1]:
        assert a[0][k] == c[0][k], k
    assert np.array_equal(ha, hc)


def _slant_vs_hierarchy(ctx, mid, energies, thetas, n, seed, **kw):
    import torch
    from paper_1806_00205_gb300 import rtmc
    out = []
    for e in energies:
        for th in thetas:
            hs = torch.zeros(n, dtype=torch.int64, device="cuda")
            hb = torch.zeros(n, dtype=torch.int64, device="cuda")
            a = ctx.run(mid, [e], [th], n, seed, desc=rtmc.run_desc(prim_hash=hs, **kw))
            b = ctx.run(mid, [e], [th], n, seed, desc=rtmc.run_desc(prim_hash=hb, traversal=2, **kw))
            out.append((th, a, b, hs, hb))
    return out


@pytest.mark.parametrize("grid,porosity,kind", [(16, 0.5, 0), (48, 0.3, 1), (48, 0.8, 2), (128, 0.6, 3)])
def test_slanted_grid_equals_hierarchy(ctx, grid, porosity, kind):
    """Oblique primaries through the slanted grid of their direction: every tally,
    histogram and per-primary hash (wraps included) equals the hierarchy's."""
    import torch
    mesh = I.grf_foam(grid, porosity)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=kind)
    n = 200_000 if grid < 128 else 1_000_000
    for th, (ra, hea, haa), (rb, heb, hab), hs, hb in _slant_vs_hierarchy(
            ctx, mid, [80.0, 500.0], [5.0, 37.0, 60.0, 80.0, 89.0], n, 17):
        for a, b in zip(ra, rb):
            # at 89 degrees a facet's slanted footprint can be wider than the cell: then no grid
            assert (a["column_rays"] == n or th > 85.0) and a["column_rays"] in (0, n), th
            assert b["column_rays"] == 0, th
            for k in INT_KEYS:
                assert a[k] == b[k], (th, k, a[k], b[k])
            assert abs(a["e_sum"] - b["e_sum"]) <= 1e-9 * max(1.0, b["e_sum"])
        assert np.array_equal(hea, heb) and np.array_equal(haa, hab)
        assert torch.equal(hs, hb), th
    ctx.unload_mesh(mid)


def test_slanted_grid_many_wraps(ctx):
    """A square well 400 nm deep in a 100 nm periodic cell at 85
    degrees: primaries wrap many times before they meet a wall or the floor; the replayed
    wraps give the hierarchy's records."""
    import torch
    from paper_1806_00205_gb300 import rtmc
    well = I.square_well(90.0, 400.0, rim=5.0)
    mid = ctx.load_mesh(well.tri, well.box)
    ctx.build_bvh(mid, kind=rtmc.BVH_W4)
    n = 100_000
    for th, (ra, _, _), (rb, _, _), hs, hb in _slant_vs_hierarchy(ctx, mid, [300.0], [45.0, 75.0, 85.0], n, 3,
                                                                    window=(0.0, 100.0, 0.0, 100.0)):
        a, b = ra[0], rb[0]
        assert a["column_rays"] == n
        for k in INT_KEYS:
            assert a[k] == b[k], (th, k, a[k], b[k])
        assert torch.equal(hs, hb), th
    assert b["wraps"] > n            # at 85 degrees primaries wrap more than once on average
    ctx.unload_mesh(mid)


def test_slanted_grid_records_match_oracle(ctx):
    """Per-ray records of oblique primaries through the slanted grid against the FP64 oracle."""
    import oracle as O
    from tests.parity import check_moments, compare_records
    mesh = I.grf_foam(16, 0.5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid)
    n = 30_000
    for th in (50.0, 80.0):
        g = ctx.run_records(mid, 300.0, th, n, seed=1806)
        assert g["column_rays"] == n
        o = O.run(mesh, TABLE, 300.0, th, n, seed=1806, records=True)
        st = compare_records(g["records"], o["records"], mesh=mesh)
        assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
        assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
        check_moments(g, o, st)
    ctx.unload_mesh(mid)


def test_slanted_grid_not_for_random_directions(ctx):
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(16, 0.5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid)
    n = 20_000
    for kw in (dict(random_azimuth=True), dict(random_polar=True), dict(traversal=1), dict(fp64_retest=True)):
        r, _, _ = ctx.run(mid, [300.0], [40.0], n, 3, desc=rtmc.run_desc(**kw))
        assert r[0]["column_rays"] == 0, kw
    ctx.unload_mesh(mid)
