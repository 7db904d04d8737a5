"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300)."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1806_00205_gb300 import inputs as I
from tests.parity import check_moments, compare_records, primary_hashes

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = I.see_table()
E47 = float(TABLE.energy_grid()[47])


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


def _mesh_id(ctx, mesh):
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid)
    return mid


@pytest.fixture(scope="module")
def tiny(ctx):
    m = I.grf_foam(16, 0.5)
    return m, _mesh_id(ctx, m)


# ------------------------------------------------------------------ RNG ----

def test_device_philox_known_answers(ctx):
    rows = []
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([int(x, 16) for x in line.split()])
    for r in rows:
        key = r[4] | (r[5] << 32)
        out = ctx.philox(np.array(r[0:4], dtype=np.uint32), key)
        assert list(out[0]) == r[6:10]


def test_device_philox_matches_oracle(ctx):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 1 << 32, (2000, 4), dtype=np.uint64).astype(np.uint32)
    key = 0x123456789ABCDEF
    dev = ctx.philox(ctr, key)
    for i in range(0, 2000, 97):
        want = O.philox(ctr[i], [key & 0xFFFFFFFF, key >> 32])
        assert list(dev[i]) == list(want)


# ------------------------------------------------------------- BVH hits ----

def _rays_for(mesh, n, rng, reach=5.0):
    box = mesh.box
    o = np.stack([rng.uniform(0, box.lx, n), rng.uniform(0, box.ly, n),
                  rng.uniform(box.z_min + 0.3 * (box.z_top - box.z_min), box.z_top, n)], axis=1)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    # rays aimed at vertices and edge midpoints (the edge cases of the test)
    tri = mesh.tri.astype(np.float64)
    k = n // 4
    pick = rng.integers(0, mesh.n_tri, k)
    tgt = np.where(rng.random(k)[:, None] < 0.5, tri[pick, 0], 0.5 * (tri[pick, 0] + tri[pick, 1]))
    o2 = tgt + rng.normal(size=(k, 3)) * reach
    d2 = tgt - o2
    d2 /= np.linalg.norm(d2, axis=1)[:, None]
    return np.concatenate([o, o2]).astype(np.float32), np.concatenate([d, d2]).astype(np.float32)


@pytest.mark.parametrize("kind,leaf,ploc", [(0, 4, False), (0, 1, False), (1, 4, False), (1, 8, False),
                                             (0, 4, True), (1, 4, True), (0, 1, True), (1, 8, True),
                                             (2, 4, False), (2, 1, False), (2, 8, True),
                                             (3, 4, False), (3, 1, False), (3, 8, True)])
@pytest.mark.parametrize("which", ["tiny", "flat", "well", "single", "foam8"])
def test_bvh_closest_hit_matches_brute_force(ctx, which, kind, leaf, ploc):
    mesh = {"tiny": lambda: I.grf_foam(16, 0.5), "flat": lambda: I.flat_plane(),
            "well": lambda: I.square_well(100.0, 60.0),
            "single": lambda: I.Mesh(I.flat_plane().tri[:1], I.flat_plane().box),
            "foam8": lambda: I.grf_foam(8, 0.7, 1.5, 3)}[which]()
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=kind, leaf=leaf, ploc=ploc)
    rng = np.random.default_rng(42)
    o, d = _rays_for(mesh, 4000, rng)
    skip = rng.integers(-1, mesh.n_tri, o.shape[0]).astype(np.int32)
    skip[rng.random(o.shape[0]) < 0.5] = -1
    hits = ctx.trace_rays(mid, o, d, skip)
    n_rand = 4000
    same_rand = 0
    for i in range(o.shape[0]):
        t, j, u, v = O.closest_hit(mesh, o[i].astype(np.float64), d[i].astype(np.float64), int(skip[i]))
        g = hits[i]
        if g["tri"] == j:
            same_rand += i < n_rand
            if j >= 0:
                assert abs(g["t"] - t) <= 1e-5 * max(t, 1.0), (i, g, t)
            continue
        # FP32 and FP64 may only disagree where the ray meets a facet edge or
        # vertex: the answer of either side then lies on a barycentric boundary
        near = []
        if j >= 0:
            near.append(min(u, v, 1 - u - v) < 1e-4)
        if g["tri"] >= 0:
            near.append(min(g["u"], g["v"], 1 - g["u"] - g["v"]) < 1e-4)
        assert any(near), (i, g, (t, j, u, v))
    assert same_rand >= 0.999 * n_rand


@pytest.mark.parametrize("kind", [2, 3])
@pytest.mark.parametrize("h", [1.0e-3, 1.0e4])
def test_four_wide_closest_hit_at_extreme_scales(ctx, kind, h):
    """The 4-wide nodes' one-FMA planes and the 8-bit codes' margins (M 2^-21 + s 2^-7) at voxel
    sizes 1e-3 and 1e4 (cells of 8e-3 and 8e4): closest hits still equal brute force."""
    mesh = I.grf_foam(8, 0.7, 1.5, 3, h=h)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=kind)
    rng = np.random.default_rng(7)
    o, d = _rays_for(mesh, 3000, rng, reach=0.5 * h)       # aimed rays start a few voxels away
    hits = ctx.trace_rays(mid, o, d, np.full(o.shape[0], -1, dtype=np.int32))
    ctx.unload_mesh(mid)
    same = 0
    for i in range(o.shape[0]):
        t, j, u, v = O.closest_hit(mesh, o[i].astype(np.float64), d[i].astype(np.float64), -1)
        g = hits[i]
        if g["tri"] == j:
            same += i < 3000                            # the random rays (the rest aim at vertices and edges)
            if j >= 0:
                assert abs(g["t"] - t) <= 1e-5 * max(t, h), (i, g, t)
            continue
        near = []
        if j >= 0:
            near.append(min(u, v, 1 - u - v) < 1e-4)
        if g["tri"] >= 0:
            near.append(min(g["u"], g["v"], 1 - g["u"] - g["v"]) < 1e-4)
        assert any(near), (i, g, (t, j, u, v))
    assert same >= 0.999 * 3000


# ---------------------------------------------------------- full runs ------

@pytest.mark.parametrize("kind", [2, 3])
def test_four_wide_nodes_records_match_oracle(ctx, kind):
    """4-wide nodes (FP32 or 8-bit boxes) change the traversal, not the answer: records on the tiny foam."""
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(16, 0.5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=kind)
    n = 30_000
    g = ctx.run_records(mid, 300.0, 0.0, n, seed=78)
    o = O.run(mesh, TABLE, 300.0, 0.0, n, seed=78, records=True)
    st = compare_records(g["records"], o["records"], mesh=mesh)
    assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
    # the same tallies through the persistent, the per-lane and the FP64 re-test kernels
    r0, _, _ = ctx.run(mid, [300.0], [0.0], n, 78)
    r1, _, _ = ctx.run(mid, [300.0], [0.0], n, 78, desc=rtmc.run_desc(traversal=1))
    r2, _, _ = ctx.run(mid, [300.0], [0.0], n, 78, desc=rtmc.run_desc(fp64_retest=True))
    for k in ("rays", "escaped", "sum_k", "wraps"):
        assert r0[0][k] == r1[0][k] == g[k], k
        assert abs(r2[0][k] - g[k]) <= 2, k
    ctx.unload_mesh(mid)


@pytest.mark.parametrize("kind", [0, 1])
def test_ploc_hierarchy_records_match_oracle(ctx, kind):
    """The clustering builder changes the tree, not the answer: records on the tiny foam."""
    mesh = I.grf_foam(16, 0.5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=kind, ploc=True)
    n = 30_000
    g = ctx.run_records(mid, 300.0, 0.0, n, seed=77)
    o = O.run(mesh, TABLE, 300.0, 0.0, n, seed=77, records=True)
    st = compare_records(g["records"], o["records"], mesh=mesh)
    assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
    ctx.unload_mesh(mid)


def test_tiny_config_records_match_oracle(ctx, tiny):
    """Tiny config: 16^3 foam, 1e5 primaries at 300 eV, normal incidence."""
    mesh, mid = tiny
    n = 100_000
    g = ctx.run_records(mid, 300.0, 0.0, n, seed=1806)
    o = O.run(mesh, TABLE, 300.0, 0.0, n, seed=1806, records=True)
    st = compare_records(g["records"], o["records"], mesh=mesh)
    assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
    # The intersection's own precision is pinned on identical rays by
    # test_bvh_closest_hit_matches_brute_force (|dt| <= 1e-5 max(t, 1 nm)).  Along
    # a full path the FP32 ray set-up (origin and direction roundings) moves the
    # ray sideways, which a facet met at incidence cosine c turns into a distance
    # error over |c|: every ray whose events agree is held to that bound
    # (tests/parity.py, t_error_bound), and 99.9 % of them to 1e-5 relative.
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
    assert st["n_t_checked"] >= 0.999 * st["n_oracle"]
    assert st["t_rel_p999"] <= 1e-5, st["t_rel_p999"]
    check_moments(g, o, st)
    for k in ("rays", "escaped", "emitted", "sum_k"):
        assert abs(g[k] - o[k]) <= 2e-4 * max(1, o[k]) + 2, k
    se = math.hypot(g["sey_se"], o["sey_se"])
    assert abs(g["sey"] - o["sey"]) < min(3 * se, 1e-3)
    assert g["lost"] == 0
    assert g["rays"] == n + g["emitted"]
    assert g["rays"] == g["escaped"] + g["absorbed_low"] + g["absorbed_other"] + g["emitters"] + g["lost"]


def test_run_tallies_equal_record_tallies(ctx, tiny):
    _, mid = tiny
    n = 20_000
    res, he, ha = ctx.run(mid, [300.0], [0.0], n, seed=5)
    rr = ctx.run_records(mid, 300.0, 0.0, n, seed=5)
    r = res[0]
    for k in ("rays", "escaped", "emitted", "sum_k", "sum_k2", "wraps", "absorbed_low"):
        assert r[k] == rr[k], k
    esc = rr["records"][rr["records"]["fate"] == O.ESCAPED]
    assert np.array_equal(np.bincount(esc["e_bin"], minlength=64), he[0].astype(np.int64))
    assert np.array_equal(np.bincount(esc["a_bin"], minlength=18), ha[0].astype(np.int64))


def test_flat_plane_gpu(ctx):
    fp = I.flat_plane()
    mid = _mesh_id(ctx, fp)
    res, he, ha = ctx.run(mid, [E47], [0.0, 60.0], 1_000_000, seed=77)
    for r, j in zip(res, (0, 12)):
        lam = float(TABLE.delta[47, j])
        assert r["lost"] == 0 and r["escaped"] == r["emitted"]
        assert abs(r["sey"] - lam) < 3 * r["sey_se"], (r["sey"], lam)


def test_square_well_view_factor_gpu(ctx):
    from tests.test_oracle_pins import view_factor_squares
    from paper_1806_00205_gb300 import rtmc
    w = I.square_well(100.0, 100.0)
    mid = _mesh_id(ctx, w)
    res, _, _ = ctx.run(mid, [E47], [0.0], 2_000_000, seed=3,
                        desc=rtmc.run_desc(window=I.opening_window(100.0)))
    expect = float(TABLE.delta[47, 0]) * view_factor_squares(1.0)
    assert abs(res[0]["sey"] - expect) < 3 * res[0]["sey_se"]


def test_multi_item_run_equals_single_items(ctx, tiny):
    _, mid = tiny
    res, he, _ = ctx.run(mid, [100.0, 700.0], [0.0, 45.0], 5000, seed=9)
    for item, (e, th) in enumerate([(100.0, 0.0), (100.0, 45.0), (700.0, 0.0), (700.0, 45.0)]):
        one = ctx.run_records(mid, e, th, 5000, seed=9, item=item)
        assert res[item]["sum_k"] == one["sum_k"] and res[item]["rays"] == one["rays"]


def test_chunking_and_edge_sizes(ctx, tiny):
    from paper_1806_00205_gb300 import rtmc
    _, mid = tiny
    ref, _, _ = ctx.run(mid, [300.0], [0.0], 2500, seed=4)
    for chunk in (1000, 999, 2500, 4096):
        r, _, _ = ctx.run(mid, [300.0], [0.0], 2500, seed=4, desc=rtmc.run_desc(chunk=chunk))
        assert r[0]["sum_k"] == ref[0]["sum_k"] and r[0]["rays"] == ref[0]["rays"]
    z, _, _ = ctx.run(mid, [300.0], [0.0], 0, seed=4)
    assert z[0]["rays"] == 0 and z[0]["sey"] == 0.0
    one = ctx.run_records(mid, 300.0, 0.0, 1, seed=4)
    assert one["records"].size == one["rays"] >= 1


def test_tertiaries_match_oracle(ctx):
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(16, 0.7, seed=4)
    em = rtmc.Emission(regen_min_ev=20.0, max_generation=2)
    c2 = rtmc.Context(0)
    try:
        c2.load_see_tables(TABLE, em)
        mid = _mesh_id(c2, mesh)
        n = 20_000
        g = c2.run_records(mid, 500.0, 0.0, n, seed=6)
        o = O.run(mesh, TABLE, 500.0, 0.0, n, seed=6, records=True,
                  emission=O.Emission(regen_min_ev=20.0, max_generation=2))
        st = compare_records(g["records"], o["records"], mesh=mesh)
        assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
        assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
        check_moments(g, o, st)
        assert g["regenerated"] > 0
    finally:
        c2.close()


def test_random_azimuth_and_window_match_oracle(ctx, tiny):
    from paper_1806_00205_gb300 import rtmc
    mesh, mid = tiny
    win = (20.0, 90.0, 30.0, 150.0)
    n = 20_000
    g = ctx.run_records(mid, 200.0, 50.0, n, seed=11, item=3,
                        desc=rtmc.run_desc(random_azimuth=True, window=win))
    o = O.run(mesh, TABLE, 200.0, 50.0, n, seed=11, item=3, random_azimuth=True, window=win, records=True)
    st = compare_records(g["records"], o["records"], mesh=mesh)
    assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])


def test_wrap_limit_counts_lost(ctx):
    from paper_1806_00205_gb300 import rtmc
    fp = I.flat_plane(160.0, height=400.0)      # tall slab: many daughters need wraps
    mid = _mesh_id(ctx, fp)
    n = 20_000
    g = ctx.run_records(mid, E47, 0.0, n, seed=2, desc=rtmc.run_desc(max_wraps=2))
    o = O.run(fp, TABLE, E47, 0.0, n, seed=2, max_wraps=2, records=True)
    assert g["lost"] > 0
    st = compare_records(g["records"], o["records"], mesh=fp)
    assert st["frac_same"] >= 0.9999
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])


def test_prim_hash_matches_oracle(ctx, tiny):
    import torch
    from paper_1806_00205_gb300 import rtmc
    mesh, mid = tiny
    n = 50_000
    h = torch.zeros(n, dtype=torch.int64, device="cuda")
    ctx.run(mid, [300.0], [0.0], n, seed=21, desc=rtmc.run_desc(prim_hash=h))
    dev = h.cpu().numpy().view(np.uint64)
    ids = np.arange(0, n, 7, dtype=np.uint64)
    o = O.run(mesh, TABLE, 300.0, 0.0, 0, seed=21, prim_ids=ids, records=True)
    want = primary_hashes(o["records"], ids)
    assert np.mean(dev[ids.astype(np.int64)] == want) >= 0.9995


def test_errors_are_reported_not_faulted(ctx):
    from paper_1806_00205_gb300 import rtmc
    with pytest.raises(rtmc.RtmcError) as e:
        ctx.run(12345, [300.0], [0.0], 10, seed=1)
    assert e.value.code == -4
    mid = ctx.load_mesh(I.flat_plane().tri, I.flat_plane().box)
    with pytest.raises(rtmc.RtmcError) as e:
        ctx.run(mid, [300.0], [0.0], 10, seed=1)
    assert e.value.code == -5
    ctx.build_bvh(mid)
    with pytest.raises(rtmc.RtmcError) as e:
        ctx.run(mid, [300.0], [95.0], 10, seed=1)
    assert e.value.code == -1
    with pytest.raises(rtmc.RtmcError):
        ctx.run(mid, [-3.0], [0.0], 10, seed=1)


@pytest.fixture(scope="module")
def paper(ctx):
    m = I.grf_foam(128, 0.6, 2.0, 1806)
    return m, _mesh_id(ctx, m)


def test_paper_scale_sampled_parity(ctx, paper):
    """128^3 foam (~1.39M triangles), 1e7 primaries at 500 eV, bench launch configuration.

    The production run (no hashing) and the hashing run must give identical
    tallies; sampled primaries replayed by the oracle must give identical
    per-primary event hashes."""
    import torch
    from paper_1806_00205_gb300 import rtmc
    mesh, mid = paper
    n = 10_000_000
    prod, he, ha = ctx.run(mid, [500.0], [0.0], n, seed=1806)
    h = torch.zeros(n, dtype=torch.int64, device="cuda")
    hashed, he2, ha2 = ctx.run(mid, [500.0], [0.0], n, seed=1806, desc=rtmc.run_desc(prim_hash=h))
    for k in ("rays", "escaped", "emitted", "sum_k", "sum_k2", "wraps", "lost", "absorbed_low"):
        assert prod[0][k] == hashed[0][k], k
    assert np.array_equal(he, he2) and np.array_equal(ha, ha2)
    r = prod[0]
    assert r["rays"] == n + r["emitted"] == r["escaped"] + r["absorbed_low"] + r["absorbed_other"] + \
        r["emitters"] + r["lost"]
    assert r["lost"] <= 1e-6 * r["rays"]
    rng = np.random.default_rng(17)
    ids = np.sort(rng.choice(n, 400, replace=False)).astype(np.uint64)
    o = O.run(mesh, TABLE, 500.0, 0.0, 0, seed=1806, prim_ids=ids, records=True)
    want = primary_hashes(o["records"], ids)
    dev = h.cpu().numpy().view(np.uint64)[ids.astype(np.int64)]
    assert np.sum(dev != want) <= 1, np.sum(dev != want)
    # the sampled SEY agrees with the full-size GPU SEY within the sample's error
    assert abs(o["sey"] - r["sey"]) < 3 * math.hypot(o["sey_se"], r["sey_se"])
    # 4-wide nodes (the bench's format) find the same closest hits: every tally and all
    # 1e7 per-primary event hashes equal the binary FP32 run's
    w4 = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(w4, kind=rtmc.BVH_W4)
    h4 = torch.zeros(n, dtype=torch.int64, device="cuda")
    r4, he4, ha4 = ctx.run(w4, [500.0], [0.0], n, seed=1806, desc=rtmc.run_desc(prim_hash=h4))
    ctx.unload_mesh(w4)
    for k in ("rays", "escaped", "emitted", "sum_k", "sum_k2", "wraps", "lost", "absorbed_low", "absorbed_other"):
        assert r4[0][k] == r[k], k
    assert np.array_equal(he4, he) and np.array_equal(ha4, ha)
    assert torch.equal(h4, h)
    # and so do the 8-bit 4-wide nodes of the precision form
    q4 = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(q4, kind=rtmc.BVH_Q4)
    hq = torch.zeros(n, dtype=torch.int64, device="cuda")
    rq, heq, haq = ctx.run(q4, [500.0], [0.0], n, seed=1806, desc=rtmc.run_desc(prim_hash=hq))
    ctx.unload_mesh(q4)
    for k in ("rays", "escaped", "emitted", "sum_k", "sum_k2", "wraps", "lost", "absorbed_low", "absorbed_other"):
        assert rq[0][k] == r[k], k
    assert np.array_equal(heq, he) and np.array_equal(haq, ha)
    assert torch.equal(hq, h)


def test_gibson_ashby_cage_records_match_oracle(ctx):
    """Open-cell cage of Section 3.1 (v_f = 4 %, C = 28) on a substrate, 600 eV, normal incidence."""
    mesh = I.gibson_ashby_cage(0.04)
    mid = _mesh_id(ctx, mesh)
    n = 30_000
    g = ctx.run_records(mid, 600.0, 0.0, n, seed=13)
    o = O.run(mesh, TABLE, 600.0, 0.0, n, seed=13, records=True)
    st = compare_records(g["records"], o["records"], mesh=mesh)
    assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
    assert g["lost"] == 0 and g["rays"] == n + g["emitted"]
    # most primaries reach the substrate through the open cage, so the yield is near the flat value
    flat = float(I.lin_joy_delta(600.0, 0.0))
    assert 0.6 * flat < g["sey"] < 1.05 * flat


def test_random_incidence_and_depth_profile_match_oracle(ctx, tiny):
    """Cosine-law incidence and the penetration-depth tally, record by record."""
    from paper_1806_00205_gb300 import rtmc
    mesh, mid = tiny
    n, nz = 20_000, 64
    g = ctx.run_records(mid, 300.0, 0.0, n, seed=21, item=2,
                        desc=rtmc.run_desc(random_polar=True, n_zbins=nz))
    o = O.run(mesh, TABLE, 300.0, 0.0, n, seed=21, item=2, random_polar=True, n_zbins=nz, records=True)
    st = compare_records(g["records"], o["records"], mesh=mesh)
    assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
    hz, oz = g["hist_z"].astype(np.int64), o["hist_z"]
    stops = g["emitters"] + g["absorbed_low"] + g["absorbed_other"]
    assert hz.sum() == stops
    # FP32 and FP64 hit points can fall on either side of a bin edge, rarely
    assert np.abs(hz - oz).sum() <= max(4, int(2e-4 * stops)), (hz, oz)


def test_depth_profile_normal_vs_random_incidence(ctx):
    """Section 3.2 on a 4 % solid foam (Fig. pen, 100 eV): normal-incidence
    electrons stop deeper than random-incidence ones."""
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(32, 0.96)
    mid = _mesh_id(ctx, mesh)
    box = mesh.box
    nz, n = 64, 500_000
    c = (np.arange(nz) + 0.5) * (box.z_top - box.z_min) / nz
    depth = {}
    for polar in (False, True):
        r, _, _ = ctx.run(mid, [100.0], [0.0], n, 9, desc=rtmc.run_desc(random_polar=polar, n_zbins=nz))
        hz = r[0]["hist_z"].astype(np.float64)
        mean = (hz * c).sum() / hz.sum()
        se = math.sqrt(((hz * c * c).sum() / hz.sum() - mean * mean) / hz.sum())
        depth[polar] = (mean, se)
    (dn, sn), (dr, sr) = depth[False], depth[True]
    assert dn - dr > 5.0 * math.hypot(sn, sr), depth
