"""rtmc_run_noalloc: the scratch-free entry point for callers that cannot
allocate device memory while they run.

Its results must equal those of rtmc_run for the same item, on two calls in a
row (the static scratch keeps the previous call's contents, so the second call
checks that everything that must start at zero is cleared).  The file is
collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_00205_gb300 import inputs as I
    from paper_1806_00205_gb300 import rtmc
    ctx = rtmc.Context(0)
    ctx.load_see_tables(I.see_table())
    mesh = I.grf_foam(16, 0.5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid)
    yield ctx, mid, rtmc
    ctx.close()


INT_KEYS = ("n_primaries", "rays", "escaped", "absorbed_low", "absorbed_other", "emitters", "emitted",
            "regenerated", "capped", "lost", "wraps", "sum_k", "sum_k2")


def test_noalloc_equals_run_on_two_calls(setup):
    ctx, mid, rtmc = setup
    n = rtmc.NOALLOC_MAX_PRIMARIES
    calls = [(300.0, 0.0, 11, 0), (700.0, 30.0, 12, 4096)]
    for energy, theta, seed, offset in calls:
        desc = rtmc.run_desc(primary_offset=offset)
        ref, he, ha = ctx.run(mid, [energy], [theta], n, seed, desc=desc)
        got, ge, ga = ctx.run_noalloc(mid, energy, theta, n, seed, item=0, desc=desc)
        for k in INT_KEYS:
            assert got[k] == ref[0][k], (k, got[k], ref[0][k])
        assert np.array_equal(ge, he[0]) and np.array_equal(ga, ha[0])
        for k in ("e_sum", "e2_sum", "sey", "sey_se"):
            assert abs(got[k] - ref[0][k]) <= 1e-12 * max(1.0, abs(ref[0][k])), k
        assert got["rays"] > n


def test_noalloc_random_incidence_depth_profile_equals_run(setup):
    ctx, mid, rtmc = setup
    n = 3000
    desc = rtmc.run_desc(random_polar=True, n_zbins=100)
    ref, _, _ = ctx.run(mid, [250.0], [0.0], n, 17, desc=desc)
    got, _, _ = ctx.run_noalloc(mid, 250.0, 0.0, n, 17, desc=desc)
    for k in INT_KEYS:
        assert got[k] == ref[0][k], (k, got[k], ref[0][k])
    assert np.array_equal(got["hist_z"], ref[0]["hist_z"]) and got["hist_z"].sum() > n


def test_noalloc_hash_equals_run_hash(setup):
    import torch
    ctx, mid, rtmc = setup
    n = 3000
    h_ref = torch.zeros(n, dtype=torch.int64, device="cuda")
    h_got = torch.full((n,), 7, dtype=torch.int64, device="cuda")
    ctx.run(mid, [450.0], [10.0], n, 5, desc=rtmc.run_desc(prim_hash=h_ref))
    ctx.run_noalloc(mid, 450.0, 10.0, n, 5, desc=rtmc.run_desc(prim_hash=h_got))
    assert torch.equal(h_ref, h_got)


def test_noalloc_fp64_retest_equals_run(setup):
    """The FP64 re-test needs no scratch, so the scratch-free entry runs it too: the same
    tallies, histograms and re-test counts as rtmc_run, call by call."""
    ctx, mid, rtmc = setup
    n = rtmc.NOALLOC_MAX_PRIMARIES
    total = 0
    for c in range(10):
        desc = rtmc.run_desc(fp64_retest=True, primary_offset=c * n)
        ref, he, ha = ctx.run(mid, [300.0], [60.0], n, 23, desc=desc)
        got, ge, ga = ctx.run_noalloc(mid, 300.0, 60.0, n, 23, desc=desc)
        for k in INT_KEYS + ("retested",):
            assert got[k] == ref[0][k], (c, k, got[k], ref[0][k])
        assert np.array_equal(ge, he[0]) and np.array_equal(ga, ha[0])
        total += got["retested"]
    assert total > 0


@pytest.mark.parametrize("opts", [dict(traversal=1), dict(traversal=2, stack_depth=8),
                                  dict(traversal=2, stack_depth=32, fetch_threshold=12, block_threads=64),
                                  dict(traversal=0, stack_depth=8, blocks_per_sm=2)])
def test_noalloc_traversal_controls_equal_run(setup, opts):
    """The traversal controls of the descriptor reach the kernels as in rtmc_run:
    the same tallies and histograms at normal incidence (where traversal 2 keeps
    generation 0 on the hierarchy) and at 40 degrees."""
    ctx, mid, rtmc = setup
    n = 3000
    for theta in (0.0, 40.0):
        desc = rtmc.run_desc(**opts)
        ref, he, ha = ctx.run(mid, [350.0], [theta], n, 29, desc=desc)
        got, ge, ga = ctx.run_noalloc(mid, 350.0, theta, n, 29, desc=desc)
        # the scratch-free entry builds no slanted grid: oblique primaries take the hierarchy
        for k in INT_KEYS + (("column_rays",) if theta == 0.0 else ()):
            assert got[k] == ref[0][k], (opts, theta, k, got[k], ref[0][k])
        assert np.array_equal(ge, he[0]) and np.array_equal(ga, ha[0])


def test_noalloc_checks_the_descriptor_as_run_does(setup):
    ctx, mid, rtmc = setup
    for bad in (dict(traversal=3), dict(stack_depth=12), dict(fetch_threshold=40), dict(chunk=-1),
                dict(traversal=1, fp64_retest=True)):
        with pytest.raises(rtmc.RtmcError) as e:
            ctx.run(mid, [300.0], [0.0], 10, 1, desc=rtmc.run_desc(**bad))
        with pytest.raises(rtmc.RtmcError) as f:
            ctx.run_noalloc(mid, 300.0, 0.0, 10, 1, desc=rtmc.run_desc(**bad))
        assert e.value.code == f.value.code == -1, bad
    # the visit bound reaches the traversal kernels of both entry points
    for opts in (dict(), dict(traversal=1)):
        with pytest.raises(rtmc.RtmcError) as e:
            ctx.run_noalloc(mid, 300.0, 30.0, 500, 1, desc=rtmc.run_desc(max_visits=2, **opts))
        assert e.value.code == -8
    ok, _, _ = ctx.run_noalloc(mid, 300.0, 30.0, 500, 1)
    assert ok["rays"] == 500 + ok["emitted"]


def test_noalloc_rejects_sizes_beyond_the_limit(setup):
    ctx, mid, rtmc = setup
    with pytest.raises(rtmc.RtmcError) as e:
        ctx.run_noalloc(mid, 300.0, 0.0, rtmc.NOALLOC_MAX_PRIMARIES + 1, 1)
    assert e.value.code == -1 and "4096" in str(e.value)
    with pytest.raises(rtmc.RtmcError):
        ctx.run_noalloc(mid, 300.0, 0.0, 10, 1, desc=rtmc.run_desc(n_ebins=1000, n_abins=100))
    # a context whose emission allows a second generation does not fit the static queues
    from paper_1806_00205_gb300 import inputs as I
    c2 = rtmc.Context(0)
    try:
        c2.load_see_tables(I.see_table(), rtmc.Emission(regen_min_ev=20.0, max_generation=2))
        m2 = c2.load_mesh(I.flat_plane().tri, I.flat_plane().box)
        c2.build_bvh(m2)
        with pytest.raises(rtmc.RtmcError):
            c2.run_noalloc(m2, 300.0, 0.0, 10, 1)
    finally:
        c2.close()
