"""Failure detection on the CUDA path, made to fire without faulting the GPU.

A daughter queue too small for a chunk's daughters must be detected on the
device (its writes are dropped and a status bit is raised), the work repeated
with more room, and the tallies must not change; when the repeats run out the
call returns RTMC_ERR_CAPACITY.  A traversal that exceeds its visit bound
abandons the ray and the call returns RTMC_ERR_DEVICE_CHECK instead of
looping; the context stays usable.  The bounds are lowered through the run
descriptor (queue_factor, max_visits), so nothing here hangs or faults."""
import numpy as np
import pytest

from paper_1806_00205_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TABLE = I.see_table()
INT_KEYS = ("n_primaries", "rays", "escaped", "absorbed_low", "absorbed_other", "emitters", "emitted",
            "regenerated", "capped", "lost", "wraps", "sum_k", "sum_k2")


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_00205_gb300 import rtmc
    ctx = rtmc.Context(0)
    ctx.load_see_tables(TABLE)
    mesh = I.grf_foam(16, 0.5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=rtmc.BVH_W4)
    yield ctx, mid, rtmc
    ctx.close()


def test_queue_overflow_is_retried_with_identical_tallies(setup):
    ctx, mid, rtmc = setup
    n = 50_000
    ref, he, ha = ctx.run(mid, [300.0, 800.0], [0.0, 45.0], n, 3)
    assert all(r["queue_retries"] == 0 for r in ref)
    got, ge, ga = ctx.run(mid, [300.0, 800.0], [0.0, 45.0], n, 3, desc=rtmc.run_desc(queue_factor=0.1))
    for a, b in zip(got, ref):
        assert a["queue_retries"] >= 2          # 0.1 and 0.2 daughters per primary cannot hold a mean near 1
        for k in INT_KEYS:
            assert a[k] == b[k], k
    assert np.array_equal(ge, he) and np.array_equal(ga, ha)


def test_queue_overflow_retries_run_out_with_capacity_error(setup):
    ctx, mid, rtmc = setup
    with pytest.raises(rtmc.RtmcError) as e:
        ctx.run(mid, [300.0], [0.0], 50_000, 3, desc=rtmc.run_desc(queue_factor=0.001))
    assert e.value.code == -6 and "overflow" in str(e.value)
    # the context is still usable and gives the reference tallies
    r, _, _ = ctx.run(mid, [300.0], [0.0], 50_000, 3)
    assert r[0]["queue_retries"] == 0 and r[0]["rays"] == 50_000 + r[0]["emitted"]


def test_batched_queue_overflow_is_retried(setup):
    ctx, mid, rtmc = setup
    n = 20_000
    ref, he, ha = ctx.run_batch([mid], [300.0, 600.0], [0.0, 30.0], n, 7)
    got, ge, ga = ctx.run_batch([mid], [300.0, 600.0], [0.0, 30.0], n, 7, desc=rtmc.run_desc(queue_factor=0.1))
    for a, b in zip(got, ref):
        assert a["queue_retries"] >= 2
        for k in INT_KEYS:
            assert a[k] == b[k], k
    assert np.array_equal(ge, he) and np.array_equal(ga, ha)
    with pytest.raises(rtmc.RtmcError) as e:
        ctx.run_batch([mid], [300.0], [0.0], n, 7, desc=rtmc.run_desc(queue_factor=0.001))
    assert e.value.code == -6


@pytest.mark.parametrize("opts", [dict(), dict(traversal=1), dict(traversal=2, fp64_retest=True)])
def test_visit_bound_ends_the_run_with_device_check(setup, opts):
    ctx, mid, rtmc = setup
    n = 5000
    with pytest.raises(rtmc.RtmcError) as e:
        ctx.run(mid, [300.0], [40.0], n, 5, desc=rtmc.run_desc(max_visits=2, **opts))
    assert e.value.code == -8
    with pytest.raises(rtmc.RtmcError) as e:
        ctx.run_batch([mid], [300.0], [40.0], n, 5, desc=rtmc.run_desc(max_visits=2, **opts))
    assert e.value.code == -8
    # the tree's own bound never fires on a correct hierarchy, and the context is intact
    ok, _, _ = ctx.run(mid, [300.0], [40.0], n, 5, desc=rtmc.run_desc(**opts))
    big, _, _ = ctx.run(mid, [300.0], [40.0], n, 5, desc=rtmc.run_desc(max_visits=1 << 30, **opts))
    for k in INT_KEYS:
        assert ok[0][k] == big[0][k], k


def test_descriptor_controls_are_checked(setup):
    ctx, mid, rtmc = setup
    for bad in (dict(max_visits=-1), dict(queue_factor=-0.5), dict(queue_factor=65.0)):
        with pytest.raises(rtmc.RtmcError) as e:
            ctx.run(mid, [300.0], [0.0], 10, 1, desc=rtmc.run_desc(**bad))
        assert e.value.code == -1, bad
