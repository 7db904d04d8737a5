"""Replica sharding on the CUDA path (the paper's Section 2.2, last paragraph:
primaries are independent, so replicas need no communication).

Two rtmc_run calls over disjoint primary-id ranges, merged by shard.merge_results,
must equal one run over the union on every integer tally and histogram, and
primaries sampled from both ranges must give the oracle's per-primary event
hashes."""
import numpy as np
import pytest

import oracle as O
from paper_1806_00205_gb300 import inputs as I
from paper_1806_00205_gb300 import shard
from tests.parity import primary_hashes

pytestmark = pytest.mark.gpu

TABLE = I.see_table()


@pytest.mark.parametrize("engine", ["run", "batch"])
def test_two_ranges_merged_equal_one_run(engine):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(24, 0.6, 2.0, seed=8)
    n = 200_000
    with rtmc.Context(0) as ctx:
        ctx.load_see_tables(TABLE)
        mid = ctx.load_mesh(mesh.tri, mesh.box)
        ctx.build_bvh(mid, kind=rtmc.BVH_W4)

        def go(count, offset, hashes=None):
            d = rtmc.run_desc(primary_offset=offset, n_zbins=32, prim_hash=hashes)
            if engine == "run" or hashes is not None:
                r, he, ha = ctx.run(mid, [450.0], [20.0], count, 1806, desc=d)
            else:
                r, he, ha = ctx.run_batch([mid], [450.0], [20.0], count, 1806, desc=d)
            out = dict(r[0])
            out.update(hist_e=he[0], hist_a=ha[0])
            return out

        parts = [go(n, shard.primary_offset(k, n)) for k in range(2)]
        whole = go(2 * n, 0)
        merged = shard.merge_results(parts)
        for k in shard.INT_KEYS:
            assert merged[k] == whole[k], k
        for h in ("hist_e", "hist_a", "hist_z"):
            assert np.array_equal(np.asarray(merged[h], dtype=np.int64), whole[h].astype(np.int64)), h
        assert merged["sey"] == whole["sey"]
        assert abs(merged["e_sum"] - whole["e_sum"]) <= 1e-9 * whole["e_sum"]
        # per-primary event hashes of rank 1's range against the oracle replaying the same ids
        h1 = torch.zeros(n, dtype=torch.int64, device="cuda")
        go(n, shard.primary_offset(1, n), hashes=h1)
        dev = h1.cpu().numpy().view(np.uint64)
        rng = np.random.default_rng(5)
        local = np.sort(rng.choice(n, 300, replace=False))
        ids = (local + shard.primary_offset(1, n)).astype(np.uint64)
        o = O.run(mesh, TABLE, 450.0, 20.0, 0, seed=1806, prim_ids=ids, records=True)
        want = primary_hashes(o["records"], ids)
        assert np.sum(dev[local] != want) <= 1
