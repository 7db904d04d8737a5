"""Precision form: 8-bit quantised nodes (binary 32-byte, 4-wide 64-byte) and the FP64 re-test (GB300)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1806_00205_gb300 import inputs as I
from tests.parity import check_moments, compare_records, primary_hashes

pytestmark = pytest.mark.gpu
TABLE = I.see_table()


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


def _decode_q8(raw):
    """Decode Q8 nodes as the device does: fmaf(2^23 + q, 2^(b-127), o'), one FP32 rounding.

    (2^23 + q) 2^e and o' are both exact in float64 and close in magnitude, so
    their float64 sum is exact and one cast to float32 is the FMA's rounding."""
    w = raw.view(np.uint32).reshape(-1, 8)
    origin = w[:, 0:3].view(np.float32).astype(np.float64)
    pk = w[:, 3]
    exps = np.stack([(pk >> (8 * k)) & 255 for k in range(3)], axis=1).astype(np.int32) - 127
    scale = np.ldexp(1.0, exps)
    meta = (pk >> 24) & 255
    qb = np.stack([(w[:, 4 + k // 4] >> (8 * (k % 4))) & 255 for k in range(12)], axis=1).astype(np.float64)
    gamma = w[:, 7].view(np.int32)
    boxes = np.empty((w.shape[0], 2, 2, 3), dtype=np.float32)      # node, child, lo/hi, axis
    for c in range(2):
        for lh in range(2):
            for ax in range(3):
                q = qb[:, 6 * c + 3 * lh + ax]
                boxes[:, c, lh, ax] = ((8388608.0 + q) * scale[:, ax] + origin[:, ax]).astype(np.float32)
    cnt0 = ((meta >> 1) & 7).astype(np.int64)
    cnt1 = ((meta >> 5) & 7).astype(np.int64)
    g = gamma.astype(np.int64)
    ref0 = np.where(meta & 1, ~(((g - cnt0) << 3) | cnt0), g)
    ref1 = np.where(meta & 16, ~(((g + 1) << 3) | cnt1), g + 1)
    return boxes, ref0.astype(np.int32), ref1.astype(np.int32)


def _decode_fp32(raw):
    f = raw.view(np.float32).reshape(-1, 16)
    i = raw.view(np.int32).reshape(-1, 16)
    boxes = np.empty((f.shape[0], 2, 2, 3), dtype=np.float32)
    boxes[:, 0, 0] = np.stack([f[:, 0], f[:, 2], f[:, 8]], axis=1)
    boxes[:, 0, 1] = np.stack([f[:, 1], f[:, 3], f[:, 9]], axis=1)
    boxes[:, 1, 0] = np.stack([f[:, 4], f[:, 6], f[:, 10]], axis=1)
    boxes[:, 1, 1] = np.stack([f[:, 5], f[:, 7], f[:, 11]], axis=1)
    return boxes, i[:, 12], i[:, 13]


@pytest.mark.parametrize("n,p,leaf", [(16, 0.5, 4), (48, 0.3, 1), (128, 0.6, 4)])
def test_q8_boxes_contain_fp32_boxes(ctx, n, p, leaf):
    """Exhaustive: every decoded 8-bit child box contains its FP32 box (both widened by M 2^-22)."""
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(n, p)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=rtmc.BVH_Q8, leaf=leaf)
    qb, q0, q1 = _decode_q8(ctx.export_bvh(mid, 1))
    fb, f0, f1 = _decode_fp32(ctx.export_bvh(mid, 0))
    ctx.unload_mesh(mid)
    assert qb.shape == fb.shape
    assert np.all(qb[:, :, 0] <= fb[:, :, 0]) and np.all(qb[:, :, 1] >= fb[:, :, 1])
    assert np.array_equal(q0, f0) and np.array_equal(q1, f1)
    # the quantised boxes stay tight: at most a few quanta looser per side
    ext = np.maximum(fb[:, :, 1] - fb[:, :, 0], 1e-6)
    grow = ((qb[:, :, 1] - qb[:, :, 0]) - (fb[:, :, 1] - fb[:, :, 0])) / ext
    assert np.median(grow) < 0.05


def _decode_q4(raw):
    """Quantised 4-wide nodes: the exact planes o' + (1 + q 2^-15) S with S = 2^15 s (float64
    holds them exactly: (m + q) s with |m + q| < 2^24 and s a power of two), the codes, the
    quanta s and the refs."""
    w = raw.view(np.uint32).reshape(-1, 16)
    f = raw.view(np.float32).reshape(-1, 16)[:, :6].astype(np.float64)
    ax = [0, 0, 1, 1, 2, 2]                                   # rows lo.x hi.x lo.y hi.y lo.z hi.z
    q = np.stack([(w[:, 6:12] >> (8 * c)) & 255 for c in range(4)], axis=2).astype(np.float64)
    planes = f[:, ax, None] + (1.0 + q * 2.0 ** -15) * f[:, [3 + a for a in ax], None]
    return planes, q, f[:, 3:6] * 2.0 ** -15, w[:, 12:16].view(np.int32)


@pytest.mark.parametrize("n,p,leaf", [(16, 0.5, 4), (48, 0.3, 1), (128, 0.6, 4)])
def test_q4_planes_enclose_four_wide_boxes(ctx, n, p, leaf):
    """Exhaustive: every quantised 4-wide child plane lies outside its FP32 4-wide plane by at
    least M 2^-22 + s 2^-8, the displacement the one-FMA evaluation may add (s the quantum);
    empty slots keep lo code 255 above hi code 0; the child refs are those of the FP32 4-wide
    nodes."""
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(n, p)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=rtmc.BVH_Q4, leaf=leaf)
    planes, q, s, refs = _decode_q4(ctx.export_bvh(mid, 4))
    w4 = ctx.export_bvh(mid, 3)
    ctx.unload_mesh(mid)
    rows = w4.view(np.float32).reshape(-1, 32)[:, :24].reshape(-1, 6, 4).astype(np.float64)
    wrefs = w4.view(np.int32).reshape(-1, 32)[:, 24:28]
    assert np.array_equal(refs, wrefs)
    box = mesh.box
    big = max(abs(box.lx), abs(box.ly), abs(box.z_min), abs(box.z_top))
    real = refs != np.iinfo(np.int32).min                      # node, child
    rows = np.where(real[:, None, :], rows, 0.0)               # empty slots: +inf boxes, not compared
    need = s[:, [0, 0, 1, 1, 2, 2], None] * 2.0 ** -8 + big * 2.0 ** -22   # node, row, 1
    lo_ok = planes[:, 0::2] <= rows[:, 0::2] - need[:, 0::2]
    hi_ok = planes[:, 1::2] >= rows[:, 1::2] + need[:, 1::2]
    assert np.all(lo_ok | ~real[:, None, :]) and np.all(hi_ok | ~real[:, None, :])
    empty = ~real[:, None, :]
    assert np.all((q[:, 0::2] == 255) | ~empty) and np.all((q[:, 1::2] == 0) | ~empty)
    assert real[:, :2].all()
    # the quantised boxes stay tight: each plane moves out by less than one quantum plus the
    # margin M 2^-21 + s 2^-7 (a plane on a grid line moves a whole quantum: the voxel-grid
    # coordinates of marching-cubes vertices often are)
    sq = s[:, [0, 0, 1, 1, 2, 2], None]
    slack = np.where(np.arange(6)[None, :, None] % 2 == 0, rows - planes, planes - rows)
    r3 = np.broadcast_to(real[:, None, :], slack.shape)
    assert np.all((slack < sq * (1.0 + 2.0 ** -7) + big * 2.0 ** -21) | ~r3)
    assert np.mean((slack / sq)[r3]) < 0.95
    ext = np.maximum(rows[:, 1::2] - rows[:, 0::2], 1e-6)
    grow = ((planes[:, 1::2] - planes[:, 0::2]) - (rows[:, 1::2] - rows[:, 0::2])) / ext
    assert np.median(grow[np.broadcast_to(real[:, None, :], grow.shape)]) < 0.1
    assert np.all(np.isfinite(planes[np.broadcast_to(np.repeat(real[:, None, :], 6, axis=1), planes.shape)]))


@pytest.mark.parametrize("kind,retest", [(1, False), (1, True), (0, True), (3, False), (3, True)])
def test_precision_form_records_match_oracle(ctx, kind, retest):
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(16, 0.5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=kind)
    n = 100_000
    g = ctx.run_records(mid, 300.0, 0.0, n, seed=1806, desc=rtmc.run_desc(fp64_retest=retest))
    ctx.unload_mesh(mid)
    o = O.run(mesh, TABLE, 300.0, 0.0, n, seed=1806, records=True)
    st = compare_records(g["records"], o["records"], mesh=mesh)
    assert st["frac_same"] >= 0.9999, {k: v for k, v in st.items() if k != "mismatch"}
    assert st["t_rel_p999"] <= 1e-5
    assert st["t_bound_violations"] == 0, (st["t_bound_ratio_max"], st["t_bound_worst"])
    check_moments(g, o, st)
    if retest:
        assert 0 < g["retested"] <= 1e-3 * g["rays"]
    else:
        assert g["retested"] == 0


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_fp64_retest_brings_records_closer_to_oracle(ctx, kind):
    """The FP64 decisions replace FP32 ones only where FP32 cannot decide (a facet within
    1e-5 of an edge, a grazing hit): the re-test run never has more per-ray record
    mismatches against the FP64 oracle than the FP32 run on the same streams."""
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(16, 0.5)
    mid = ctx.load_mesh(mesh.tri, mesh.box)
    ctx.build_bvh(mid, kind=kind)
    n = 100_000
    plain = ctx.run_records(mid, 300.0, 60.0, n, seed=1806)
    rt = ctx.run_records(mid, 300.0, 60.0, n, seed=1806, desc=rtmc.run_desc(fp64_retest=True))
    ctx.unload_mesh(mid)
    o = O.run(mesh, TABLE, 300.0, 60.0, n, seed=1806, records=True)
    sp, sr = compare_records(plain["records"], o["records"]), compare_records(rt["records"], o["records"])
    miss_p, miss_r = sp["n_oracle"] - sp["n_same"], sr["n_oracle"] - sr["n_same"]
    assert 0 < rt["retested"] <= 1e-3 * rt["rays"]
    assert miss_r <= miss_p, (miss_r, miss_p)
    assert sr["frac_same"] >= 0.9999


def test_precision_config_sey_vs_plain_and_oracle(ctx):
    """Precision config: 128^3 foams at porosity 0.4 / 0.6 / 0.8, E in {100, 300, 700} eV,
    incidence 0 and 60 deg.  Q8 nodes + FP64 re-test against FP32 nodes (same streams),
    and sampled primaries against the oracle."""
    import torch
    from paper_1806_00205_gb300 import rtmc
    n = 1_000_000
    for porosity in (0.4, 0.6, 0.8):
        mesh = I.grf_foam(128, porosity)
        m32 = ctx.load_mesh(mesh.tri, mesh.box)
        ctx.build_bvh(m32, kind=rtmc.BVH_FP32)
        mq = ctx.load_mesh(mesh.tri, mesh.box)
        ctx.build_bvh(mq, kind=rtmc.BVH_Q8)
        plain, _, _ = ctx.run(m32, [100.0, 300.0, 700.0], [0.0, 60.0], n, 1806)
        prec, _, _ = ctx.run(mq, [100.0, 300.0, 700.0], [0.0, 60.0], n, 1806, desc=rtmc.run_desc(fp64_retest=True))
        for a, b in zip(plain, prec):
            assert abs(a["sey"] - b["sey"]) <= 1e-3
            assert b["retested"] <= 1e-3 * b["rays"]
        h = torch.zeros(n, dtype=torch.int64, device="cuda")
        ctx.run(mq, [300.0], [60.0], n, 1806, desc=rtmc.run_desc(fp64_retest=True, prim_hash=h))
        ids = np.sort(np.random.default_rng(3).choice(n, 150, replace=False)).astype(np.uint64)
        o = O.run(mesh, TABLE, 300.0, 60.0, 0, seed=1806, prim_ids=ids, records=True)
        dev = h.cpu().numpy().view(np.uint64)[ids.astype(np.int64)]
        assert np.sum(dev != primary_hashes(o["records"], ids)) <= 1
        ctx.unload_mesh(m32)
        ctx.unload_mesh(mq)


def test_large_config_tertiaries_sampled(ctx):
    """Large config: 256^3 foam at porosity 0.7 (~8M triangles, Q8 BVH), tertiaries above
    20 eV, 1e8 primaries at 500 eV x 9 angles, 128 / 36 bins -- the launch configuration of
    `bench.py --config large`.  Invariants at full size; sampled primaries vs the oracle."""
    import torch
    from paper_1806_00205_gb300 import rtmc
    mesh = I.grf_foam(256, 0.7)
    assert 6e6 < mesh.n_tri < 1.2e7
    em = rtmc.Emission(regen_min_ev=20.0, max_generation=2)
    c2 = rtmc.Context(0)
    try:
        c2.load_see_tables(TABLE, em)
        mid = c2.load_mesh(mesh.tri, mesh.box)
        c2.build_bvh(mid, kind=rtmc.BVH_Q8)
        n = 100_000_000
        thetas = [10.0 * j for j in range(9)]
        res, he, ha = c2.run(mid, [500.0], thetas, n, 1806, desc=rtmc.run_desc(n_ebins=128, n_abins=36))
        assert he.shape == (9, 128) and ha.shape == (9, 36)
        for r, h in zip(res, he):
            assert r["rays"] == n + r["emitted"]
            assert r["rays"] == r["escaped"] + r["absorbed_low"] + r["absorbed_other"] + r["emitters"] + r["lost"]
            assert r["regenerated"] > 0 and r["lost"] <= 1e-6 * r["rays"]
            assert int(h.sum()) == r["escaped"]
        h = torch.zeros(n, dtype=torch.int64, device="cuda")
        one, _, _ = c2.run(mid, [500.0], [40.0], n, 1806,
                           desc=rtmc.run_desc(n_ebins=128, n_abins=36, prim_hash=h))
        ids = np.sort(np.random.default_rng(8).choice(n, 40, replace=False)).astype(np.uint64)
        o = O.run(mesh, TABLE, 500.0, 40.0, 0, seed=1806, prim_ids=ids, records=True, n_ebins=128, n_abins=36,
                  emission=O.Emission(regen_min_ev=20.0, max_generation=2))
        dev = h.cpu().numpy().view(np.uint64)[ids.astype(np.int64)]
        assert np.sum(dev != primary_hashes(o["records"], ids)) <= 1
        # 4-wide FP32 nodes on the same 9.9M-triangle mesh: the same tallies and the same
        # per-primary event hashes as the Q8 hierarchy (first 1e7 primaries of the 40-degree item)
        m4 = c2.load_mesh(mesh.tri, mesh.box)
        c2.build_bvh(m4, kind=rtmc.BVH_W4)
        n4 = 10_000_000
        hq = torch.zeros(n4, dtype=torch.int64, device="cuda")
        h4 = torch.zeros(n4, dtype=torch.int64, device="cuda")
        rq, _, _ = c2.run(mid, [500.0], [40.0], n4, 1806, desc=rtmc.run_desc(n_ebins=128, n_abins=36, prim_hash=hq))
        r4, _, _ = c2.run(m4, [500.0], [40.0], n4, 1806, desc=rtmc.run_desc(n_ebins=128, n_abins=36, prim_hash=h4))
        for k in ("rays", "escaped", "emitted", "regenerated", "sum_k", "sum_k2", "wraps", "lost"):
            assert rq[0][k] == r4[0][k], k
        assert torch.equal(hq, h4)
        assert torch.equal(hq, h[:n4])          # the prefix of the full 1e8 run
    finally:
        c2.close()
