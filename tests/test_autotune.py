"""Autotuner host logic on a fake context (no GPU): the search visits every
allowed candidate on a sample of the batch, keeps the fastest, skips launch
shapes beyond 2048 threads per SM, and caches the choice per device, node
format and mesh sizes."""
import pytest


@pytest.fixture(scope="module")
def autotune():
    from paper_1806_00205_gb300 import build
    build.build()
    from paper_1806_00205_gb300 import autotune as A
    return A


class FakeCtx:
    """run_batch returns a time that is smallest at stack 16, threshold 20, 64 threads, 0 blocks/SM
    (the library defaults use threshold 28, 2 ms slower here)."""

    def __init__(self):
        self.calls = []

    def run_batch(self, ids, energies, thetas, n, seed, desc):
        p = (desc.stack_depth, desc.fetch_threshold, desc.block_threads, desc.blocks_per_sm)
        self.calls.append((list(ids), list(energies), list(thetas), n, seed, p, desc.fp64_retest))
        ms = abs(p[0] - 16) + abs(p[1] - 20) / 4 + (0.5 if p[2] == 128 else 0.0) + 0.01 * p[3]
        ms += 0.25 * (len(self.calls) % 2)          # the second timing of each candidate is faster
        return [{"gpu_ms": ms}], None, None


def test_tune_picks_the_fastest_candidate_on_a_sample(autotune, tmp_path):
    ctx = FakeCtx()
    ids, n_tris = [7, 3, 9, 4], [5000, 200, 90000, 1200]
    energies, thetas = [50.0, 100.0, 300.0, 600.0, 1000.0], [0.0, 20.0, 40.0, 80.0]
    best = autotune.tune(ctx, ids, n_tris, energies, thetas, kind=2, n_sample=1000,
                         cache_path=str(tmp_path / "c.json"), device_name="dev")
    assert best == {"stack_depth": 16, "fetch_threshold": 20, "block_threads": 64, "blocks_per_sm": 0}
    n_cand = 3 * 3 * 2 * 2
    assert len(ctx.calls) == 2 * n_cand                          # every candidate timed twice
    for c in ctx.calls:
        assert c[0] == [3, 9]                                    # smallest and largest mesh
        assert c[1] == [50.0, 300.0, 1000.0] and c[2] == [0.0, 80.0] and c[3] == 1000
    assert {c[5] for c in ctx.calls} == {(s, t, b, k) for s in (8, 16, 32) for t in (12, 20, 28)
                                         for b in (64, 128) for k in (0, 12)}


def test_tune_skips_launch_shapes_beyond_the_sm_thread_limit(autotune):
    ctx = FakeCtx()
    space = {"stack_depth": (16,), "fetch_threshold": (20,), "block_threads": (64, 128),
             "blocks_per_sm": (0, 16, 24)}
    best = autotune.tune(ctx, [0], [100], [300.0], [0.0], cache_path=None, space=space, fp64_retest=True)
    shapes = {c[5][2:] for c in ctx.calls}
    assert shapes == {(64, 0), (64, 16), (64, 24), (128, 0), (128, 16)}     # 128 x 24 > 2048 threads
    assert all(c[6] == 1 for c in ctx.calls)                                 # the re-test flag is passed on
    assert best["blocks_per_sm"] == 0 and best["block_threads"] == 64


def test_tune_caches_per_device_format_and_sizes(autotune, tmp_path):
    path = str(tmp_path / "cache.json")
    ctx = FakeCtx()
    first = autotune.tune(ctx, [0, 1], [100, 5000], [300.0], [0.0], kind=1, cache_path=path, device_name="a")
    n = len(ctx.calls)
    assert autotune.tune(ctx, [0, 1], [100, 5000], [300.0], [0.0], kind=1, cache_path=path,
                         device_name="a") == first
    assert len(ctx.calls) == n                                   # served from the cache
    autotune.tune(ctx, [0, 1], [100, 5000], [300.0], [0.0], kind=3, cache_path=path, device_name="a")
    assert len(ctx.calls) == 2 * n                               # another node format is tuned anew
    autotune.tune(ctx, [0, 1], [100, 7000], [300.0], [0.0], kind=1, cache_path=path, device_name="a")
    assert len(ctx.calls) == 3 * n                               # so are other mesh sizes


class FlatCtx:
    """The defaults take 10 ms, every other candidate 10.05 ms, except (8, 12, 128, 0): `fast` ms."""

    def __init__(self, defaults, fast):
        self.defaults, self.fast = defaults, fast

    def run_batch(self, ids, energies, thetas, n, seed, desc):
        p = (desc.stack_depth, desc.fetch_threshold, desc.block_threads, desc.blocks_per_sm)
        ms = 10.0 if p == self.defaults else (self.fast if p == (8, 12, 128, 0) else 10.05)
        return [{"gpu_ms": ms}], None, None


def test_tune_keeps_the_defaults_unless_clearly_faster(autotune):
    d = autotune.DEFAULTS
    defaults = (d["stack_depth"], d["fetch_threshold"], d["block_threads"], d["blocks_per_sm"])
    assert autotune.MARGIN == 0.02
    kept = autotune.tune(FlatCtx(defaults, 9.9), [0], [100], [300.0], [0.0], cache_path=None)
    assert kept == d                                              # 1 % faster: within the margin
    moved = autotune.tune(FlatCtx(defaults, 9.7), [0], [100], [300.0], [0.0], cache_path=None)
    assert moved == {"stack_depth": 8, "fetch_threshold": 12, "block_threads": 128, "blocks_per_sm": 0}
