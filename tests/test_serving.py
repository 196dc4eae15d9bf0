"""Continuous batching (the serving loop): requests of different sizes that
arrive while others are on the GPU are packed into shared launches on
co-resident slots, and each result equals the same request served alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_14306_gb300 import scenes  # noqa: E402


@pytest.mark.parametrize("solo", [None, 100_000])
def test_served_results_equal_standalone_calls(solo):
    # solo: clouds of at least that many points get a call of their own
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_14306_gb300 import build, hav, serving
    build.build()
    hav.load()
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.integers(3000, 150000, size=24)]
    reqs = []
    for i, n in enumerate(sizes):
        pts = scenes.lidar_exact(n, 100 + i) if n > 20000 else scenes.uniform_box(n, i)
        m = [n // 4, n // 16, min(4096, n)][i % 3]
        reqs.append(serving.Request(i, arrival=0.002 * (i // 6), points=torch.from_numpy(pts).pin_memory(), m=m))
    srv = serving.Server(slots=3, slot_points=400_000, max_segments=16, solo_points=solo)
    try:
        res = srv.serve(reqs)
    finally:
        srv.close()
    assert sorted(res) == list(range(len(reqs)))
    assert max(r.batch for r in res.values()) > 1  # requests really shared launches
    if solo:
        assert all(res[r.rid].batch == 1 for r in reqs if r.points.shape[0] >= solo)
    ctx = hav.Context(150000, 1)
    try:
        for r in reqs:
            alone = hav.hav_sample(ctx, r.points.cuda(), r.m).cpu().numpy()
            assert np.array_equal(res[r.rid].indices, alone), r.rid
    finally:
        ctx.close()


def test_served_c5_requests_match_the_oracle_and_contain_errors():
    """C5-shaped requests (N log-uniform in [10k, 1M]; LiDAR up to 200k, indoor
    rooms above, one room well above 200k; m in {N/4, N/16, 4,096}), one of
    them with a NaN coordinate, served by the continuous-batching loop: every
    good request's indices equal the CPU oracle's, and the bad request alone
    reports HAV_ERR_NONFINITE."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import _gpu_helpers as G
    from paper_2305_14306_gb300 import build, hav, serving
    build.build()
    hav.load()
    sizes = [int(x) for x in scenes.log_uniform_sizes(9, 10_000, 1_000_000, seed=77)] + [650_000]
    clouds = [scenes.scene_for(n, seed=900 + i) for i, n in enumerate(sizes)]
    bad = 3
    clouds[bad] = clouds[bad].copy()
    clouds[bad][clouds[bad].shape[0] // 2, 2] = np.nan
    budgets = [[n // 4, n // 16, min(4096, n)][i % 3] for i, n in enumerate(sizes)]
    reqs = [serving.Request(i, arrival=0.001 * (i // 3), points=torch.from_numpy(c).pin_memory(), m=m)
            for i, (c, m) in enumerate(zip(clouds, budgets))]
    srv = serving.Server(slots=2, slot_points=2 * max(sizes), max_segments=16)
    try:
        res = srv.serve(reqs)
    finally:
        srv.close()
    assert sorted(res) == list(range(len(reqs)))
    good = [i for i in range(len(reqs)) if i != bad]
    ref = G.oracle_many([clouds[i] for i in good], [[budgets[i]] for i in good])
    for i, (levels, _) in zip(good, ref):
        assert res[i].status == hav.HAV_OK, (i, res[i].status)
        assert np.array_equal(res[i].indices, levels[0]), i
    assert res[bad].status == hav.HAV_ERR_NONFINITE
    assert res[bad].indices.shape == (budgets[bad],)
