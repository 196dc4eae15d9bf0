"""Continuous batching (the serving loop): requests of different sizes that
arrive while others are on the GPU are packed into shared launches on
co-resident slots, and each result equals the same request served alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_14306_gb300 import scenes  # noqa: E402


def test_served_results_equal_standalone_calls():
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
    srv = serving.Server(slots=3, slot_points=400_000, max_segments=16)
    try:
        res = srv.serve(reqs)
    finally:
        srv.close()
    assert sorted(res) == list(range(len(reqs)))
    assert max(r.batch for r in res.values()) > 1  # requests really shared launches
    ctx = hav.Context(150000, 1)
    try:
        for r in reqs:
            alone = hav.hav_sample(ctx, r.points.cuda(), r.m).cpu().numpy()
            assert np.array_equal(res[r.rid].indices, alone), r.rid
    finally:
        ctx.close()
