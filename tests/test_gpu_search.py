"""GPU parity of the guided search start (HAV_SEARCH_GUIDED, the start of the
Section 3.3 search from the cloud's previous search) through the C ABI:
indices and every evaluated size and count identical to the oracle's guided
mode, on the benchmark shapes, level chains, batches, every speculation depth
and the allocation-free entry point."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(__file__))
import _gpu_helpers as G  # noqa: E402
from paper_2305_14306_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu
GUIDED = {"search": "guided"}


@pytest.fixture(scope="module")
def hv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_14306_gb300 import build, hav
    build.build()
    hav.load()
    return hav


@pytest.fixture(scope="module")
def ctx(hv):
    c = hv.Context(1 << 20, 64)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def run_levels(hv, ctx, pts, ml, pkw):
    p = hv.params(**pkw)
    outs = hv.hav_sample_levels(ctx, dev(pts), ml, p)
    st, _ = hv.hav_status_get(ctx, 1)
    tr = hv.hav_trace_get(ctx, len(ml) * p.layers)
    return [o.cpu().numpy() for o in outs], st, tr, p.layers


def check_levels(hv, ctx, pts, ml, pkw=GUIDED):
    res, st, tr, layers = run_levels(hv, ctx, pts, ml, pkw)
    assert st == 0
    (ora, tr_o), = G.oracle_many([pts], [ml], pkw)
    for j in range(len(ml)):
        assert np.array_equal(res[j], ora[j]), j
        for l in range(layers):
            why = G.traces_equal(tr[j * layers + l], tr_o[j][l])
            assert why is None, (j, l, why)
    return tr


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_c1_guided(hv, ctx, seed):
    check_levels(hv, ctx, scenes.uniform_box(16384, seed), [4096])


@pytest.mark.parametrize("seed,shuffle", [(0, False), (1, True), (2, False)])
def test_c2_chain_guided(hv, ctx, seed, shuffle):
    pts = scenes.lidar_min(16384, seed)[0]
    if shuffle:
        pts = pts[np.random.default_rng(seed).permutation(pts.shape[0])]
    check_levels(hv, ctx, pts, [16384, 4096, 1024, 512])


def test_c3_chain_guided(hv, ctx):
    tr = check_levels(hv, ctx, scenes.room_scene(1 << 20, 0), [1 << 18, 1 << 16, 1 << 14, 1 << 12])
    # the later searches start near s*: fewer steps than the first one's bracket
    assert sum(int(t["iters"]) for t in tr) < 100


@pytest.mark.parametrize("pkw", [{"layers": 3}, {"layers": 1}, {"aspect": (1.0, 1.0, 0.88)},
                                 {"sigma": (0, 1)}, {"t_max": 3}, {"select": 1, "seed": 9}])
def test_guided_with_other_parameters(hv, ctx, pkw):
    check_levels(hv, ctx, scenes.lidar_min(16384, 3)[0], [4096, 1024], {**GUIDED, **pkw})


def test_batched_guided(hv, ctx):
    sizes = [20000, 1, 0, 513, 70000, 4096, 33333, 12, 150000, 999]
    clouds = [scenes.lidar_exact(n, 10 + i) if n >= 20000 else scenes.uniform_box(n, i)
              for i, n in enumerate(sizes)]
    pts, offs = scenes.concat(clouds)
    seg_m = np.array([[n // 4 for n in sizes], [n // 16 for n in sizes]], dtype=np.int64)
    p = hv.params(**GUIDED)
    outs = hv.hav_sample_batched(ctx, dev(pts), offs, seg_m, p)
    st, per = hv.hav_status_get(ctx, len(sizes))
    assert st == 0, per
    tr = hv.hav_trace_get(ctx, 2 * len(sizes) * p.layers)
    ora = G.oracle_many(clouds, [seg_m[:, s] for s in range(len(sizes))], GUIDED)
    S = len(sizes)
    for j in range(2):
        cut = np.concatenate([[0], np.cumsum(seg_m[j])])
        got = outs[j].cpu().numpy()
        for s in range(S):
            assert np.array_equal(got[cut[s]:cut[s + 1]], ora[s][0][j]), (j, s)
            for l in range(p.layers):
                why = G.traces_equal(tr[(j * S + s) * p.layers + l], ora[s][1][j][l])
                assert why is None, (j, s, l, why)


TUNINGS = [
    {"spec_points": [0, 0, 0], "chunk_min": 64},
    {"spec_points": [1 << 31, 1 << 31, 1 << 31], "chunk_min": 32},
    {"spec_points": [65536, 262144, 524288], "chunk_min": 1024},
    {"spec_points": [32768, 131072, 262144], "chunk_min": 64, "nblocks": 5},
]


@pytest.mark.parametrize("t", TUNINGS)
def test_every_speculation_depth_walks_the_guided_search(hv, t):
    # a pass evaluates a subtree of the guided search (doubling, then
    # bisection); every depth must land on the oracle's sizes
    c = hv.Context(1 << 18, 16)
    try:
        c.set_tuning(**t)
        check_levels(hv, c, scenes.room_scene(200_000, 6), [50_000, 12_500, 3_125])
        check_levels(hv, c, scenes.lidar_min(16384, 5)[0], [16384, 4096, 1024, 512])
    finally:
        c.close()


def test_noalloc_guided(hv):
    pts = scenes.lidar_min(16384, 4)[0][:20000]
    p = hv.params(**GUIDED)
    out = hv.hav_sample_noalloc(dev(pts), 5000, p).cpu().numpy()
    (ora, _), = G.oracle_many([pts], [[5000]], GUIDED)
    assert np.array_equal(out, ora[0])


@pytest.mark.parametrize("small,solo,q", [(0, 0, 0), (0, 4096, 0), (32768, 0, 8), (32768, 0, 16),
                                          (32768, 4096, 0), (32768, 4096, 16)])
def test_small_level_engines_run_the_guided_search(hv, small, solo, q):
    # the cluster and single-CTA engines take the guided start too, with the
    # previous search handed on from the kernel that ran the earlier levels;
    # every engine combination lands on the oracle's sizes and indices
    c = hv.Context(1 << 18, 16)
    try:
        if small and c.get_tuning()["small_points"] == 0:
            pytest.skip("no cluster launch on this device")
        c.set_tuning(small_points=small, solo_points=solo, cluster_ctas=q)
        check_levels(hv, c, scenes.lidar_min(16384, 6)[0], [16384, 4096, 1024, 512])
        check_levels(hv, c, scenes.room_scene(60000, 9), [30000, 7500, 1875, 400])
        check_levels(hv, c, scenes.uniform_box(16384, 4), [4096], {**GUIDED, "layers": 3})
    finally:
        c.close()
