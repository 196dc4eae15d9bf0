"""GPU parity of the subset point spacing (Fig. 3, Section 3.1) through the C
ABI: bit-identical squared nearest-neighbour distances to the oracle's."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(__file__))
from paper_2305_14306_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu


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
    c = hv.Context(1 << 17, 4)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def check(hv, ctx, oracle_mod, pts, idx):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    got = hv.hav_spacing(ctx, dev(pts), torch.from_numpy(idx).cuda()).cpu().numpy()
    st, _ = hv.hav_status_get(ctx, 1)
    assert st == 0
    want = oracle_mod.spacing(pts, idx)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), np.nonzero(got != want)[0][:5]
    return got


def test_spacing_of_samplers(hv, ctx, oracle_mod):
    pts = scenes.uniform_box(16384, seed=3)
    d = dev(pts)
    hav_idx = hv.hav_sample(ctx, d, 4096).cpu().numpy()
    fps_idx = hv.hav_fps(ctx, d, 1500).cpu().numpy()
    rnd_idx = np.random.default_rng(0).choice(16384, size=5000, replace=False)
    for idx in (hav_idx, fps_idx, rnd_idx):
        check(hv, ctx, oracle_mod, pts, idx)


def test_spacing_lidar_subset_and_order(hv, ctx, oracle_mod):
    pts = scenes.lidar_min(16384, seed=2)[0]
    idx = hv.hav_sample(ctx, dev(pts), 8192).cpu().numpy()
    a = check(hv, ctx, oracle_mod, pts, idx)
    perm = np.random.default_rng(1).permutation(len(idx))
    b = check(hv, ctx, oracle_mod, pts, idx[perm])
    assert np.array_equal(a[perm], b)


def test_spacing_edges(hv, ctx, oracle_mod):
    pts = np.array([[0, 0, 0], [1, 0, 0], [3, 0, 0], [7, 0, 0], [7, 0, 0]], dtype=np.float32)
    got = check(hv, ctx, oracle_mod, pts, [0, 1, 2, 3, 4])
    assert got.tolist() == [1.0, 1.0, 4.0, 0.0, 0.0]
    got = check(hv, ctx, oracle_mod, pts, [2, 2, 1])  # a repeated index is at distance 0
    assert got.tolist() == [0.0, 0.0, 4.0]
    assert np.isinf(check(hv, ctx, oracle_mod, pts, [3])[0])
    out = hv.hav_spacing(ctx, dev(pts), torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert out.shape == (0,)
    # ragged sizes around the tile and block sizes
    big = scenes.uniform_box(9000, seed=5)
    for m in (1023, 1024, 1025, 4097, 8999):
        check(hv, ctx, oracle_mod, big, np.arange(m))


def test_spacing_rejects_bad_indices(hv, ctx):
    pts = dev(scenes.uniform_box(100, seed=1))
    hv.hav_spacing(ctx, pts, torch.tensor([0, 5, 100, 7], dtype=torch.int32, device="cuda"))
    st, _ = hv.hav_status_get(ctx, 1)
    assert st == hv.HAV_ERR_INVALID
    hv.hav_spacing(ctx, pts, torch.tensor([0, 5, 7], dtype=torch.int32, device="cuda"))
    st, _ = hv.hav_status_get(ctx, 1)
    assert st == 0


def numpy_counts(d2, edges):
    """below, numpy.histogram's bins, above: the layout hav_spacing_histogram writes."""
    d2 = np.asarray(d2, dtype=np.float32)
    e = np.asarray(edges, dtype=np.float32)
    hist, _ = np.histogram(d2, bins=e)
    return np.concatenate([[int((d2 < e[0]).sum())], hist, [int((d2 > e[-1]).sum())]]).astype(np.int64)


@pytest.mark.parametrize("sampler", ["hav", "random", "fps"])
def test_spacing_histogram_matches_numpy_on_the_oracle_spacings(hv, ctx, oracle_mod, sampler):
    # Fig. 3's distributions as integer counts: the GPU histogram of the
    # spacings equals numpy.histogram of the oracle's spacings, with edges that
    # include some spacings exactly (the half-open bins and the closed last bin)
    pts = scenes.uniform_box(16384, 3)
    rng = np.random.default_rng(8)
    if sampler == "hav":
        idx = oracle_mod.sample(pts, 4096)
    elif sampler == "fps":
        idx = oracle_mod.fps(pts, 4096)
    else:
        idx = np.sort(rng.choice(16384, size=4096, replace=False))
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    d2 = oracle_mod.spacing(pts, idx)
    geo = np.geomspace(max(float(d2.min()), 1e-6) * 0.5, float(d2.max()) * 0.9, 30)
    exact = rng.choice(d2, size=6, replace=False)
    edges = np.unique(np.concatenate([geo.astype(np.float32), exact, [d2.max()]]).astype(np.float32))
    got_d2, counts = hv.hav_spacing_histogram(ctx, dev(pts), torch.from_numpy(idx).cuda(), edges)
    st, _ = hv.hav_status_get(ctx, 1)
    assert st == 0
    assert np.array_equal(got_d2.cpu().numpy().view(np.uint32), d2.view(np.uint32))
    want = numpy_counts(d2, edges)
    assert np.array_equal(counts.cpu().numpy(), want)
    assert int(want.sum()) == 4096 and want[-1] == 0  # the largest spacing is the closed last edge


def test_spacing_histogram_edge_cases(hv, ctx, oracle_mod):
    pts = scenes.uniform_box(2000, 4)
    idx = np.arange(0, 2000, 7, dtype=np.int32)
    d2 = oracle_mod.spacing(pts, idx)
    # every value below the first edge, every value above the last one, one bin
    for edges in ([float(d2.max()) * 2, float(d2.max()) * 3], [0.0, float(d2.min()) * 0.5], [0.0, 1e9]):
        e = np.asarray(edges, dtype=np.float32)
        _, counts = hv.hav_spacing_histogram(ctx, dev(pts), torch.from_numpy(idx).cuda(), e)
        assert np.array_equal(counts.cpu().numpy(), numpy_counts(d2, e))
    # a subset of one point: +inf spacing, counted above the last edge
    _, counts = hv.hav_spacing_histogram(ctx, dev(pts), torch.from_numpy(idx[:1].copy()).cuda(),
                                         np.array([0.0, 1.0], np.float32))
    assert counts.cpu().numpy().tolist() == [0, 0, 1]
    # edges must be finite and strictly ascending
    for bad in ([1.0, 1.0], [2.0, 1.0], [0.0, np.inf]):
        with pytest.raises(hv.HavError):
            hv.hav_spacing_histogram(ctx, dev(pts), torch.from_numpy(idx).cuda(), np.array(bad, np.float32))


def test_spacing_on_the_grid(hv, ctx, oracle_mod):
    # subsets of 32,768 points and more are searched on a grid, shell by shell
    # around each point's cell, with an exact stopping bound: bit-identical to
    # the oracle's all-pairs minimum on a room, a LiDAR scan (cells near the
    # sensor hold thousands of returns), repeated indices, a NaN point, and a
    # far isolated point that scans the whole subset
    room = scenes.room_scene(120000, 4)
    rng = np.random.default_rng(2)
    check(hv, ctx, oracle_mod, room, rng.choice(120000, 40000, replace=False))
    lidar = scenes.lidar_exact(40000, 2)
    check(hv, ctx, oracle_mod, lidar, np.arange(lidar.shape[0]))
    box = scenes.uniform_box(60000, seed=6)
    idx = rng.choice(60000, 40000, replace=False)
    idx[100:200] = idx[:100]  # repeated indices: spacing 0
    got = check(hv, ctx, oracle_mod, box, idx)
    assert (got[:100] == 0).all()
    nan = box.copy()
    nan[idx[5], 2] = np.nan
    got = check(hv, ctx, oracle_mod, nan, idx[:32768])
    assert np.isinf(got[5])
    far = np.concatenate([scenes.uniform_box(32768, seed=7), np.array([[1e6, 1e6, 1e6]], np.float32)])
    check(hv, ctx, oracle_mod, far, np.arange(far.shape[0]))
