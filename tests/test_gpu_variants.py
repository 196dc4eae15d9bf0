"""GPU parity of the Table 6 variants (Section 4.5) through the C ABI: random
selection, fixed voxel size, and the representative coordinates of the mean,
centre, centre-closest and random strategies, bit-identical to the oracle."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(__file__))
import _gpu_helpers as G  # noqa: E402
from paper_2305_14306_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

CC, RA, ME, CE = 0, 1, 2, 3


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


def gpu_levels(hv, ctx, pts, ml, **kw):
    p = hv.params(**kw)
    outs = hv.hav_sample_levels(ctx, dev(pts), ml, p)
    st, _ = hv.hav_status_get(ctx, 1)
    tr = hv.hav_trace_get(ctx, len(ml) * p.layers)
    return [o.cpu().numpy() for o in outs], st, tr


def check_levels(hv, ctx, pts, ml, **kw):
    res, st, tr = gpu_levels(hv, ctx, pts, ml, **kw)
    assert st == 0
    ora_res, ora_tr = G.oracle_many([pts], [ml], kw)[0]
    layers = kw.get("layers", 2)
    for j in range(len(ml)):
        assert np.array_equal(res[j], ora_res[j]), (kw, j)
        for l in range(layers):
            why = G.traces_equal(tr[j * layers + l], ora_tr[j][l])
            assert why is None, (kw, j, l, why)


@pytest.mark.parametrize("seed", [0, 1, 12345])
@pytest.mark.parametrize("layers", [1, 2])
def test_random_selection_c1(hv, ctx, seed, layers):
    check_levels(hv, ctx, scenes.uniform_box(16384, seed=seed), [4096], layers=layers, select=RA, seed=seed * 7 + 1)


def test_random_selection_lidar_chain(hv, ctx):
    pts = scenes.lidar_min(16384, seed=3)[0]
    check_levels(hv, ctx, pts, [16384, 4096, 1024, 512], select=RA, seed=99)


def test_random_selection_batched(hv, ctx):
    # draws count from each segment's own first point
    sizes = [20000, 513, 0, 7000, 1]
    clouds = [scenes.lidar_exact(n, 70 + i) if n >= 20000 else scenes.uniform_box(n, 70 + i)
              for i, n in enumerate(sizes)]
    pts, offs = scenes.concat(clouds)
    seg_m = np.array([[n // 4 for n in sizes]], dtype=np.int64)
    p = hv.params(select=RA, seed=5)
    outs = hv.hav_sample_batched(ctx, dev(pts), offs, seg_m, p)
    st, _ = hv.hav_status_get(ctx, len(sizes))
    assert st == 0
    got = outs[0].cpu().numpy()
    ora = G.oracle_many(clouds, [[n // 4] for n in sizes], {"select": RA, "seed": 5})
    cut = np.concatenate([[0], np.cumsum(seg_m[0])])
    for s in range(len(sizes)):
        assert np.array_equal(got[cut[s]:cut[s + 1]], ora[s][0][0]), s


@pytest.mark.parametrize("fixed_s,m", [(1.0, 4096), (3.0, 4096), (10.0, 256), (0.5, 16000)])
def test_fixed_voxel_c1(hv, ctx, fixed_s, m):
    check_levels(hv, ctx, scenes.uniform_box(16384, seed=2), [m], layers=1, fixed_s=fixed_s)


def test_fixed_voxel_room(hv, ctx):
    pts = scenes.room_scene(100_000, seed=4)
    check_levels(hv, ctx, pts, [25000], layers=1, fixed_s=0.05)
    check_levels(hv, ctx, pts, [25000], layers=1, fixed_s=0.05, select=RA, seed=3)


XYZ_CASES = [
    ("uniform cut-off", lambda: scenes.uniform_box(16384, seed=8), 4096),
    ("uniform shortfall", lambda: scenes.uniform_box(16384, seed=8), 15000),
    ("room", lambda: scenes.room_scene(65536, seed=5), 16384),
    ("lattice duplicates", lambda: np.repeat(np.stack(np.meshgrid(*[np.arange(12, dtype=np.float32)] * 3),
                                                      -1).reshape(-1, 3), 3, axis=0), 500),
]


@pytest.mark.parametrize("select", [CC, RA, ME, CE])
@pytest.mark.parametrize("name,make,m", XYZ_CASES)
def test_representative_coordinates(hv, ctx, oracle_mod, select, name, make, m):
    pts = np.ascontiguousarray(make(), dtype=np.float32)
    p = hv.params(layers=1, select=select, seed=17)
    idx, xyz = hv.hav_sample_xyz(ctx, dev(pts), m, p)
    st, _ = hv.hav_status_get(ctx, 1)
    assert st == 0
    o_idx, o_xyz = oracle_mod.sample_xyz(pts, m, oracle_mod.params(layers=1, select=select, seed=17))
    assert np.array_equal(idx.cpu().numpy(), o_idx), name
    got = xyz.cpu().numpy()
    bad = np.nonzero((got.view(np.uint32) != o_xyz.view(np.uint32)).any(axis=1))[0]
    assert bad.size == 0, (name, bad[:5], got[bad[:3]], o_xyz[bad[:3]])
    # the tables are left empty: an ordinary call right after is still exact
    check_levels(hv, ctx, pts, [m], layers=1)


def test_xyz_after_an_error_reports_the_points(hv, ctx):
    pts = scenes.uniform_box(3000, seed=1)
    pts[10, 1] = np.nan
    idx, xyz = hv.hav_sample_xyz(ctx, dev(pts), 500, hv.params(layers=1, select=ME))
    st, _ = hv.hav_status_get(ctx, 1)
    assert st == hv.HAV_ERR_NONFINITE
    got = xyz.cpu().numpy()
    want = pts[idx.cpu().numpy()]
    assert np.array_equal(np.nan_to_num(got, nan=-7), np.nan_to_num(want, nan=-7))
    check_levels(hv, ctx, scenes.uniform_box(3000, seed=1), [500], layers=1)


def test_variant_parameters_rejected(hv, ctx):
    pts = dev(scenes.uniform_box(1000, seed=1))
    for kw in ({"layers": 2, "select": ME}, {"layers": 2, "select": CE}, {"layers": 2, "fixed_s": 1.0},
               {"layers": 1, "select": 4}, {"layers": 1, "select": -1}, {"layers": 1, "fixed_s": -1.0},
               {"layers": 1, "fixed_s": float("nan")}, {"layers": 1, "fixed_s": float("inf")}):
        with pytest.raises(hv.HavError):
            hv.hav_sample(ctx, pts, 100, hv.params(**kw))
    with pytest.raises(hv.HavError):
        hv.hav_sample_xyz(ctx, pts, 100, hv.params(layers=2))


# ------------------------------------------- small levels on thread-block clusters
def test_cluster_levels_match_the_oracle(hv, oracle_mod):
    # the same sampler on clusters (opt-in): identical indices and traces
    c = hv.Context(1 << 20, 16)
    try:
        c.set_tuning(small_points=32768)
        check_levels(hv, c, scenes.uniform_box(16384, seed=0), [4096])
        check_levels(hv, c, scenes.uniform_box(16384, seed=1), [4096], layers=1, select=RA, seed=4)
        check_levels(hv, c, scenes.lidar_min(16384, seed=2)[0], [16384, 4096, 1024, 512])
        check_levels(hv, c, scenes.room_scene(1 << 18, seed=1), [1 << 16, 1 << 14, 1 << 12])  # split launch
        check_levels(hv, c, scenes.uniform_box(16384, seed=3), [4096], layers=1, fixed_s=3.0)
        for n, m in ((1, 1), (7, 3), (513, 100), (1000, 1000), (2049, 1)):
            check_levels(hv, c, scenes.uniform_box(n, seed=n), [m])
        sizes = [20000, 1, 0, 513, 7000, 4096]
        clouds = [scenes.lidar_exact(n, 90 + i) if n >= 20000 else scenes.uniform_box(n, 90 + i)
                  for i, n in enumerate(sizes)]
        pts, offs = scenes.concat(clouds)
        seg_m = np.array([[n // 4 for n in sizes], [n // 16 for n in sizes]], dtype=np.int64)
        outs = hv.hav_sample_batched(c, dev(pts), offs, seg_m, hv.params())
        st, _ = hv.hav_status_get(c, len(sizes))
        assert st == 0
        ora = G.oracle_many(clouds, [seg_m[:, s] for s in range(len(sizes))])
        for j in range(2):
            cut = np.concatenate([[0], np.cumsum(seg_m[j])])
            got = outs[j].cpu().numpy()
            for s in range(len(sizes)):
                assert np.array_equal(got[cut[s]:cut[s + 1]], ora[s][0][j]), (j, s)
        bad = scenes.uniform_box(3000, seed=1)
        bad[5, 2] = np.nan
        outs = hv.hav_sample_levels(c, dev(bad), [700], hv.params())
        st, _ = hv.hav_status_get(c, 1)
        assert st == hv.HAV_ERR_NONFINITE and outs[0].cpu().numpy().tolist() == list(range(700))
    finally:
        c.close()
