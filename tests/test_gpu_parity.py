"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element, bit-exact (integer indices; binary32 voxel sizes compared
by their bits), on seeded inputs shaped like the paper's workloads."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import _gpu_helpers as G  # noqa: E402
from paper_2305_14306_gb300 import scenes  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))


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
    c = hv.Context(1 << 21, 256)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def run_levels(hv, ctx, pts, ml, pkw=None):
    p = hv.params(**(pkw or {}))
    outs = hv.hav_sample_levels(ctx, dev(pts), ml, p)
    st, per = hv.hav_status_get(ctx, 1)
    tr = hv.hav_trace_get(ctx, len(ml) * p.layers)
    return [o.cpu().numpy() for o in outs], st, tr, p.layers


def assert_parity(res_gpu, tr_gpu, layers, res_ora, tr_ora):
    for j, (a, b) in enumerate(zip(res_gpu, res_ora)):
        assert a.shape == b.shape, (j, a.shape, b.shape)
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError(f"level {j}: {len(bad)} mismatches, first at {bad[0]}: {a[bad[0]]} vs {b[bad[0]]}")
    for j, lev in enumerate(tr_ora):
        for l, rec in enumerate(lev):
            why = G.traces_equal(tr_gpu[j * layers + l], rec)
            assert why is None, f"level {j} layer {l}: {why}"


# ------------------------------------------------------------------ Cnt
@pytest.mark.parametrize("gen", ["c1", "c2", "c3"])
def test_count_matches_oracle(hv, ctx, oracle_mod, gen):
    pts = {"c1": lambda: scenes.uniform_box(16384, 0),
           "c2": lambda: scenes.lidar_min(16384, 0)[0],
           "c3": lambda: scenes.room_scene(1 << 18, 3)}[gen]()
    d = dev(pts)
    for s in [0.05, 0.21, 0.5, 1.3, 7.0]:
        assert hv.hav_count(ctx, d, s) == oracle_mod.count(pts, s), s
    assert hv.hav_count(ctx, d, 0.3, (1.0, 1.0, 0.88)) == oracle_mod.count(pts, 0.3, (1.0, 1.0, 0.88))


# ----------------------------------------------------------- hand cases
@pytest.mark.parametrize("name", ["line4_m2", "line8_two_layers", "identical_shortfall"])
def test_hand_cases(hv, ctx, name):
    c = GOLD[name]
    pts = np.asarray(c["points"], dtype=np.float32)
    res, st, tr, K = run_levels(hv, ctx, pts, [c["m"]], {"t_max": c["t_max"], "layers": c["layers"]})
    assert st == 0
    assert list(res[0]) == c["out"]
    for l, s_star in enumerate(c["s_star"]):
        assert tr[l]["s_star"] == np.float32(s_star)
    for l, steps in enumerate(c.get("trace", [])):
        assert [float(s) for s in tr[l]["s"]] == [float(x[0]) for x in steps]
        for t, (k, x) in enumerate(zip(tr[l]["K"], steps)):
            if (tr[l]["bounded"] >> t) & 1:  # settled by an earlier layer's count: a bound below m_l
                assert int(x[1]) <= int(k) < tr[l]["m_l"], (l, t)
            else:
                assert int(k) == int(x[1]), (l, t)


# -------------------------------------------------------- full configs
@pytest.mark.parametrize("seed", range(10))
def test_c1_uniform_16k_to_4096(hv, ctx, seed):
    pts = scenes.uniform_box(16384, seed)
    res, st, tr, K = run_levels(hv, ctx, pts, [4096])
    assert st == 0
    (ora, tr_o), = G.oracle_many([pts], [[4096]])
    assert_parity(res, tr, K, ora, tr_o)


@pytest.mark.parametrize("seed,shuffle", [(0, False), (1, False), (2, True), (5, False)])
def test_c2_lidar_chain(hv, ctx, seed, shuffle):
    pts, _ = scenes.lidar_min(16384, seed)
    if shuffle:
        pts = pts[np.random.default_rng(seed).permutation(pts.shape[0])]
    ml = [16384, 4096, 1024, 512]
    res, st, tr, K = run_levels(hv, ctx, pts, ml)
    assert st == 0
    (ora, tr_o), = G.oracle_many([pts], [ml])
    assert_parity(res, tr, K, ora, tr_o)


@pytest.mark.parametrize("seed", [0, 1])
def test_c3_indoor_1m_four_levels(hv, ctx, seed):
    pts = scenes.room_scene(1 << 20, seed)
    ml = [1 << 18, 1 << 16, 1 << 14, 1 << 12]
    res, st, tr, K = run_levels(hv, ctx, pts, ml)
    assert st == 0
    (ora, tr_o), = G.oracle_many([pts], [ml])
    assert_parity(res, tr, K, ora, tr_o)


# ---------------------------------------------------------- edge cases
@pytest.mark.parametrize("n,m", [(1, 1), (7, 3), (513, 100), (1000, 1000), (1000, 999), (2049, 1)])
def test_ragged_sizes(hv, ctx, n, m):
    pts = scenes.uniform_box(n, n + m)
    res, st, tr, K = run_levels(hv, ctx, pts, [m])
    assert st == 0
    (ora, tr_o), = G.oracle_many([pts], [[m]])
    assert_parity(res, tr, K, ora, tr_o)


def test_m_zero_writes_nothing(hv, ctx):
    pts = dev(scenes.uniform_box(100, 1))
    out = torch.full((4,), -7, dtype=torch.int32, device="cuda")
    hv.hav_sample(ctx, pts, 0, out=out)
    assert hv.hav_status_get(ctx)[0] == 0
    assert (out.cpu() == -7).all()


@pytest.mark.parametrize("pkw", [{"t_max": 0}, {"t_max": 1}, {"t_max": 3}, {"layers": 1}, {"layers": 3},
                                 {"aspect": (1.0, 1.0, 0.88)}, {"sigma": (0, 1)}, {"sigma": (1, 2)}])
def test_parameter_variants(hv, ctx, pkw):
    pts = scenes.lidar_min(16384, 3)[0]
    ml = [4096, 1024]
    res, st, tr, K = run_levels(hv, ctx, pts, ml, pkw)
    assert st == 0
    (ora, tr_o), = G.oracle_many([pts], [ml], pkw)
    assert_parity(res, tr, K, ora, tr_o)


@pytest.mark.parametrize("n", [1000, 20000, 150000])  # one CTA, a cluster, the grid kernel
@pytest.mark.parametrize("scale", [2.0 ** -23, 1e-30])
def test_range_error_matches_the_oracle(hv, ctx, oracle_mod, n, scale):
    # a fixed voxel size (Table 6 "Fix") far below the cloud's extent: the cell
    # indices need more than 21 bits (extent / 2^23), or the quotient of the
    # box's minimum is no usable integer (1e-30 times the extent); the library
    # reports HAV_ERR_RANGE where the oracle does, and the segment takes its
    # first m points
    pts = scenes.uniform_box(n, 11)
    ext = float(np.max(pts.max(axis=0) - pts.min(axis=0)))
    pkw = {"fixed_s": float(np.float32(ext * scale)), "layers": 1}
    m = n // 4
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.sample_levels(pts, [m], oracle_mod.params(**pkw))
    assert e.value.status == hv.HAV_ERR_RANGE
    res, st, tr, K = run_levels(hv, ctx, pts, [m], pkw)
    assert st == hv.HAV_ERR_RANGE
    assert np.array_equal(res[0], np.arange(m, dtype=np.int32))


def test_duplicates_and_lattice(hv, ctx):
    rng = np.random.default_rng(0)
    base = rng.uniform(0, 4, size=(300, 3)).astype(np.float32)
    pts = np.concatenate([base, base, np.round(base), np.full((50, 3), 2.0, np.float32)])
    for m in [10, 100, 500, 900]:
        res, st, tr, K = run_levels(hv, ctx, pts, [m])
        assert st == 0
        (ora, tr_o), = G.oracle_many([pts], [[m]])
        assert_parity(res, tr, K, ora, tr_o)


@pytest.mark.parametrize("shift,aspect", [(0.0, (1.0, 1.0, 1.0)), (-8.0, (1.0, 1.0, 0.88))])
def test_bucketed_lattice_on_cell_boundaries(hv, ctx, shift, aspect):
    # a cloud large enough for the Morton bucketing whose box is [shift, shift + 16]
    # on every axis: a 16^3 cell is one unit, and a quarter of the lattice planes
    # lie exactly on cell faces, where voxels counted without the global table
    # would first go wrong
    g = np.arange(65, dtype=np.float32) * np.float32(0.25)
    zz = np.arange(33, dtype=np.float32) * np.float32(0.5)
    x, y, z = np.meshgrid(g, g, zz, indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.float32) + np.float32(shift)
    pts = np.concatenate([pts, pts[::7]])
    assert pts.shape[0] >= 1 << 17
    ml = [40000, 10000, 2500]
    res, st, tr, K = run_levels(hv, ctx, pts, ml, {"aspect": aspect})
    assert st == 0
    (ora, tr_o), = G.oracle_many([pts], [ml], {"aspect": aspect})
    assert_parity(res, tr, K, ora, tr_o)


def test_nonfinite_reports_status(hv, ctx):
    pts = scenes.uniform_box(5000, 2)
    pts[1234, 2] = np.inf
    res, st, tr, K = run_levels(hv, ctx, pts, [100])
    assert st == hv.HAV_ERR_NONFINITE
    assert list(res[0]) == list(range(100))  # documented fill for a segment in error


def test_repeat_is_deterministic(hv, ctx):
    pts = scenes.room_scene(200000, 4)
    a, _, _, _ = run_levels(hv, ctx, pts, [50000, 12500])
    b, _, _, _ = run_levels(hv, ctx, pts, [50000, 12500])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_permutation_invariance_gpu(hv, ctx):
    pts = scenes.uniform_box(16384, 6)
    perm = np.random.default_rng(1).permutation(pts.shape[0])
    a, _, tr, _ = run_levels(hv, ctx, pts, [4096])
    b, _, _, _ = run_levels(hv, ctx, pts[perm], [4096])
    assert all(r["accepted"] for r in tr)
    assert np.array_equal(np.sort(perm[b[0]]), a[0])


# ------------------------------------------------------------- batched
def _batched(hv, ctx, clouds, ml_per_level, pkw=None):
    pts, offs = scenes.concat(clouds)
    S = len(clouds)
    seg_m = np.array(ml_per_level, dtype=np.int64).reshape(-1, S)
    p = hv.params(**(pkw or {}))
    outs = hv.hav_sample_batched(ctx, dev(pts), offs, seg_m, p)
    st, per = hv.hav_status_get(ctx, S)
    tr = hv.hav_trace_get(ctx, seg_m.shape[0] * S * p.layers)
    return [o.cpu().numpy() for o in outs], st, per, tr, seg_m, p.layers


def _split(out, seg_m_level):
    offs = np.concatenate([[0], np.cumsum(seg_m_level)])
    return [out[offs[s]:offs[s + 1]] for s in range(len(seg_m_level))]


def check_batched(hv, ctx, clouds, seg_m, pkw=None):
    outs, st, per, tr, seg_m, layers = _batched(hv, ctx, clouds, seg_m, pkw)
    assert st == 0, per
    S, L = len(clouds), seg_m.shape[0]
    ora = G.oracle_many(clouds, [seg_m[:, s] for s in range(S)], pkw)
    for j in range(L):
        parts = _split(outs[j], seg_m[j])
        for s in range(S):
            assert np.array_equal(parts[s], ora[s][0][j]), (j, s)
            for l in range(layers):
                why = G.traces_equal(tr[(j * S + s) * layers + l], ora[s][1][j][l])
                assert why is None, (j, s, l, why)


def test_batched_mixed_segments(hv, ctx):
    sizes = [20000, 1, 0, 513, 70000, 4096, 33333, 12, 150000, 999]
    clouds = [scenes.lidar_exact(n, 10 + i) if n >= 20000 else scenes.uniform_box(n, i)
              for i, n in enumerate(sizes)]
    m1 = [n // 4 for n in sizes]
    m2 = [n // 16 for n in sizes]
    check_batched(hv, ctx, clouds, [m1, m2])


@pytest.mark.parametrize("knobs", [{}, {"nblocks": 17}])
def test_batched_bucketed_segments_on_cell_boundaries(hv, ctx, knobs):
    # large shuffled segments of a batch are sorted by Morton cell and counted
    # with the ownership test item by item: two lattices whose planes lie on
    # their 16^3 cell faces (boxes [0, 16] and [-8, 8]), a shuffled room and a
    # scan-ordered LiDAR cloud, and between them small clouds that keep their
    # order; 17 blocks give each block several items
    g = np.arange(65, dtype=np.float32) * np.float32(0.25)
    zz = np.arange(33, dtype=np.float32) * np.float32(0.5)
    x, y, z = np.meshgrid(g, g, zz, indexing="ij")
    lat = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.float32)
    lat = np.concatenate([lat, lat[::7]])
    rng = np.random.default_rng(5)
    clouds = [lat[rng.permutation(lat.shape[0])], scenes.uniform_box(3000, 1),
              scenes.lidar_exact(140000, 2), lat[rng.permutation(lat.shape[0])] - np.float32(8.0),
              scenes.room_scene(150000, 3), scenes.uniform_box(20000, 4)]
    sizes = [c.shape[0] for c in clouds]
    old = ctx.get_tuning()
    try:
        ctx.set_tuning(**knobs)
        check_batched(hv, ctx, clouds, [[n // 4 for n in sizes], [n // 16 for n in sizes]])
    finally:
        ctx.set_tuning(**old)


def test_batched_error_is_contained(hv, ctx):
    clouds = [scenes.uniform_box(3000, i) for i in range(4)]
    clouds[2] = clouds[2].copy()
    clouds[2][5, 0] = np.nan
    m = [[700] * 4]
    outs, st, per, tr, seg_m, layers = _batched(hv, ctx, clouds, m)
    assert st == hv.HAV_ERR_NONFINITE
    assert per == [0, 0, hv.HAV_ERR_NONFINITE, 0]
    parts = _split(outs[0], seg_m[0])
    ora = G.oracle_many([clouds[s] for s in (0, 1, 3)], [[700]] * 3)
    for k, s in enumerate((0, 1, 3)):
        assert np.array_equal(parts[s], ora[k][0][0])
    assert list(parts[2]) == list(range(700))


def test_batched_error_in_a_sorted_segment_is_contained(hv, ctx):
    # a NaN in a segment large enough to be sorted by Morton cell: that segment
    # reports HAV_ERR_NONFINITE and takes its first m points, the others stay
    # exact; segments of 2^17 - 1 and 2^17 points sit on either side of the
    # sorting threshold
    bad = scenes.room_scene(140000, 12)
    bad[70000, 1] = np.nan
    clouds = [scenes.uniform_box((1 << 17) - 1, 13), bad, scenes.uniform_box(1 << 17, 14),
              scenes.uniform_box(5000, 15)]
    sizes = [c.shape[0] for c in clouds]
    outs, st, per, tr, seg_m, layers = _batched(hv, ctx, clouds, [[n // 4 for n in sizes], [n // 16 for n in sizes]])
    assert st == hv.HAV_ERR_NONFINITE
    assert per == [0, hv.HAV_ERR_NONFINITE, 0, 0]
    keep = (0, 2, 3)
    ora = G.oracle_many([clouds[s] for s in keep], [[sizes[s] // 4, sizes[s] // 16] for s in keep])
    for j in range(2):
        parts = _split(outs[j], seg_m[j])
        for k, s in enumerate(keep):
            assert np.array_equal(parts[s], ora[k][0][j]), (j, s)
        assert list(parts[1]) == list(range(int(seg_m[j][1]))), j
    # one sorted cloud alone with the same NaN
    res, st1, _, _ = run_levels(hv, ctx, bad, [35000])
    assert st1 == hv.HAV_ERR_NONFINITE
    assert list(res[0]) == list(range(35000))


TUNINGS = [
    {"spec_points": [0, 0, 0], "chunk_min": 64},                       # plain bisection
    {"spec_points": [1 << 31, 1 << 31, 1 << 31], "chunk_min": 32},     # depth 4 wherever it fits
    {"spec_points": [65536, 262144, 524288], "chunk_min": 1024},
    {"spec_points": [32768, 131072, 262144], "chunk_min": 64, "nblocks": 5},
    {"spec_points": [0, 16384, 262144], "chunk_min": 128, "nblocks": 17},
    # emptier tables (the workspace grows on the first of these) and the other
    # pass shapes of the grid kernel
    {"table_log2": 2},
    {"table_log2": 3, "pass_shape": 2},
    {"pass_shape": 1, "spec_points": [0, 0, 0]},
    {"pass_shape": 3, "nblocks": 40},
]


def test_tuning_never_changes_results(hv):
    # the launch-shape knobs cut the work differently; indices, status and
    # traces stay those of the default tuning (which the oracle pins above)
    sizes = [20000, 1, 0, 513, 70000, 4096, 33333, 12, 150000, 999]
    clouds = [scenes.lidar_exact(n, 40 + i) if n >= 20000 else scenes.uniform_box(n, 40 + i)
              for i, n in enumerate(sizes)]
    ms = [[n // 4 for n in sizes], [n // 16 for n in sizes]]
    big = scenes.room_scene(300_000, seed=3)
    c = hv.Context(1 << 20, 16)
    try:
        ref_b = _batched(hv, c, clouds, ms)
        ref_c = run_levels(hv, c, big, [75_000, 18_750, 4_687])
        for t in TUNINGS:
            c.set_tuning(**t)
            got_b = _batched(hv, c, clouds, ms)
            got_c = run_levels(hv, c, big, [75_000, 18_750, 4_687])
            for a, b in zip(got_b[0], ref_b[0]):
                assert np.array_equal(a, b), t
            assert got_b[1] == ref_b[1] and got_b[2] == ref_b[2], t
            for j in range(len(ref_c[0])):
                assert np.array_equal(got_c[0][j], ref_c[0][j]), (t, j)
            assert len(got_b[3]) == len(ref_b[3]) and len(got_c[2]) == len(ref_c[2])
            for x, y in zip(got_b[3] + got_c[2], ref_b[3] + ref_c[2]):
                assert G.traces_equal(x, y) is None, (t, G.traces_equal(x, y))
            c.set_tuning(spec_points=[0, 4096, 65536], chunk_min=64, nblocks=0, table_log2=1, pass_shape=0)
        assert c.get_tuning()["chunk_min"] == 64 and c.get_tuning()["table_log2"] == 1
        with pytest.raises(hv.HavError):
            c.set_tuning(spec_points=[3, 2, 1])
        with pytest.raises(hv.HavError):
            c.set_tuning(chunk_min=0)
        for bad in ({"table_log2": 0}, {"table_log2": 4}, {"pass_shape": 4}, {"pass_shape": -1}):
            with pytest.raises(hv.HavError):
                c.set_tuning(**bad)
    finally:
        c.close()


def test_many_segments_on_few_blocks(hv):
    # 200 segments on a context limited to one block: the call widens to
    # ceil(200 / 7) blocks so that no block owns more work items than it tracks
    clouds = [scenes.uniform_box(300 + 37 * i, 500 + i) for i in range(200)]
    total = sum(c.shape[0] for c in clouds)
    c = hv.Context(total, 200)
    try:
        c.set_blocks(1)
        check_batched(hv, c, clouds, [[x.shape[0] // 4 for x in clouds]])
    finally:
        c.close()


@pytest.mark.slow
def test_c4_batch_64_lidar_clouds(hv):
    clouds = scenes.lidar_batch(64, seed=0)
    total = sum(c.shape[0] for c in clouds)
    ctx = hv.Context(total, 64)
    try:
        sizes = [c.shape[0] for c in clouds]
        check_batched(hv, ctx, clouds, [[n // 4 for n in sizes], [n // 16 for n in sizes]])
    finally:
        ctx.close()


# ------------------------------------------------------ FPS comparator
# up to 32,768 points on one 8-CTA cluster (some CTAs empty for tiny clouds),
# above it on the cooperative grid
@pytest.mark.parametrize("n,m,seed", [(16384, 512, 0), (16384, 4096, 1), (1000, 100, 2), (5, 5, 3), (3000, 1, 4),
                                      (7, 7, 7), (32768, 700, 8), (32769, 700, 9)])
def test_fps_matches_oracle(hv, ctx, oracle_mod, n, m, seed):
    pts = scenes.uniform_box(n, seed)
    got = hv.hav_fps(ctx, dev(pts), m).cpu().numpy()
    assert hv.hav_status_get(ctx)[0] == 0
    assert np.array_equal(got, oracle_mod.fps(pts, m))


@pytest.mark.parametrize("n,m", [(1_000_003, 64), (2_000_003, 48)])
def test_fps_large_clouds(hv, oracle_mod, n, m):
    # a million points: each block's share held in shared memory; two
    # million: too many for that, read from global memory in every round
    pts = scenes.uniform_box(n, 6)
    ctx = hv.Context(n, 1)
    try:
        got = hv.hav_fps(ctx, dev(pts), m).cpu().numpy()
        assert hv.hav_status_get(ctx)[0] == 0
    finally:
        ctx.close()
    assert np.array_equal(got, oracle_mod.fps(pts, m))


def test_fps_hand_case_and_duplicates(hv, ctx, oracle_mod):
    line = np.array([[x, 0, 0] for x in range(11)], dtype=np.float32)
    assert list(hv.hav_fps(ctx, dev(line), 4).cpu().numpy()) == [0, 10, 5, 2]
    dup = np.repeat(scenes.uniform_box(50, 8), 4, axis=0)
    assert np.array_equal(hv.hav_fps(ctx, dev(dup), 120).cpu().numpy(), oracle_mod.fps(dup, 120))


def test_coverage_fps_vs_hav(hv, ctx):
    # informative comparison (Section 3.1): FPS bounds the covering radius best;
    # HAV is close to it, a uniform random subset is far worse
    pts = scenes.uniform_box(16384, 3)
    d = dev(pts)
    hav_idx = hv.hav_sample(ctx, d, 4096)
    fps_idx = hv.hav_fps(ctx, d, 4096)
    rnd = torch.from_numpy(np.sort(np.random.default_rng(0).choice(16384, 4096, replace=False))).cuda()
    c_hav, c_fps, c_rnd = hv.coverage(d, hav_idx), hv.coverage(d, fps_idx), hv.coverage(d, rnd)
    assert c_fps <= c_hav < c_rnd


@pytest.mark.parametrize("spec", [[0, 4096, 65536], [0, 0, 0], [1 << 31, 1 << 31, 1 << 31]])
def test_small_level_engines_match_the_grid_kernel(hv, spec):
    # levels within 32,768 points per segment run on clusters of 16 or 8 CTAs
    # and levels within 4,096 on one CTA each by default; every combination,
    # the grid kernel alone included, gives the same indices and traces (the
    # grid kernel and the small engines settle the same steps by the same
    # bounds), whatever the grid kernel's speculation depth
    c = hv.Context(1 << 18, 16)
    try:
        c.set_tuning(spec_points=spec)
        t = c.get_tuning()
        assert t["solo_points"] == 4096 and t["small_points"] in (0, 32768) and t["cluster_ctas"] == 0
        pts = scenes.lidar_min(16384, 7)[0]
        sizes = [3000, 1, 0, 700, 4096, 9000]
        clouds = [scenes.uniform_box(n, 30 + i) for i, n in enumerate(sizes)]
        big = scenes.room_scene(60000, 8)
        combos = [(0, 0, 0), (0, 4096, 0)]
        if t["small_points"]:
            combos += [(32768, solo, q) for solo in (0, 4096) for q in (0, 8, 16)]
        res = {}
        for small, solo, q in combos:
            c.set_tuning(small_points=small, solo_points=solo, cluster_ctas=q)
            chain = run_levels(hv, c, pts, [16384, 4096, 1024, 512])
            batch = _batched(hv, c, clouds, [[n // 4 for n in sizes], [n // 16 for n in sizes]])
            chain2 = run_levels(hv, c, big, [30000, 7500, 1875])
            res[(small, solo, q)] = (chain, batch, chain2)
        ref = res[(0, 0, 0)]
        for key, (ch, ba, ch2) in res.items():
            for a, b in ((ch, ref[0]), (ch2, ref[2])):
                for j in range(len(a[0])):
                    assert np.array_equal(a[0][j], b[0][j]), (key, j)
                for x, y in zip(a[2], b[2]):
                    assert G.traces_equal(x, y) is None, (key, G.traces_equal(x, y))
            for a, b in zip(ba[0], ref[1][0]):
                assert np.array_equal(a, b), key
            assert ba[1] == 0, key
            for x, y in zip(ba[3], ref[1][3]):
                assert G.traces_equal(x, y) is None, (key, G.traces_equal(x, y))
        with pytest.raises(hv.HavError):
            c.set_tuning(solo_points=4097)
        for q in (1, 4, 12, 32, -8):
            with pytest.raises(hv.HavError):
                c.set_tuning(cluster_ctas=q)
    finally:
        c.close()


# ------------------------------------------------------ limits of the boundary
def test_maximum_segment_count(hv, ctx):
    # 256 segments, the most a call takes: two large clouds that are sorted by
    # Morton cell (one at exactly 2^17 points, where that starts), the others
    # small, empty or single points
    rng = np.random.default_rng(77)
    sizes = [int(x) for x in rng.integers(0, 2500, size=256)]
    sizes[3], sizes[200], sizes[17], sizes[90] = 131072, 140000, 0, 1
    clouds = [scenes.room_scene(n, 40 + i) if n >= 131072 else scenes.uniform_box(n, 40 + i)
              for i, n in enumerate(sizes)]
    check_batched(hv, ctx, clouds, [[n // 4 for n in sizes], [n // 16 for n in sizes]])
    with pytest.raises(hv.HavError):
        hv.Context(1000, 257)


@pytest.mark.parametrize("pkw,ml", [
    ({"layers": 8, "layer_ratio": 2}, [16384]),  # the most layers
    ({"layers": 8}, [16384, 4096]),  # ratio 4: the first layers get no budget and are skipped
    ({}, [32768, 16384, 8192, 4096, 2048, 1024, 512, 256]),  # the most levels
])
def test_maximum_layers_and_levels(hv, ctx, pkw, ml):
    pts = scenes.room_scene(65536, 12)
    res, st, tr, K = run_levels(hv, ctx, pts, ml, pkw)
    assert st == 0
    (ora, tr_o), = G.oracle_many([pts], [ml], pkw)
    assert_parity(res, tr, K, ora, tr_o)
    with pytest.raises(hv.HavError):
        hv.hav_sample_levels(ctx, dev(pts[:4096]), [256] * 9)


@pytest.mark.slow
def test_eight_million_points(hv, oracle_mod):
    # a room of 2^23 points to 2^21 in one call (one level, two layers)
    n, m = 1 << 23, 1 << 21
    pts = scenes.room_scene(n, 9)
    c = hv.Context(n, 1)
    try:
        got = hv.hav_sample(c, dev(pts), m).cpu().numpy()
        assert hv.hav_status_get(c)[0] == 0
    finally:
        c.close()
    ref = oracle_mod.sample(pts, m)
    assert np.array_equal(got, ref)
