"""Pins of the oracle's guided search start (Section 3.3; the paper bounds the
search by ceil(log 1/sigma) steps but does not say where it starts): the oracle
against an independent numpy restatement with brute-force counts, exact counts
along the trace at scale, the tolerance of every accepted size, the case that
reduces to the plain bisection, and fewer steps on the benchmark shapes."""
import numpy as np
import pytest

import _indep as ind
from paper_2305_14306_gb300 import scenes

F32 = np.float32


def _trace_pairs(t):
    return [(F32(s), int(k)) for s, k in zip(t["s"], t["K"])]


@pytest.mark.parametrize("seed,m,layers", [(0, 400, 2), (1, 900, 2), (2, 1500, 3), (3, 700, 1)])
def test_guided_matches_numpy_restatement(oracle_mod, seed, m, layers):
    pts = scenes.uniform_box(3000, seed=60 + seed)
    got, tr = oracle_mod.sample_levels(pts, [m], oracle_mod.params(layers=layers, search="guided"),
                                       want_trace=True)
    want, wtr = ind.hav_reference_levels_small(pts, [m], search="guided", layers=layers)
    assert np.array_equal(got[0], want[0])
    for l in range(layers):
        assert _trace_pairs(tr[0][l]) == [(F32(s), int(k)) for s, k in wtr[0][l]], l


@pytest.mark.parametrize("m", [4, 16])
def test_guided_doubling_stops_below_the_top(oracle_mod, m):
    # m a power of 4: the first guess s_hi / sqrt(m) = s_hi / 2^j is exact, and
    # with few voxels wanted every doubling stays above k_max up to s_hi / 2;
    # there 2 lo equals s_hi, which is not below the top, so the search bisects
    pts = scenes.uniform_box(3000, seed=70)
    got, tr = oracle_mod.sample_levels(pts, [m], oracle_mod.params(layers=1, search="guided"),
                                       want_trace=True)
    want, wtr = ind.hav_reference_levels_small(pts, [m], search="guided", layers=1)
    pairs = _trace_pairs(tr[0][0])
    assert np.array_equal(got[0], want[0])
    assert pairs == [(F32(s), int(k)) for s, k in wtr[0][0]]
    _, s_hi = ind.bbox_s_hi(pts)
    assert all(s < s_hi for s, _ in pairs)  # the top itself is never evaluated
    assert any(s == F32(s_hi * F32(0.5)) for s, _ in pairs)  # the doubling reached s_hi / 2


@pytest.mark.parametrize("seed", [0, 1])
def test_guided_level_chain_matches_numpy_restatement(oracle_mod, seed):
    # the start of every later search comes from the previous one, across levels
    pts = scenes.lidar_min(4096, seed=seed)[0][:4500]
    ml = [2048, 512, 128]
    got, tr = oracle_mod.sample_levels(pts, ml, oracle_mod.params(search="guided"), want_trace=True)
    want, wtr = ind.hav_reference_levels_small(pts, ml, search="guided")
    for j in range(len(ml)):
        assert np.array_equal(got[j], want[j]), j
        for l in range(2):
            assert _trace_pairs(tr[j][l]) == [(F32(s), int(k)) for s, k in wtr[j][l]], (j, l)


def test_guided_counts_are_exact_at_scale(oracle_mod):
    # every size the first search evaluates on 200k room points, recounted in numpy
    pts = scenes.room_scene(200_000, seed=7)
    _, tr = oracle_mod.sample_levels(pts, [50_000], oracle_mod.params(search="guided"), want_trace=True)
    t0 = tr[0][0]
    _, s_hi = ind.bbox_s_hi(pts)
    assert F32(t0["s_hi"]) == s_hi
    assert F32(t0["s"][0]) == F32(s_hi / np.sqrt(F32(t0["m_l"])))
    for s, K in zip(t0["s"], t0["K"]):
        assert ind.count_unique(pts, F32(s)) == K


@pytest.mark.parametrize("gen", ["uniform", "lidar", "room"])
def test_guided_accepts_within_the_tolerance(oracle_mod, gen):
    pts = {"uniform": lambda: scenes.uniform_box(16384, 3), "lidar": lambda: scenes.lidar_min(16384, 2)[0],
           "room": lambda: scenes.room_scene(1 << 17, 5)}[gen]()
    ml = [pts.shape[0] // 4, pts.shape[0] // 16, pts.shape[0] // 64]
    _, tr = oracle_mod.sample_levels(pts, ml, oracle_mod.params(search="guided"), want_trace=True)
    for j in range(len(ml)):
        for t in tr[j]:
            assert t["accepted"], (j, t["iters"])
            assert t["m_l"] <= t["k_star"] <= t["k_max"]
            assert t["K"][-1] == t["k_star"]


def test_guided_reduces_to_bisection_when_the_start_reaches_the_top(oracle_mod):
    # m_l = 1: the first guess s_hi / sqrt(1) is not below s_hi
    pts = scenes.uniform_box(500, seed=4)
    a, ta = oracle_mod.sample_levels(pts, [1], oracle_mod.params(layers=1, search="bisect"), want_trace=True)
    b, tb = oracle_mod.sample_levels(pts, [1], oracle_mod.params(layers=1, search="guided"), want_trace=True)
    assert np.array_equal(a[0], b[0])
    assert _trace_pairs(ta[0][0]) == _trace_pairs(tb[0][0])
    # no search at all: identical too
    for search in ("bisect", "guided"):
        out = oracle_mod.sample(pts, 100, oracle_mod.params(t_max=0, search=search))
        assert np.array_equal(out, oracle_mod.sample(pts, 100, oracle_mod.params(t_max=0)))


def test_guided_takes_fewer_steps_on_the_benchmark_shapes(oracle_mod):
    cases = [(scenes.uniform_box(16384, 0), [4096]),
             (scenes.lidar_min(16384, 0)[0], [16384, 4096, 1024, 512]),
             (scenes.room_scene(1 << 18, 1), [1 << 16, 1 << 14, 1 << 12])]
    for pts, ml in cases:
        steps = {}
        for search in ("bisect", "guided"):
            _, tr = oracle_mod.sample_levels(pts, ml, oracle_mod.params(search=search), want_trace=True)
            steps[search] = sum(t["iters"] for lev in tr for t in lev)
        assert steps["guided"] < steps["bisect"], steps


def test_search_mode_is_validated(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.sample(scenes.uniform_box(100, 1), 10, oracle_mod.params(search=2))
