"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, never against the oracle itself.

* hand-derived cases (tests/golden/hand_cases.json, each with its citation);
* Eq. 2 cells against an independent numpy float32 computation;
* Cnt against closed-form lattice counts and np.unique;
* S(P, v) against O(n^2) brute-force grouping and a lexsort dedupe;
* the Section 3.3 bisection trace against a numpy re-run;
* nested-grid monotonicity K(2^j s) <= K(s);
* output invariants (exactly m distinct indices, per-layer voxel distinctness,
  centre-closest argmin over untaken points, cut-off keeps smallest priority);
* permutation invariance;
* the published SplitMix64 vectors for the cut-off priority;
* farthest point sampling on hand cases.
"""
import json
import os

import numpy as np
import pytest

import _indep as ind
from paper_2305_14306_gb300 import scenes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))
F32 = np.float32


def P(rows):
    return np.asarray(rows, dtype=np.float32).reshape(-1, 3)


# --------------------------------------------------------------- hand cases
def test_floor_cells_eq2(oracle_mod):
    for x, v, g in GOLD["floor_cells"]["rows"]:
        # a point at x on every axis, plus the origin so the bbox minimum is known
        pts = P([[x, x, x], [min(x, 0.0)] * 3])
        keys = oracle_mod.keys(pts, v)
        gmin = int(np.floor(F32(min(x, 0.0)) / F32(v)))
        u = g - gmin
        assert int(keys[0]) == u | (u << 21) | (u << 42), (x, v, g)
        assert int(np.floor(F32(x) / F32(v))) == g


def test_tie_goes_to_lowest_index(oracle_mod):
    c = GOLD["tie_lowest_index"]
    pts = P(c["points"])
    assert list(oracle_mod.select(pts, c["s"])) == c["reps"]
    # reversed order: the (new) lowest index wins again
    assert list(oracle_mod.select(pts[::-1].copy(), c["s"])) == c["reps"]


@pytest.mark.parametrize("name", ["line4_m2", "line8_two_layers", "identical_shortfall"])
def test_hand_derived_sampler_cases(oracle_mod, name):
    c = GOLD[name]
    p = oracle_mod.params(t_max=c["t_max"], layers=c["layers"])
    out, tr = oracle_mod.sample(P(c["points"]), c["m"], p, want_trace=True)
    assert list(out) == c["out"]
    for l, s_star in enumerate(c["s_star"]):
        assert tr[l]["s_star"] == F32(s_star)
    for l, steps in enumerate(c.get("trace", [])):
        assert [(float(s), int(k)) for s, k in zip(tr[l]["s"], tr[l]["K"])] == [tuple(x) for x in steps]


def test_splitmix64_published_vectors(oracle_mod):
    c = GOLD["splitmix64_seed0"]
    for x, y in zip(c["inputs"], c["outputs"]):
        assert oracle_mod.priority(int(x, 16)) == int(y, 16)
        assert ind.splitmix64_finalise(int(x, 16)) == int(y, 16)


def test_priority_is_a_bijection_sample(oracle_mod):
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 1 << 63, size=2000, dtype=np.int64).astype(np.uint64)
    hs = {oracle_mod.priority(int(x)) for x in xs}
    assert len(hs) == len(set(int(x) for x in xs))


def test_layer_budgets_eq3():
    # m = 4096, k = 2: 819 + 3277 (the 4:1 ratio rounded down, remainder to the last layer)
    assert ind.budgets(4096, 2, 4) == [819, 3277]
    for m in [1, 5, 100, 4096, 262144]:
        for k in [1, 2, 3]:
            b = ind.budgets(m, k, 4)
            assert sum(b) == m and all(x >= 0 for x in b)


# ----------------------------------------------------------------- Eq. 2 / Cnt
@pytest.mark.parametrize("seed", [0, 1])
def test_keys_match_numpy(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    pts = (rng.normal(size=(3000, 3)) * [20, 5, 1]).astype(np.float32)
    pts[:50] = np.round(pts[:50])  # exact multiples of v
    for s in [F32(0.37), F32(1.0), F32(2.5), F32(0.05)]:
        assert np.array_equal(oracle_mod.keys(pts, s), ind.packed_keys(pts, s))
        asp = (1.0, 0.5, 0.25)
        assert np.array_equal(oracle_mod.keys(pts, s, asp), ind.packed_keys(pts, s, asp))


@pytest.mark.parametrize("abc", [(4, 4, 4), (7, 3, 5), (16, 16, 1)])
def test_count_lattice_closed_form(oracle_mod, abc):
    a, b, c = abc
    rng = np.random.default_rng(sum(abc))
    g = np.stack(np.meshgrid(np.arange(a), np.arange(b), np.arange(c), indexing="ij"), -1).reshape(-1, 3)
    pts = (g + rng.uniform(0.25, 0.75, size=g.shape)).astype(np.float32)
    assert oracle_mod.count(pts, 1.0) == a * b * c
    # cells of size 2 anchored at the origin: ceil(a/2) * ceil(b/2) * ceil(c/2)
    assert oracle_mod.count(pts, 2.0) == -(-a // 2) * -(-b // 2) * -(-c // 2)


@pytest.mark.parametrize("gen", ["box", "lidar", "room"])
def test_count_matches_unique_and_nested_monotone(oracle_mod, gen):
    pts = {"box": lambda: scenes.uniform_box(4000, 5),
           "lidar": lambda: scenes.lidar_scene(2)[:5000],
           "room": lambda: scenes.room_scene(5000, 1)}[gen]()
    for s in [F32(0.1), F32(0.33), F32(1.7)]:
        K = oracle_mod.count(pts, s)
        assert K == ind.count_unique(pts, s)
        # nested grids: K(2^j s) <= K(s) (scaling by 2 is exact, floor(q/2) = floor(floor(q)/2))
        prev = K
        for j in range(1, 5):
            Kj = oracle_mod.count(pts, F32(s * (1 << j)))
            assert Kj <= prev
            prev = Kj


# ------------------------------------------------------------------ S(P, v)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_select_equals_brute_force_grouping(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = 1500
    pts = rng.uniform(-3, 3, size=(n, 3)).astype(np.float32)
    pts[n // 2:] = np.round(pts[n // 2:] * 4) / 4  # many exact ties and cell-boundary points
    for s in [F32(0.5), F32(1.0), F32(1.3)]:
        got = oracle_mod.select(pts, s)
        assert np.array_equal(got, ind.brute_force_select(pts, s))
        assert np.array_equal(got, ind.lexsort_select(pts, s))


def test_fixed_size_select_is_textbook_dedupe(oracle_mod):
    pts = scenes.uniform_box(20000, 9)
    s = F32(2.0)
    assert np.array_equal(oracle_mod.select(pts, s), ind.lexsort_select(pts, s))


# ------------------------------------------------------------- bisection
@pytest.mark.parametrize("seed,m", [(0, 200), (1, 500), (2, 1000)])
def test_bisection_trace_matches_numpy(oracle_mod, seed, m):
    pts = scenes.uniform_box(3000, seed)
    p = oracle_mod.params(layers=1)
    _, tr = oracle_mod.sample(pts, m, p, want_trace=True)
    _, s_hi = ind.bbox_s_hi(pts)
    trace, s_star, acc = ind.bisection(pts, m, s_hi)
    assert tr[0]["s_hi"] == s_hi
    assert [(F32(s), int(k)) for s, k in zip(tr[0]["s"], tr[0]["K"])] == trace
    assert tr[0]["s_star"] == s_star and tr[0]["accepted"] == acc


@pytest.mark.parametrize("m,t_max", [(4, 1), (100, 1), (6, 3), (2000, 3)])
def test_unfinished_search_ends_at_the_bracket(oracle_mod, m, t_max):
    # Section 3.3 with no size accepted within t_max steps (sigma = 0): s* is
    # the last lower end when one was found (too many voxels there), else the
    # last upper end; both branches are taken by these cases
    pts = scenes.uniform_box(3000, 5)
    p = oracle_mod.params(layers=1, t_max=t_max, sigma=(0, 1))
    _, tr = oracle_mod.sample(pts, m, p, want_trace=True)
    _, s_hi = ind.bbox_s_hi(pts)
    trace, s_star, acc = ind.bisection(pts, m, s_hi, sigma=(0, 1), t_max=t_max)
    assert not acc and tr[0]["accepted"] == 0
    assert [(F32(s), int(k)) for s, k in zip(tr[0]["s"], tr[0]["K"])] == trace
    assert tr[0]["s_star"] == s_star
    lo_found = any(k > m for _, k in trace)
    assert (s_star < s_hi) if lo_found else (s_star == trace[-1][0])


@pytest.mark.parametrize("seed,m,k", [(0, 300, 2), (1, 800, 2), (2, 100, 3), (3, 1000, 1)])
def test_sampler_matches_numpy_restatement(oracle_mod, seed, m, k):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0, 10, size=(2500, 3)).astype(np.float32)
    pts[:300] = np.round(pts[:300])
    p = oracle_mod.params(layers=k)
    assert np.array_equal(oracle_mod.sample(pts, m, p), ind.hav_reference_small(pts, m, layers=k))


# -------------------------------------------------------------- invariants
def _check_invariants(oracle_mod, pts, m, p):
    out, tr = oracle_mod.sample(pts, m, p, want_trace=True)
    n = pts.shape[0]
    assert out.shape == (m,) and np.all(np.diff(out) > 0) and out.min() >= 0 and out.max() < n
    taken = np.zeros(n, dtype=bool)
    for l, rec in enumerate(tr):
        if rec["m_l"] == 0:
            continue
        active = np.nonzero(~taken)[0]
        assert rec["n_in"] == len(active)
        s = rec["s_star"]
        u, f, v = ind.rel_cells(pts, s)
        d2 = ind.centre_d2(pts, f, v)
        reps_all = ind.lexsort_select(pts, s, active=active)
        assert rec["k_star"] == len(reps_all)
        # layer l's picks: taken after the layer minus taken before
        taken_after = np.zeros(n, dtype=bool)
        taken_after[out] = True
        # reconstruct this layer's picks as the oracle defines them
        if rec["k_star"] >= rec["m_l"]:
            keys = ind.packed_keys(pts, s)
            pr = np.array([ind.splitmix64_finalise(int(keys[i])) for i in reps_all], dtype=np.uint64)
            picks = np.sort(reps_all[np.argsort(pr)[: rec["m_l"]]])
            # distinct voxels at s*, each the centre-closest untaken point of its voxel
            cells = {tuple(u[i]) for i in picks}
            assert len(cells) == len(picks)
            for i in picks:
                same = active[(u[active] == u[i]).all(axis=1)]
                best = same[np.lexsort((same, d2[same]))[0]]
                assert best == i
            assert taken_after[picks].all()
            taken[picks] = True
        else:
            taken[reps_all] = True
            need = rec["m_l"] - rec["k_star"]
            for i in active:
                if need == 0:
                    break
                if not taken[i]:
                    taken[i] = True
                    need -= 1
    assert np.array_equal(np.nonzero(taken)[0], out)
    return out, tr


@pytest.mark.parametrize("case", ["c1", "lidar", "room"])
def test_output_invariants(oracle_mod, case):
    if case == "c1":
        pts, m = scenes.uniform_box(16384, 0), 4096
    elif case == "lidar":
        pts, m = scenes.lidar_scene(1), 4096
    else:
        pts, m = scenes.room_scene(30000, 2), 7500
    _check_invariants(oracle_mod, pts, m, oracle_mod.params())


def test_permutation_invariance(oracle_mod):
    pts = scenes.uniform_box(16384, 4)
    out, tr = oracle_mod.sample(pts, 4096, want_trace=True)
    assert all(r["accepted"] and r["k_star"] >= r["m_l"] for r in tr)  # no shortfall
    perm = np.random.default_rng(11).permutation(pts.shape[0])
    out2 = oracle_mod.sample(pts[perm], 4096)
    a = {tuple(x) for x in pts[out].tolist()}
    b = {tuple(x) for x in pts[perm][out2].tolist()}
    assert a == b
    # index map applied: the same original points
    assert np.array_equal(np.sort(perm[out2]), out)


def test_levels_compose(oracle_mod):
    pts, _ = scenes.lidar_min(16384, 0)
    ml = [16384, 4096, 1024, 512]
    levels = oracle_mod.sample_levels(pts, ml)
    cur_pts, cur_idx = pts, np.arange(pts.shape[0])
    for j, m in enumerate(ml):
        # nested: each level is a subset of the previous one
        assert set(levels[j].tolist()) <= set(cur_idx.tolist())
        sub = oracle_mod.sample(cur_pts, m)
        assert np.array_equal(cur_idx[sub], levels[j])
        cur_pts, cur_idx = cur_pts[sub], cur_idx[sub]


def test_edge_cases(oracle_mod):
    pts = scenes.uniform_box(100, 1)
    assert oracle_mod.sample(pts, 0).shape == (0,)
    assert np.array_equal(oracle_mod.sample(pts, 100), np.arange(100))
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.sample(pts, 101)
    bad = pts.copy()
    bad[7, 1] = np.nan
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.sample(bad, 10)
    assert e.value.status == oracle_mod.ERR_NONFINITE
    one = P([[1, 2, 3]])
    assert list(oracle_mod.sample(one, 1)) == [0]


# --------------------------------------------------------------------- FPS
def test_fps_hand_cases(oracle_mod):
    line = P([[x, 0, 0] for x in range(11)])
    # start at 0, farthest is 10, then the midpoint 5, then 2 (ties 2/3 and 7/8 -> lowest index)
    assert list(oracle_mod.fps(line, 4)) == [0, 10, 5, 2]
    sq = P([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0.5, 0.5, 0]])
    assert list(oracle_mod.fps(sq, 3)) == [0, 3, 1]


def test_fps_covering_property(oracle_mod):
    pts = scenes.uniform_box(1500, 3)
    m = 64
    idx = oracle_mod.fps(pts, m)
    assert len(set(idx.tolist())) == m
    S = pts[idx].astype(np.float64)
    d = np.sqrt(((pts[:, None, :] - S[None, :, :]) ** 2).sum(-1)).min(1)
    cover = d.max()
    sp = np.sqrt(((S[:, None, :] - S[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(sp, np.inf)
    # the greedy farthest-point rule: every pair of samples is at least the final covering radius apart
    assert sp.min() >= cover * (1 - 1e-5)
