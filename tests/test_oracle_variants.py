"""Pins of the oracle's Table 6 variants (Section 4.5): random, mean and centre
point selection and the fixed voxel size, against published generator outputs,
numpy restatements of the grouping, closed forms and exact rational means."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import _indep as ind
from paper_2305_14306_gb300 import scenes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))
F32 = np.float32


def test_random_draws_are_the_published_splitmix64(oracle_mod):
    want = [int(x, 16) for x in GOLD["splitmix64_seed0"]["outputs"]]
    assert [oracle_mod.random_draw(0, k) for k in range(3)] == want
    assert [ind.splitmix64_draw(0, k) for k in range(3)] == want
    for seed in (1, 77, 2 ** 32 - 1):
        for k in (0, 5, 123456):
            assert oracle_mod.random_draw(seed, k) == ind.splitmix64_draw(seed, k)


@pytest.mark.parametrize("select", ["cc", "random"])
@pytest.mark.parametrize("seed,m", [(0, 300), (1, 900), (2, 1900)])
def test_selection_matches_numpy_restatement(oracle_mod, select, seed, m):
    pts = scenes.uniform_box(2500, seed=40 + seed)
    for layers in (1, 2):
        p = oracle_mod.params(layers=layers, select=select, seed=seed * 11 + 3)
        got = oracle_mod.sample(pts, m, p)
        want = ind.hav_reference_small(pts, m, layers=layers, select=select, seed=seed * 11 + 3)
        assert np.array_equal(got, want), (select, layers)


def test_random_selection_is_uniform_within_a_voxel(oracle_mod):
    # four points in one cell of a coarse fixed grid, plus points in other cells
    pts = np.array([[0.1, 0.1, 0.1], [0.2, 0.3, 0.1], [0.4, 0.2, 0.3], [0.3, 0.4, 0.2],
                    [5.5, 5.5, 5.5], [9.5, 0.5, 0.5]], dtype=np.float32)
    hits = np.zeros(4, dtype=int)
    for seed in range(400):
        idx = oracle_mod.sample(pts, 3, oracle_mod.params(layers=1, select="random", seed=seed, fixed_s=1.0))
        chosen = [i for i in idx if i < 4]
        assert len(chosen) == 1
        hits[chosen[0]] += 1
    assert hits.sum() == 400 and hits.min() >= 60 and hits.max() <= 140, hits  # ~binomial(400, 1/4)


@pytest.mark.parametrize("s,m", [(4.0, 200), (9.0, 50), (2.5, 1500)])
def test_fixed_voxel_size(oracle_mod, s, m):
    pts = scenes.uniform_box(2500, seed=5)
    idx, tr = oracle_mod.sample(pts, m, oracle_mod.params(layers=1, fixed_s=s), want_trace=True)
    assert tr[0]["iters"] == 0 and tr[0]["s_star"] == F32(s) and not tr[0]["accepted"]
    assert tr[0]["k_star"] == ind.count_unique(pts, F32(s))
    assert np.array_equal(idx, ind.hav_reference_small(pts, m, layers=1, fixed_s=s))


def test_centre_and_mean_coordinates(oracle_mod):
    pts = scenes.uniform_box(3000, seed=9)
    for m in (400, 2800):  # cut-off, then shortfall (fill points report themselves)
        idx_cc, xyz_cc, tr = oracle_mod.sample_xyz(pts, m, oracle_mod.params(layers=1), want_trace=True)
        assert np.array_equal(xyz_cc, pts[idx_cc])
        s_star = tr[0]["s_star"]
        g, f, v = ind.cells(pts, s_star)
        reps = set(ind.lexsort_select(pts, s_star).tolist())
        idx_ce, xyz_ce = oracle_mod.sample_xyz(pts, m, oracle_mod.params(layers=1, select="centre"))
        idx_me, xyz_me = oracle_mod.sample_xyz(pts, m, oracle_mod.params(layers=1, select="mean"))
        assert np.array_equal(idx_ce, idx_cc) and np.array_equal(idx_me, idx_cc)
        M = float(np.abs(pts).max())
        k = int(np.frexp(M)[1])
        quantum = 2.0 ** (k - 30)
        groups = {}
        for i in range(pts.shape[0]):
            groups.setdefault(tuple(g[i]), []).append(i)
        fills = 0
        for r, i in enumerate(idx_cc):
            if i not in reps:
                fills += 1
                assert np.array_equal(xyz_ce[r], pts[i]) and np.array_equal(xyz_me[r], pts[i])
                continue
            cen = (v * (f[i] + F32(0.5)).astype(F32)).astype(F32)  # closed form v (g + 1/2)
            assert np.array_equal(xyz_ce[r], cen)
            members = groups[tuple(g[i])]
            for a in range(3):
                exact = sum(Fraction(float(pts[j, a])) for j in members) / len(members)
                err = abs(Fraction(float(xyz_me[r, a])) - exact)
                tol = Fraction(quantum) + Fraction(float(np.spacing(np.abs(xyz_me[r, a]).astype(F32))))
                assert err <= tol, (r, a, float(err))
        assert (fills > 0) == (m > tr[0]["k_star"])


def test_mean_is_exact_on_a_binary_grid(oracle_mod):
    # coordinates on a 1/8 grid and four points per voxel: the fixed-point sums and
    # the division by 4 are exact, so the mean is the rational mean exactly
    rng = np.random.default_rng(3)
    cellc = rng.integers(0, 8, size=(60, 3))
    pts = []
    for c in cellc:
        for _ in range(4):
            pts.append(c * 4.0 + rng.integers(0, 32, size=3) / 8.0)
    pts = np.unique(np.asarray(pts, dtype=np.float32), axis=0)
    idx, xyz, tr = oracle_mod.sample_xyz(pts, 20, oracle_mod.params(layers=1, select="mean", fixed_s=4.0),
                                         want_trace=True)
    g, _, _ = ind.cells(pts, F32(4.0))
    for r, i in enumerate(idx):
        members = np.nonzero((g == g[i]).all(axis=1))[0]
        if len(members) & (len(members) - 1):
            continue  # only power-of-two member counts are exact in binary
        want = pts[members].astype(np.float64).mean(axis=0).astype(np.float32)
        assert np.array_equal(xyz[r], want)


def test_variants_reject_several_layers(oracle_mod):
    pts = scenes.uniform_box(500, seed=1)
    for kw in ({"select": "mean"}, {"select": "centre"}, {"fixed_s": 3.0}):
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.sample(pts, 100, oracle_mod.params(layers=2, **kw))
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.sample(pts, 100, oracle_mod.params(layers=1, select=4))


# ------------------------------------------------------------ Fig. 3 spacing
def test_spacing_hand_case(oracle_mod):
    # a line 0, 1, 3, 7 and a duplicate of 7: spacings 1, 1, 2, 0, 0 (squared)
    pts = np.array([[0, 0, 0], [1, 0, 0], [3, 0, 0], [7, 0, 0], [7, 0, 0], [50, 50, 50]], dtype=np.float32)
    d2 = oracle_mod.spacing(pts, [0, 1, 2, 3, 4])
    assert d2.tolist() == [1.0, 1.0, 4.0, 0.0, 0.0]
    assert np.isinf(oracle_mod.spacing(pts, [5])[0])
    assert oracle_mod.spacing(pts, []).shape == (0,)


@pytest.mark.parametrize("seed", [0, 1])
def test_spacing_matches_kdtree(oracle_mod, seed):
    spatial = pytest.importorskip("scipy.spatial")
    pts = scenes.uniform_box(4000, seed=seed)
    idx = np.sort(np.random.default_rng(seed).choice(4000, size=1500, replace=False)).astype(np.int32)
    d2 = oracle_mod.spacing(pts, idx)
    sub = pts[idx].astype(np.float64)
    dist, _ = spatial.cKDTree(sub).query(sub, k=2)
    assert np.allclose(np.sqrt(d2.astype(np.float64)), dist[:, 1], rtol=2e-6, atol=1e-6)


def test_fps_spacing_lower_bound(oracle_mod):
    # the FPS property behind Fig. 3's red line: every spacing is at least the
    # distance at which the last point was added
    pts = scenes.uniform_box(3000, seed=4)
    idx = oracle_mod.fps(pts, 400)
    d2 = oracle_mod.spacing(pts, idx)
    last = pts[idx[-1]]
    reach = min(float(np.sum((pts[i].astype(np.float64) - last) ** 2)) for i in idx[:-1])
    assert d2.min() >= np.float32(reach) * (1 - 1e-5)


# --------------------------------------------------- grouping (ball query)
def test_ball_query_hand_case(oracle_mod):
    # a line at x = 0, 1, 2, 5, 5.5; radius 1.5: strict inequality, index order, padding
    pts = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [5, 0, 0], [5.5, 0, 0]], dtype=np.float32)
    idx, xyz = oracle_mod.ball_query(pts, [1, 3, 0], 1.5, 4)
    assert idx.tolist() == [[0, 1, 2, 0], [3, 4, 3, 3], [0, 1, 0, 0]]
    assert xyz[0, :, 0].tolist() == [-1.0, 0.0, 1.0, -1.0]
    assert xyz[1, :, 0].tolist() == [0.0, 0.5, 0.0, 0.0]
    # a point exactly at the radius is outside (d^2 < r^2)
    idx, _ = oracle_mod.ball_query(pts, [0], 1.0, 3)
    assert idx.tolist() == [[0, 0, 0]]


@pytest.mark.parametrize("radius,nsample", [(2.0, 16), (4.5, 64), (0.5, 8)])
def test_ball_query_matches_kdtree(oracle_mod, radius, nsample):
    spatial = pytest.importorskip("scipy.spatial")
    pts = scenes.uniform_box(6000, seed=2)
    centres = oracle_mod.sample(pts, 500, oracle_mod.params(layers=1))
    idx, xyz = oracle_mod.ball_query(pts, centres, radius, nsample)
    tree = spatial.cKDTree(pts.astype(np.float64))
    r2 = np.float32(radius) * np.float32(radius)
    for j, c in enumerate(centres):
        near = sorted(tree.query_ball_point(pts[c].astype(np.float64), radius * (1 + 1e-5)))
        # drop the points whose binary32 distance is not strictly inside
        d = pts[near] - pts[c]
        d2 = ((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]).astype(np.float32) + d[:, 2] * d[:, 2]).astype(np.float32)
        inside = [k for k, q in zip(near, d2) if q < r2]
        want = inside[:nsample] + [inside[0]] * max(0, nsample - len(inside))
        assert idx[j].tolist() == want
        assert np.array_equal(xyz[j], (pts[idx[j]] - pts[c]).astype(np.float32))
