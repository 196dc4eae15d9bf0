"""The seeded synthetic inputs keep the recipe they state: sizes, ranges, order
and determinism of the stand-ins for the paper's datasets (no GPU)."""
import numpy as np

from paper_2305_14306_gb300 import scenes


def test_uniform_box_is_the_kitti_range_and_deterministic():
    p = scenes.uniform_box(16384, 3)
    assert p.shape == (16384, 3) and p.dtype == np.float32 and p.flags.c_contiguous
    lo, hi = np.array(scenes.KITTI_LO, np.float32), np.array(scenes.KITTI_HI, np.float32)
    assert (p >= lo).all() and (p <= hi).all()
    assert np.array_equal(p, scenes.uniform_box(16384, 3)) and not np.array_equal(p, scenes.uniform_box(16384, 4))


def test_lidar_scene_returns_and_geometry():
    sizes = [scenes.lidar_scene(seed=s).shape[0] for s in range(4)]
    assert all(14_000 <= n <= 22_000 for n in sizes), sizes  # the "kitti-fov" reading: about 16-20k
    p = scenes.lidar_scene(seed=0)
    r = np.linalg.norm(p.astype(np.float64), axis=1)
    assert r.max() <= 80.0 + 0.1  # range cut (plus noise along the ray)
    assert p[:, 0].min() > 0  # the front 90 degrees only
    assert p[:, 2].min() > -1.73 - 0.1  # nothing below the ground plane beyond the noise
    # ring-major scan order: elevation angle never decreases by more than the noise
    elev = np.arcsin(p[:, 2] / r)
    assert np.all(np.diff(elev) > -0.01)
    q = scenes.lidar_scene(seed=0, shuffle=True)
    assert q.shape == p.shape and not np.array_equal(p, q)
    assert np.array_equal(np.sort(p, axis=0), np.sort(q, axis=0))


def test_lidar_min_and_exact_sizes():
    p, s = scenes.lidar_min(16384, 0)
    assert p.shape[0] >= 16384 and np.array_equal(p, scenes.lidar_scene(seed=s))
    e = scenes.lidar_exact(50_000, 9)
    assert e.shape == (50_000, 3) and np.array_equal(e, scenes.lidar_exact(50_000, 9))
    dense = scenes.lidar_scene(seed=9, rings=64, az_steps=2048, keep=1.0)
    # a subset of the dense scan, kept in scan order
    pos = {tuple(x): i for i, x in enumerate(dense.tolist())}
    idx = np.array([pos[tuple(x)] for x in e.tolist()])
    assert np.all(np.diff(idx) > 0)


def test_room_scene_bounds_size_and_shuffle():
    p = scenes.room_scene(200_000, 2)
    assert p.shape == (200_000, 3) and p.dtype == np.float32
    tol = 6 * 0.005  # six standard deviations of the coordinate noise
    assert (p >= -tol).all() and (p <= np.array([10.0, 10.0, 3.0]) + tol).all()
    # floor and ceiling hold a visible share of the points (area-uniform surfaces)
    on_floor = np.abs(p[:, 2]) < tol
    on_ceiling = np.abs(p[:, 2] - 3.0) < tol
    assert 0.1 < on_floor.mean() < 0.5 and 0.05 < on_ceiling.mean() < 0.5
    assert np.array_equal(p, scenes.room_scene(200_000, 2))
    # shuffled: no spatial order survives in the index order
    assert abs(np.corrcoef(np.arange(len(p)), p[:, 0])[0, 1]) < 0.05


def test_batch_sizes_and_segment_offsets():
    sizes = scenes.log_uniform_sizes(64, 20_000, 200_000, 0)
    assert sizes.min() >= 20_000 and sizes.max() <= 200_000
    # log-uniform: about half below the geometric mean
    gm = np.sqrt(20_000 * 200_000)
    assert 0.3 < (sizes < gm).mean() < 0.7
    clouds = [scenes.uniform_box(n, i) for i, n in enumerate([5, 0, 7])]
    pts, offs = scenes.concat(clouds)
    assert pts.shape == (12, 3) and offs.tolist() == [0, 5, 5, 12]


def test_request_stream():
    t, n, m = scenes.request_stream(2000, 1000.0, seed=1)
    assert t[0] == 0 and np.all(np.diff(t) >= 0)
    assert abs(len(t) / t[-1] - 1000.0) / 1000.0 < 0.1  # Poisson rate
    assert n.min() >= 10_000 and n.max() <= 1_000_000
    ok = (m == n // 4) | (m == n // 16) | (m == np.minimum(4096, n))
    assert ok.all()
