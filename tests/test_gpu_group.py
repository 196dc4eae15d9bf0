"""GPU parity of the grouping around sampled centres (the ball query after
sampling, Section 3.1) through the C ABI: indices and offsets bit-identical to
the oracle's."""
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


def check(hv, ctx, oracle_mod, pts, centres, radius, nsample):
    centres = np.ascontiguousarray(centres, dtype=np.int32)
    idx, xyz = hv.hav_ball_query(ctx, dev(pts), torch.from_numpy(centres).cuda(), radius, nsample)
    st, _ = hv.hav_status_get(ctx, 1)
    assert st == 0
    o_idx, o_xyz = oracle_mod.ball_query(pts, centres, radius, nsample)
    got = idx.cpu().numpy()
    bad = np.nonzero((got != o_idx).any(axis=1))[0]
    assert bad.size == 0, (bad[:3], got[bad[:1]], o_idx[bad[:1]])
    assert np.array_equal(xyz.cpu().numpy().view(np.uint32), o_xyz.view(np.uint32))
    return got


@pytest.mark.parametrize("radius,nsample", [(2.0, 16), (5.0, 64), (0.7, 8), (100.0, 32)])
def test_group_uniform(hv, ctx, oracle_mod, radius, nsample):
    pts = scenes.uniform_box(16384, seed=1)
    centres = hv.hav_sample(ctx, dev(pts), 4096).cpu().numpy()
    check(hv, ctx, oracle_mod, pts, centres, radius, nsample)


def test_group_lidar_and_room(hv, ctx, oracle_mod):
    pts = scenes.lidar_min(16384, seed=1)[0]
    centres = hv.hav_sample(ctx, dev(pts), 4096).cpu().numpy()
    check(hv, ctx, oracle_mod, pts, centres, 0.8, 32)
    room = scenes.room_scene(65536, seed=2)
    centres = hv.hav_sample(ctx, dev(room), 4096).cpu().numpy()
    check(hv, ctx, oracle_mod, room, centres, 0.2, 32)
    check(hv, ctx, oracle_mod, room, centres[:500], 0.05, 256)


def test_group_edges(hv, ctx, oracle_mod):
    # duplicates: the first nsample copies by index; a tiny radius: only the centre (and its copies)
    base = scenes.uniform_box(300, seed=3)
    pts = np.concatenate([base, base, base[:50]])
    check(hv, ctx, oracle_mod, pts, [0, 7, 310, 649], 1e-3, 4)
    check(hv, ctx, oracle_mod, pts, np.arange(0, 650, 3), 6.0, 1)
    out, offs = hv.hav_ball_query(ctx, dev(pts), torch.zeros(0, dtype=torch.int32, device="cuda"), 1.0, 8)
    assert out.shape == (0, 8) and offs.shape == (0, 8, 3)
    idx, _ = hv.hav_ball_query(ctx, dev(pts), torch.tensor([0, 5], dtype=torch.int32, device="cuda"), 2.0, 4,
                               xyz=False)
    assert idx.shape == (2, 4)


def test_group_rejects(hv, ctx):
    pts = dev(scenes.uniform_box(100, seed=1))
    c = torch.tensor([0, 1000, 3], dtype=torch.int32, device="cuda")
    idx, _ = hv.hav_ball_query(ctx, pts, c, 1.0, 4)
    st, _ = hv.hav_status_get(ctx, 1)
    assert st == hv.HAV_ERR_INVALID and idx[1].tolist() == [0, 0, 0, 0]
    ok = torch.tensor([0, 3], dtype=torch.int32, device="cuda")
    for radius, ns in ((0.0, 4), (-1.0, 4), (float("nan"), 4), (1.0, 0), (1.0, 257)):
        with pytest.raises(hv.HavError):
            hv.hav_ball_query(ctx, pts, ok, radius, ns)
    big = dev(scenes.uniform_box((1 << 17) + 1, seed=1))
    with pytest.raises(hv.HavError):
        hv.hav_ball_query(ctx, big, ok, 1.0, 4)
