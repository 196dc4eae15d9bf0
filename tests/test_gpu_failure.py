"""Failure detection on the GPU without a fault: the bounded device waits.
HAV_FLAG_TEST_TIMEOUT makes the call's first grid barrier wait for a block
the launch does not have; every block gives up after its bounded wait, the
host reads HAV_ERR_TIMEOUT, and the same context then samples exactly again."""
import os
import sys
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(__file__))
import _gpu_helpers as G  # noqa: E402
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_bounded_wait_reports_a_timeout_and_the_context_recovers(hv):
    pts = scenes.uniform_box(16384, 3)
    c = hv.Context(1 << 16, 8)
    try:
        t0 = time.perf_counter()
        hv.hav_sample_levels(c, dev(pts), [4096], hv.params(flags=hv.HAV_FLAG_TEST_TIMEOUT))
        st, _ = hv.hav_status_get(c, 1)
        dt = time.perf_counter() - t0
        assert st == hv.HAV_ERR_TIMEOUT
        assert dt < 60.0  # the wait is bounded (about 2 s)
        # the next call on the same context is exact again
        out = hv.hav_sample_levels(c, dev(pts), [4096, 1024], hv.params())
        st, _ = hv.hav_status_get(c, 1)
        assert st == 0
        (ora, _), = G.oracle_many([pts], [[4096, 1024]])
        for j in range(2):
            assert np.array_equal(out[j].cpu().numpy(), ora[j]), j
    finally:
        c.close()


def test_timeout_on_a_batch_and_on_a_cluster_context(hv):
    # batched launch, and a context whose small levels would run on clusters:
    # the hook still reaches the grid kernel's barrier
    sizes = [5000, 700, 12000]
    clouds = [scenes.uniform_box(n, 20 + i) for i, n in enumerate(sizes)]
    pts, offs = scenes.concat(clouds)
    seg_m = np.array([[n // 4 for n in sizes]], dtype=np.int64)
    c = hv.Context(1 << 16, 8)
    try:
        for tuning in ({}, {"small_points": 32768}):
            if tuning:
                c.set_tuning(**tuning)
            hv.hav_sample_batched(c, dev(pts), offs, seg_m, hv.params(flags=hv.HAV_FLAG_TEST_TIMEOUT))
            st, _ = hv.hav_status_get(c, len(sizes))
            assert st == hv.HAV_ERR_TIMEOUT, tuning
            outs = hv.hav_sample_batched(c, dev(pts), offs, seg_m, hv.params())
            st, _ = hv.hav_status_get(c, len(sizes))
            assert st == 0, tuning
            ora = G.oracle_many(clouds, [[int(seg_m[0, s])] for s in range(len(sizes))])
            cut = np.concatenate([[0], np.cumsum(seg_m[0])])
            got = outs[0].cpu().numpy()
            for s in range(len(sizes)):
                assert np.array_equal(got[cut[s]:cut[s + 1]], ora[s][0][0]), (tuning, s)
    finally:
        c.close()


def test_full_table_is_reported_and_contained(hv):
    # segment 0 keeps a 64-slot table: more than 64 occupied voxels fill it;
    # the segment reports HAV_ERR_TABLE_FULL and takes indices 0..m-1, while the
    # other segments of the same launch stay exact
    sizes = [3000, 5000, 700, 12000]
    clouds = [scenes.uniform_box(n, 40 + i) for i, n in enumerate(sizes)]
    pts, offs = scenes.concat(clouds)
    seg_m = np.array([[n // 4 for n in sizes], [n // 16 for n in sizes]], dtype=np.int64)
    ora = G.oracle_many(clouds, [seg_m[:, s] for s in range(len(sizes))])
    c = hv.Context(1 << 16, 8)
    try:
        outs = hv.hav_sample_batched(c, dev(pts), offs, seg_m, hv.params(flags=hv.HAV_FLAG_TEST_TABLE_FULL))
        st, per = hv.hav_status_get(c, len(sizes))
        assert st == hv.HAV_ERR_TABLE_FULL
        assert list(per) == [hv.HAV_ERR_TABLE_FULL, 0, 0, 0]
        for j in range(2):
            cut = np.concatenate([[0], np.cumsum(seg_m[j])])
            got = outs[j].cpu().numpy()
            assert got[cut[0]:cut[1]].tolist() == list(range(int(seg_m[j, 0])))
            for s in range(1, len(sizes)):
                assert np.array_equal(got[cut[s]:cut[s + 1]], ora[s][0][j]), (j, s)
        # a cloud that never has more than 64 occupied voxels is exact under the hook,
        # and the context is exact again without it
        tiny = scenes.uniform_box(50, 9)
        out = hv.hav_sample_levels(c, dev(tiny), [10], hv.params(flags=hv.HAV_FLAG_TEST_TABLE_FULL))
        assert hv.hav_status_get(c, 1)[0] == 0
        assert np.array_equal(out[0].cpu().numpy(), G.oracle_many([tiny], [[10]])[0][0][0])
        outs = hv.hav_sample_batched(c, dev(pts), offs, seg_m, hv.params())
        assert hv.hav_status_get(c, len(sizes))[0] == 0
        for j in range(2):
            cut = np.concatenate([[0], np.cumsum(seg_m[j])])
            got = outs[j].cpu().numpy()
            for s in range(len(sizes)):
                assert np.array_equal(got[cut[s]:cut[s + 1]], ora[s][0][j]), (j, s)
    finally:
        c.close()
