"""The context's kernel-launch count (hav_context_launches) through the C ABI:
how many kernels each call enqueues under the default tuning, so that a
reported launch count is the library's own."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def launched(ctx, fn):
    k0 = ctx.launches()
    fn()
    torch.cuda.synchronize()
    return ctx.launches() - k0


def test_level_chains_launch_one_kernel_per_engine(hv):
    ctx = hv.Context(1 << 17, 4)
    try:
        assert ctx.get_tuning()["small_points"] == 32768 and ctx.get_tuning()["solo_points"] == 4096
        big = dev(scenes.uniform_box(100_000, seed=1))
        p = hv.params()
        # one level above 32,768 points: the grid kernel alone
        assert launched(ctx, lambda: hv.hav_sample(ctx, big, 25_000, p)) == 1
        # grid kernel, then clusters from the first level within 32,768 points
        assert launched(ctx, lambda: hv.hav_sample_levels(ctx, big, [25_000, 6_250, 1_562], p)) == 2
        # ... then one CTA per segment from the first level of at most 1,024 points
        assert launched(ctx, lambda: hv.hav_sample_levels(ctx, big, [25_000, 4_000, 1_000, 250], p)) == 3
        # small clouds skip the grid kernel
        mid = dev(scenes.uniform_box(3_000, seed=2))
        assert launched(ctx, lambda: hv.hav_sample(ctx, mid, 700, p)) == 1
        tiny = dev(scenes.uniform_box(800, seed=3))
        assert launched(ctx, lambda: hv.hav_sample(ctx, tiny, 200, p)) == 1
        # the phase timer does not change which kernel runs a level
        pt = hv.params(flags=hv.HAV_FLAG_PHASE_TIMES)
        assert launched(ctx, lambda: hv.hav_sample_levels(ctx, big, [25_000, 4_000, 1_000, 250], pt)) == 3
        # nothing to select: nothing launched
        assert launched(ctx, lambda: hv.hav_sample(ctx, big, 0, p)) == 0
        st, _ = hv.hav_status_get(ctx, 1)
        assert st == hv.HAV_OK
    finally:
        ctx.close()


def test_other_calls_count_their_kernels(hv):
    ctx = hv.Context(1 << 16, 1)
    try:
        big = dev(scenes.uniform_box(50_000, seed=4))
        p1 = hv.params(layers=1)
        assert launched(ctx, lambda: hv.hav_sample(ctx, big, 12_000, p1)) == 1
        # the representative coordinates: one more kernel, four with the voxel table
        assert launched(ctx, lambda: hv.hav_sample_xyz(ctx, big, 12_000, p1)) == 2
        assert launched(ctx, lambda: hv.hav_sample_xyz(ctx, big, 12_000, hv.params(layers=1, select="mean"))) == 5
        idx = hv.hav_sample(ctx, big, 12_000, p1)
        torch.cuda.synchronize()
        assert launched(ctx, lambda: hv.hav_fps(ctx, big, 500)) == 1
        assert launched(ctx, lambda: hv.hav_spacing(ctx, big, idx)) == 2
        # a subset from 32,768 points: gathered, a grid built over it, searched
        assert launched(ctx, lambda: hv.hav_spacing(ctx, big, torch.arange(40_000, dtype=torch.int32,
                                                                          device="cuda"))) == 3
        assert launched(ctx, lambda: hv.hav_ball_query(ctx, big, idx[:100], 0.05, 16)) == 2
        st, _ = hv.hav_status_get(ctx, 1)
        assert st == hv.HAV_OK
    finally:
        ctx.close()


def test_phase_timer_spans_every_kernel_of_a_chain(hv):
    """The grid kernel's records, then those of the cluster and single-CTA
    kernels that continue the chain: one start record, times in order, one
    record per evaluated bisection step on the small levels (the trace's
    steps less those settled by bounds), the bbox, selection and compaction
    records of each small level, and the same indices as without the timer."""
    ctx = hv.Context(1 << 17, 1)
    try:
        big = dev(scenes.uniform_box(100_000, seed=1))
        ml = [25_000, 4_000, 1_000, 250]
        ref = [o.cpu().numpy() for o in hv.hav_sample_levels(ctx, big, ml, hv.params())]
        pt = hv.params(flags=hv.HAV_FLAG_PHASE_TIMES)
        k0 = ctx.launches()
        out = [o.cpu().numpy() for o in hv.hav_sample_levels(ctx, big, ml, pt)]
        assert ctx.launches() - k0 == 3
        assert all(np.array_equal(a, b) for a, b in zip(out, ref))
        rec = hv.hav_phase_times_get(ctx)
        trace = hv.hav_trace_get(ctx, len(ml) * 2)
        st, _ = hv.hav_status_get(ctx, 1)
        assert st == hv.HAV_OK
    finally:
        ctx.close()
    assert rec[0][1] == 0 and sum(1 for _, g in rec if g == 0) == 1
    times = [t for t, _ in rec]
    assert times == sorted(times)
    tags = [((g >> 24), (g >> 16) & 255, (g >> 8) & 255) for _, g in rec]
    assert any(ph == 2 and lv == 0 for ph, lv, _ in tags)  # the grid kernel's passes come first
    first_small = next(k for k, (ph, lv, _) in enumerate(tags) if lv == 1)
    assert all(lv == 0 for _, lv, _ in tags[1:first_small])
    for j in (1, 2, 3):  # levels of at most 32,768 points: the small-level kernels
        for ph in (1, 3, 7, 8):  # bbox, and per layer selection; compaction count and write
            want = 2 if ph == 3 else 1
            assert sum(1 for p2, lv, _ in tags if p2 == ph and lv == j) == want, (j, ph)
        for l in range(2):
            tr = trace[j * 2 + l]
            steps = tr["iters"] - bin(tr["bounded"]).count("1")
            assert sum(1 for ph, lv, ly in tags if ph == 2 and lv == j and ly == l) == steps
