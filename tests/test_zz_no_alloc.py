"""hav_sample_noalloc: the context-free entry point for callers that may not
allocate device memory (framework memory pools, fixed budgets, plugin hosts,
real-time loops).  It must give exactly what hav_sample gives, call after
call, out of its static scratch array, and refuse clouds larger than that
array holds.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_14306_gb300 import scenes  # noqa: E402


@pytest.fixture(scope="module")
def hv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_14306_gb300 import build, hav
    build.build()
    hav.load()
    return hav


def test_noalloc_matches_hav_sample_on_two_calls_in_a_row(hv):
    a = torch.from_numpy(scenes.uniform_box(16384, 21)).cuda()
    b = torch.from_numpy(scenes.lidar_min(16384, 4)[0][:20000].copy()).cuda()
    ma, mb = 4096, 5000
    st_a = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st_b = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    # two calls back to back on one stream, no synchronisation between them
    out_a = hv.hav_sample_noalloc(a, ma, status_out=st_a)
    out_b = hv.hav_sample_noalloc(b, mb, status_out=st_b)
    torch.cuda.synchronize()
    assert int(st_a.item()) == hv.HAV_OK and int(st_b.item()) == hv.HAV_OK

    ctx = hv.Context(32768, 1)
    try:
        ref_a = hv.hav_sample(ctx, a, ma)
        ref_b = hv.hav_sample(ctx, b, mb)
        assert hv.hav_status_get(ctx)[0] == hv.HAV_OK
    finally:
        ctx.close()
    # the tests' tolerance for indices: bit-exact
    assert torch.equal(out_a.cpu(), ref_a.cpu())
    assert torch.equal(out_b.cpu(), ref_b.cpu())
    # and again, reusing the shared scratch that still holds the last call's contents
    again = hv.hav_sample_noalloc(a, ma)
    torch.cuda.synchronize()
    assert torch.equal(again.cpu(), ref_a.cpu())


def test_noalloc_refuses_clouds_beyond_its_scratch(hv):
    n = hv.NOALLOC_MAX_POINTS + 1
    pts = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    out = torch.full((8,), -3, dtype=torch.int32, device="cuda")
    p = hv.params()
    st = hv.load().hav_sample_noalloc(ctypes.c_void_p(pts.data_ptr()), n, 8, ctypes.byref(p),
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == hv.HAV_ERR_NOMEM
    torch.cuda.synchronize()
    assert (out.cpu() == -3).all()  # nothing was enqueued


def test_noalloc_allocates_nothing(hv):
    """The property the entry point exists for: with the output and status
    tensors passed in, a call allocates no device memory at all."""
    pts = torch.from_numpy(scenes.uniform_box(16384, 5)).cuda()
    out = torch.empty(4096, dtype=torch.int32, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    hv.hav_sample_noalloc(pts, 4096, out=out, status_out=st)  # first call: set-up on this device
    torch.cuda.synchronize()
    before_torch = torch.cuda.memory_allocated()
    before_free = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        hv.hav_sample_noalloc(pts, 4096, out=out, status_out=st)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before_torch
    # the driver's free-memory figure moves in pages; no call may take more
    assert before_free - torch.cuda.mem_get_info()[0] <= (2 << 20)
    assert int(st.item()) == hv.HAV_OK


def _ctx_reference(hv, pts, m, p):
    ctx = hv.Context(32768, 1)
    try:
        ref = hv.hav_sample(ctx, pts, m, p)
        status = hv.hav_status_get(ctx)[0]
    finally:
        ctx.close()
    return ref, status


def test_noalloc_m_zero_reports_ok(hv):
    pts = torch.from_numpy(scenes.uniform_box(1000, 6)).cuda()
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    out = hv.hav_sample_noalloc(pts, 0, status_out=st)
    torch.cuda.synchronize()
    assert out.numel() == 0
    assert int(st.item()) == hv.HAV_OK


def test_noalloc_nonfinite_reaches_status_out(hv):
    """A data-dependent error is written to status_out, and the indices are
    those hav_sample gives for a cloud in error (its first m points)."""
    a = scenes.uniform_box(8000, 7)
    a[1234, 1] = np.nan
    pts = torch.from_numpy(a).cuda()
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    out = hv.hav_sample_noalloc(pts, 2000, status_out=st)
    torch.cuda.synchronize()
    assert int(st.item()) == hv.HAV_ERR_NONFINITE
    ref, ref_status = _ctx_reference(hv, pts, 2000, hv.params())
    assert ref_status == hv.HAV_ERR_NONFINITE
    assert torch.equal(out.cpu(), ref.cpu())
    # the next call on the shared scratch starts clean
    ok = torch.from_numpy(scenes.uniform_box(8000, 8)).cuda()
    out2 = hv.hav_sample_noalloc(ok, 2000, status_out=st)
    torch.cuda.synchronize()
    assert int(st.item()) == hv.HAV_OK
    ref2, _ = _ctx_reference(hv, ok, 2000, hv.params())
    assert torch.equal(out2.cpu(), ref2.cpu())


@pytest.mark.parametrize("kw", [dict(layers=1, select="centre"), dict(layers=1, select="random", seed=9),
                                dict(search="guided"), dict(layers=3)])
def test_noalloc_variants_match_hav_sample(hv, kw):
    """The parameter variants reach other code in the grid kernel (which this
    entry point always runs, one step per pass): bit-exact with hav_sample."""
    pts = torch.from_numpy(scenes.lidar_min(16384, 11)[0][:24000].copy()).cuda()
    p = hv.params(**kw)
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    got = hv.hav_sample_noalloc(pts, 6000, p, status_out=st)
    torch.cuda.synchronize()
    assert int(st.item()) == hv.HAV_OK
    ref, ref_status = _ctx_reference(hv, pts, 6000, p)
    assert ref_status == hv.HAV_OK
    assert torch.equal(got.cpu(), ref.cpu())
