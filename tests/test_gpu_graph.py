"""The batched call captured in a CUDA graph: a replay of the captured
segmented launch gives, cloud by cloud, the CPU oracle's indices, replay
after replay (the plan travels in the captured launch's parameters)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import _gpu_helpers as G  # noqa: E402
from paper_2305_14306_gb300 import scenes  # noqa: E402


def test_graph_replay_of_batched_call_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_14306_gb300 import build, hav
    build.build()
    hav.load()
    sizes = [int(x) for x in scenes.log_uniform_sizes(10, 20_000, 200_000, seed=31)]
    clouds = [scenes.lidar_exact(n, 4000 + i) for i, n in enumerate(sizes)]
    pts, offs = scenes.concat(clouds)
    seg_m = np.stack([np.diff(offs) // 4, np.diff(offs) // 16]).astype(np.int64)
    ctx = hav.Context(int(offs[-1]), len(clouds))
    d_pts = torch.from_numpy(pts).cuda()
    outs = [torch.full((int(seg_m[j].sum()),), -1, dtype=torch.int32, device="cuda") for j in range(2)]
    p = hav.params()
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):  # one eager call first: the library's launch set-up
            hav.hav_sample_batched(ctx, d_pts, offs, seg_m, p, outs=outs, stream=side)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            hav.hav_sample_batched(ctx, d_pts, offs, seg_m, p, outs=outs, stream=torch.cuda.current_stream())
        ref = G.oracle_many(clouds, [seg_m[:, s] for s in range(len(clouds))])
        cut = [np.concatenate([[0], np.cumsum(seg_m[j])]) for j in range(2)]
        for rep in range(2):
            for o in outs:
                o.fill_(-1)
            graph.replay()
            torch.cuda.synchronize()
            st, per = hav.hav_status_get(ctx, len(clouds))
            assert st == hav.HAV_OK and all(int(x) == hav.HAV_OK for x in per[:len(clouds)])
            for j in range(2):
                got = outs[j].cpu().numpy()
                for s in range(len(clouds)):
                    assert np.array_equal(got[cut[j][s]:cut[j][s + 1]], ref[s][0][j]), (rep, j, s)
    finally:
        ctx.close()
