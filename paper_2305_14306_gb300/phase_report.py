"""Per-phase device time of one sampler call, from the kernel's phase timer.

With HAV_FLAG_PHASE_TIMES, block 0 of the persistent grid kernel records a
device timestamp after every grid-wide phase (bounding box, Morton
bucketing, each bisection pass, selection, classification, cut-off
resolution, shortfall fill, compaction), and the first cluster of the
small-level kernel that continues the chain appends its own after every
cluster-wide phase.  This tool runs a workload a few times and prints the
median time per phase and level, and the bisection passes per level.

    python -m paper_2305_14306_gb300.phase_report [--workload indoor-1m|lidar-chain|uniform-16k|batch64] [--runs 20]

Timestamps come from %globaltimer; the recording itself adds well under a
microsecond per phase.
"""
from __future__ import annotations

import argparse
import collections
import statistics

import numpy as np

from . import build, hav, scenes

PHASES = {0: "start", 1: "bbox", 2: "pass", 3: "select", 4: "classify", 5: "resolve", 6: "shortfall",
          7: "compact-count", 8: "compact-write", 9: "bucket-count", 10: "bucket-scatter"}

WORKLOADS = {
    "indoor-1m": (lambda: scenes.room_scene(1 << 20, seed=0), [1 << 18, 1 << 16, 1 << 14, 1 << 12]),
    "lidar-chain": (lambda: scenes.lidar_min(16384, seed=0)[0], [16384, 4096, 1024, 512]),
    "uniform-16k": (lambda: scenes.uniform_box(16384, seed=0), [4096]),
    # 64 LiDAR clouds in one segmented call, each to N/4 then N/16
    "batch64": (lambda: scenes.lidar_batch(64, seed=0), None),
}


def phase_durations(records):
    """(level, phase name) -> microseconds, and (level, phase name) -> count, for one call."""
    dur = collections.defaultdict(float)
    cnt = collections.defaultdict(int)
    for (t0, _), (t1, g1) in zip(records[:-1], records[1:]):
        ph, lev = g1 >> 24, (g1 >> 16) & 255
        name = PHASES.get(ph, str(ph))
        dur[(lev, name)] += (t1 - t0) / 1e3
        cnt[(lev, name)] += 1
    return dur, cnt


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="indoor-1m", choices=sorted(WORKLOADS))
    ap.add_argument("--runs", type=int, default=20)
    args = ap.parse_args(argv)
    import torch

    build.build()
    hav.load()
    make, ml = WORKLOADS[args.workload]
    p = hav.params(flags=hav.HAV_FLAG_PHASE_TIMES)
    if ml is None:  # a batch: one segmented call
        clouds = make()
        pts, offs = scenes.concat(clouds)
        sizes = np.diff(offs)
        seg_m = np.stack([sizes // 4, sizes // 16]).astype(np.int64)
        ml = [int(x) for x in seg_m.sum(axis=1)]
        ctx = hav.Context(pts.shape[0], len(clouds))
        d = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float32)).cuda()
        outs = [torch.empty(m, dtype=torch.int32, device="cuda") for m in ml]

        def call():
            hav.hav_sample_batched(ctx, d, offs, seg_m, p, outs=outs)
    else:
        pts = make()
        ctx = hav.Context(pts.shape[0], 1)
        d = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float32)).cuda()
        outs = [torch.empty(m, dtype=torch.int32, device="cuda") for m in ml]

        def call():
            hav.hav_sample_levels(ctx, d, ml, p, outs=outs)
    for _ in range(5):
        call()
    per = collections.defaultdict(list)
    counts = None
    totals = []
    for _ in range(args.runs):
        torch.cuda.synchronize()
        call()
        rec = hav.hav_phase_times_get(ctx)
        dur, counts = phase_durations(rec)
        for k, v in dur.items():
            per[k].append(v)
        totals.append((rec[-1][0] - rec[0][0]) / 1e3)
    print(f"workload {args.workload}: {pts.shape[0]} points, levels {ml}; median of {args.runs} calls")
    print(f"{'level':>5} {'phase':>15} {'count':>6} {'us':>9}")
    by_phase = collections.defaultdict(float)
    for k in sorted(per, key=lambda k: (k[0], k[1])):
        med = statistics.median(per[k])
        by_phase[k[1]] += med
        print(f"{k[0]:>5} {k[1]:>15} {counts[k]:>6} {med:>9.1f}")
    print("all levels:")
    for name, v in sorted(by_phase.items(), key=lambda kv: -kv[1]):
        print(f"      {name:>15} {v:>9.1f}")
    print(f"total (first to last timestamp) {statistics.median(totals):.1f} us")
    ctx.close()


if __name__ == "__main__":
    main()
