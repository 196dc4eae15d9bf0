#!/usr/bin/env python3
"""Benchmark of the HAVSampler hot path on GB300.

A step is one whole sampler call on one synthetic scene: every level of the
chain, every layer, every bisection pass, selection, cut-off and compaction.
Default workload: the indoor room of N = 1,048,576 points sampled through
four levels of N/4 each (262,144 -> 65,536 -> 16,384 -> 4,096), the
single-cloud HBM-roofline case.  Other workloads (--workload) exist for
exploration; the default line is the one to read.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hav|reference]

N > 1 runs one replica per GPU (torchrun), each on its own scene; no data
moves between ranks ("replicas only": the sampler does not shard a cloud).
--impl reference times the CPU oracle (test infrastructure, never the product
path) on bounded samples of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2305_14306_gb300 import scenes  # noqa: E402

WORKLOADS = {
    "indoor-1m": {"desc": "indoor room, N=1,048,576 FP32 xyz, 4 levels of N/4 (to 4,096), k=2 layers",
                  "n": 1 << 20, "levels": [1 << 18, 1 << 16, 1 << 14, 1 << 12]},
    "lidar-chain": {"desc": "64-ring LiDAR scene (~16-20k returns), levels 16,384 -> 4,096 -> 1,024 -> 512",
                    "n": None, "levels": [16384, 4096, 1024, 512]},
    "uniform-16k": {"desc": "16,384 uniform points in the KITTI range, one level to 4,096",
                    "n": 16384, "levels": [4096]},
    "serving": {"desc": "Poisson arrivals of scenes with N log-uniform in [10k, 1M] (LiDAR up to 200k, room above), "
                        "M in {N/4, N/16, 4096}; continuous batching on co-resident slots vs the plain per-cloud path",
                "n": None, "levels": None},
    "compare": {"desc": "HAV vs the plain GPU FPS comparator (Eq. 1): C1 16,384 -> 4,096; C2 LiDAR returns -> 16,384; "
                        "C4 64 LiDAR clouds -> N/4 each; C3 1,048,576 -> 262,144 (level 1); time and coverage",
                "n": None, "levels": None},
    "variants": {"desc": "Table 6 strategies, one layer: centre-closest / random / mean / centre representatives, "
                         "adaptive and fixed voxel size, on C1 16,384 -> 4,096 and C3 1,048,576 -> 262,144",
                 "n": None, "levels": None},
    "spacing": {"desc": "Fig. 3 point spacing of HAV, random-voxel (RA + fixed size), FPS and random subsets: "
                        "C1 16,384 -> 4,096; C2 LiDAR returns -> 16,384; C3 1,048,576 -> 262,144",
                "n": None, "levels": None},
    "grouping": {"desc": "grouping after sampling (ball query, fused offset gather): C2 LiDAR 4,096 centres r = 0.8 m, "
                         "C3 262,144 centres of 1,048,576 r = 0.1 m and 65,536 centres r = 0.2 m, 32 samples",
                 "n": None, "levels": None},
    "batch64": {"desc": "64 LiDAR clouds, N log-uniform in [20k, 200k], per cloud M = N/4 then N/16, "
                        "one persistent segmented launch (also replayed from a CUDA graph) vs 64 per-cloud calls",
                "n": None, "levels": None},
}
FLUSH_BYTES = 256 << 20  # > 129 MB L2
L2_NOTE = "flushed before every step (256 MB read sweep: L2 holds no dirty lines when a step starts)"


class L2Flush:
    """Evicts L2 between timed steps by reading a 256 MB buffer (twice the L2).
    A read sweep leaves only clean lines behind, so no write-back of earlier
    data is charged to the next step's kernels (a write sweep would leave
    about 129 MB of dirty lines that the step itself then writes back)."""

    def __init__(self, torch):
        self.buf = torch.zeros(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.acc = torch.zeros((), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()  # the zero-fill's dirty lines go out before any timing

    def sweep(self):
        self.acc.add_(self.buf.sum())


def make_scene(name: str, seed: int) -> np.ndarray:
    if name == "indoor-1m":
        return scenes.room_scene(1 << 20, seed=seed)
    if name == "lidar-chain":
        return scenes.lidar_min(16384, seed=seed)[0]
    if name == "uniform-16k":
        return scenes.uniform_box(16384, seed=seed)
    raise ValueError(name)


def algorithmic_bytes(traces, level_inputs, level_budgets, layers):
    """Bytes the paper's procedure must move per call: each bisection pass and
    the selection pass read the layer's points (12 B each) plus, from the
    second layer on, the taken bitmask (n/8 B); the output writes 4 B per index.
    B = sum_levels [ sum_l (t_l + 1) (12 n_l + [l >= 2] n / 8) + 4 m ]."""
    B = 0
    for j, (n, m) in enumerate(zip(level_inputs, level_budgets)):
        for l in range(layers):
            tr = traces[j * layers + l]
            if tr["m_l"] == 0:
                continue
            passes = tr["iters"] + 1
            B += passes * 12 * tr["n_in"]
            if l >= 1:
                B += passes * (n // 8)
        B += 4 * m
    return B


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments and with whitespace runs collapsed,
    so that edits of comments alone leave the hash (and a capture) valid."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":  # string or character literal, copied whole
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


# the files the sampler's kernels (hav_chain_kernel, hav_small_kernel) and
# their launch are built from; the other kernels (grouping, spacing, FPS,
# representatives, the allocation-free entry) do not change the profiled call
SAMPLER_SOURCES = ("hav_api.cu", "hav_device.cuh", "hav_internal.h", "hav_sampler.cu", "hav_small.cu")


def source_hash() -> str:
    """Hash of the sampler kernels' source code (comments and layout ignored)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2305_14306_gb300", "csrc")
    for f in SAMPLER_SOURCES + ("../../include/hav.h",):
        h.update(os.path.basename(f).encode() + b"\0" +
                 _code_only(open(os.path.join(csrc, f)).read()).encode() + b"\0")
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes (read + write) per sampler call, summed over the call's
    kernels, from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"hav_chain_kernel_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    mh = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    mt = re.search(r"dram_bytes_per_call:\s*([0-9]+)", text)
    if not mh or not mt or mh.group(1) != source_hash():
        return None
    return int(mt.group(1))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            self.f.close()
            os.unlink(self.f.name)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def clocks_bad(c) -> bool:
    if any(r in c["reasons"] for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")):
        return True
    if c["sm_mhz"] and c["sm_max_mhz"] and not c["reasons"] and c["sm_mhz"] < 0.6 * c["sm_max_mhz"]:
        return True
    return False


def whole_job(local_seconds: float, points_per_rank: int, world: int, device=None) -> tuple:
    """Replicas: every rank timed its own steps; the job takes as long as the
    slowest rank, and `value` counts every rank's points.  Returns
    (max seconds over ranks, whole-job Mpoints/s)."""
    t = local_seconds
    if world > 1:
        import torch
        import torch.distributed as dist
        x = torch.tensor([local_seconds], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, points_per_rank * world / t / 1e6


def host_cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    """The CPU oracle timed as it stands, on bounded samples of the workload."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = WORKLOADS[args.workload]
    pts = make_scene(args.workload, 0)
    n_full = pts.shape[0]
    ratios = [m / n_full for m in w["levels"]] if w["n"] else None

    def levels_for(n):
        if ratios is None:
            return [min(m, n) for m in w["levels"]]
        return [max(1, int(round(r * n))) for r in ratios]

    # calibrate: per-point time on a 16k prefix (the scenes are shuffled or scan-ordered clouds)
    n_cal = min(16384, n_full)
    t0 = time.perf_counter()
    op = oracle.params(search=args.search)
    oracle.sample_levels(pts[:n_cal], levels_for(n_cal), op)
    per_pt = (time.perf_counter() - t0) / n_cal
    budget_s = 90.0
    n_s = int(budget_s / max(1, args.steps + args.warmup) / per_pt)
    n_s = max(min(4096, n_full), min(n_full, n_s))
    sample = pts[:n_s]
    ml = levels_for(n_s)
    for _ in range(args.warmup):
        oracle.sample_levels(sample, ml, op)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sample_levels(sample, ml, op)
    dt = time.perf_counter() - t0
    value = n_s * args.steps / dt / 1e6
    desc = f"first {n_s} points of the {args.workload} scene, levels {ml}, per step"
    line = {
        "impl": "reference", "metric": "input Mpoints/s", "value": value, "unit": "Mpoints/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "sample": desc, "search": args.search},
        "cpu_baseline": {"value": value, "unit": "Mpoints/s", "cores": 1, "kind": "oracle", "sample": desc,
                         "cpu_model": host_cpu_model()},
        "e2e": {"value": value, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- batched arm
def _oracle_cloud(job):
    """One cloud of a batch on one host core (a spawned pool worker)."""
    import oracle
    pts, ml, search = job
    return oracle.sample_levels(pts, ml, oracle.params(search=search))


def scene_parallel_oracle(clouds, m_levels, search, reps=3):
    """The oracle over a batch, one cloud per host core (spawned processes, so
    that no worker inherits the CUDA context); m_levels[s] is cloud s's level
    budgets.  Returns (Mpoints/s, cores, per-cloud outputs)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    jobs = [(c, [int(x) for x in m_levels[s]], search) for s, c in enumerate(clouds)]
    total = sum(c.shape[0] for c in clouds)
    with mp.get_context("spawn").Pool(cores) as pool:
        # bounded waits: a pool whose workers cannot start would wait forever
        pool.map_async(_oracle_cloud, jobs[:cores]).get(timeout=300)  # workers up, library loaded
        t0 = time.perf_counter()
        for _ in range(reps):
            res = pool.map_async(_oracle_cloud, jobs, chunksize=1).get(timeout=600)
        dt = time.perf_counter() - t0
    return total * reps / dt / 1e6, cores, res
def run_batched(args, world, rank, local, sub=False):
    """64 clouds per step: one hav_sample_batched call, the same call from a
    CUDA graph, and 64 plain per-cloud hav_sample_levels calls, at identical outputs.
    sub=True: return rank 0's result (no print, no host-core oracle) for the
    default line's "batch64" object."""
    import torch
    import torch.distributed as dist
    from paper_2305_14306_gb300 import hav

    clouds = scenes.lidar_batch(64, seed=rank)
    pts, offs = scenes.concat(clouds)
    sizes = np.diff(offs)
    seg_m = np.stack([sizes // 4, sizes // 16]).astype(np.int64)
    total = int(offs[-1])
    p = hav.params(search=args.search)
    ctx = hav.Context(total, 64)
    ctx1 = hav.Context(int(sizes.max()), 1)
    stream = torch.cuda.current_stream()
    d_pts = torch.from_numpy(pts).cuda()
    outs = [torch.empty(int(seg_m[j].sum()), dtype=torch.int32, device="cuda") for j in range(2)]
    per_outs = [[torch.empty(int(seg_m[j, s]), dtype=torch.int32, device="cuda") for j in range(2)]
                for s in range(64)]
    views = [d_pts[int(offs[s]):int(offs[s + 1])] for s in range(64)]
    flush = L2Flush(torch)

    def step_batched(strm=stream):
        hav.hav_sample_batched(ctx, d_pts, offs, seg_m, p, outs=outs, stream=strm)

    def step_per_cloud():
        for s in range(64):
            hav.hav_sample_levels(ctx1, views[s], seg_m[:, s], p, outs=per_outs[s], stream=stream)

    for _ in range(args.warmup):
        step_batched()
        step_per_cloud()
    st, per = hav.hav_status_get(ctx, 64)
    if st != hav.HAV_OK:
        raise SystemExit(f"batched status {st}")
    # identical outputs, cloud by cloud
    cut = [np.concatenate([[0], np.cumsum(seg_m[j])]) for j in range(2)]
    for j in range(2):
        got = outs[j].cpu().numpy()
        for s in range(64):
            if not np.array_equal(got[cut[j][s]:cut[j][s + 1]], per_outs[s][j].cpu().numpy()):
                raise SystemExit(f"batched and per-cloud outputs differ at level {j}, cloud {s}")

    # autotune the batched launch (the knobs never change a result)
    from paper_2305_14306_gb300 import tuning
    ref = [o.clone() for o in outs]
    gpu_name = torch.cuda.get_device_name(local)
    tuned, tune_report = tuning.autotune(ctx, step_batched, tuning.signature(sizes, 2), gpu_name,
                                         cache=args.tuning_cache, force=args.tuning_cache is None)
    step_batched()
    st, _ = hav.hav_status_get(ctx, 64)
    if st != hav.HAV_OK or not all(torch.equal(a, b) for a, b in zip(outs, ref)):
        raise SystemExit("tuned batched outputs differ")

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_batched(torch.cuda.current_stream())  # the capturing stream
    for o in outs:
        o.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    st, _ = hav.hav_status_get(ctx, 64)
    if st != hav.HAV_OK or not all(torch.equal(a, b) for a, b in zip(outs, ref)):
        raise SystemExit("graph replay outputs differ")

    def time_it(fn, steps):
        ms = []
        for _ in range(steps):
            flush.sweep()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ms.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ms]

    gpu_index = local
    steps = max(10, min(args.steps, 200))
    clk = Clocks(gpu_index)
    time.sleep(0.3)
    k0 = ctx.launches()
    ms_b = time_it(step_batched, steps)
    launches_b = ctx.launches() - k0
    ms_g = time_it(graph.replay, steps)
    k1 = ctx1.launches()
    ms_p = time_it(step_per_cloud, max(5, steps // 4))
    launches_p = ctx1.launches() - k1
    clocks = clk.stop()
    tb, value = whole_job(sum(ms_b) / 1e3, total * len(ms_b), world, device="cuda")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not sub:
        try:
            v_cpu, cores, res = scene_parallel_oracle(clouds, [seg_m[:, s] for s in range(64)], args.search)
        except Exception as e:  # reported, never silently replaced
            raise SystemExit(f"scene-parallel oracle failed: {e!r}")
        same = all(np.array_equal(outs[j].cpu().numpy()[cut[j][s]:cut[j][s + 1]], res[s][j])
                   for j in range(2) for s in range(64))
        if not same:
            raise SystemExit("the GPU batch and the scene-parallel oracle differ")
        cpu = {"value": v_cpu, "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
               "sample": "the same 64 clouds, 3 times, one cloud per process (spawned pool)",
               "identical_outputs": True, "cpu_model": host_cpu_model()}
    v_graph = total * len(ms_g) / (sum(ms_g) / 1e3) / 1e6
    v_per = total * len(ms_p) / (sum(ms_p) / 1e3) / 1e6
    if rank == 0:
        srt = sorted(ms_b)
        line = {
            "metric": "input Mpoints/s", "value": value, "unit": "Mpoints/s", "n_gpus": world,
            "steps": len(ms_b), "warmup": args.warmup, "ms_per_step": statistics.fmean(ms_b),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batch64", "desc": WORKLOADS["batch64"]["desc"], "points": total,
                       "segments": 64, "levels": 2, "l2": L2_NOTE,
                       "search": args.search},
            "scenes_per_s": 64 * len(ms_b) / (sum(ms_b) / 1e3),
            "p50_ms": srt[len(srt) // 2], "p99_ms": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
            "graph": {"value": v_graph, "ms_per_step": statistics.fmean(ms_g)},
            "per_cloud": {"value": v_per, "ms_per_step": statistics.fmean(ms_p),
                          "launches_per_step": launches_p / len(ms_p)},
            "speedup_vs_per_cloud": value / v_per,
            "identical_outputs": True,
            "cpu_baseline": cpu,
            "tuning": {"batched": tuned, **tune_report,
                       "per_cloud": "default knobs (one call per cloud)"},
            "gpu_launches": launches_b,  # counted by the library over the timed batched steps
            "launches_per_step": launches_b / len(ms_b),
            "clocks": clocks,
        }
        if not sub:
            print(json.dumps(line), flush=True)
    ctx.close()
    ctx1.close()
    if sub:
        return line if rank == 0 else None
    return 0


# ----------------------------------------------------------------- comparator arm
def coverage_fast(pts, idx, queries=None, chunk=2048):
    """max over query points of the distance to the nearest selected point, fp32 on
    centred coordinates with matmul distances (about 1e-4 m error at these extents)."""
    import torch
    c = pts - pts.mean(dim=0, keepdim=True)
    sel = c[idx.long()]
    q = c if queries is None else c[queries]
    worst = 0.0
    for a in range(0, q.shape[0], chunk):
        d = torch.cdist(q[a:a + chunk], sel, compute_mode="use_mm_for_euclid_dist")
        worst = max(worst, float(d.min(dim=1).values.max()))
    return worst


def run_compare(args, world, rank, local):
    import torch
    from paper_2305_14306_gb300 import hav

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = fn()
        b.record()
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    rng = np.random.default_rng(11)
    p = hav.params(search=args.search)
    cases = []

    def single(name, pts_np, m, exact_cov, sample_q=None):
        n = pts_np.shape[0]
        ctx = hav.Context(n, 1)
        d = torch.from_numpy(pts_np).cuda()
        out = torch.empty(m, dtype=torch.int32, device="cuda")
        fout = torch.empty(m, dtype=torch.int32, device="cuda")
        for _ in range(3):
            hav.hav_sample_levels(ctx, d, [m], p, outs=[out])
        hav.hav_fps(ctx, d, min(m, 64), out=fout[:min(m, 64)])
        ms_h = min(timed(lambda: hav.hav_sample_levels(ctx, d, [m], p, outs=[out]))[1] for _ in range(5))
        _, ms_f = timed(lambda: hav.hav_fps(ctx, d, m, out=fout))
        st, _ = hav.hav_status_get(ctx, 1)
        rnd = torch.from_numpy(rng.choice(n, size=m, replace=False).astype(np.int32)).cuda()
        q = None if sample_q is None else torch.from_numpy(rng.choice(n, size=sample_q, replace=False)).cuda()
        if exact_cov:
            cov = [hav.coverage(d, x) for x in (out, fout, rnd)]
        else:
            cov = [coverage_fast(d, x, q) for x in (out, fout, rnd)]
        ctx.close()
        cases.append({"case": name, "n": n, "m": m, "hav_ms": ms_h, "fps_ms": ms_f, "fps_over_hav": ms_f / ms_h,
                      "coverage_m": {"hav": cov[0], "fps": cov[1], "random": cov[2]},
                      "coverage": "exact (fp64)" if exact_cov else
                      ("fp32, all points" if q is None else f"fp32, {sample_q} sampled query points"),
                      "status": st})

    single("C1 uniform", scenes.uniform_box(16384, seed=0), 4096, True)
    single("C2 LiDAR first level", scenes.lidar_min(16384, seed=0)[0], 16384, True)
    single("C3 indoor level 1", scenes.room_scene(1 << 20, seed=0), 1 << 18, False, sample_q=65536)

    # C4: 64 clouds, M = N/4: one batched HAV call vs 64 FPS calls
    clouds = scenes.lidar_batch(64, seed=0)
    pts, offs = scenes.concat(clouds)
    sizes = np.diff(offs)
    ms4 = (sizes // 4).astype(np.int64)
    ctx = hav.Context(int(offs[-1]), 64)
    d = torch.from_numpy(pts).cuda()
    out = torch.empty(int(ms4.sum()), dtype=torch.int32, device="cuda")
    for _ in range(3):
        hav.hav_sample_batched(ctx, d, offs, ms4[None, :], p, outs=[out])
    k0 = ctx.launches()
    hav.hav_sample_batched(ctx, d, offs, ms4[None, :], p, outs=[out])
    hav_launches = ctx.launches() - k0
    ms_h = min(timed(lambda: hav.hav_sample_batched(ctx, d, offs, ms4[None, :], p, outs=[out]))[1] for _ in range(5))
    fouts = [torch.empty(int(ms4[s]), dtype=torch.int32, device="cuda") for s in range(64)]
    views = [d[int(offs[s]):int(offs[s + 1])] for s in range(64)]

    def fps_all():
        for s in range(64):
            hav.hav_fps(ctx, views[s], int(ms4[s]), out=fouts[s])
    k0 = ctx.launches()
    _, ms_f = timed(fps_all)
    fps_launches = ctx.launches() - k0
    cut = np.concatenate([[0], np.cumsum(ms4)])
    covs = {"hav": [], "fps": [], "random": []}
    for s in range(64):
        n = int(sizes[s])
        rnd = torch.from_numpy(rng.choice(n, size=int(ms4[s]), replace=False).astype(np.int32)).cuda()
        covs["hav"].append(coverage_fast(views[s], out[int(cut[s]):int(cut[s + 1])]))
        covs["fps"].append(coverage_fast(views[s], fouts[s]))
        covs["random"].append(coverage_fast(views[s], rnd))
    ctx.close()
    cases.append({"case": "C4 64 LiDAR clouds, N/4 each", "n": int(offs[-1]), "m": int(ms4.sum()), "hav_ms": ms_h,
                  "fps_ms": ms_f, "fps_over_hav": ms_f / ms_h,
                  "coverage_m": {k: float(np.mean(v)) for k, v in covs.items()},
                  "coverage": "fp32, all points; mean over the 64 clouds",
                  "hav_launches": hav_launches, "fps_launches": fps_launches})
    if rank == 0:
        tot_n = sum(c["n"] for c in cases)
        tot_ms = sum(c["hav_ms"] for c in cases)
        line = {"metric": "input Mpoints/s", "value": tot_n / tot_ms / 1e3, "unit": "Mpoints/s", "n_gpus": world,
                "steps": 5, "warmup": 3, "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "compare", "desc": WORKLOADS["compare"]["desc"],
                           "l2": "not flushed (each case timed as the best of 5 calls)"},
                "cases": cases}
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- Table 6 variants
def run_variants(args, world, rank, local):
    import torch
    from paper_2305_14306_gb300 import hav

    flush = L2Flush(torch)
    steps = max(5, min(args.steps, 100))
    rows = []
    for case, pts_np, m in (("C1 uniform 16,384 -> 4,096", scenes.uniform_box(16384, seed=0), 4096),
                            ("C3 indoor 1,048,576 -> 262,144", scenes.room_scene(1 << 20, seed=0), 1 << 18)):
        n = pts_np.shape[0]
        ctx = hav.Context(n, 1)
        d = torch.from_numpy(pts_np).cuda()
        base = hav.params(layers=1)
        _ = hav.hav_sample_levels(ctx, d, [m], base)
        s_star = float(hav.hav_trace_get(ctx, 1)[0]["s_star"])
        idx = torch.empty(m, dtype=torch.int32, device="cuda")
        xyz = torch.empty((m, 3), dtype=torch.float32, device="cuda")
        for sel in ("centre-closest", "random", "mean", "centre"):
            for fixed in (0.0, s_star):
                p = hav.params(layers=1, select=sel, seed=1, fixed_s=fixed)
                for _ in range(3):
                    hav.hav_sample_xyz(ctx, d, m, p, out=idx, xyz=xyz)
                ev = []
                for _ in range(steps):
                    flush.sweep()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    hav.hav_sample_xyz(ctx, d, m, p, out=idx, xyz=xyz)
                    b.record()
                    ev.append((a, b))
                torch.cuda.synchronize()
                ms = sorted(a.elapsed_time(b) for a, b in ev)
                st, _ = hav.hav_status_get(ctx, 1)
                tr = hav.hav_trace_get(ctx, 1)[0]
                rows.append({"case": case, "select": sel, "voxel": "fixed" if fixed else "adaptive",
                             "fixed_s": fixed or None, "ms_p50": ms[len(ms) // 2], "k_star": int(tr["k_star"]),
                             "iters": int(tr["iters"]), "status": st})
        ctx.close()
    if rank == 0:
        main_rows = [r for r in rows if r["select"] == "centre-closest" and r["voxel"] == "adaptive"]
        tot_n = 16384 + (1 << 20)
        tot_ms = sum(r["ms_p50"] for r in main_rows)
        line = {"metric": "input Mpoints/s", "value": tot_n / tot_ms / 1e3, "unit": "Mpoints/s", "n_gpus": world,
                "steps": steps, "warmup": 3, "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "variants", "desc": WORKLOADS["variants"]["desc"],
                           "l2": L2_NOTE,
                           "fixed_s": "the adaptive search's s* of the same cloud"},
                "rows": rows}
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- Fig. 3 spacing
def run_spacing(args, world, rank, local):
    import torch
    from paper_2305_14306_gb300 import hav

    rng = np.random.default_rng(21)
    cases = []
    for case, pts_np, m in (("C1 uniform 16,384 -> 4,096", scenes.uniform_box(16384, seed=0), 4096),
                            ("C2 LiDAR returns -> 16,384", scenes.lidar_min(16384, seed=0)[0], 16384),
                            ("C3 indoor 1,048,576 -> 262,144", scenes.room_scene(1 << 20, seed=0), 1 << 18)):
        n = pts_np.shape[0]
        ctx = hav.Context(n, 1)
        d = torch.from_numpy(pts_np).cuda()
        subsets = {}
        subsets["HAV"] = hav.hav_sample_levels(ctx, d, [m], hav.params())[0]
        hav.hav_sample_levels(ctx, d, [m], hav.params(layers=1))
        s1 = float(hav.hav_trace_get(ctx, 1)[0]["s_star"])  # the one-layer search's size
        subsets["RVS (random voxel point, fixed size)"] = hav.hav_sample_levels(
            ctx, d, [m], hav.params(layers=1, select="random", seed=1, fixed_s=s1))[0]
        subsets["FPS"] = hav.hav_fps(ctx, d, m)
        subsets["RPS"] = torch.from_numpy(rng.choice(n, size=m, replace=False).astype(np.int32)).cuda()
        res = {}
        fps_min = None
        for name in ("FPS", "HAV", "RVS (random voxel point, fixed size)", "RPS"):
            idx = subsets[name]
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            d2 = hav.hav_spacing(ctx, d, idx)
            b.record()
            torch.cuda.synchronize()
            sp = np.sqrt(d2.cpu().numpy().astype(np.float64))
            if fps_min is None:
                fps_min = float(sp.min())
            # Fig. 3 as integer counts on the GPU: 24 bins of 1/8 of FPS's
            # minimum spacing (edges as binary32 squared distances)
            edges = (np.linspace(0.0, 3.0, 25) * fps_min) ** 2
            _, counts = hav.hav_spacing_histogram(ctx, d, idx, edges.astype(np.float32))
            counts = counts.cpu().numpy()
            res[name] = {"min": float(sp.min()), "p10": float(np.percentile(sp, 10)),
                         "median": float(np.median(sp)), "mean": float(sp.mean()),
                         "below_fps_min": float((sp < fps_min).mean()),
                         "hist_fps_min_units_0_to_3": counts[1:-1].tolist(), "above_3_fps_min": int(counts[-1]),
                         "spacing_ms": a.elapsed_time(b)}
        st, _ = hav.hav_status_get(ctx, 1)
        ctx.close()
        cases.append({"case": case, "n": n, "m": m, "fps_min_spacing": fps_min, "samplers": res, "status": st})
    if rank == 0:
        tot = sum(c["m"] for c in cases)
        tms = sum(c["samplers"]["HAV"]["spacing_ms"] for c in cases)
        line = {"metric": "subset points/s (spacing)", "value": tot / tms * 1e3, "unit": "points/s", "n_gpus": world,
                "steps": 1, "warmup": 0, "ms_per_step": tms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "spacing", "desc": WORKLOADS["spacing"]["desc"]}, "cases": cases}
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- grouping
def run_grouping(args, world, rank, local):
    import torch
    from paper_2305_14306_gb300 import hav

    flush = L2Flush(torch)
    steps = max(5, min(args.steps, 50))
    rows = []
    for case, pts_np, m, radius, ns in (
            ("C2 LiDAR, 4,096 centres, r 0.8 m", scenes.lidar_min(16384, seed=0)[0], 4096, 0.8, 32),
            ("C3 indoor, 262,144 centres, r 0.1 m", scenes.room_scene(1 << 20, seed=0), 1 << 18, 0.1, 32),
            ("C3 indoor, 65,536 centres, r 0.2 m", scenes.room_scene(1 << 20, seed=0), 1 << 16, 0.2, 32)):
        n = pts_np.shape[0]
        ctx = hav.Context(n, 1)
        d = torch.from_numpy(pts_np).cuda()
        centres = hav.hav_sample(ctx, d, m)
        out = torch.empty((m, ns), dtype=torch.int32, device="cuda")
        for _ in range(3):
            hav.hav_ball_query(ctx, d, centres, radius, ns, out=out)
        ev = []
        for _ in range(steps):
            flush.sweep()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            hav.hav_ball_query(ctx, d, centres, radius, ns, out=out)
            b.record()
            ev.append((a, b))
        torch.cuda.synchronize()
        ms = sorted(a.elapsed_time(b) for a, b in ev)
        st, _ = hav.hav_status_get(ctx, 1)
        filled = float((out[:, 1:] != out[:, :1]).any(dim=1).float().mean())
        rows.append({"case": case, "n": n, "m": m, "radius": radius, "nsample": ns, "ms_p50": ms[len(ms) // 2],
                     "centres_per_s": m / ms[len(ms) // 2] * 1e3, "share_with_neighbours": filled, "status": st})
        ctx.close()
    if rank == 0:
        tot_m = sum(r["m"] for r in rows)
        tot_ms = sum(r["ms_p50"] for r in rows)
        line = {"metric": "centres/s (grouping)", "value": tot_m / tot_ms * 1e3, "unit": "centres/s",
                "n_gpus": world, "steps": steps, "warmup": 3, "ms_per_step": tot_ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "grouping", "desc": WORKLOADS["grouping"]["desc"],
                           "l2": L2_NOTE}, "rows": rows}
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- serving arm
def run_serving(args, world, rank, local, sub=False, requests=None):
    """C5: closed-loop capacity and open-loop latency (Poisson arrivals at 0.5, 0.8
    and 0.95 x the plain path's capacity) of the served path vs the plain per-cloud path.
    sub=True: `requests` requests, rank 0's result returned (no print, no
    host-core oracle) for the default line's "serving" object."""
    import torch
    from paper_2305_14306_gb300 import hav, serving

    rng = np.random.default_rng(1000 + rank)
    pool_n = scenes.log_uniform_sizes(16, 10_000, 1_000_000, seed=1000 + rank)
    pool = [torch.from_numpy(scenes.scene_for(int(n), seed=5000 + i)).pin_memory() for i, n in enumerate(pool_n)]
    R = int(requests) if requests else max(20, min(args.steps, 2000))
    picks = rng.integers(0, len(pool), size=R)
    choice = rng.integers(0, 3, size=R)

    def make(arrivals):
        out = []
        for i in range(len(arrivals)):
            pts = pool[picks[i]]
            n = pts.shape[0]
            m = [n // 4, n // 16, min(4096, n)][choice[i]]
            out.append(serving.Request(i, float(arrivals[i]), pts, int(m)))
        return out

    slot_points = int(pool_n.max()) * args.serve_slot_scale
    sp = hav.params(search=args.search)
    served = serving.Server(slots=args.serve_slots, slot_points=slot_points, max_segments=64, params=sp,
                            solo_points=args.serve_solo_points or None)
    plain = serving.Server(slots=1, slot_points=int(pool_n.max()), max_segments=1, share_sms=False, params=sp)
    try:
        zero = np.zeros(R)
        plain.serve(make(zero[:min(R, 8)]))  # warm-up
        served.serve(make(zero[:min(R, 8)]))
        # closed-loop capacity: the better of two runs of each path (a host
        # hiccup in one run would otherwise move the ratio)
        cap_plain = cap_served = 0.0
        for _ in range(2):
            t0 = time.perf_counter()
            res_p = plain.serve(make(zero))
            cap_plain = max(cap_plain, R / (time.perf_counter() - t0))
            t0 = time.perf_counter()
            res_s = served.serve(make(zero))
            cap_served = max(cap_served, R / (time.perf_counter() - t0))
        same = all(np.array_equal(res_p[i].indices, res_s[i].indices) for i in range(R))
        clk = Clocks(local)
        open_loop = []
        for load in (0.5, 0.8, 0.95):  # Poisson arrivals at these fractions of the plain capacity
            lam = load * cap_plain
            arr = np.cumsum(np.random.default_rng(7 + rank).exponential(1.0 / lam, size=R))
            arr -= arr[0]
            lat_p = [r.latency for r in plain.serve(make(arr)).values()]
            res_s2 = served.serve(make(arr))
            lat_s = [r.latency for r in res_s2.values()]
            same = same and all(np.array_equal(res_p[i].indices, res_s2[i].indices) for i in range(R))
            open_loop.append({
                "load": load, "arrival_rate_hz": lam,
                "served": {"p50_ms": 1e3 * serving.percentile(lat_s, 0.5),
                           "p99_ms": 1e3 * serving.percentile(lat_s, 0.99)},
                "plain": {"p50_ms": 1e3 * serving.percentile(lat_p, 0.5),
                          "p99_ms": 1e3 * serving.percentile(lat_p, 0.99)},
                "mean_batch": float(np.mean([r.batch for r in res_s2.values()]))})
        clocks = clk.stop()
    finally:
        served.close()
        plain.close()
    pts_total = int(sum(pool[picks[i]].shape[0] for i in range(R)))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not sub:
        # the first 48 requests on the host cores, one scene per process
        k = min(R, 48)
        reqs = [(pool[picks[i]].numpy(), [[n // 4, n // 16, min(4096, n)][choice[i]]])
                for i in range(k) for n in [pool[picks[i]].shape[0]]]
        try:
            v_cpu, cores, res = scene_parallel_oracle([r[0] for r in reqs], [r[1] for r in reqs],
                                                      args.search, reps=1)
        except Exception as e:
            raise SystemExit(f"scene-parallel oracle failed: {e!r}")
        pts_k = sum(r[0].shape[0] for r in reqs)
        same = same and all(np.array_equal(res[i][0], res_p[i].indices) for i in range(k))
        cpu = {"value": v_cpu, "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
               "scenes_per_s": v_cpu * 1e6 / (pts_k / k),
               "sample": f"the first {k} requests ({pts_k} points), one scene per process (spawned pool)",
               "cpu_model": host_cpu_model()}
    if rank == 0:
        line = {
            "metric": "input Mpoints/s", "value": pts_total / R * cap_served / 1e6, "unit": "Mpoints/s",
            "n_gpus": world, "steps": R, "warmup": 8, "ms_per_step": 1e3 / cap_served,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving", "desc": WORKLOADS["serving"]["desc"], "requests": R,
                       "slots": args.serve_slots, "slot_points": slot_points, "pool_scenes": len(pool),
                       "solo_points": args.serve_solo_points or None,
                       "search": args.search},
            "scenes_per_s": cap_served,
            "plain": {"scenes_per_s": cap_plain, "value": pts_total / R * cap_plain / 1e6},
            "speedup_vs_per_cloud": cap_served / cap_plain,
            "open_loop": open_loop,
            "identical_outputs": bool(same),
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        if not sub:
            print(json.dumps(line), flush=True)
    if sub:
        return line if rank == 0 else None
    return 0


# ----------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["hav", "reference"], default="hav")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="indoor-1m")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-slots", type=int, default=2,
                    help="co-resident serving slots (GB300 at 800 requests: 2 slots of 4x the largest "
                         "scene 4.79x the plain path, 3 of 2x 4.8x)")
    ap.add_argument("--no-search-compare", action="store_true",
                    help="skip timing the guided search start beside the default one")
    ap.add_argument("--search", choices=["bisect", "guided"], default="bisect",
                    help="start of the voxel-size search: bisection over (0, s_hi] (default), or "
                         "guided by the cloud's previous search")
    ap.add_argument("--no-sub-workloads", action="store_true",
                    help="default workload only: skip the batch64 and serving objects of the line")
    ap.add_argument("--serve-slot-scale", type=int, default=4,
                    help="points a serving slot holds, in units of the largest scene of the pool")
    ap.add_argument("--serve-solo-points", type=int, default=0,
                    help="served path: clouds of at least this many points get a call of their own "
                         "(lower p99, lower throughput: GB300 at 2^17, p99 at 0.95 load 2.6 -> 1.5 ms, "
                         "3.08x -> 2.2-2.8x the plain path); 0: batch every cloud")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving object in the default line")
    ap.add_argument("--tuning-cache", default=None,
                    help="JSON cache of autotuned knobs (default: always sweep, write nothing)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()

    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2305_14306_gb300 import build as cuda_build
    from paper_2305_14306_gb300 import hav
    if rank == 0 or world == 1:
        cuda_build.build()
    if world > 1:
        dist.barrier()
    hav.load()
    arms = {"batch64": run_batched, "serving": run_serving, "compare": run_compare,
            "variants": run_variants, "spacing": run_spacing, "grouping": run_grouping}
    if args.workload in arms:
        rc = arms[args.workload](args, world, rank, local)
        if world > 1:
            dist.destroy_process_group()
        return rc

    w = WORKLOADS[args.workload]
    pts = make_scene(args.workload, seed=rank)
    n = pts.shape[0]
    ml = [min(m, n) for m in w["levels"]]
    p = hav.params(search=args.search)
    ctx = hav.Context(n, 1)
    stream = torch.cuda.current_stream()
    d_pts = torch.from_numpy(pts).cuda()
    outs = [torch.empty(m, dtype=torch.int32, device="cuda") for m in ml]
    flush = L2Flush(torch)

    def step(pp=p):
        hav.hav_sample_levels(ctx, d_pts, ml, pp, outs=outs, stream=stream)

    for _ in range(args.warmup):
        step()
    st, _ = hav.hav_status_get(ctx, 1)
    if st != hav.HAV_OK:
        raise SystemExit(f"hav status {st} on the warm-up call")
    traces = hav.hav_trace_get(ctx, len(ml) * p.layers)
    level_inputs = [n] + ml[:-1]
    B = algorithmic_bytes(traces, level_inputs, ml, p.layers)

    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except ValueError:
            pass

    def timed(pp=p, steps=args.steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = Clocks(gpu_index)
        time.sleep(0.3)
        k0 = ctx.launches()
        t0 = time.perf_counter()
        for k in range(steps):
            flush.sweep()
            evs[k][0].record(stream)
            step(pp)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        launched = ctx.launches() - k0
        if world > 1:
            dist.barrier()
        clocks = clk.stop()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, wall, clocks, launched

    ms, wall, clocks, launched = timed()
    if clocks_bad(clocks):
        ms, wall, clocks, launched = timed()
        clocks["remeasured"] = True
    st, _ = hav.hav_status_get(ctx, 1)
    if st != hav.HAV_OK:
        raise SystemExit(f"hav status {st} in the timed region")

    total_s, value = whole_job(sum(ms) / 1e3, n * args.steps, world, device="cuda")
    mean_ms = statistics.fmean(ms)
    ms_sorted = sorted(ms)
    p50 = ms_sorted[len(ms) // 2]
    p99 = ms_sorted[min(len(ms) - 1, int(0.99 * len(ms)))]

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    h_pts = torch.from_numpy(pts).pin_memory()
    h_outs = [torch.empty(m, dtype=torch.int32).pin_memory() for m in ml]
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    e2e_ms = []
    for k in range(e2e_steps + 3):
        flush.sweep()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        d_pts.copy_(h_pts, non_blocking=True)
        step()
        for o, h in zip(outs, h_outs):
            h.copy_(o, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if k >= 3:
            e2e_ms.append(a.elapsed_time(b))
    e2e_total, e2e_value = whole_job(sum(e2e_ms) / 1e3, n * len(e2e_ms), world, device="cuda")

    # the same calls pipelined: step k + 1's input copy and step k's result
    # copy run on a second stream while step k computes (two input and two
    # output buffers, ordered by events)
    def e2e_overlapped(steps):
        cs = torch.cuda.Stream()
        d_in = [d_pts, torch.empty_like(d_pts)]
        o2 = [outs, [torch.empty_like(o) for o in outs]]
        h2 = [h_outs, [torch.empty(m, dtype=torch.int32).pin_memory() for m in ml]]
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(cs)
        with torch.cuda.stream(cs):
            d_in[0].copy_(h_pts, non_blocking=True)
        ev_in[0].record(cs)
        for k in range(steps):
            x = k & 1
            stream.wait_event(ev_in[x])
            if k >= 2:
                stream.wait_event(ev_out[x])  # step k - 2's result has left this buffer
            hav.hav_sample_levels(ctx, d_in[x], ml, p, outs=o2[x], stream=stream)
            ev_done[x].record(stream)
            if k + 1 < steps:
                if k >= 1:
                    cs.wait_event(ev_done[1 - x])  # step k - 1 has read this input buffer
                with torch.cuda.stream(cs):
                    d_in[1 - x].copy_(h_pts, non_blocking=True)
                ev_in[1 - x].record(cs)
            cs.wait_event(ev_done[x])
            with torch.cuda.stream(cs):
                for o, h in zip(o2[x], h2[x]):
                    h.copy_(o, non_blocking=True)
            ev_out[x].record(cs)
        b.record(cs)
        b.synchronize()
        return a.elapsed_time(b)

    e2e_overlapped(4)
    ov_ms = e2e_overlapped(e2e_steps)
    _, ov_value = whole_job(ov_ms / 1e3, n * e2e_steps, world, device="cuda")
    if hav.hav_status_get(ctx, 1)[0] != hav.HAV_OK:
        raise SystemExit("hav status in the overlapped end-to-end run")

    peak, peak_kind = read_peaks()
    achieved = B / (mean_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic(args.workload + ("-guided" if args.search == "guided" else "")),
                "peak_kind": peak_kind,
                # one sampler call: the grid kernel, plus the small-level kernel
                # when the last levels fit it; achieved and traffic cover the call
                "kernel": "hav_chain_kernel" if launched == args.steps else "hav_chain_kernel + hav_small_kernel",
                "launches_per_call": launched / args.steps,
                "algorithmic_bytes_per_launch": B}

    # the other search start on the same workload, timed the same way
    other = None
    if args.search == "bisect" and not args.no_search_compare:
        pg = hav.params(search="guided")
        for _ in range(args.warmup):
            step(pg)
        st, _ = hav.hav_status_get(ctx, 1)
        tr_g = hav.hav_trace_get(ctx, len(ml) * pg.layers)
        B_g = algorithmic_bytes(tr_g, level_inputs, ml, pg.layers)
        g_steps = min(args.steps, 200)
        ms_g, _, clk_g, _ = timed(pg, g_steps)
        if st == hav.HAV_OK and hav.hav_status_get(ctx, 1)[0] == hav.HAV_OK:
            _, v_g = whole_job(sum(ms_g) / 1e3, n * g_steps, world, device="cuda")
            mg = statistics.fmean(ms_g)
            peak_g, _ = read_peaks()
            other = {"search": "guided", "value": v_g, "unit": "Mpoints/s", "ms_per_step": mg,
                     "p50_ms": sorted(ms_g)[len(ms_g) // 2], "steps": g_steps,
                     "bisection_steps": int(sum(int(t["iters"]) for t in tr_g)),
                     "roofline_frac": B_g / (mg / 1e3) / 1e9 / peak_g,
                     "algorithmic_bytes_per_launch": B_g, "sm_mhz": clk_g.get("sm_mhz"),
                     "traffic": profiled_traffic(args.workload + "-guided")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        op = oracle.params(search=args.search)
        runs, t_cpu = 0, 0.0
        while runs < 30 and (runs < 3 or t_cpu < 10.0):
            t0 = time.perf_counter()
            oracle.sample_levels(pts, ml, op)
            t_cpu += time.perf_counter() - t0
            runs += 1
        cpu = {"value": n * runs / t_cpu / 1e6, "unit": "Mpoints/s", "cores": 1, "kind": "oracle",
               "sample": f"{runs} full run(s) of the same scene and level chain ({t_cpu:.1f} s), single thread",
               "cpu_model": host_cpu_model()}

    if rank == 0:
        line = {
            "metric": "input Mpoints/s", "value": value, "unit": "Mpoints/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "n": n, "levels": ml,
                       "layers": p.layers, "sigma": "5/100", "t_max": p.t_max, "search": args.search,
                       "bisection_steps": int(sum(int(t["iters"]) for t in traces)),
                       "l2": L2_NOTE,
                       "parallelism": "replicas" if world > 1 else "single"},
            "scenes_per_s": world * args.steps / total_s,
            "p50_ms": p50, "p99_ms": p99,
            "hbm_gbs_effective": achieved,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "Mpoints/s", "h2d_bytes_per_step": int(pts.nbytes),
                    "d2h_bytes_per_step": int(4 * sum(ml)), "steps": len(e2e_ms),
                    "overlapped": {"value": ov_value, "unit": "Mpoints/s", "steps": e2e_steps,
                                   "how": "the same copies and calls, step k + 1's input copy and step k's "
                                          "result copy on a second stream during step k's call; L2 not "
                                          "flushed (each step's input arrives by its own copy)"}},
            "gpu_launches": launched,  # counted by the library over the timed steps
            "launches_per_step": launched / args.steps,
            "clocks": clocks,
            "wall_s_timed": wall,
        }
        if other is not None:
            line["search_guided"] = other
    ctx.close()
    subs = {}
    if world == 1 and args.workload == "indoor-1m" and not args.no_sub_workloads:
        # the batched (C4) and served (C5) forms against the plain per-cloud
        # path, on the same GPU in the same run, summarised beside the headline
        b = run_batched(args, world, rank, local, sub=True)
        subs["batch64"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "scenes_per_s", "p50_ms", "p99_ms",
                                             "graph", "per_cloud", "speedup_vs_per_cloud", "identical_outputs",
                                             "tuning", "gpu_launches", "launches_per_step", "clocks")}
        subs["batch64"]["config"] = b["config"]
        srv = run_serving(args, world, rank, local, sub=True, requests=args.serve_requests)
        subs["serving"] = {k: srv[k] for k in ("value", "unit", "scenes_per_s", "plain", "speedup_vs_per_cloud",
                                               "open_loop", "identical_outputs", "clocks")}
        subs["serving"]["config"] = srv["config"]
    if rank == 0:
        line.update(subs)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
