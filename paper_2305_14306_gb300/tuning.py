"""Autotuner for the sampler's launch shape.

A context's knobs (``hav_tuning`` in include/hav.h) that the tuner searches:

* ``spec_points`` -- the level sizes up to which one bisection pass evaluates
  4, 3 or 2 steps of the search at once (Section 3.3 run speculatively: on a
  small level a pass is mostly fixed latency, so evaluating several sizes per
  pass means fewer grid-wide passes, until the work per candidate catches up);
* ``chunk_min`` -- the smallest work item, in points;
* ``table_log2`` -- the hash-table load factor: a segment's voxel table has
  nextpow2(2^f n) slots for n points (f = 1, 2, 3: at most 1/2, 1/4, 1/8 full;
  a flush waits for its longest probe chain, so emptier tables can pay);
* ``pass_shape`` -- points each thread loads ahead and global probes it keeps
  in flight in a pass, one instantiation of the grid kernel each (the block
  shape itself is fixed: one 1024-thread block per SM);
* ``small_points`` -- the level size up to which levels run on thread-block
  clusters (0: never).

The number of blocks is left as it is.  No knob changes a result.  The tuner
therefore times the caller's own workload under a short list of settings (a
coordinate search, one knob after the other, each from the best so far) and
keeps the fastest.  The choice is cached in a JSON file under the GPU's name
and a signature of the workload (segment count, total points and level count,
each rounded to a power of two), so the next process with the same kind of
workload skips the sweep.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "hav_tuning.json")
BASE_SPEC = (0, 4096, 65536)
# speculation thresholds tried (depth 4 up to [0], 3 up to [1], 2 up to [2] points)
SPEC_CHOICES = (
    (0, 0, 0), (0, 4096, 65536), (0, 0, 65536), (0, 0, 262144), (0, 8192, 131072), (0, 16384, 262144),
    (0, 32768, 262144), (0, 65536, 524288), (8192, 16384, 262144), (32768, 131072, 262144),
)
CHUNK_MINS = (32, 64, 128, 256, 512, 1024)
TABLE_LOG2 = (1, 2, 3)
PASS_SHAPES = (0, 1, 2, 3)
SMALL_POINTS = (0, 32768)
# the knobs the search visits, in order, and their defaults where a context
# (or an older cache entry) does not report one
STAGES = (("spec_points", SPEC_CHOICES), ("chunk_min", CHUNK_MINS), ("table_log2", TABLE_LOG2),
          ("pass_shape", PASS_SHAPES), ("small_points", SMALL_POINTS))
DEFAULTS = {"spec_points": list(BASE_SPEC), "chunk_min": 64, "table_log2": 1, "pass_shape": 0, "small_points": 0}


def signature(seg_sizes, levels: int) -> str:
    """Workload key: segments, total points and levels, rounded to powers of two."""
    sizes = [int(x) for x in seg_sizes]
    S = max(1, len(sizes))
    N = max(1, sum(sizes))
    return f"S{1 << math.ceil(math.log2(S))}-N{1 << round(math.log2(N))}-L{int(levels)}"


def spec_for(scale: float, base=BASE_SPEC):
    """The thresholds scaled (clamped to 2^31)."""
    return [min(1 << 31, int(round(b * scale))) for b in base]


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: dict) -> None:
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".hav_tuning.")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)  # readers never see a half-written file


def cuda_timer(run, reps: int = 3):
    """Milliseconds per call of run() on the current stream (CUDA events, after one warm-up)."""
    import torch
    run()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        run()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _same(a, b) -> bool:
    return list(a) == list(b) if isinstance(a, (list, tuple)) else a == b


def autotune(ctx, run, key: str, gpu: str, cache: str | None = DEFAULT_CACHE, force: bool = False,
             timer=None, reps: int = 3):
    """Pick the fastest knobs for run() (one call of the workload on ctx).

    ctx: an object with get_tuning() / set_tuning(**knobs) (a hav.Context).
    Returns (tuning dict, report dict); the context is left with the chosen
    tuning.  cache=None: neither read nor write a cache.  A setting the
    context refuses (e.g. clusters on a device without them) is skipped.
    """
    timer = timer or (lambda: cuda_timer(run, reps))
    entry_key = f"{gpu}|{key}"
    data = load_cache(cache) if cache else {}
    if not force and entry_key in data:
        t = {**DEFAULTS, **data[entry_key]["tuning"]}
        ctx.set_tuning(**t)
        return t, {"cached": True, **data[entry_key].get("report", {})}

    start = ctx.get_tuning()
    best = {k: (list(start[k]) if k == "spec_points" else int(start[k])) if k in start else DEFAULTS[k]
            for k, _ in STAGES}
    tried = []

    def measure(setting):
        try:
            ctx.set_tuning(**setting)
        except Exception:  # refused by the context: not a candidate
            return None
        ms = float(timer())
        tried.append({**setting, "ms": ms})
        return ms

    default_ms = measure(best)
    best_ms = default_ms
    for knob, choices in STAGES:  # coordinate search, each knob from the best so far
        for choice in choices:
            if _same(choice, best[knob]):
                continue
            cand = {**best, knob: list(choice) if knob == "spec_points" else int(choice)}
            ms = measure(cand)
            if ms is not None and ms < best_ms:
                best, best_ms = cand, ms
    ctx.set_tuning(**best)
    report = {"cached": False, "default_ms": default_ms, "tuned_ms": best_ms, "tried": len(tried)}
    if cache:
        data = load_cache(cache)  # re-read: another process may have added entries
        data[entry_key] = {"tuning": best, "report": {k: v for k, v in report.items() if k != "cached"}}
        save_cache(cache, data)
    return best, report
