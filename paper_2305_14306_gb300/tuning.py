"""Autotuner for the sampler's launch shape.

A context has three knobs (``hav_tuning`` in include/hav.h):

* the level sizes up to which one bisection pass evaluates 4, 3 or 2 steps of
  the search at once (Section 3.3 run speculatively: on a small level a pass
  is mostly fixed latency, so evaluating several sizes per pass means fewer
  grid-wide passes, until the work per candidate catches up);
* the smallest work item, in points;
* the number of blocks (one per SM);
* the level size up to which levels run on thread-block clusters (0: never).

No knob changes a result.  The tuner therefore times the caller's own
workload under a short list of settings (a coordinate search: first the
speculation thresholds, then the work-item size) and keeps the fastest.  The
choice is cached in a JSON file under the GPU's name and a signature of the
workload (segment count, total points and level count, each rounded to a
power of two), so the next process with the same kind of workload skips the
sweep.
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
SMALL_POINTS = (0, 32768)


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


def autotune(ctx, run, key: str, gpu: str, cache: str | None = DEFAULT_CACHE, force: bool = False,
             timer=None, reps: int = 3):
    """Pick the fastest knobs for run() (one call of the workload on ctx).

    ctx: an object with get_tuning() / set_tuning(spec_points=, chunk_min=)
    (a hav.Context).  Returns (tuning dict, report dict); the context is left
    with the chosen tuning.  cache=None: neither read nor write a cache.
    """
    timer = timer or (lambda: cuda_timer(run, reps))
    entry_key = f"{gpu}|{key}"
    data = load_cache(cache) if cache else {}
    if not force and entry_key in data:
        t = data[entry_key]["tuning"]
        ctx.set_tuning(spec_points=t["spec_points"], chunk_min=t["chunk_min"],
                       small_points=t.get("small_points", 0))
        return t, {"cached": True, **data[entry_key].get("report", {})}

    start = ctx.get_tuning()
    tried = []

    def measure(spec, chunk):
        ctx.set_tuning(spec_points=spec, chunk_min=chunk)
        ms = float(timer())
        tried.append({"spec_points": list(spec), "chunk_min": int(chunk), "ms": ms})
        return ms

    default_ms = measure(start["spec_points"], start["chunk_min"])
    best = (default_ms, list(start["spec_points"]), int(start["chunk_min"]))
    for choice in SPEC_CHOICES:  # stage 1: speculation thresholds at the current work-item size
        spec = list(choice)
        if spec == best[1]:
            continue
        ms = measure(spec, best[2])
        if ms < best[0]:
            best = (ms, spec, best[2])
    for ch in CHUNK_MINS:  # stage 2: work-item size at the best thresholds
        if ch == best[2]:
            continue
        ms = measure(best[1], ch)
        if ms < best[0]:
            best = (ms, best[1], ch)
    small = int(start.get("small_points", 0))
    for sp in SMALL_POINTS:  # stage 3: small levels on clusters or not
        if sp == small:
            continue
        try:
            ctx.set_tuning(spec_points=best[1], chunk_min=best[2], small_points=sp)
        except Exception:  # no cluster launch on this device
            continue
        ms = float(timer())
        tried.append({"spec_points": list(best[1]), "chunk_min": int(best[2]), "small_points": sp, "ms": ms})
        if ms < best[0]:
            best = (ms, best[1], best[2])
            small = sp
    tuning = {"spec_points": best[1], "chunk_min": best[2], "small_points": small}
    ctx.set_tuning(spec_points=tuning["spec_points"], chunk_min=tuning["chunk_min"], small_points=small)
    report = {"cached": False, "default_ms": default_ms, "tuned_ms": best[0], "tried": len(tried)}
    if cache:
        data = load_cache(cache)  # re-read: another process may have added entries
        data[entry_key] = {"tuning": tuning, "report": {k: v for k, v in report.items() if k != "cached"}}
        save_cache(cache, data)
    return tuning, report
