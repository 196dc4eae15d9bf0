"""Helpers for the GPU parity tests: a shared libhav context and an oracle
process pool (spawn start method, so it is safe after CUDA is initialised)."""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

_pool = None


def oracle_levels(args):
    """Worker: oracle level chain of one cloud; plain picklable arguments."""
    import oracle
    pts, m_levels, pkw = args
    p = oracle.params(**pkw)
    res, tr = oracle.sample_levels(pts, m_levels, p, want_trace=True)
    return res, tr


def pool():
    global _pool
    if _pool is None:
        workers = max(1, min(16, (os.cpu_count() or 2) - 1))
        _pool = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    return _pool


def oracle_many(clouds, m_levels_per_cloud, pkw=None):
    pkw = pkw or {}
    jobs = [(c, list(map(int, ml)), pkw) for c, ml in zip(clouds, m_levels_per_cloud)]
    if len(jobs) == 1:
        return [oracle_levels(jobs[0])]
    return list(pool().map(oracle_levels, jobs))


def traces_equal(gpu_tr, ora_tr):
    """Compare one layer's GPU trace record with the oracle's; returns a reason or None."""
    if int(gpu_tr["m_l"]) != int(ora_tr["m_l"]):
        return f"m_l: gpu {gpu_tr['m_l']} oracle {ora_tr['m_l']}"
    if gpu_tr["m_l"] == 0:
        return None
    for key in ("k_max", "k_star", "n_in", "iters", "accepted"):
        if int(gpu_tr[key]) != int(ora_tr[key]):
            return f"{key}: gpu {gpu_tr[key]} oracle {ora_tr[key]}"
    for key in ("s_hi", "s_star"):
        if np.float32(gpu_tr[key]).tobytes() != np.float32(ora_tr[key]).tobytes():
            return f"{key}: gpu {gpu_tr[key]!r} oracle {ora_tr[key]!r}"
    if not np.array_equal(gpu_tr["s"].view(np.uint32), ora_tr["s"].view(np.uint32)):
        return f"s: gpu {gpu_tr['s']} oracle {ora_tr['s']}"
    # steps the device settled from an earlier layer's count (bit t of "bounded"):
    # that count bounds the exact one from above and is below m_l (too few voxels,
    # the outcome the oracle's exact count also gives); every other step is exact
    bounded = int(gpu_tr.get("bounded", 0))
    for t in range(int(gpu_tr["iters"])):
        kg, ko = int(gpu_tr["K"][t]), int(ora_tr["K"][t])
        if (bounded >> t) & 1:
            if not (ko <= kg < int(gpu_tr["m_l"])):
                return f"bounded step {t}: gpu bound {kg}, oracle count {ko}, m_l {gpu_tr['m_l']}"
        elif kg != ko:
            return f"K: gpu {gpu_tr['K']} oracle {ora_tr['K']} (step {t})"
    if bounded >> int(gpu_tr["iters"]):
        return f"bounded bits beyond the evaluated steps: {bounded:#x}"
    return None
