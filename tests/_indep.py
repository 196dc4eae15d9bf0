"""Independent numpy restatements used only to pin the oracle.

These take a different route from the oracle (numpy float32 vector arithmetic,
np.unique / lexsort grouping, O(n^2) pairwise comparison) so that a slip in
the oracle's C++ (a dropped term, a wrong index, a wrong sign) shows up as a
mismatch.  Nothing here is called by the oracle or by the CUDA library.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def bbox_s_hi(p: np.ndarray, aspect=(1.0, 1.0, 1.0)):
    mn = p.min(axis=0)
    mx = p.max(axis=0)
    ext = (mx - mn).astype(F32)
    s_hi = F32(np.max(ext / np.asarray(aspect, dtype=F32)))
    if s_hi == 0:
        s_hi = F32(1.0)
    return mn.astype(F32), s_hi


def cells(p: np.ndarray, s, aspect=(1.0, 1.0, 1.0)):
    """Eq. 2: absolute cells floor(x / v) (int64) and the float floors, v = s * r."""
    v = (F32(s) * np.asarray(aspect, dtype=F32)).astype(F32)
    q = (p.astype(F32) / v[None, :]).astype(F32)
    f = np.floor(q).astype(F32)
    return f.astype(np.int64), f, v


def rel_cells(p: np.ndarray, s, aspect=(1.0, 1.0, 1.0)):
    mn, _ = bbox_s_hi(p, aspect)
    g, f, v = cells(p, s, aspect)
    gmin = np.floor((mn / v).astype(F32)).astype(np.int64)
    return g - gmin[None, :], f, v


def packed_keys(p, s, aspect=(1.0, 1.0, 1.0)):
    u, _, _ = rel_cells(p, s, aspect)
    assert (u >= 0).all() and (u < (1 << 21)).all()
    u = u.astype(np.uint64)
    return u[:, 0] | (u[:, 1] << np.uint64(21)) | (u[:, 2] << np.uint64(42))


def centre_d2(p, f, v):
    """Section 3.2 distance to v * (g + 0.5), squared, binary32, fixed order."""
    half = (f + F32(0.5)).astype(F32)
    c = (v[None, :] * half).astype(F32)
    d = (p.astype(F32) - c).astype(F32)
    sq = (d * d).astype(F32)
    return ((sq[:, 0] + sq[:, 1]).astype(F32) + sq[:, 2]).astype(F32)


def count_unique(p, s, aspect=(1.0, 1.0, 1.0), active=None):
    u, _, _ = rel_cells(p, s, aspect)
    if active is not None:
        u = u[active]
    return int(np.unique(u, axis=0).shape[0])


def brute_force_select(p, s, aspect=(1.0, 1.0, 1.0), active=None):
    """O(n^2) grouping by pairwise cell equality, then a linear argmin of d^2
    (ties to the lowest index) per group; returns the representatives, ascending."""
    idx = np.arange(p.shape[0]) if active is None else np.asarray(active)
    g, f, v = cells(p, s, aspect)
    d2 = centre_d2(p, f, v)
    g = g[idx]
    d2 = d2[idx]
    same = (g[:, None, :] == g[None, :, :]).all(axis=2)
    reps = set()
    for a in range(len(idx)):
        members = np.nonzero(same[a])[0]
        best = members[0]
        for b in members[1:]:
            if d2[b] < d2[best] or (d2[b] == d2[best] and idx[b] < idx[best]):
                best = b
        reps.add(int(idx[best]))
    return np.array(sorted(reps), dtype=np.int32)


def lexsort_select(p, s, aspect=(1.0, 1.0, 1.0), active=None):
    """Textbook dedupe: sort by (cell, d^2, index) and keep the first of each cell."""
    idx = np.arange(p.shape[0]) if active is None else np.asarray(active)
    u, f, v = rel_cells(p, s, aspect)
    d2 = centre_d2(p, f, v)
    u, d2 = u[idx], d2[idx]
    order = np.lexsort((idx, d2, u[:, 2], u[:, 1], u[:, 0]))
    us = u[order]
    first = np.ones(len(order), dtype=bool)
    first[1:] = (us[1:] != us[:-1]).any(axis=1)
    return np.sort(idx[order[first]]).astype(np.int32)


def select_by_word(p, s, word, aspect=(1.0, 1.0, 1.0), active=None):
    """Per occupied cell, the point with the smallest (word, index): sort by
    (cell, word, index) and keep the first of each cell; ascending."""
    idx = np.arange(p.shape[0]) if active is None else np.asarray(active)
    u, _, _ = rel_cells(p, s, aspect)
    u, w = u[idx], np.asarray(word, dtype=np.uint64)[idx]
    order = np.lexsort((idx, w, u[:, 2], u[:, 1], u[:, 0]))
    us = u[order]
    first = np.ones(len(order), dtype=bool)
    first[1:] = (us[1:] != us[:-1]).any(axis=1)
    return np.sort(idx[order[first]]).astype(np.int32)


def splitmix64_draw(seed: int, counter: int) -> int:
    """SplitMix64 as published: the state starts at `seed` and advances by the
    golden-ratio step before each output; draw `counter` (0-based)."""
    M = (1 << 64) - 1
    return splitmix64_finalise((seed + (counter + 1) * 0x9E3779B97F4A7C15) & M)


def splitmix64_finalise(z: int) -> int:
    M = (1 << 64) - 1
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def budgets(m: int, layers: int, ratio: int):
    w = [ratio ** l for l in range(layers)]
    S = sum(w)
    ml = [m * w[l] // S for l in range(layers - 1)]
    ml.append(m - sum(ml))
    return ml


def bisection(p, m_l, s_hi, sigma=(5, 100), t_max=20, aspect=(1.0, 1.0, 1.0), active=None, start=None):
    """Section 3.3 search with numpy counting; returns (trace [(s, K)], s*, accepted).
    start: the guided search's first size; from it the size doubles while every
    count so far was above k_max and twice the lower end stays below the top,
    and bisects otherwise."""
    k_max = m_l + (m_l * sigma[0]) // sigma[1]
    lo, hi = F32(0.0), F32(s_hi)
    up = start is not None
    trace = []
    for t in range(t_max):
        if t == 0 and start is not None:
            s = F32(start)
        elif up and F32(lo * F32(2.0)) < hi:
            s = F32(lo * F32(2.0))
        else:
            s = F32((lo + hi) * F32(0.5))
        K = count_unique(p, s, aspect, active)
        trace.append((s, K))
        if K > k_max:
            lo = s
        elif K < m_l:
            hi = s
            up = False
        else:
            return trace, s, True
    return trace, (lo if lo > 0 else hi), False


def guided_start(s_hi, m_l, prev):
    """First size of a guided search: s_hi / sqrt(m_l) without a previous search,
    else s_prev * sqrt(m_prev / m_l); None when it is not below s_hi."""
    if prev is None:
        g = F32(F32(s_hi) / np.sqrt(F32(m_l)))
    else:
        g = F32(F32(prev[0]) * np.sqrt(F32(F32(prev[1]) / F32(m_l))))
    return g if (g > 0 and g < F32(s_hi)) else None


def hav_reference_small(p, m, layers=2, ratio=4, sigma=(5, 100), t_max=20, aspect=(1.0, 1.0, 1.0),
                        select="cc", seed=0, fixed_s=0.0, search="bisect", guide=None, traces=None):
    """Whole sampler on a tiny cloud with numpy pieces (bisection + lexsort select +
    priority truncation + shortfall), for cross-checking the oracle end to end.
    select "random": per cell the smallest SplitMix64 draw (high 32 bits) wins;
    fixed_s > 0: no search, s* = fixed_s.  search "guided": each search starts at
    guided_start(); `guide` (a one-element list) carries (s*, m_l) of the previous
    search between calls; `traces` collects each layer's [(s, K)]."""
    n = p.shape[0]
    taken = np.zeros(n, dtype=bool)
    _, s_hi = bbox_s_hi(p, aspect)
    if guide is None:
        guide = [None]
    word = None
    if select == "random":
        word = np.array([splitmix64_draw(seed, i) >> 32 for i in range(n)], dtype=np.uint64)
    for m_l in budgets(m, layers, ratio):
        if m_l == 0:
            if traces is not None:
                traces.append([])
            continue
        active = np.nonzero(~taken)[0]
        if fixed_s > 0:
            s_star = F32(fixed_s)
            tr = []
        else:
            start = guided_start(s_hi, m_l, guide[0]) if search == "guided" else None
            tr, s_star, _ = bisection(p, m_l, s_hi, sigma, t_max, aspect, active, start)
            if t_max > 0:
                guide[0] = (s_star, m_l)
        if traces is not None:
            traces.append(tr)
        if word is None:
            reps = lexsort_select(p, s_star, aspect, active)
        else:
            reps = select_by_word(p, s_star, word, aspect, active)
        K = len(reps)
        if K > m_l:
            u, _, _ = rel_cells(p, s_star, aspect)
            u = u.astype(np.uint64)
            keys = u[:, 0] | (u[:, 1] << np.uint64(21)) | (u[:, 2] << np.uint64(42))
            pr = np.array([splitmix64_finalise(int(keys[i])) for i in reps], dtype=np.uint64)
            reps = reps[np.argsort(pr, kind="stable")[:m_l]]
        taken[reps] = True
        if K < m_l:
            need = m_l - K
            for i in active:
                if need == 0:
                    break
                if not taken[i]:
                    taken[i] = True
                    need -= 1
    return np.nonzero(taken)[0].astype(np.int32)


def hav_reference_levels_small(p, m_levels, search="bisect", **kw):
    """Level chain of hav_reference_small: level j + 1 samples level j's points in
    ascending order; indices refer to the original cloud.  Returns (levels, traces),
    traces[j][l] the [(s, K)] of level j, layer l."""
    cur = np.asarray(p, dtype=F32)
    orig = np.arange(cur.shape[0], dtype=np.int32)
    guide = [None]
    out, traces = [], []
    for m in m_levels:
        tr = []
        idx = hav_reference_small(cur, m, search=search, guide=guide, traces=tr, **kw) if m > 0 else \
            np.zeros(0, dtype=np.int32)
        out.append(orig[idx])
        traces.append(tr)
        cur, orig = cur[idx], orig[idx]
    return out, traces
