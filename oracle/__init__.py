"""HAVSampler CPU oracle -- test infrastructure only.

Plain C++ restatement of the sampler of arXiv 2305.14306, Section 3 (Eq. 2
voxel coordinates, the centre-closest rule of Section 3.2, the adaptive voxel
search of Section 3.3 and the k-layer paradigm of Eq. 3), loaded through
ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package; the CUDA library never does, and the
two share no code.

Every function takes and returns numpy arrays; points are (n, 3) float32,
C-contiguous, x/y/z interleaved.

HAV_ORACLE_LIB, when set, names a prebuilt library of a modified copy of
hav_oracle.cpp to load instead of this one (the planted-mistake tests use it
to check that the pins catch each mistake); it is never rebuilt.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hav_oracle.cpp")
_LIB = os.environ.get("HAV_ORACLE_LIB") or os.path.join(_HERE, "libhav_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_NONFINITE, ERR_RANGE = 0, 1, 2, 7
MAX_ITERS = 20


class Params(C.Structure):
    _fields_ = [
        ("sigma_num", C.c_int32),
        ("sigma_den", C.c_int32),
        ("t_max", C.c_int32),
        ("layers", C.c_int32),
        ("layer_ratio", C.c_int32),
        ("aspect", C.c_float * 3),
        ("flags", C.c_uint32),
        ("select", C.c_int32),
        ("seed", C.c_uint32),
        ("fixed_s", C.c_float),
        ("search", C.c_int32),
    ]


SELECT = {"cc": 0, "random": 1, "mean": 2, "centre": 3}
SEARCH = {"bisect": 0, "guided": 1}


class LayerTrace(C.Structure):
    _fields_ = [
        ("m_l", C.c_int64),
        ("k_max", C.c_int64),
        ("k_star", C.c_int64),
        ("n_in", C.c_int64),
        ("iters", C.c_int32),
        ("accepted", C.c_int32),
        ("s_hi", C.c_float),
        ("s_star", C.c_float),
        ("s", C.c_float * MAX_ITERS),
        ("K", C.c_int64 * MAX_ITERS),
    ]


def params(sigma=(5, 100), t_max=20, layers=2, layer_ratio=4, aspect=(1.0, 1.0, 1.0),
           select="cc", seed=0, fixed_s=0.0, search="bisect"):
    """Paper defaults (Section 4.1): sigma = 0.05, t_max = 20, k = 2, centre-closest
    selection, adaptive voxel.  select / fixed_s: the Table 6 variants.
    search: "bisect" (over (0, s_hi]) or "guided" (from the previous search)."""
    p = Params()
    p.sigma_num, p.sigma_den = sigma
    p.t_max, p.layers, p.layer_ratio = t_max, layers, layer_ratio
    for a in range(3):
        p.aspect[a] = aspect[a]
    p.flags = 0
    p.select = SELECT[select] if isinstance(select, str) else int(select)
    p.seed = int(seed)
    p.fixed_s = float(fixed_s)
    p.search = SEARCH[search] if isinstance(search, str) else int(search)
    return p


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain IEEE binary32, no contraction)."""
    if os.environ.get("HAV_ORACLE_LIB"):
        return _LIB
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            fp, i64, i32 = C.POINTER(C.c_float), C.c_int64, C.c_int32
            L.hor_sample.argtypes = [fp, i64, i64, C.POINTER(Params), C.POINTER(C.c_int32),
                                     C.POINTER(LayerTrace)]
            L.hor_sample.restype = C.c_int
            L.hor_sample_levels.argtypes = [fp, i64, C.POINTER(C.c_int64), i32, C.POINTER(Params),
                                            C.POINTER(C.c_int32), C.POINTER(LayerTrace)]
            L.hor_sample_levels.restype = C.c_int
            L.hor_count.argtypes = [fp, i64, C.c_float, fp, C.POINTER(C.c_int64)]
            L.hor_count.restype = C.c_int
            L.hor_keys.argtypes = [fp, i64, C.c_float, fp, C.POINTER(C.c_uint64)]
            L.hor_keys.restype = C.c_int
            L.hor_select.argtypes = [fp, i64, C.c_float, fp, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int64)]
            L.hor_select.restype = C.c_int
            L.hor_priority.argtypes = [C.c_uint64]
            L.hor_priority.restype = C.c_uint64
            L.hor_s_hi.argtypes = [fp, i64, fp]
            L.hor_s_hi.restype = C.c_float
            L.hor_fps.argtypes = [fp, i64, i64, C.POINTER(C.c_int32)]
            L.hor_fps.restype = C.c_int
            L.hor_ball_query.argtypes = [fp, i64, C.POINTER(C.c_int32), i64, C.c_float, C.c_int32,
                                         C.POINTER(C.c_int32), fp]
            L.hor_ball_query.restype = C.c_int
            L.hor_spacing.argtypes = [fp, i64, C.POINTER(C.c_int32), i64, fp]
            L.hor_spacing.restype = C.c_int
            L.hor_random.argtypes = [C.c_uint32, C.c_uint64]
            L.hor_random.restype = C.c_uint64
            L.hor_sample_xyz.argtypes = [fp, i64, i64, C.POINTER(Params), C.POINTER(C.c_int32), fp,
                                         C.POINTER(LayerTrace)]
            L.hor_sample_xyz.restype = C.c_int
            _lib = L
    return _lib


def _pts(points):
    a = np.ascontiguousarray(points, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("points must be (n, 3) float32")
    return a


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _aspect(aspect):
    return np.ascontiguousarray(aspect, dtype=np.float32)


def trace_dict(t: LayerTrace) -> dict:
    it = t.iters
    return {
        "m_l": t.m_l, "k_max": t.k_max, "k_star": t.k_star, "n_in": t.n_in,
        "iters": it, "accepted": bool(t.accepted),
        "s_hi": np.float32(t.s_hi), "s_star": np.float32(t.s_star),
        "s": np.array(t.s[:it], dtype=np.float32), "K": np.array(t.K[:it], dtype=np.int64),
    }


def sample(points, m, p: Params | None = None, want_trace: bool = False):
    """One HAVSampler call; returns ascending int32 indices (and the per-layer trace)."""
    p = p or params()
    a = _pts(points)
    out = np.zeros(max(int(m), 1), dtype=np.int32)
    tr = (LayerTrace * max(p.layers, 1))()
    st = lib().hor_sample(_fp(a), a.shape[0], int(m), C.byref(p),
                          out.ctypes.data_as(C.POINTER(C.c_int32)), tr)
    if st != OK:
        raise OracleError(st)
    out = out[: int(m)]
    if want_trace:
        return out, [trace_dict(tr[l]) for l in range(p.layers)]
    return out


def sample_levels(points, m_levels, p: Params | None = None, want_trace: bool = False):
    """Level chain; returns a list of per-level index arrays into the original cloud."""
    p = p or params()
    a = _pts(points)
    ml = np.ascontiguousarray(m_levels, dtype=np.int64)
    out = np.zeros(max(int(ml.sum()), 1), dtype=np.int32)
    tr = (LayerTrace * (len(ml) * p.layers))()
    st = lib().hor_sample_levels(_fp(a), a.shape[0], ml.ctypes.data_as(C.POINTER(C.c_int64)),
                                 len(ml), C.byref(p), out.ctypes.data_as(C.POINTER(C.c_int32)), tr)
    if st != OK:
        raise OracleError(st)
    res, off = [], 0
    for m in ml:
        res.append(out[off: off + int(m)].copy())
        off += int(m)
    if want_trace:
        traces = [[trace_dict(tr[j * p.layers + l]) for l in range(p.layers)] for j in range(len(ml))]
        return res, traces
    return res


def count(points, s, aspect=(1.0, 1.0, 1.0)) -> int:
    """Cnt(P, v) of Section 3.3 at v = s * aspect, over all points."""
    a = _pts(points)
    asp = _aspect(aspect)
    K = C.c_int64(0)
    st = lib().hor_count(_fp(a), a.shape[0], float(np.float32(s)), _fp(asp), C.byref(K))
    if st != OK:
        raise OracleError(st)
    return int(K.value)


def keys(points, s, aspect=(1.0, 1.0, 1.0)):
    a = _pts(points)
    asp = _aspect(aspect)
    out = np.zeros(a.shape[0], dtype=np.uint64)
    st = lib().hor_keys(_fp(a), a.shape[0], float(np.float32(s)), _fp(asp),
                        out.ctypes.data_as(C.POINTER(C.c_uint64)))
    if st != OK:
        raise OracleError(st)
    return out


def select(points, s, aspect=(1.0, 1.0, 1.0)):
    """S(P, v) of Section 3.2 at v = s * aspect: centre-closest point per voxel, ascending."""
    a = _pts(points)
    out = np.zeros(a.shape[0], dtype=np.int32)
    K = C.c_int64(0)
    st = lib().hor_select(_fp(a), a.shape[0], float(np.float32(s)), _fp(_aspect(aspect)),
                          out.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(K))
    if st != OK:
        raise OracleError(st)
    return out[: K.value].copy()


def priority(key: int) -> int:
    return int(lib().hor_priority(C.c_uint64(int(key))))


def ball_query(points, centres, radius, nsample):
    """Grouping around centres (indices into points): (m, nsample) int32 indices and
    (m, nsample, 3) float32 offsets p_k - c_j."""
    a = _pts(points)
    c = np.ascontiguousarray(centres, dtype=np.int32)
    m = len(c)
    idx = np.zeros((max(m, 1), nsample), dtype=np.int32)
    xyz = np.zeros((max(m, 1), nsample, 3), dtype=np.float32)
    st = lib().hor_ball_query(_fp(a), a.shape[0], c.ctypes.data_as(C.POINTER(C.c_int32)), m,
                              float(np.float32(radius)), int(nsample), idx.ctypes.data_as(C.POINTER(C.c_int32)),
                              _fp(xyz))
    if st != OK:
        raise OracleError(st)
    return idx[:m], xyz[:m]


def spacing(points, idx):
    """Squared nearest-neighbour distance of every subset point within the subset (Fig. 3)."""
    a = _pts(points)
    ix = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.zeros(max(len(ix), 1), dtype=np.float32)
    st = lib().hor_spacing(_fp(a), a.shape[0], ix.ctypes.data_as(C.POINTER(C.c_int32)), len(ix), _fp(out))
    if st != OK:
        raise OracleError(st)
    return out[: len(ix)]


def random_draw(seed: int, counter: int) -> int:
    """Draw `counter` of the counter-based SplitMix64 generator started at `seed`."""
    return int(lib().hor_random(C.c_uint32(int(seed)), C.c_uint64(int(counter))))


def sample_xyz(points, m, p: Params | None = None, want_trace: bool = False):
    """One-layer call returning (ascending indices, representative coordinates (m, 3))."""
    p = p or params(layers=1)
    a = _pts(points)
    out = np.zeros(max(int(m), 1), dtype=np.int32)
    xyz = np.zeros((max(int(m), 1), 3), dtype=np.float32)
    tr = LayerTrace()
    st = lib().hor_sample_xyz(_fp(a), a.shape[0], int(m), C.byref(p), out.ctypes.data_as(C.POINTER(C.c_int32)),
                              _fp(xyz), C.byref(tr))
    if st != OK:
        raise OracleError(st)
    res = (out[: int(m)], xyz[: int(m)])
    if want_trace:
        return res + ([trace_dict(tr)],)
    return res


def s_hi(points, aspect=(1.0, 1.0, 1.0)) -> np.float32:
    a = _pts(points)
    return np.float32(lib().hor_s_hi(_fp(a), a.shape[0], _fp(_aspect(aspect))))


def fps(points, m):
    a = _pts(points)
    out = np.zeros(max(int(m), 1), dtype=np.int32)
    st = lib().hor_fps(_fp(a), a.shape[0], int(m), out.ctypes.data_as(C.POINTER(C.c_int32)))
    if st != OK:
        raise OracleError(st)
    return out[: int(m)]


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle status {status}")
        self.status = status
