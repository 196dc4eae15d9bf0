"""Python binding of libhav.so (include/hav.h): argument marshalling only.

Every step of the sampler runs in the library's CUDA kernels; this module
only passes device pointers, sizes and the current CUDA stream.  PyTorch
supplies device memory and streams.  If the library is missing the calls
raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhav.so")

HAV_OK, HAV_ERR_INVALID, HAV_ERR_NONFINITE, HAV_ERR_TABLE_FULL = 0, 1, 2, 3
HAV_ERR_TIMEOUT, HAV_ERR_NOMEM, HAV_ERR_CUDA, HAV_ERR_RANGE = 4, 5, 6, 7
HAV_MAX_ITERS = 20
MAX_SEGMENTS = 256
MAX_LEVELS = 8


class hav_params(C.Structure):
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


# start of the Section 3.3 search: bisection over (0, s_hi], or guided by the
# cloud's previous search (HAV_SEARCH_GUIDED in hav.h)
SEARCH = {"bisect": 0, "guided": 1}

# voxel representatives (Table 6): the method's centre-closest point, a random
# point, the voxel mean, the voxel centre
SELECT = {"centre-closest": 0, "random": 1, "mean": 2, "centre": 3}


class hav_layer_trace(C.Structure):
    _fields_ = [
        ("m_l", C.c_int64),
        ("k_max", C.c_int64),
        ("k_star", C.c_int64),
        ("n_in", C.c_int64),
        ("iters", C.c_int32),
        ("accepted", C.c_int32),
        ("s_hi", C.c_float),
        ("s_star", C.c_float),
        ("s", C.c_float * HAV_MAX_ITERS),
        ("K", C.c_int64 * HAV_MAX_ITERS),
        ("bounded", C.c_uint32),
        ("reserved", C.c_int32),
    ]


class hav_tuning(C.Structure):
    _fields_ = [
        ("spec_points", C.c_int64 * 3),
        ("chunk_min", C.c_int32),
        ("nblocks", C.c_int32),
        ("small_points", C.c_int32),
        ("solo_points", C.c_int32),
        ("cluster_ctas", C.c_int32),
        ("table_log2", C.c_int32),
        ("pass_shape", C.c_int32),
    ]


class HavError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = _lib_or_none().hav_status_string(status).decode() if _lib_or_none() else str(status)
        super().__init__(f"{where}: {msg} ({status})")


_lock = threading.Lock()
_lib = None

EXPORTS = [
    "hav_params_default", "hav_context_create", "hav_context_destroy", "hav_workspace_bytes",
    "hav_sample", "hav_sample_levels", "hav_sample_batched", "hav_status_get", "hav_trace_get",
    "hav_count", "hav_status_string", "hav_sample_noalloc", "hav_phase_times_get", "hav_fps",
    "hav_context_set_blocks", "hav_context_get_tuning", "hav_context_set_tuning", "hav_sample_xyz",
    "hav_spacing", "hav_spacing_histogram", "hav_ball_query", "hav_context_launches",
]
HAV_FLAG_PHASE_TIMES = 1
HAV_FLAG_TEST_TIMEOUT = 2
HAV_FLAG_TEST_TABLE_FULL = 4


def _lib_or_none():
    return _lib


def load(path: str = LIB_PATH):
    """Load libhav.so and declare its signatures (no device work)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2305_14306_gb300.build.build() first")
        L = C.CDLL(path)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        P = C.POINTER
        L.hav_params_default.argtypes = [P(hav_params)]
        L.hav_params_default.restype = None
        L.hav_context_create.argtypes = [P(vp), i64, i32]
        L.hav_context_create.restype = C.c_int
        L.hav_context_destroy.argtypes = [vp]
        L.hav_context_destroy.restype = None
        L.hav_workspace_bytes.argtypes = [i64, i32]
        L.hav_workspace_bytes.restype = C.c_size_t
        L.hav_sample.argtypes = [vp, vp, i64, i64, P(hav_params), vp, vp]
        L.hav_sample.restype = C.c_int
        L.hav_ball_query.argtypes = [vp, vp, i64, vp, i64, C.c_float, i32, vp, vp, vp]
        L.hav_ball_query.restype = C.c_int
        L.hav_spacing.argtypes = [vp, vp, i64, vp, i64, vp, vp]
        L.hav_spacing.restype = C.c_int
        L.hav_spacing_histogram.argtypes = [vp, vp, i64, vp, i64, P(C.c_float), C.c_int32, vp, vp, vp]
        L.hav_spacing_histogram.restype = C.c_int
        L.hav_sample_xyz.argtypes = [vp, vp, i64, i64, P(hav_params), vp, vp, vp]
        L.hav_sample_xyz.restype = C.c_int
        L.hav_sample_levels.argtypes = [vp, vp, i64, P(C.c_int64), i32, P(hav_params), P(vp), vp]
        L.hav_sample_levels.restype = C.c_int
        L.hav_sample_batched.argtypes = [vp, vp, P(C.c_int64), P(C.c_int64), i32, i32, P(hav_params),
                                         P(vp), vp]
        L.hav_sample_batched.restype = C.c_int
        L.hav_status_get.argtypes = [vp, vp, P(C.c_int32)]
        L.hav_status_get.restype = C.c_int
        L.hav_trace_get.argtypes = [vp, vp, P(hav_layer_trace), i32]
        L.hav_trace_get.restype = C.c_int32
        L.hav_count.argtypes = [vp, vp, i64, C.c_float, P(C.c_float), P(C.c_int64), vp]
        L.hav_count.restype = C.c_int
        L.hav_status_string.argtypes = [C.c_int]
        L.hav_status_string.restype = C.c_char_p
        L.hav_context_set_blocks.argtypes = [vp, i32]
        L.hav_context_set_blocks.restype = C.c_int
        L.hav_context_get_tuning.argtypes = [vp, P(hav_tuning)]
        L.hav_context_get_tuning.restype = C.c_int
        L.hav_context_set_tuning.argtypes = [vp, P(hav_tuning)]
        L.hav_context_set_tuning.restype = C.c_int
        L.hav_context_launches.argtypes = [vp, P(C.c_uint64)]
        L.hav_context_launches.restype = C.c_int
        L.hav_fps.argtypes = [vp, vp, i64, i64, vp, vp]
        L.hav_fps.restype = C.c_int
        L.hav_phase_times_get.argtypes = [vp, vp, P(C.c_uint64), P(C.c_uint32), i32]
        L.hav_phase_times_get.restype = C.c_int32
        L.hav_sample_noalloc.argtypes = [vp, i64, i64, P(hav_params), vp, vp, vp]
        L.hav_sample_noalloc.restype = C.c_int
        _lib = L
        return L


def params(sigma=(5, 100), t_max=20, layers=2, layer_ratio=4, aspect=(1.0, 1.0, 1.0),
           flags=0, select="centre-closest", seed=0, fixed_s=0.0, search="bisect") -> hav_params:
    p = hav_params()
    load().hav_params_default(C.byref(p))
    p.sigma_num, p.sigma_den = sigma
    p.t_max, p.layers, p.layer_ratio = t_max, layers, layer_ratio
    for a in range(3):
        p.aspect[a] = aspect[a]
    p.flags = flags
    p.select = SELECT[select] if isinstance(select, str) else int(select)
    p.seed = int(seed)
    p.fixed_s = float(fixed_s)
    p.search = SEARCH[search] if isinstance(search, str) else int(search)
    return p


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check(st, where):
    if st != HAV_OK:
        raise HavError(st, where)


def _points(points):
    import torch
    if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dtype == torch.float32
            and points.dim() == 2 and points.shape[1] == 3 and points.is_contiguous()):
        raise ValueError("points must be a contiguous (n, 3) float32 CUDA tensor")
    return points


def _out(t, numel: int, dtype, like, name: str, shape=None):
    """A caller-provided output tensor, checked before the device writes into
    it (the library cannot see its size), or a new one of `shape`."""
    import torch
    if t is None:
        return torch.empty(shape if shape is not None else (int(numel),), dtype=dtype, device=like.device)
    if not (isinstance(t, torch.Tensor) and t.device == like.device and t.dtype == dtype and t.is_contiguous()
            and t.numel() >= int(numel)):
        raise ValueError(f"{name} must be a contiguous {dtype} tensor on {like.device} with at least "
                         f"{int(numel)} elements")
    return t


class Context:
    """A libhav context: device workspace for calls of up to max_points points
    in total and max_segments segments."""

    def __init__(self, max_points: int, max_segments: int = 1):
        L = load()
        h = C.c_void_p()
        _check(L.hav_context_create(C.byref(h), int(max_points), int(max_segments)), "hav_context_create")
        self.handle = h
        self.max_points = int(max_points)
        self.max_segments = int(max_segments)

    def set_blocks(self, nblocks: int):
        """Limit the sampler launches of this context to nblocks SMs (0: all)."""
        _check(load().hav_context_set_blocks(self.handle, int(nblocks)), "hav_context_set_blocks")

    def get_tuning(self) -> dict:
        """The context's launch-shape knobs (no knob changes a result)."""
        t = hav_tuning()
        _check(load().hav_context_get_tuning(self.handle, C.byref(t)), "hav_context_get_tuning")
        return {"spec_points": list(t.spec_points), "chunk_min": t.chunk_min, "nblocks": t.nblocks,
                "small_points": t.small_points, "solo_points": t.solo_points, "cluster_ctas": t.cluster_ctas,
                "table_log2": t.table_log2, "pass_shape": t.pass_shape}

    def set_tuning(self, spec_points=None, chunk_min=None, nblocks=None, small_points=None, solo_points=None,
                   cluster_ctas=None, table_log2=None, pass_shape=None):
        """Change some of the knobs; the others keep their values."""
        cur = self.get_tuning()
        t = hav_tuning()
        sp = cur["spec_points"] if spec_points is None else list(spec_points)
        for k in range(3):
            t.spec_points[k] = int(sp[k])
        t.chunk_min = int(cur["chunk_min"] if chunk_min is None else chunk_min)
        t.nblocks = int(cur["nblocks"] if nblocks is None else nblocks)
        t.small_points = int(cur["small_points"] if small_points is None else small_points)
        t.solo_points = int(cur["solo_points"] if solo_points is None else solo_points)
        t.cluster_ctas = int(cur["cluster_ctas"] if cluster_ctas is None else cluster_ctas)
        t.table_log2 = int(cur["table_log2"] if table_log2 is None else table_log2)
        t.pass_shape = int(cur["pass_shape"] if pass_shape is None else pass_shape)
        _check(load().hav_context_set_tuning(self.handle, C.byref(t)), "hav_context_set_tuning")

    def launches(self) -> int:
        """Device kernels this context's calls have enqueued since creation."""
        n = C.c_uint64()
        _check(load().hav_context_launches(self.handle, C.byref(n)), "hav_context_launches")
        return int(n.value)

    def close(self):
        if self.handle:
            load().hav_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hav_sample(ctx: Context, points, m: int, p: hav_params | None = None, out=None, stream=None):
    """One cloud, one level: returns (or fills) an int32 CUDA tensor of m ascending indices."""
    import torch
    points = _points(points)
    p = p or params()
    out = _out(out, max(0, int(m)), torch.int32, points, "out")
    st = load().hav_sample(ctx.handle, C.c_void_p(points.data_ptr()), points.shape[0], int(m), C.byref(p),
                           C.c_void_p(out.data_ptr()), _stream_handle(stream))
    _check(st, "hav_sample")
    return out


def hav_sample_xyz(ctx: Context, points, m: int, p: hav_params | None = None, out=None, xyz=None, stream=None):
    """One cloud, one layer: (m ascending int32 indices, (m, 3) float32 coordinates
    standing for them: the point, the voxel centre or the voxel mean, by p.select)."""
    import torch
    points = _points(points)
    p = p or params(layers=1)
    out = _out(out, max(0, int(m)), torch.int32, points, "out")
    xyz = _out(xyz, 3 * max(0, int(m)), torch.float32, points, "xyz", shape=(max(0, int(m)), 3))
    st = load().hav_sample_xyz(ctx.handle, C.c_void_p(points.data_ptr()), points.shape[0], int(m), C.byref(p),
                               C.c_void_p(out.data_ptr()), C.c_void_p(xyz.data_ptr()), _stream_handle(stream))
    _check(st, "hav_sample_xyz")
    return out, xyz


def hav_sample_levels(ctx: Context, points, m_levels, p: hav_params | None = None, outs=None, stream=None):
    """Level chain on one cloud: returns one int32 tensor per level (indices into the original cloud)."""
    import torch
    points = _points(points)
    p = p or params()
    ml = np.ascontiguousarray(m_levels, dtype=np.int64)
    if outs is None:
        outs = [None] * len(ml)
    if len(outs) != len(ml):
        raise ValueError("outs must hold one tensor per level")
    outs = [_out(o, max(0, int(m)), torch.int32, points, f"outs[{j}]") for j, (o, m) in enumerate(zip(outs, ml))]
    ptrs = (C.c_void_p * len(ml))(*[o.data_ptr() for o in outs])
    st = load().hav_sample_levels(ctx.handle, C.c_void_p(points.data_ptr()), points.shape[0],
                                  ml.ctypes.data_as(C.POINTER(C.c_int64)), len(ml), C.byref(p), ptrs,
                                  _stream_handle(stream))
    _check(st, "hav_sample_levels")
    return outs


def hav_sample_batched(ctx: Context, points, seg_offsets, seg_m, p: hav_params | None = None, outs=None,
                       stream=None):
    """Segmented batch: seg_offsets (S+1,), seg_m (L, S) host arrays.  Returns one int32
    tensor per level holding each segment's segment-local indices back to back."""
    import torch
    points = _points(points)
    p = p or params()
    offs = np.ascontiguousarray(seg_offsets, dtype=np.int64)
    m = np.ascontiguousarray(np.atleast_2d(seg_m), dtype=np.int64)
    S, L = len(offs) - 1, m.shape[0]
    if m.shape[1] != S:
        raise ValueError("seg_m must be (levels, segments)")
    if outs is None:
        outs = [None] * L
    if len(outs) != L:
        raise ValueError("outs must hold one tensor per level")
    outs = [_out(outs[j], max(0, int(m[j].sum())), torch.int32, points, f"outs[{j}]") for j in range(L)]
    ptrs = (C.c_void_p * L)(*[o.data_ptr() for o in outs])
    st = load().hav_sample_batched(ctx.handle, C.c_void_p(points.data_ptr()),
                                   offs.ctypes.data_as(C.POINTER(C.c_int64)),
                                   m.ctypes.data_as(C.POINTER(C.c_int64)), S, L, C.byref(p), ptrs,
                                   _stream_handle(stream))
    _check(st, "hav_sample_batched")
    return outs


def hav_status_get(ctx: Context, num_segments: int = 1, stream=None):
    """Synchronise and return (status, per-segment statuses) of the last call."""
    # the library writes one entry per segment of the last call (at most the
    # context's segment limit)
    per = (C.c_int32 * max(1, int(num_segments), ctx.max_segments))()
    st = load().hav_status_get(ctx.handle, _stream_handle(stream), per)
    return int(st), [int(x) for x in per[:num_segments]]


def hav_trace_get(ctx: Context, num_records: int, stream=None):
    """Per-layer traces of the last call, [level][segment][layer] flattened, as dicts."""
    buf = (hav_layer_trace * max(1, num_records))()
    w = load().hav_trace_get(ctx.handle, _stream_handle(stream), buf, num_records)
    if w < 0:
        raise HavError(HAV_ERR_CUDA, "hav_trace_get")
    out = []
    for r in buf[:w]:
        it = r.iters
        out.append({
            "m_l": r.m_l, "k_max": r.k_max, "k_star": r.k_star, "n_in": r.n_in, "iters": it,
            "accepted": bool(r.accepted), "s_hi": np.float32(r.s_hi), "s_star": np.float32(r.s_star),
            "s": np.array(r.s[:it], dtype=np.float32), "K": np.array(r.K[:it], dtype=np.int64),
            "bounded": int(r.bounded),
        })
    return out


def hav_phase_times_get(ctx: Context, max_records: int = 4096, stream=None):
    """Phase timer of the last call made with flags=HAV_FLAG_PHASE_TIMES: list of (ns, tag)."""
    t = (C.c_uint64 * max_records)()
    g = (C.c_uint32 * max_records)()
    w = load().hav_phase_times_get(ctx.handle, _stream_handle(stream), t, g, max_records)
    if w < 0:
        raise HavError(HAV_ERR_CUDA, "hav_phase_times_get")
    return [(int(t[k]), int(g[k])) for k in range(w)]


def hav_fps(ctx: Context, points, m: int, out=None, stream=None):
    """Farthest point sampling (the paper's comparator): m int32 indices in selection order."""
    import torch
    points = _points(points)
    out = _out(out, max(0, int(m)), torch.int32, points, "out")
    st = load().hav_fps(ctx.handle, C.c_void_p(points.data_ptr()), points.shape[0], int(m),
                        C.c_void_p(out.data_ptr()), _stream_handle(stream))
    _check(st, "hav_fps")
    return out


def hav_spacing(ctx: Context, points, idx, out=None, stream=None):
    """Squared distance from each subset point to its nearest other subset point (Fig. 3)."""
    import torch
    points = _points(points)
    if idx.dim() != 1:
        raise ValueError("idx must be one-dimensional")
    idx = idx.to(dtype=torch.int32, device=points.device).contiguous()
    m = idx.shape[0]
    out = _out(out, m, torch.float32, points, "out")
    st = load().hav_spacing(ctx.handle, C.c_void_p(points.data_ptr()), points.shape[0],
                            C.c_void_p(idx.data_ptr()), m, C.c_void_p(out.data_ptr()), _stream_handle(stream))
    _check(st, "hav_spacing")
    return out


SPACING_MAX_BINS = 1024


def hav_spacing_histogram(ctx: Context, points, idx, edges_d2, out=None, counts=None, stream=None):
    """hav_spacing and the histogram of the spacings over the given bin edges
    (squared distances, binary32, ascending): returns (d2, counts) with counts
    an int64 CUDA tensor of len(edges_d2) + 1 entries: below the first edge,
    the bins (numpy.histogram's), above the last edge."""
    import torch
    points = _points(points)
    if idx.dim() != 1:
        raise ValueError("idx must be one-dimensional")
    idx = idx.to(dtype=torch.int32, device=points.device).contiguous()
    e = np.ascontiguousarray(edges_d2, dtype=np.float32)
    if e.ndim != 1 or not (2 <= e.shape[0] <= SPACING_MAX_BINS + 1):
        raise ValueError("edges_d2 must hold 2 .. 1025 edges")
    nb = e.shape[0] - 1
    m = idx.shape[0]
    out = _out(out, m, torch.float32, points, "out")
    counts = _out(counts, nb + 2, torch.int64, points, "counts")
    st = load().hav_spacing_histogram(ctx.handle, C.c_void_p(points.data_ptr()), points.shape[0],
                                      C.c_void_p(idx.data_ptr()), m,
                                      e.ctypes.data_as(C.POINTER(C.c_float)), nb, C.c_void_p(out.data_ptr()),
                                      C.c_void_p(counts.data_ptr()), _stream_handle(stream))
    _check(st, "hav_spacing_histogram")
    return out, counts


def hav_ball_query(ctx: Context, points, centres, radius: float, nsample: int, out=None, xyz=True, stream=None):
    """Grouping around centres (indices into points): (m, nsample) int32 indices and,
    if xyz, (m, nsample, 3) float32 offsets p_k - c_j (else None)."""
    import torch
    points = _points(points)
    if centres.dim() != 1:
        raise ValueError("centres must be one-dimensional")
    centres = centres.to(dtype=torch.int32, device=points.device).contiguous()
    m = centres.shape[0]
    out = _out(out, m * max(0, int(nsample)), torch.int32, points, "out", shape=(m, int(nsample)))
    offs = torch.empty((m, int(nsample), 3), dtype=torch.float32, device=points.device) if xyz else None
    st = load().hav_ball_query(ctx.handle, C.c_void_p(points.data_ptr()), points.shape[0],
                               C.c_void_p(centres.data_ptr()), m, float(np.float32(radius)), int(nsample),
                               C.c_void_p(out.data_ptr()), C.c_void_p(offs.data_ptr() if xyz else None),
                               _stream_handle(stream))
    _check(st, "hav_ball_query")
    return out, offs


def coverage(points, idx, chunk: int = 8192) -> float:
    """Subset coverage: the largest distance from any input point to its nearest
    selected point (a measurement for the comparison, computed with torch)."""
    import torch
    pts = points.double()
    sel = pts[idx.long()]
    worst = torch.zeros((), dtype=torch.float64, device=pts.device)
    for a in range(0, pts.shape[0], chunk):
        d = torch.cdist(pts[a:a + chunk], sel)
        worst = torch.maximum(worst, d.min(dim=1).values.max())
    return float(worst.item())


def hav_count(ctx: Context, points, s: float, aspect=(1.0, 1.0, 1.0), stream=None) -> int:
    """Cnt(P, v) at v = s * aspect (synchronous test hook)."""
    points = _points(points)
    asp = (C.c_float * 3)(*[float(a) for a in aspect])
    K = C.c_int64(0)
    st = load().hav_count(ctx.handle, C.c_void_p(points.data_ptr()), points.shape[0],
                          float(np.float32(s)), asp, C.byref(K), _stream_handle(stream))
    _check(st, "hav_count")
    return int(K.value)


NOALLOC_MAX_POINTS = 32768


def hav_sample_noalloc(points, m: int, p: hav_params | None = None, out=None, status_out=None, stream=None):
    """hav_sample for callers that cannot allocate device memory: no context,
    scratch in the library's static device array (clouds of up to 32,768
    points).  `out` and `status_out` (an int32 CUDA tensor of one element, or
    None) are caller-provided; calls on one device must not overlap."""
    import torch
    points = _points(points)
    p = p or params()
    out = _out(out, max(0, int(m)), torch.int32, points, "out")
    if status_out is not None:
        status_out = _out(status_out, 1, torch.int32, points, "status_out")
    sp = C.c_void_p(status_out.data_ptr()) if status_out is not None else C.c_void_p()
    st = load().hav_sample_noalloc(C.c_void_p(points.data_ptr()), points.shape[0], int(m), C.byref(p),
                                   C.c_void_p(out.data_ptr()), sp, _stream_handle(stream))
    _check(st, "hav_sample_noalloc")
    return out


def workspace_bytes(max_points: int, max_segments: int = 1) -> int:
    return int(load().hav_workspace_bytes(int(max_points), int(max_segments)))
