// HAVSampler hot path for sm_103a: one persistent cooperative kernel runs a
// batched level chain, every level of it or the large levels up to the first
// one the small-level kernels take (hav_small.cu).
//
// Per level j, for every segment (cloud) of the batch at once:
//   bbox    per-axis min/max and finiteness (the bracket of the Section 3.3
//           search); the level's points are laid out as float4 (x, y, z, g)
//           with g the point's level index
//   bucket  (one large cloud, first level) a counting sort by a 16^3 Morton
//           cell of the bounding box, so that each block's share of the points
//           is a compact region; later levels inherit the order
//   layer l = 1..k (Section 3.4, Eq. 3):
//     pass p   Cnt(P_l, s_p): Eq. 2 voxel keys are first deduplicated in a
//              block-local shared-memory set, and only keys new to the block
//              probe the global open-addressed table (atomicCAS); every fresh
//              global insert is logged so the table can be cleaned slot by slot;
//              the bisection of Section 3.3 is decided identically by every
//              block from the pass counts (no leader, no host round trip)
//     select   centre-closest representative per voxel at s*: a block-local
//              shared-memory argmin of packed (d^2 bits, index), then one global
//              64-bit atomicMin per block-distinct voxel (Section 3.2); the
//              first touch of a slot feeds the cut-off histogram
//     cut      voxels below the boundary priority bin are taken, the boundary
//              bin's voxels are ranked exactly, or the shortfall is filled
//   compact taken bitmask -> ascending indices composed to the segment's
//           original cloud; the kept points are also gathered, in the current
//           processing order, as the next level's input
// Phases are separated by a grid barrier whose wait is bounded in time; a
// timeout sets an abort flag every block honours and the host reads
// HAV_ERR_TIMEOUT.  Every loop has a fixed bound.  Control flow depends only
// on values that no block can change while others read them, so every block
// executes the same sequence of barriers.
//
// Arithmetic: voxel keys and distances use explicitly rounded binary32
// intrinsics (__fdiv_rn, __fmul_rn, __fadd_rn, __fsub_rn), so the compiler
// cannot contract or reassociate them.

#include <cuda_runtime.h>

#include "hav_device.cuh"
#include "hav_internal.h"

namespace havk {
namespace {

#define TAG(phase, level, layer, pass)                                            \
    ((static_cast<unsigned>(phase) << 24) | (static_cast<unsigned>(level) << 16) | \
     (static_cast<unsigned>(layer) << 8) | static_cast<unsigned>(pass))

static_assert(kHistBins % kThreads == 0, "the cut-off scan gives each thread whole bins");
constexpr int kSetSlots = 16384;   // block-local dedupe set of a bisection pass (128 KB + 32 KB list)
constexpr size_t kPassSmem = static_cast<size_t>(kSetSlots) * 10;
constexpr int kSelSlots = 8192;    // block-local argmin table of the selection (128 KB + 16 KB list)
constexpr size_t kSelSmem = static_cast<size_t>(kSelSlots) * 20;  // + the list of keys that go global
constexpr size_t kDynSmem = kPassSmem > kSelSmem ? kPassSmem : kSelSmem;
constexpr int kBucketMin = 1 << 17;
// Loads and probes in flight per thread (the kernel's template arguments,
// one instantiation per pass shape): with 64 registers a thread (one
// 1024-thread block per SM), deeper batches spill more than they hide
// (measured on GB300: 4 and 2 made the 1M-point chain 5 % slower than the
// default 2 and 1).
template <int IF, int PR>
struct PassShape {
    static constexpr int kInFlight = IF;  // points loaded ahead per thread
    static constexpr int kProbes = PR;    // global first probes issued together per thread
    static_assert(kSetSlots % (PR * kThreads) == 0 && kSelSlots % (PR * kThreads) == 0,
                  "flush loops take kProbes slots per thread per step");
};

enum : int { F_ACTIVE = 1, F_SEARCH = 2, F_ACCEPT = 4, F_UP = 8, F_PRE = 16 };

struct Smem {
    // level layout
    long long off[kMaxSegments + 1];
    long long tab_off[kMaxSegments];
    long long cand_off[kMaxSegments];
    int n[kMaxSegments];
    int m[kMaxSegments];
    int cap_log2[kMaxSegments];
    int item0[kMaxSegments + 1];
    int err[kMaxSegments];
    // bracket
    float mn[kMaxSegments][3];
    float mx[kMaxSegments][3];
    float s_hi[kMaxSegments];
    // controller of the current layer
    float lo[kMaxSegments], hi[kMaxSegments], s_star[kMaxSegments];
    // guided search: the pending first size of the current search, and the
    // segment's previous search in this call (its s*, its budget; 0: none)
    float first[kMaxSegments];
    float gs[kMaxSegments];
    int gm[kMaxSegments];
    Grid grid[kMaxSegments];
    int iters[kMaxSegments];
    int sel_cand[kMaxSegments];
    int ml[kMaxSegments];
    int kmax[kMaxSegments];
    int flags[kMaxSegments];
    int sel[kMaxSegments];
    int kstar[kMaxSegments];
    int cprefix[kMaxSegments + 1];
    // per-block logs of fresh global inserts, one per (table set, owned item, candidate)
    int dcnt[kTableSets][kLocalItems][kMaxCand];
    // candidate grids of a speculative pass, per owned item
    Grid cgrid[kLocalItems][kMaxCand];
    int cvalid[kLocalItems][kMaxCand];
    unsigned rbits;
    int ncand;
    int setc_log2;
    long long tab_stride;
    // scratch
    long long scan_ll[32];
    int scan_i[32];
    unsigned scan_u[32];
    float redf[6][32];
    unsigned epoch;
    unsigned list_n;
    int set_clean;  // 1 when every slot of the block set is empty
    // a bucketed segment (level 0, and for one cloud the levels that keep its
    // order): per work item of the block, the Morton cells [own_lo, own_hi]
    // of the level-0 bucketing (its box own_mn, own_k[a] = 16 / extent) whose
    // points all lie in the item (own_on); per pass the keys that go to the
    // global table (rest_n) and the owned ones counted here.  b0_*: one
    // bucketed cloud's level-0 box, kept for its later levels.
    int own_on[kLocalItems], own_lo[kLocalItems], own_hi[kLocalItems], bucketed;
    float own_k[kLocalItems][3], own_mn[kLocalItems][3];
    float b0_mn[3], b0_mx[3], b0_k[3];
    unsigned rest_n;
    unsigned xcnt[kMaxCand];
    int ocnt[kLocalItems];  // owned voxels the selection listed for the classification, per item
    unsigned gl_n;          // keys of the selection that go to the global table
    unsigned bh[kHistBins]; // this block's cut-off histogram of a selection (added to the global one once)
    int ntimes;
    int was_clean;
    int cut_seg;
    int cut_bin;
    int cut_below;
    int flag;
    int any;
    int items_total;
    int chunk;
    // counting barrier of single-cloud passes
    unsigned fused_uses[2];
    unsigned long long fused_last[2];
    unsigned long long fused_delta;
    unsigned long long pass_cnt;
    int pass_err;
    long long n_level;
    long long m_total;
};

struct Dev {
    Barrier* bar;
    GlobalHdr* gh;
    SegHdr* sh;
    unsigned* clean;
    LayerState* ls;        // [2][S]
    uint32_t* hist;        // [2][S][kHistBins]
    int32_t* psf;          // [S][kMaxBlocks]
    int32_t* pcmp;         // [kMaxBlocks]
    int32_t* pitem;        // [kMaxItems]
    hav_layer_trace* tr;   // [L][S][kMaxLayers]
    float4* ord[2];        // level input in processing order: x, y, z, level index
    int32_t* orig[2];      // original (segment-local) index by level index
    int32_t* posof;        // staged position by level index (current level)
    uint32_t* taken[2];    // by level index
    uint32_t* wpre;        // block-local prefix of taken bits per mask word
    uint32_t* dirty[kTableSets];  // fresh-insert logs, item-owned ranges of the level index space
    uint32_t* bkt;         // [2][4096] bucket counts, bucket cursors
    int32_t* prefix;       // [S][kMaxIters] counts at s_hi / 2^(k+1) of this level (-1: none)
    unsigned long long* tk[kTableSets];
    unsigned long long* tv;
    Cand* cand;
    unsigned long long* ptimes;
    int ptimes_cap;
};

// Barrier plus, when phase timing is on, a (time, tag) record from block 0.
// A pass of one cloud with one candidate: the pass count travels with the
// barrier (fused_sync_impl).  A block that met an out-of-range key adds
// kFusedErr, which no count reaches (counts stay below 2^31); it happens at
// most once per call, as the search of the cloud stops there, so the low
// field stays below 2^48 (at most 640 passes per word, each below 2^31).
constexpr unsigned long long kFusedErr = 1ull << 36;

__device__ __forceinline__ void phase_record(Dev& d, Smem& st, unsigned tag) {
    if (d.ptimes && blockIdx.x == 0 && threadIdx.x == 0 && st.ntimes < d.ptimes_cap) {
        d.ptimes[2 * st.ntimes] = globaltimer();
        d.ptimes[2 * st.ntimes + 1] = tag;
        st.ntimes += 1;
    }
}

__device__ __forceinline__ void fused_arrive(Dev& d, Smem& st, int par, unsigned long long add) {
    fused_arrive_impl(&d.bar->fused[par], &st.fused_uses[par], add);
}

__device__ __forceinline__ bool fused_wait(Dev& d, unsigned nblocks, Smem& st, int par, unsigned tag) {
    const bool ok = fused_wait_impl(&d.bar->fused[par], d.gh, nblocks, &st.fused_uses[par], &st.fused_last[par],
                                    &st.fused_delta, &st.flag);
    phase_record(d, st, tag);
    return ok;
}

__device__ __forceinline__ void grid_arrive(Dev& d, Smem& st) { grid_arrive_impl(d.bar, &st.epoch); }

__device__ __forceinline__ bool grid_wait(Dev& d, unsigned nblocks, Smem& st, unsigned tag) {
    const bool ok = grid_wait_impl(d.bar, d.gh, nblocks, &st.epoch, &st.flag);
    phase_record(d, st, tag);
    return ok;
}

__device__ __forceinline__ bool grid_sync(Dev& d, unsigned nblocks, Smem& st, unsigned tag) {
    const bool ok = grid_sync_impl(d.bar, d.gh, nblocks, &st.epoch, &st.flag);
    phase_record(d, st, tag);
    return ok;
}

__device__ __forceinline__ void seg_error(Dev& d, int s, int code) {
    atomicCAS(&d.sh[s].status, 0, code);
    atomicCAS(&d.gh->status, 0, code);
}

// largest s with prefix[s] <= t (prefix has S+1 entries, prefix[0] = 0)
template <typename T>
__device__ __forceinline__ int find_seg(const T* prefix, int S, long long t) {
    int lo = 0, hi = S;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool is_taken(const uint32_t* tk, int g) {
    return (tk[g >> 5] >> (g & 31)) & 1u;
}
__device__ __forceinline__ void set_taken(uint32_t* tk, int g) {
    atomicOr(&tk[g >> 5], 1u << (g & 31));
}
// A taken point also carries -(g + 2) in its staged entry, so that later
// layers skip it without reading the mask.
__device__ __forceinline__ void mark_taken(uint32_t* tk, float4* ord, const int32_t* posof, int g) {
    set_taken(tk, g);
    reinterpret_cast<int*>(ord + posof[g])[3] = -(g + 2);
}
__device__ __forceinline__ int level_index(float w) {
    const int x = __float_as_int(w);
    return x >= 0 ? x : -x - 2;
}

template <typename T>
__device__ __forceinline__ void fill(T* p, long long count, T v, long long gtid, long long gstride) {
    for (long long i = gtid; i < count; i += gstride) p[i] = v;
}

__device__ __forceinline__ void clear_layer_state(Dev& d, int S, int q, long long gtid, long long gstride) {
    fill<uint32_t>(reinterpret_cast<uint32_t*>(d.ls + q * S), static_cast<long long>(S) * (sizeof(LayerState) / 4),
                   0u, gtid, gstride);
    fill<uint32_t>(d.hist + static_cast<long long>(q) * S * kHistBins, static_cast<long long>(S) * kHistBins, 0u,
                   gtid, gstride);
}

// Item `it` of the level: segment and point range [a, b).
// (A level holds fewer than 2^30 points, so point indices fit 32 bits.)
__device__ __forceinline__ int item_range(const Smem& st, int S, int it, int* a, int* b) {
    const int s = find_seg(st.item0, S, it);
    const int k = it - st.item0[s];
    *a = static_cast<int>(st.off[s]) + k * st.chunk;
    const int e = *a + st.chunk;
    const int end = static_cast<int>(st.off[s]) + st.n[s];
    *b = e < end ? e : end;
    return s;
}

// 16^3 Morton cell of a point inside its segment's bounding box (layout only).
// The cell index along an axis is a non-decreasing function of the
// coordinate (every rounded step is monotone), which the ownership test of
// the bisection passes relies on.
__device__ __forceinline__ unsigned bucket_axis(float x, float mn, float mx) {
    const float e = __fsub_rn(mx, mn);
    if (!(e > 0.0f)) return 0u;
    float q = __fmul_rn(__fdiv_rn(__fsub_rn(x, mn), e), 16.0f);
    q = fminf(fmaxf(q, -1.0f), 16.0f);  // (NaN-free: x, mn, mx finite)
    const int c = static_cast<int>(q);
    return static_cast<unsigned>(c < 0 ? 0 : (c > 15 ? 15 : c));
}
__device__ __forceinline__ unsigned morton16(unsigned cx, unsigned cy, unsigned cz) {
    unsigned id = 0;
#pragma unroll
    for (int bit = 0; bit < 4; ++bit)
        id |= (((cx >> bit) & 1u) << (3 * bit)) | (((cy >> bit) & 1u) << (3 * bit + 1)) |
              (((cz >> bit) & 1u) << (3 * bit + 2));
    return id;
}
__device__ __forceinline__ unsigned bucket_of(const float p[3], const float mn[3], const float mx[3]) {
    return morton16(bucket_axis(p[0], mn[0], mx[0]), bucket_axis(p[1], mn[1], mx[1]), bucket_axis(p[2], mn[2], mx[2]));
}

// Whether every point of the voxel `key` (Eq. 2 cell of grid g) lies in Morton
// cells [own_lo, own_hi] of its segment's bucketing, all of whose points one
// work item of this block processes: then no other item has a point in the
// voxel, and the item counts it without the global table.  The test may answer no for an owned
// voxel (the key then goes to the global table), never yes for another one.
// A point x of the voxel along an axis has f <= RN(x / v) < f + 1, so
// v (f - ulp(f) / 2) <= x < v (f + 1); the box [v f, v (f + 1)] is widened by
// 2^-20 (|end| + v) on both sides, which covers that half ulp and the
// rounding of the products.  Along each axis the box's ends are mapped to
// cell coordinates by t = (end - mn) * (16 / e): within the box [0, 16] of the
// points this differs from bucket_axis's rounded (x - mn) / e * 16 by less
// than 1e-5, so widening the ends by 0.01 cells yields every cell a point of
// the voxel can fall in (outside [0, 16] the clamp to the end cells decides).
// Morton order is monotone in each cell coordinate, so those cells lie
// between the codes of the two corner cells.  k[a] = RN(16 / e_a), 0 if e_a = 0.
__device__ __forceinline__ bool voxel_owned(unsigned long long key, const Grid& g, const float mn[3],
                                            const float k[3], int own_lo, int own_hi) {
    unsigned c0[3], c1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float f = __fadd_rn(static_cast<float>(static_cast<unsigned>((key >> (21 * a)) & 0x1fffffull)), g.fmin[a]);
        const float v = g.v[a];
        float lo = __fmul_rn(v, f);
        float hi = __fmul_rn(v, __fadd_rn(f, 1.0f));
        lo = __fsub_rn(lo, __fmul_rn(__fadd_rn(fabsf(lo), v), 9.5367431640625e-07f));
        hi = __fadd_rn(hi, __fmul_rn(__fadd_rn(fabsf(hi), v), 9.5367431640625e-07f));
        float tl = __fsub_rn(__fmul_rn(__fsub_rn(lo, mn[a]), k[a]), 0.01f);
        float th = __fadd_rn(__fmul_rn(__fsub_rn(hi, mn[a]), k[a]), 0.01f);
        tl = fminf(fmaxf(tl, 0.0f), 15.0f);  // NaN-free: finite inputs
        th = fminf(fmaxf(th, 0.0f), 15.0f);
        c0[a] = static_cast<unsigned>(tl);
        c1[a] = static_cast<unsigned>(th);
    }
    return static_cast<int>(morton16(c0[0], c0[1], c0[2])) >= own_lo &&
           static_cast<int>(morton16(c1[0], c1[1], c1[2])) <= own_hi;
}

// The Morton cells a work item [ia, ib) of a bucketed segment holds whole,
// from the bucket bases hb (position of each cell's first point; the
// segment's points end at `end`): from the first cell starting at or after
// ia to the last one ending at or before ib.  Stored as item li's owned
// range with the bucketing's box mn and k = RN(16 / extent).
__device__ void own_cells(const uint32_t* hb, int ia, int ib, unsigned end, const float mn[3], const float k[3],
                          Smem& st, int li) {
    int lo = 0, hi = 4096;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (hb[mid] >= static_cast<unsigned>(ia)) hi = mid; else lo = mid + 1;
    }
    const int c_lo = lo;
    lo = 0;
    hi = 4096;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const unsigned e = (mid + 1 < 4096) ? hb[mid + 1] : end;
        if (e > static_cast<unsigned>(ib)) hi = mid; else lo = mid + 1;
    }
    st.own_lo[li] = c_lo;
    st.own_hi[li] = lo - 1;
    st.own_on[li] = (c_lo <= lo - 1) ? 1 : 0;
    for (int a3 = 0; a3 < 3; ++a3) {
        st.own_mn[li][a3] = mn[a3];
        st.own_k[li][a3] = k[a3];
    }
}

// Level layout of every segment, computed identically by every block.
__device__ void level_setup(const Plan& P, int j, Smem& st) {
    const int S = P.S;
    const int s = threadIdx.x;
    long long n = 0, C = 0, mm = 0;
    int lg = kMinCapLog2;
    if (s < S) {
        n = (j == 0) ? (P.off0[s + 1] - P.off0[s]) : P.m[j - 1][s];
        mm = P.m[j][s];
        // (test hook: segment 0's tables keep the smallest capacity)
        // (the load factor: capacity nextpow2(2^f n), f = table_log2, at least 1)
        const int tl = P.table_log2 > 0 ? P.table_log2 : 1;
        if (!(P.test_table_full && s == 0))
            while ((1ll << lg) < (n << tl)) ++lg;
        C = 1ll << lg;
        st.n[s] = static_cast<int>(n);
        st.m[s] = static_cast<int>(mm);
        st.cap_log2[s] = lg;
    }
    long long tot;
    long long o = block_excl_scan<long long>(n, &tot, st.scan_ll);
    if (s < S) st.off[s] = o;
    if (s == 0) {
        st.off[S] = tot;
        st.n_level = tot;
    }
    __syncthreads();
    const long long nl = st.n_level;
    o = block_excl_scan<long long>(mm, &tot, st.scan_ll);
    if (s == 0) st.m_total = tot;
    o = block_excl_scan<long long>(C, &tot, st.scan_ll);
    if (s < S) {
        st.tab_off[s] = o;
        st.cand_off[s] = o / 2;
    }
    for (int k = s; k < kTableSets * kLocalItems * kMaxCand; k += kThreads) (&st.dcnt[0][0][0])[k] = 0;
    __syncthreads();
    const long long stride = st.tab_off[S - 1] + (1ll << st.cap_log2[S - 1]);
    // speculation depth: deeper on small levels, where a pass is latency-bound;
    // a shallower one wherever the candidate tables, their logs or the work
    // items a block tracks would not fit
    int depth = nl <= P.spec_n[0] ? 4 : nl <= P.spec_n[1] ? 3 : nl <= P.spec_n[2] ? 2 : 1;
    while (depth > 1 && (((1ll << depth) - 1) * stride > P.lay.tab_slots ||
                         ((1ll << depth) - 1) * nl > P.lay.dirty_slots))
        --depth;
    for (;; --depth) {
        long long chunk = (nl + P.nblocks - 1) / P.nblocks;  // every block gets a share
        if (chunk < P.chunk_min) chunk = P.chunk_min;
        const int ncand = (1 << depth) - 1;
        int lg2 = 0;
        while ((1 << (lg2 + 1)) * ncand <= kSetSlots) ++lg2;
        // a candidate's share of the block set must stay at most half full
        const long long half = (1ll << lg2) / 2;
        if (depth > 1 && chunk > half) chunk = half;
        long long items = (s < S) ? (n + chunk - 1) / chunk : 0;
        if (depth == 1 && chunk > half) {
            // several smaller items per block, evenly spread, where they fit
            const long long k = (chunk + half - 1) / half;
            long long c2 = (nl + k * P.nblocks - 1) / (k * P.nblocks);
            if (c2 < P.chunk_min) c2 = P.chunk_min;
            const long long items2 = (s < S) ? (n + c2 - 1) / c2 : 0;
            block_excl_scan<long long>(items2, &tot, st.scan_ll);
            if (tot <= static_cast<long long>(kLocalItems) * P.nblocks && tot <= kMaxItems) {
                chunk = c2;
                items = items2;
            }
        }
        o = block_excl_scan<long long>(items, &tot, st.scan_ll);
        // (depth 1 always fits: chunk >= nl / nblocks gives at most nblocks + S
        // items, and the host keeps S <= (kLocalItems - 1) * nblocks)
        if (depth == 1 || (tot <= static_cast<long long>(kLocalItems) * P.nblocks && tot <= kMaxItems)) {
            if (s < S) st.item0[s] = static_cast<int>(o);
            if (s == 0) {
                st.item0[S] = static_cast<int>(tot);
                st.items_total = static_cast<int>(tot);
                st.chunk = static_cast<int>(chunk);
                st.tab_stride = stride;
                st.ncand = ncand;
                st.setc_log2 = lg2;
            }
            break;
        }
    }
    __syncthreads();
}

}  // namespace

template <int IF, int PR>
__global__ void __launch_bounds__(kThreads, 1) hav_chain_kernel(const __grid_constant__ Plan P) {
    constexpr int kInFlight = PassShape<IF, PR>::kInFlight;
    constexpr int kProbes = PassShape<IF, PR>::kProbes;
    __shared__ Smem st;
    extern __shared__ __align__(16) unsigned char dyn[];
    const int S = P.S;
    const int tid = threadIdx.x;
    const unsigned nb = static_cast<unsigned>(P.nblocks);
    const long long gtid = static_cast<long long>(blockIdx.x) * kThreads + tid;
    const long long gstride = static_cast<long long>(P.nblocks) * kThreads;

    Dev d;
    unsigned char* ws = P.ws;
    d.bar = reinterpret_cast<Barrier*>(ws + P.lay.barrier);
    d.gh = reinterpret_cast<GlobalHdr*>(ws + P.lay.ghdr);
    d.sh = reinterpret_cast<SegHdr*>(ws + P.lay.seghdr);
    d.clean = reinterpret_cast<unsigned*>(ws + P.lay.clean);
    d.ls = reinterpret_cast<LayerState*>(ws + P.lay.lstate);
    d.hist = reinterpret_cast<uint32_t*>(ws + P.lay.hist);
    d.psf = reinterpret_cast<int32_t*>(ws + P.lay.partial_sf);
    d.pcmp = reinterpret_cast<int32_t*>(ws + P.lay.partial_cmp);
    d.pitem = reinterpret_cast<int32_t*>(ws + P.lay.pitem);
    d.tr = reinterpret_cast<hav_layer_trace*>(ws + P.lay.trace);
    for (int b = 0; b < 2; ++b) {
        d.ord[b] = reinterpret_cast<float4*>(ws + P.lay.ord[b]);
        d.orig[b] = reinterpret_cast<int32_t*>(ws + P.lay.orig[b]);
    d.posof = reinterpret_cast<int32_t*>(ws + P.lay.posof);
        d.taken[b] = reinterpret_cast<uint32_t*>(ws + P.lay.taken[b]);
    }
    for (int b = 0; b < kTableSets; ++b) {
        d.dirty[b] = reinterpret_cast<uint32_t*>(ws + P.lay.dirty[b]);
        d.tk[b] = reinterpret_cast<unsigned long long*>(ws + P.lay.tabk[b]);
    }
    d.wpre = reinterpret_cast<uint32_t*>(ws + P.lay.wpre);
    d.bkt = reinterpret_cast<uint32_t*>(ws + P.lay.bkt);
    d.prefix = reinterpret_cast<int32_t*>(ws + P.lay.prefix);
    d.tv = reinterpret_cast<unsigned long long*>(ws + P.lay.tabv);
    d.cand = reinterpret_cast<Cand*>(ws + P.lay.cand);
    d.ptimes = P.ptimes;
    d.ptimes_cap = P.ptimes_cap;
    for (int k = tid; k < P.S; k += kThreads) st.gm[k] = 0;  // no previous search yet
    if (tid == 0) st.bucketed = 0;
    if (tid == 0) {
        st.fused_uses[0] = st.fused_uses[1] = 0u;
        st.fused_last[0] = st.fused_last[1] = 0ull;
        st.epoch = 0u;
        st.set_clean = 0;
        st.ntimes = 0;
        // every block reads this before block 0 may change it (after the first barrier)
        st.was_clean = static_cast<int>(ld_volatile_u(d.clean));
        if (d.ptimes && blockIdx.x == 0) {
            d.ptimes[0] = globaltimer();
            d.ptimes[1] = 0;
            st.ntimes = 1;
        }
    }
    __syncthreads();

    for (int j = 0; j < P.L; ++j) {
        level_setup(P, j, st);
        if (tid < kLocalItems) st.own_on[tid] = 0;
        float4* ord = d.ord[j & 1];
        const int32_t* orig_in = (j == 0) ? nullptr : d.orig[(j - 1) & 1];
        uint32_t* taken = d.taken[j & 1];
        const long long NL = st.n_level;
        // level 0: every segment of at least kBucketMin points is sorted by
        // Morton cell (one cloud: the whole level; a batch: each such segment
        // within its own range)
        bool bucketing = false;
        if (j == 0)
            for (int s2 = 0; s2 < S; ++s2) bucketing = bucketing || st.n[s2] >= kBucketMin;

        // ------------------------------------------------ bbox, layout, clears
        // (a later level's box, masks and states were prepared by the previous
        // level's compaction, which wrote its points)
        if (j == 0) {
            const int par = j & 1;
            for (int it = blockIdx.x; it < st.items_total; it += nb) {
                int a, b;
                const int s = item_range(st, S, it, &a, &b);
                float mnv[3] = {INFINITY, INFINITY, INFINITY}, mxv[3] = {-INFINITY, -INFINITY, -INFINITY};
                int bad = 0;
                for (int i = a + tid; i < b; i += kThreads) {
                    float p[3];
                    if (j == 0) {
                        const float* q = P.points + 3 * i;
                        p[0] = q[0];
                        p[1] = q[1];
                        p[2] = q[2];
                        if (st.n[s] < kBucketMin) {  // (a bucketed segment is placed by its scatter)
                            ord[i] = make_float4(p[0], p[1], p[2], __int_as_float(static_cast<int>(i)));
                            d.posof[i] = static_cast<int32_t>(i);
                        }
                    } else {
                        const float4 q = ord[i];
                        p[0] = q.x;
                        p[1] = q.y;
                        p[2] = q.z;
                    }
#pragma unroll
                    for (int a3 = 0; a3 < 3; ++a3) {
                        if (!isfinite(p[a3])) bad = 1;
                        mnv[a3] = fminf(mnv[a3], p[a3]);
                        mxv[a3] = fmaxf(mxv[a3], p[a3]);
                    }
                }
#pragma unroll
                for (int a3 = 0; a3 < 3; ++a3) {
                    for (int o = 16; o > 0; o >>= 1) {
                        mnv[a3] = fminf(mnv[a3], __shfl_xor_sync(0xffffffffu, mnv[a3], o));
                        mxv[a3] = fmaxf(mxv[a3], __shfl_xor_sync(0xffffffffu, mxv[a3], o));
                    }
                }
                if ((tid & 31) == 0) {
                    for (int a3 = 0; a3 < 3; ++a3) {
                        st.redf[a3][tid >> 5] = mnv[a3];
                        st.redf[3 + a3][tid >> 5] = mxv[a3];
                    }
                }
                bad = __syncthreads_or(bad);
                if (tid < 6) {
                    float r = st.redf[tid][0];
                    for (int w = 1; w < kThreads / 32; ++w)
                        r = (tid < 3) ? fminf(r, st.redf[tid][w]) : fmaxf(r, st.redf[tid][w]);
                    if (isfinite(r)) {
                        if (tid < 3) atomicMax(&d.sh[s].bbox[par][tid], ~enc_f(r));
                        else atomicMax(&d.sh[s].bbox[par][tid], enc_f(r));
                    }
                }
                if (tid == 0 && bad) {
                    atomicExch(&d.sh[s].nonfinite, 1);
                    seg_error(d, s, HAV_ERR_NONFINITE);
                }
                __syncthreads();
            }
            fill<uint32_t>(taken, NL / 32 + 1, 0u, gtid, gstride);
            fill<int32_t>(d.prefix, static_cast<long long>(S) * kMaxIters, -1, gtid, gstride);
            clear_layer_state(d, S, 0, gtid, gstride);
            clear_layer_state(d, S, 1, gtid, gstride);
            if (j == 0 && !st.was_clean) {
                // first call on this workspace, or the previous call was cut short
                for (int b = 0; b < kTableSets; ++b)
                    fill<unsigned long long>(d.tk[b], P.lay.tab_slots, kEmptyKey, gtid, gstride);
                fill<unsigned long long>(d.tv, P.lay.tab_slots, kEmptyVal, gtid, gstride);
            }
            if (bucketing) fill<uint32_t>(d.bkt, 2 * 4096ll * S, 0u, gtid, gstride);
            // (test hook: one arrival more than the launch has blocks never comes,
            // so every block's bounded wait gives up and the call reports a timeout)
            if (!grid_sync(d, nb + ((j == 0 && P.test_timeout) ? 1u : 0u), st, TAG(1, j, 0, 0))) return;
            if (j == 0 && blockIdx.x == 0 && tid == 0) *(volatile unsigned*)d.clean = 0u;
        }

        // --------------------------------------------------- search bracket
        if (tid < S) {
            const int par = j & 1;
            // control flow uses only values that no block can change while
            // others read them: the error carried from the previous level's
            // compaction, and the non-finite flag of this level's bbox phase
            int err = (j == 0) ? 0 : st.err[tid];
            if (!err && ld_volatile(&d.sh[tid].nonfinite)) err = HAV_ERR_NONFINITE;
            float s_hi = 0.0f;
            for (int a = 0; a < 3; ++a) {
                float mn = dec_f(~d.sh[tid].bbox[par][a]);
                float mx = dec_f(d.sh[tid].bbox[par][3 + a]);
                if (st.n[tid] == 0 || err) mn = mx = 0.0f;
                st.mn[tid][a] = mn;
                st.mx[tid][a] = mx;
                const float e = __fsub_rn(mx, mn);
                s_hi = fmaxf(s_hi, __fdiv_rn(e, P.aspect[a]));
            }
            if (s_hi == 0.0f) s_hi = 1.0f;
            if (!err && !isfinite(s_hi)) {
                err = HAV_ERR_RANGE;
                seg_error(d, tid, err);
            }
            st.s_hi[tid] = s_hi;
            st.err[tid] = err;
        }
        __syncthreads();

        // A later level of a bucketed cloud keeps the bucketing's order (each
        // level's points are a subsequence of the previous level's, in order),
        // so its points are sorted by their level-0 Morton cell: the cells this
        // block's item holds whole run from the first cell starting in it to
        // the last cell ending in it, read off the cells of the points at and
        // beside the item's two ends.
        // The same for a batch's segments sorted at level 0 (their level-0
        // boxes are in the segment headers), item by item within the segment.
        if (j > 0 && S > 1 && tid < kLocalItems &&
            static_cast<long long>(blockIdx.x) + static_cast<long long>(tid) * nb < st.items_total) {
            const int li = tid;
            int ia, ib;
            const int s = item_range(st, S, static_cast<int>(blockIdx.x + tid * nb), &ia, &ib);
            if (ld_volatile(&d.sh[s].b0_on) && ib > ia) {
                float mn3[3], mx3[3], k3[3];
                for (int a3 = 0; a3 < 3; ++a3) {
                    mn3[a3] = d.sh[s].b0[a3];
                    mx3[a3] = d.sh[s].b0[3 + a3];
                    const float e = __fsub_rn(mx3[a3], mn3[a3]);
                    k3[a3] = (e > 0.0f) ? __fdiv_rn(16.0f, e) : 0.0f;
                }
                auto cell = [&](int i) {
                    const float4 q = ord[i];
                    const float p3[3] = {q.x, q.y, q.z};
                    return static_cast<int>(bucket_of(p3, mn3, mx3));
                };
                const int sa = static_cast<int>(st.off[s]), se = static_cast<int>(st.off[s + 1]);
                const int cf = cell(ia), cl = cell(ib - 1);
                const int lo = (ia == sa || cell(ia - 1) < cf) ? cf : cf + 1;
                const int hi = (ib == se || cell(ib) > cl) ? cl : cl - 1;
                st.own_lo[li] = lo;
                st.own_hi[li] = hi;
                st.own_on[li] = (lo <= hi) ? 1 : 0;
                for (int a3 = 0; a3 < 3; ++a3) {
                    st.own_mn[li][a3] = mn3[a3];
                    st.own_k[li][a3] = k3[a3];
                }
            }
        }
        if (j > 0 && st.bucketed && S == 1 && tid < kLocalItems &&
            static_cast<long long>(blockIdx.x) + static_cast<long long>(tid) * nb < st.items_total) {
            const int li = tid;  // one thread per item of the block
            int ia, ib;
            item_range(st, S, static_cast<int>(blockIdx.x + tid * nb), &ia, &ib);
            auto cell = [&](int i) {
                const float4 q = ord[i];
                const float p3[3] = {q.x, q.y, q.z};
                return static_cast<int>(bucket_of(p3, st.b0_mn, st.b0_mx));
            };
            if (ib > ia) {
                const int cf = cell(ia), cl = cell(ib - 1);
                const int lo = (ia == 0 || cell(ia - 1) < cf) ? cf : cf + 1;
                const int hi = (ib == NL || cell(ib) > cl) ? cl : cl - 1;
                st.own_lo[li] = lo;
                st.own_hi[li] = hi;
                st.own_on[li] = (lo <= hi) ? 1 : 0;
                for (int a3 = 0; a3 < 3; ++a3) {
                    st.own_mn[li][a3] = st.b0_mn[a3];
                    st.own_k[li][a3] = st.b0_k[a3];
                }
            }
        }
        __syncthreads();

        // ---------------------------------------- bucketing (one large cloud)
        if (bucketing && S == 1) {
            if (tid == 0) st.set_clean = 0;
            uint32_t* h = reinterpret_cast<uint32_t*>(dyn);          // this block's counts
            uint32_t* hb = reinterpret_cast<uint32_t*>(dyn) + 4096;  // global bucket bases
            for (int b = tid; b < 4096; b += kThreads) h[b] = 0u;
            __syncthreads();
            for (int it = blockIdx.x; it < st.items_total; it += nb) {
                int a, b;
                item_range(st, S, it, &a, &b);
                for (int i = a + tid; i < b; i += kThreads) {
                    const float* q = P.points + 3 * i;
                    const float p[3] = {q[0], q[1], q[2]};
                    atomicAdd(&h[bucket_of(p, st.mn[0], st.mx[0])], 1u);
                }
            }
            __syncthreads();
            for (int b = tid; b < 4096; b += kThreads)
                if (h[b]) atomicAdd(&d.bkt[b], h[b]);
            if (!grid_sync(d, nb, st, TAG(9, j, 0, 0))) return;
            {
                // exclusive prefix over the 4096 global counts (whole bins per thread)
                constexpr int kPerT = 4096 / kThreads;
                static_assert(4096 % kThreads == 0, "bucket bins per thread");
                uint32_t c4[kPerT], sum = 0;
#pragma unroll
                for (int k = 0; k < kPerT; ++k) {
                    c4[k] = d.bkt[kPerT * tid + k];
                    sum += c4[k];
                }
                unsigned tot;
                unsigned before = block_excl_scan<unsigned>(sum, &tot, st.scan_u);
#pragma unroll
                for (int k = 0; k < kPerT; ++k) {
                    hb[kPerT * tid + k] = before;
                    before += c4[k];
                }
                __syncthreads();
                // the Morton cells each of this block's work items holds whole
                // (one thread per item; the items are the same in every pass of
                // this level), and the bucketing's box, kept for the levels
                // that inherit its order
                if (tid == 0) {
                    st.bucketed = 1;
                    for (int a3 = 0; a3 < 3; ++a3) {
                        st.b0_mn[a3] = st.mn[0][a3];
                        st.b0_mx[a3] = st.mx[0][a3];
                        const float e = __fsub_rn(st.mx[0][a3], st.mn[0][a3]);
                        st.b0_k[a3] = (e > 0.0f) ? __fdiv_rn(16.0f, e) : 0.0f;
                    }
                }
                __syncthreads();
                if (tid < kLocalItems &&
                    static_cast<long long>(blockIdx.x) + static_cast<long long>(tid) * nb < st.items_total) {
                    int ia, ib;
                    item_range(st, S, static_cast<int>(blockIdx.x + tid * nb), &ia, &ib);
                    own_cells(hb, ia, ib, static_cast<unsigned>(NL), st.b0_mn, st.b0_k, st, tid);
                }
                for (int b = tid; b < 4096; b += kThreads)
                    if (h[b]) h[b] = hb[b] + atomicAdd(&d.bkt[4096 + b], h[b]);
                __syncthreads();
                for (int it = blockIdx.x; it < st.items_total; it += nb) {
                    int a, b;
                    item_range(st, S, it, &a, &b);
                    for (int i = a + tid; i < b; i += kThreads) {
                        const float* q = P.points + 3 * i;
                        const float p[3] = {q[0], q[1], q[2]};
                        const unsigned r = atomicAdd(&h[bucket_of(p, st.mn[0], st.mx[0])], 1u);
                        if (r < static_cast<unsigned>(NL)) {
                            ord[r] = make_float4(p[0], p[1], p[2], __int_as_float(static_cast<int>(i)));
                            d.posof[i] = static_cast<int32_t>(r);
                        }
                    }
                }
            }
            if (!grid_sync(d, nb, st, TAG(10, j, 0, 0))) return;
        } else if (bucketing) {
            // ------------------------------- bucketing (large clouds of a batch)
            // The same counting sort per segment of at least kBucketMin points,
            // within the segment's range: counts [S][4096] and cursors [S][4096]
            // in the workspace.  A block's items may belong to several
            // segments: the counts are gathered per run of items of one
            // segment, and every item counts its points again before it takes
            // its places.  The smaller segments kept their order in the bbox
            // phase.  (Leaving a segment that comes in a coherent order, a
            // LiDAR scan, unsorted measured 0.9 % slower on 64 LiDAR clouds:
            // the ownership test needs the sort.)
            if (tid == 0) st.set_clean = 0;
            uint32_t* h = reinterpret_cast<uint32_t*>(dyn);          // counts of one segment's items
            uint32_t* hb = reinterpret_cast<uint32_t*>(dyn) + 4096;  // bases of one segment's buckets
            uint32_t* bcnt = d.bkt;
            uint32_t* bcur = d.bkt + 4096ll * S;
            if (blockIdx.x == 0)  // the boxes of the sorted segments, for their later levels
                for (int s2 = tid; s2 < S; s2 += kThreads)
                    if (st.n[s2] >= kBucketMin) {
                        for (int a3 = 0; a3 < 3; ++a3) {
                            d.sh[s2].b0[a3] = st.mn[s2][a3];
                            d.sh[s2].b0[3 + a3] = st.mx[s2][a3];
                        }
                        d.sh[s2].b0_on = 1;
                    }
            int hs = -1;  // the segment whose counts h holds
            for (int b = tid; b < 4096; b += kThreads) h[b] = 0u;
            __syncthreads();
            for (int it = blockIdx.x; it < st.items_total; it += nb) {  // (block-uniform)
                int a, b;
                const int s = item_range(st, S, it, &a, &b);
                if (st.n[s] < kBucketMin) continue;
                if (hs >= 0 && hs != s) {
                    for (int k = tid; k < 4096; k += kThreads)
                        if (h[k]) {
                            atomicAdd(&bcnt[4096ll * hs + k], h[k]);
                            h[k] = 0u;
                        }
                    __syncthreads();
                }
                hs = s;
                for (int i = a + tid; i < b; i += kThreads) {
                    const float* q = P.points + 3 * i;
                    const float p3[3] = {q[0], q[1], q[2]};
                    atomicAdd(&h[bucket_of(p3, st.mn[s], st.mx[s])], 1u);
                }
                __syncthreads();
            }
            if (hs >= 0)
                for (int k = tid; k < 4096; k += kThreads)
                    if (h[k]) atomicAdd(&bcnt[4096ll * hs + k], h[k]);
            if (!grid_sync(d, nb, st, TAG(9, j, 0, 0))) return;
            int bs = -1;  // the segment whose bases hb holds
            for (int it = blockIdx.x; it < st.items_total; it += nb) {  // (block-uniform)
                int a, b;
                const int s = item_range(st, S, it, &a, &b);
                if (st.n[s] < kBucketMin) continue;
                const int li = static_cast<int>((it - static_cast<int>(blockIdx.x)) / static_cast<int>(nb));
                if (bs != s) {
                    // exclusive prefix of the segment's 4096 counts, from its first position
                    constexpr int kPerT = 4096 / kThreads;
                    uint32_t c4[kPerT], sum = 0;
#pragma unroll
                    for (int k = 0; k < kPerT; ++k) {
                        c4[k] = bcnt[4096ll * s + kPerT * tid + k];
                        sum += c4[k];
                    }
                    unsigned tot;
                    unsigned before = static_cast<unsigned>(st.off[s]) + block_excl_scan<unsigned>(sum, &tot, st.scan_u);
#pragma unroll
                    for (int k = 0; k < kPerT; ++k) {
                        hb[kPerT * tid + k] = before;
                        before += c4[k];
                    }
                    bs = s;
                }
                for (int k = tid; k < 4096; k += kThreads) h[k] = 0u;
                __syncthreads();
                if (tid == 0) {  // the cells this item holds whole, in its segment's box
                    float k3[3];
                    for (int a3 = 0; a3 < 3; ++a3) {
                        const float e = __fsub_rn(st.mx[s][a3], st.mn[s][a3]);
                        k3[a3] = (e > 0.0f) ? __fdiv_rn(16.0f, e) : 0.0f;
                    }
                    own_cells(hb, a, b, static_cast<unsigned>(st.off[s + 1]), st.mn[s], k3, st, li);
                }
                for (int i = a + tid; i < b; i += kThreads) {
                    const float* q = P.points + 3 * i;
                    const float p3[3] = {q[0], q[1], q[2]};
                    atomicAdd(&h[bucket_of(p3, st.mn[s], st.mx[s])], 1u);
                }
                __syncthreads();
                for (int k = tid; k < 4096; k += kThreads)
                    if (h[k]) h[k] = hb[k] + atomicAdd(&bcur[4096ll * s + k], h[k]);
                __syncthreads();
                const unsigned end = static_cast<unsigned>(st.off[s + 1]);
                for (int i = a + tid; i < b; i += kThreads) {
                    const float* q = P.points + 3 * i;
                    const float p3[3] = {q[0], q[1], q[2]};
                    const unsigned r = atomicAdd(&h[bucket_of(p3, st.mn[s], st.mx[s])], 1u);
                    if (r < end) {
                        ord[r] = make_float4(p3[0], p3[1], p3[2], __int_as_float(static_cast<int>(i)));
                        d.posof[i] = static_cast<int32_t>(r);
                    }
                }
                __syncthreads();
            }
            if (!grid_sync(d, nb, st, TAG(10, j, 0, 0))) return;
        }

        // ------------------------------------------------------------ layers
        long long taken_before = 0;  // thread s: budgets of earlier layers of segment s
        const int ncand = st.ncand;
        const long long tstride = st.tab_stride;  // table slots of one candidate (all segments)
        const long long dstride = NL;             // log entries of one candidate
        for (int l = 0; l < P.layers; ++l) {
            const int q = l & 1;
            LayerState* ls = d.ls + q * S;
            uint32_t* hist = d.hist + static_cast<long long>(q) * S * kHistBins;

            if (tid < S) {
                const long long ml = layer_budget(st.m[tid], P.layers, P.ratio, l);
                const long long kmax = ml + ml * P.sigma_num / P.sigma_den;
                const bool active = ml > 0 && st.err[tid] == 0;
                st.ml[tid] = static_cast<int>(ml);
                st.kmax[tid] = static_cast<int>(kmax);
                st.lo[tid] = 0.0f;
                st.hi[tid] = st.s_hi[tid];
                st.sel[tid] = 0;
                st.sel_cand[tid] = 0;
                st.iters[tid] = 0;
                st.kstar[tid] = 0;
                // a fixed voxel size (Table 6 "Fix") skips the search
                const bool fixed = P.fixed_s > 0.0f;
                int fl = active ? F_ACTIVE : 0;
                if (active && P.t_max > 0 && !fixed) fl |= F_SEARCH;
                // guided start: g from the previous search, or from s_hi for the
                // first; doubling up from it while the counts stay too high
                st.first[tid] = 0.0f;
                if ((fl & F_SEARCH) && P.search == HAV_SEARCH_GUIDED) {
                    const float g =
                        (st.gm[tid] > 0)
                            ? __fmul_rn(st.gs[tid], __fsqrt_rn(__fdiv_rn(__int2float_rn(st.gm[tid]), __ll2float_rn(ml))))
                            : __fdiv_rn(st.s_hi[tid], __fsqrt_rn(__ll2float_rn(ml)));
                    if (g > 0.0f && g < st.s_hi[tid]) {
                        st.first[tid] = g;
                        fl |= F_UP;
                    }
                }
                if (active && (P.t_max == 0 || fixed)) {
                    st.s_star[tid] = fixed ? P.fixed_s : st.s_hi[tid];
                    if (!make_grid(st.s_star[tid], P.aspect, st.mn[tid], &st.grid[tid])) {
                        seg_error(d, tid, HAV_ERR_RANGE);
                        st.err[tid] = HAV_ERR_RANGE;
                        fl = 0;
                    }
                }
                st.flags[tid] = fl;
                if (blockIdx.x == 0) {
                    hav_layer_trace* tr = d.tr + (static_cast<long long>(j) * S + tid) * kMaxLayers + l;
                    tr->m_l = ml;
                    tr->k_max = kmax;
                    tr->k_star = 0;
                    tr->n_in = st.n[tid] - taken_before;
                    tr->iters = 0;
                    tr->accepted = 0;
                    tr->s_hi = st.s_hi[tid];
                    tr->s_star = (P.t_max == 0 && (fl & F_ACTIVE)) ? st.s_hi[tid] : 0.0f;
                    tr->bounded = 0u;
                }
                taken_before += ml;
            }
            __syncthreads();
            // bisection: the leading steps whose outcome is already settled are
            // taken without a pass: at the size s_hi / 2^(k+1) either an earlier
            // layer of this level counted fewer than m_l voxels on a superset of
            // this layer's points, or the bounding box spans fewer than m_l grid
            // cells.  The trace keeps the smaller bound.  One warp per searching
            // segment, lane k the step k (the same k + 1 halvings of s_hi).
            if (P.search == HAV_SEARCH_BISECT && P.t_max > 0) {
                static_assert(kMaxIters <= 32, "one lane per step");
                const int lane = tid & 31;
                for (int s = tid >> 5; s < S; s += kThreads / 32) {  // (warp-uniform)
                    if (!(st.flags[s] & F_SEARCH)) continue;
                    const long long ml = st.ml[s];
                    float sv = st.s_hi[s];
                    for (int h = 0; h <= lane; ++h) sv = __fmul_rn(__fadd_rn(0.0f, sv), 0.5f);
                    long long bd = LLONG_MAX;
                    if (lane < P.t_max) {
                        bd = cell_bound(sv, P.aspect, st.mn[s], st.mx[s]);
                        const int pk = ld_volatile(d.prefix + s * kMaxIters + lane);
                        if (pk >= 0 && pk < bd) bd = pk;
                    }
                    const unsigned settled = __ballot_sync(0xffffffffu, lane < P.t_max && bd < ml);
                    const int nskip = __ffs(~settled) - 1;  // leading settled steps
                    const float hi_ff = __shfl_sync(0xffffffffu, sv, nskip > 0 ? nskip - 1 : 0);
                    int fl = st.flags[s] | F_PRE;
                    const float hi_s = nskip > 0 ? hi_ff : st.s_hi[s];
                    if (nskip >= P.t_max) fl = F_ACTIVE;  // every step settled: no acceptance, s* = hi
                    if (lane == 0) {
                        st.hi[s] = hi_s;
                        st.iters[s] = nskip;
                        if (nskip >= P.t_max) {
                            st.s_star[s] = hi_s;
                            if (!make_grid(hi_s, P.aspect, st.mn[s], &st.grid[s])) {
                                seg_error(d, s, HAV_ERR_RANGE);
                                st.err[s] = HAV_ERR_RANGE;
                                fl = 0;
                            }
                        }
                        st.flags[s] = fl;
                    }
                    if (blockIdx.x == 0) {
                        hav_layer_trace* tr = d.tr + (static_cast<long long>(j) * S + s) * kMaxLayers + l;
                        if (lane < nskip) {
                            tr->s[lane] = sv;
                            tr->K[lane] = bd;
                        }
                        if (lane == 0) {
                            tr->iters = nskip;
                            tr->s_star = (nskip >= P.t_max && (fl & F_ACTIVE)) ? hi_s : 0.0f;
                            tr->bounded = nskip ? (0xffffffffu >> (32 - nskip)) : 0u;
                        }
                    }
                }
                __syncthreads();
            }

            // --------------------------------------- Section 3.3 bisection
            // One pass evaluates the whole depth-D subtree of the bisection below
            // each segment's current (lo, hi): ncand = 2^D - 1 candidate sizes,
            // each with its own table and count.  The decision then walks the
            // subtree exactly as the sequential search does, so the sizes
            // evaluated on the path, their counts and the outcome are those of the
            // plain bisection; D = 1 is the plain bisection.
            // one cloud, one candidate per pass: the count rides on the barrier
            const bool fused = (S == 1 && ncand == 1);
            for (int p = 0; p < P.t_max; ++p) {
                const int searching = (tid < S && (st.flags[tid] & F_SEARCH)) ? 1 : 0;
                if (tid == 0) {
                    st.pass_cnt = 0ull;
                    st.pass_err = 0;
                }
                if (!__syncthreads_or(searching)) break;
                // table sets: X this pass, Z the previous pass (emptied after this
                // pass's arrival), F the next pass (empty since the last barrier)
                const int X = p % kTableSets;
                const int Z = (p + kTableSets - 1) % kTableSets;
                const int F = (p + 1) % kTableSets;

                // candidate grids of the owned items' segments
                {
                    int li = 0;
                    for (int it = blockIdx.x; it < st.items_total; it += nb, ++li) {
                        const int s = find_seg(st.item0, S, it);
                        if (tid < ncand && (st.flags[s] & F_SEARCH)) {
                            const float sc = cand_size(st.lo[s], st.hi[s], (st.flags[s] & F_UP) != 0,
                                                       st.first[s], tid);
                            st.cvalid[li][tid] = make_grid(sc, P.aspect, st.mn[s], &st.cgrid[li][tid]) ? 1 : 0;
                        }
                    }
                }
                __syncthreads();

                // Cnt(P_l, s_c) for every candidate c: (a) every point's key into the
                // candidate's part of the block set, keys new to the block listed
                // densely; (b) the listed keys into the candidates' global tables,
                // kProbes compare-and-swaps in flight per thread
                unsigned long long* set = reinterpret_cast<unsigned long long*>(dyn);
                unsigned short* list = reinterpret_cast<unsigned short*>(dyn + kSetSlots * sizeof(unsigned long long));
                const int setc_log2 = st.setc_log2;
                int li = 0;
                for (int it = blockIdx.x; it < st.items_total; it += nb, ++li) {
                    int a, b;
                    const int s = item_range(st, S, it, &a, &b);
                    if (!(st.flags[s] & F_SEARCH)) continue;
                    if (!st.set_clean)  // otherwise every slot is already empty
                        for (int k = tid; k < kSetSlots; k += kThreads) set[k] = kEmptyKey;
                    if (tid == 0) {
                        st.list_n = 0u;
                        st.rbits = 0u;
                        st.rest_n = 0u;
                    }
                    if (tid < kMaxCand) st.xcnt[tid] = 0u;
                    __syncthreads();
                    const int cap = st.cap_log2[s];
                    unsigned long long* Tb = d.tk[X] + st.tab_off[s];
                    int bad = 0;
                    unsigned rbits = 0;  // candidates with a key out of range
                    // log a fresh insert (whole warp calls, converged): one shared
                    // counter add per candidate present in the warp, and the warp's
                    // log entries of a candidate land side by side.  The set X logs
                    // are empty when a pass starts, so dcnt[X] ends as the count.
                    auto log_fresh = [&](bool fresh, int c, long long slot) {
                        const int k = (ncand == 1) ? warp_append(fresh, &st.dcnt[X][li][0])
                                                   : warp_append_keyed(fresh, c, st.dcnt[X][li]);
                        if (fresh)
                            d.dirty[X][c * dstride + a + k] = static_cast<uint32_t>(c * tstride + st.tab_off[s] + slot);
                    };
                    // work units are (candidate, point) pairs, point-minor, so that a
                    // warp reads consecutive points and the candidates run in parallel
                    const int lane = tid & 31;
                    const int L = b - a;
                    const int units = L * ncand;
                    for (int base = tid - lane; base < units; base += kInFlight * kThreads) {  // warp-uniform
                        float4 q4[kInFlight];
                        int cu[kInFlight];
#pragma unroll
                        for (int u = 0; u < kInFlight; ++u) {
                            const int w = base + lane + u * kThreads;
                            cu[u] = (ncand == 1) ? 0 : w / L;
                            q4[u] = (w < units) ? ord[a + (w - cu[u] * L)]
                                                : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                        }
                        // the keys of all units first (independent arithmetic), then
                        // their inserts one after the other
                        unsigned long long key[kInFlight];
#pragma unroll
                        for (int u = 0; u < kInFlight; ++u) {
                            key[u] = kEmptyKey;
                            const int c = cu[u];
                            // w < 0: padding, or taken by an earlier layer
                            if (__float_as_int(q4[u].w) >= 0 && st.cvalid[li][c]) {
                                const float p3[3] = {q4[u].x, q4[u].y, q4[u].z};
                                float f[3];
                                if (!cell_key(p3, st.cgrid[li][c], &key[u], f)) {
                                    rbits |= 1u << c;
                                    key[u] = kEmptyKey;
                                }
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kInFlight; ++u) {
                            const int c = cu[u];
                            int r = -2;
                            bool nw = false;
                            if (key[u] != kEmptyKey) r = smem_insert_n(set + (c << setc_log2), setc_log2, key[u], &nw);
                            const int pos = warp_append(r >= 0 && nw, &st.list_n);
                            if (pos >= 0) list[pos] = static_cast<unsigned short>((c << setc_log2) + r);
                            bool fr = false;
                            long long slot = -1;
                            if (r == -1) {  // block set saturated: straight to the global table
                                slot = find_or_insert(Tb + c * tstride, cap, key[u], &fr);
                                if (slot < 0) bad = HAV_ERR_TABLE_FULL;
                            }
                            log_fresh(r == -1 && slot >= 0 && fr, c, slot);
                        }
                    }
                    __syncthreads();
                    const int nl = static_cast<int>(st.list_n);
                    // a voxel whose every point lies in cells this block holds
                    // whole is counted here; the other keys go to the global table
                    const unsigned short* gl = list;
                    int ng = nl;
                    // (below 256 listed keys the test costs about what it saves)
                    if (st.own_on[li] && nl >= 256 && nl <= kSetSlots / 2) {
                        unsigned short* rest = list + kSetSlots / 2;
                        unsigned mine = 0;  // owned keys of this thread (one candidate)
                        for (int k0 = tid - lane; k0 < nl; k0 += kThreads) {  // warp-uniform
                            const int k = k0 + lane;
                            bool glob = false;
                            int c = 0;
                            if (k < nl) {
                                const int idx = list[k];
                                c = idx >> setc_log2;
                                glob = !voxel_owned(set[idx], st.cgrid[li][c], st.own_mn[li], st.own_k[li],
                                                    st.own_lo[li], st.own_hi[li]);
                            }
                            const int pos = warp_append(glob, &st.rest_n);
                            if (pos >= 0) rest[pos] = list[k];
                            if (ncand == 1) mine += (k < nl && !glob) ? 1u : 0u;
                            else warp_append_keyed(k < nl && !glob, c, st.xcnt);
                        }
                        if (ncand == 1) {
                            const unsigned w = __reduce_add_sync(0xffffffffu, mine);
                            if (lane == 0 && w) atomicAdd(&st.xcnt[0], w);
                        }
                        __syncthreads();
                        gl = rest;
                        ng = static_cast<int>(st.rest_n);
                    }
                    for (int k0 = tid - lane; k0 < ng; k0 += kProbes * kThreads) {  // warp-uniform
                        unsigned long long key[kProbes];
                        unsigned long long* Tp[kProbes];
                        int cc[kProbes];
                        long long slot[kProbes];
                        bool fr[kProbes];
#pragma unroll
                        for (int u = 0; u < kProbes; ++u) {
                            const int k = k0 + lane + u * kThreads;
                            const int idx = (k < ng) ? static_cast<int>(gl[k]) : 0;
                            cc[u] = idx >> setc_log2;
                            key[u] = (k < ng) ? set[idx] : kEmptyKey;
                            Tp[u] = Tb + cc[u] * tstride;
                        }
                        find_or_insert_batch<kProbes>(Tp, cap, key, slot, fr);
#pragma unroll
                        for (int u = 0; u < kProbes; ++u) {
                            if (key[u] != kEmptyKey && slot[u] < 0) bad = HAV_ERR_TABLE_FULL;
                            log_fresh(key[u] != kEmptyKey && slot[u] >= 0 && fr[u], cc[u], slot[u]);
                        }
                    }
                    // empty the set again: exactly the listed slots are occupied
                    __syncthreads();
                    for (int k = tid; k < nl; k += kThreads) set[list[k]] = kEmptyKey;
                    if (tid == 0) st.set_clean = 1;
                    if (rbits) atomicOr(&st.rbits, rbits);
                    if (bad) seg_error(d, s, bad);
                    __syncthreads();
                    if (fused) {
                        if (tid == 0) {
                            st.pass_cnt += static_cast<unsigned long long>(st.dcnt[X][li][0]) + st.xcnt[0];
                            if (st.rbits) st.pass_err = 1;
                        }
                    } else {
                        if (tid < ncand && (st.dcnt[X][li][tid] || st.xcnt[tid]))
                            atomicAdd(&ls[s].count[p % 3][tid], static_cast<unsigned>(st.dcnt[X][li][tid]) + st.xcnt[tid]);
                        if (tid == 0 && st.rbits) atomicOr(&ls[s].cerr[p % 3], st.rbits);
                    }
                }
                if (fused) {
                    const unsigned long long add = st.pass_cnt + (st.pass_err ? kFusedErr : 0ull);
                    fused_arrive(d, st, p & 1, add);
                } else {
                    if (p >= 1 && blockIdx.x == 0)
                        for (int k = tid; k < S * (kMaxCand + 1); k += kThreads) {
                            const int s = k / (kMaxCand + 1), c = k % (kMaxCand + 1);
                            if (c < kMaxCand) ls[s].count[(p + 1) % 3][c] = 0u;
                            else ls[s].cerr[(p + 1) % 3] = 0u;
                        }
                    grid_arrive(d, st);
                }
                // while the other blocks arrive: empty set Z, slot by slot, from this
                // block's logs (segments still searching only: an accepted segment's
                // tables stay for its selection).  This block's next arrival
                // publishes the stores, before pass p + 2 inserts into set Z.
                if (p >= 1) {
                    int li = 0;
                    for (int it = blockIdx.x; it < st.items_total; it += nb, ++li) {
                        int a, b;
                        const int s = item_range(st, S, it, &a, &b);
                        if (!(st.flags[s] & F_SEARCH)) continue;
                        for (int c = 0; c < ncand; ++c) {
                            const int cnt = st.dcnt[Z][li][c];
                            const uint32_t* lg = d.dirty[Z] + c * dstride + a;
                            for (int k = tid; k < cnt; k += kThreads) d.tk[Z][lg[k]] = kEmptyKey;
                        }
                    }
                    __syncthreads();
                    li = 0;
                    for (int it = blockIdx.x; it < st.items_total; it += nb, ++li) {
                        const int s = find_seg(st.item0, S, it);
                        if (tid < ncand && (st.flags[s] & F_SEARCH)) st.dcnt[Z][li][tid] = 0;
                    }
                }
                if (fused) {
                    if (!fused_wait(d, nb, st, p & 1, TAG(2, j, l, p))) return;
                } else {
                    if (!grid_wait(d, nb, st, TAG(2, j, l, p))) return;
                }

                // decide (identically in every block): walk the evaluated subtree
                if (searching) {
                    float lo = st.lo[tid], hi = st.hi[tid];
                    bool up = (st.flags[tid] & F_UP) != 0;
                    bool pre = (st.flags[tid] & F_PRE) != 0;  // every step so far too few
                    float first = st.first[tid];
                    int node = 0;
                    int t = st.iters[tid];
                    const unsigned cerr = fused ? (st.fused_delta >= kFusedErr ? 1u : 0u)
                                                : ld_volatile_u(&ls[tid].cerr[p % 3]);
                    // every candidate's count in one round trip, before the walk
                    unsigned cnt[kMaxCand];
#pragma unroll
                    for (int c = 0; c < kMaxCand; ++c)
                        cnt[c] = (!fused && c < ncand) ? ld_volatile_u(&ls[tid].count[p % 3][c]) : 0u;
                    hav_layer_trace* tr = d.tr + (static_cast<long long>(j) * S + tid) * kMaxLayers + l;
                    while (node < ncand && t < P.t_max) {
                        const float sv = next_size(lo, hi, up, first);
                        first = 0.0f;
                        Grid gv;
                        if ((cerr >> node) & 1u || !make_grid(sv, P.aspect, st.mn[tid], &gv)) {
                            seg_error(d, tid, HAV_ERR_RANGE);
                            st.err[tid] = HAV_ERR_RANGE;
                            st.flags[tid] = 0;
                            break;
                        }
                        unsigned kn = cnt[0];
#pragma unroll
                        for (int c = 1; c < kMaxCand; ++c)
                            if (c == node) kn = cnt[c];
                        const long long K = fused ? static_cast<long long>(st.fused_delta) : static_cast<long long>(kn);
                        if (blockIdx.x == 0) {
                            tr->s[t] = sv;
                            tr->K[t] = K;
                            tr->iters = t + 1;
                        }
                        if (pre) {  // sv = s_hi / 2^(t+1): later layers of the level may reuse K
                            if (blockIdx.x == 0) d.prefix[tid * kMaxIters + t] = static_cast<int32_t>(K);
                            if (K >= st.ml[tid]) pre = false;
                        }
                        ++t;
                        if (K > st.kmax[tid]) {
                            lo = sv;
                            node = 2 * node + 2;
                        } else if (K < st.ml[tid]) {
                            hi = sv;
                            up = false;
                            node = 2 * node + 1;
                        } else {
                            st.s_star[tid] = sv;
                            st.grid[tid] = gv;
                            st.sel[tid] = X;
                            st.sel_cand[tid] = node;
                            st.flags[tid] = F_ACTIVE | F_ACCEPT;
                            break;
                        }
                    }
                    st.lo[tid] = lo;
                    st.hi[tid] = hi;
                    st.iters[tid] = t;
                    st.first[tid] = first;
                    if (st.flags[tid] & F_SEARCH)
                        st.flags[tid] = (st.flags[tid] & ~(F_UP | F_PRE)) | (up ? F_UP : 0) | (pre ? F_PRE : 0);
                    if ((st.flags[tid] & F_SEARCH) && t >= P.t_max) {
                        // no acceptance within t_max steps: set F is empty for this
                        // segment (emptied before this pass's arrival, or unused)
                        const float sv = (lo > 0.0f) ? lo : hi;
                        st.s_star[tid] = sv;
                        st.sel[tid] = F;
                        st.sel_cand[tid] = 0;
                        st.flags[tid] = F_ACTIVE;
                        if (!make_grid(sv, P.aspect, st.mn[tid], &st.grid[tid])) {
                            seg_error(d, tid, HAV_ERR_RANGE);
                            st.flags[tid] = 0;
                            st.err[tid] = HAV_ERR_RANGE;
                        }
                    }
                }
                __syncthreads();
            }
            // (every searching segment takes at least one step per pass, so none is
            // still searching after t_max passes)
            // the guided start of the segment's next search follows this one
            if (P.search == HAV_SEARCH_GUIDED && tid < S && st.ml[tid] > 0 && P.t_max > 0 &&
                !(P.fixed_s > 0.0f) && st.err[tid] == 0) {
                st.gs[tid] = st.s_star[tid];
                st.gm[tid] = st.ml[tid];
                if (blockIdx.x == 0) {  // for a small-level launch that continues the chain
                    d.sh[tid].guide_s = st.gs[tid];
                    d.sh[tid].guide_m = st.gm[tid];
                }
            }

            // ------------------------------------- Section 3.2 selection at s*
            {
                if (tid == 0) st.set_clean = 0;
                unsigned long long* skey = reinterpret_cast<unsigned long long*>(dyn);
                unsigned long long* sval = skey + kSelSlots;
                unsigned short* list = reinterpret_cast<unsigned short*>(sval + kSelSlots);
                int li = 0;
                for (int it = blockIdx.x; it < st.items_total; it += nb, ++li) {
                    int a, b;
                    const int s = item_range(st, S, it, &a, &b);
                    if (!(st.flags[s] & F_ACTIVE)) continue;
                    for (int k = tid; k < kSelSlots; k += kThreads) {
                        skey[k] = kEmptyKey;
                        sval[k] = kEmptyVal;
                    }
                    for (int k = tid; k < kHistBins; k += kThreads) st.bh[k] = 0u;
                    if (tid == 0) {
                        st.list_n = 0u;
                        st.rest_n = 0u;
                        st.gl_n = 0u;
                    }
                    __syncthreads();
                    const Grid& G = st.grid[s];
                    // level 0 of a bucketed cloud: a voxel the block owns whole has its
                    // representative in the block's own minimum; it skips the global
                    // table and is listed for the classification (in the next level's
                    // staged-point array, not written before this level's compaction)
                    const bool owning = st.own_on[li] != 0;
                    Cand* olist = reinterpret_cast<Cand*>(d.ord[(j + 1) & 1]) + a;
                    const int sel = st.sel[s];
                    const int sc = st.sel_cand[s];
                    unsigned long long* T = d.tk[sel] + sc * tstride + st.tab_off[s];
                    unsigned long long* V = d.tv + st.tab_off[s];
                    const int cap = st.cap_log2[s];
                    unsigned first = 0;
                    int bad = 0;
                    auto global_min = [&](unsigned long long key, long long slot, bool fr, unsigned long long packed) {
                        if (fr) {
                            const int k = atomicAdd(&st.dcnt[sel][li][sc], 1);
                            d.dirty[sel][sc * dstride + a + k] =
                                static_cast<uint32_t>(sc * tstride + st.tab_off[s] + slot);
                        }
                        if (atomicMin(V + slot, packed) == kEmptyVal) {
                            ++first;
                            atomicAdd(&st.bh[priority(key) >> (64 - kHistBits)], 1u);
                        }
                    };
                    const int lane = tid & 31;
                    for (int base = a + (tid - lane); base < b; base += kInFlight * kThreads) {  // warp-uniform
                        float4 q4[kInFlight];
#pragma unroll
                        for (int u = 0; u < kInFlight; ++u) {
                            const int i = base + lane + u * kThreads;
                            q4[u] = (i < b) ? ord[i] : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                        }
#pragma unroll
                        for (int u = 0; u < kInFlight; ++u) {
                            const int g = __float_as_int(q4[u].w);  // < 0: padding, or taken by an earlier layer
                            bool ok = g >= 0;
                            unsigned long long key = kEmptyKey, packed = kEmptyVal;
                            if (ok) {
                                const float p3[3] = {q4[u].x, q4[u].y, q4[u].z};
                                float f[3];
                                if (cell_key(p3, G, &key, f)) {
                                    // the voxel keeps the smallest (word, index): the squared
                                    // distance to the centre, or a random draw (Table 6 "RA")
                                    const unsigned word =
                                        (P.select == HAV_SELECT_RANDOM)
                                            ? static_cast<unsigned>(random_draw(P.seed, static_cast<unsigned long long>(
                                                                                            g - st.off[s])) >>
                                                                    32)
                                            : __float_as_uint(centre_d2(p3, G, f));
                                    packed = (static_cast<unsigned long long>(word) << 32) | static_cast<unsigned>(g);
                                } else {
                                    bad = HAV_ERR_RANGE;
                                    ok = false;
                                }
                            }
                            int r = -2;
                            bool nw = false;
                            if (ok) r = smem_insert<kSelSlots>(skey, key, &nw);
                            const int pos = warp_append(r >= 0 && nw, &st.list_n);
                            if (pos >= 0) list[pos] = static_cast<unsigned short>(r);
                            if (r >= 0) {
                                atomicMin(sval + r, packed);
                            } else if (r == -1) {  // block table saturated: straight to the global table
                                bool fr;
                                const long long slot = find_or_insert(T, cap, key, &fr);
                                if (slot < 0) bad = HAV_ERR_TABLE_FULL;
                                else global_min(key, slot, fr, packed);
                            }
                        }
                    }
                    __syncthreads();
                    const int nl = static_cast<int>(st.list_n);
                    // owned voxels first: listed for the classification, counted here;
                    // the other keys are packed into a second list for the global table
                    const unsigned short* gl = list;
                    int ng = nl;
                    if (owning) {
                        unsigned short* glist = list + kSelSlots;
                        for (int k0 = tid - lane; k0 < nl; k0 += kThreads) {  // warp-uniform
                            const int k = k0 + lane;
                            const int si = (k < nl) ? static_cast<int>(list[k]) : 0;
                            const unsigned long long key = (k < nl) ? skey[si] : kEmptyKey;
                            const bool own = key != kEmptyKey &&
                                             voxel_owned(key, G, st.own_mn[li], st.own_k[li], st.own_lo[li],
                                                         st.own_hi[li]);
                            const int opos = warp_append(own, &st.rest_n);
                            if (opos >= 0) {
                                const unsigned long long h = priority(key);
                                olist[opos].h = h;
                                olist[opos].g = static_cast<uint32_t>(sval[si] & 0xffffffffull);
                                ++first;
                                atomicAdd(&st.bh[h >> (64 - kHistBits)], 1u);
                            }
                            const int gpos = warp_append(key != kEmptyKey && !own, &st.gl_n);
                            if (gpos >= 0) glist[gpos] = static_cast<unsigned short>(si);
                        }
                        __syncthreads();
                        gl = glist;
                        ng = static_cast<int>(st.gl_n);
                    }
                    for (int k0 = tid - lane; k0 < ng; k0 += kProbes * kThreads) {  // warp-uniform
                        unsigned long long key[kProbes];
                        unsigned long long* Tp[kProbes];
                        long long slot[kProbes];
                        bool fr[kProbes];
                        int sidx[kProbes];
#pragma unroll
                        for (int u = 0; u < kProbes; ++u) {
                            const int k = k0 + lane + u * kThreads;
                            sidx[u] = (k < ng) ? static_cast<int>(gl[k]) : 0;
                            key[u] = (k < ng) ? skey[sidx[u]] : kEmptyKey;
                            Tp[u] = T;
                        }
                        find_or_insert_batch<kProbes>(Tp, cap, key, slot, fr);
#pragma unroll
                        for (int u = 0; u < kProbes; ++u) {
                            const bool ok = key[u] != kEmptyKey && slot[u] >= 0;
                            if (key[u] != kEmptyKey && slot[u] < 0) bad = HAV_ERR_TABLE_FULL;
                            // a fresh insert (a voxel no count pass put in this table) is
                            // logged, warp-aggregated
                            const int pos = warp_append(ok && fr[u], &st.dcnt[sel][li][sc]);
                            if (pos >= 0)
                                d.dirty[sel][sc * dstride + a + pos] =
                                    static_cast<uint32_t>(sc * tstride + st.tab_off[s] + slot[u]);
                            if (ok) global_min(key[u], slot[u], false, sval[sidx[u]]);
                        }
                    }
                    if (bad) seg_error(d, s, bad);
                    const unsigned total = block_sum(first, st.scan_u);  // (its barriers order bh)
                    for (int k = tid; k < kHistBins; k += kThreads)
                        if (st.bh[k]) atomicAdd(&hist[static_cast<long long>(s) * kHistBins + k], st.bh[k]);
                    if (tid == 0) st.ocnt[li] = owning ? static_cast<int>(st.rest_n) : 0;
                    if (tid == 0 && total) atomicAdd(&ls[s].kstar, total);
                }
            }
            if (!grid_sync(d, nb, st, TAG(3, j, l, 0))) return;

            // ------------------------------------------- cut-off: classify
            if (tid < S) {
                st.kstar[tid] = static_cast<int>(ld_volatile(reinterpret_cast<const int*>(&ls[tid].kstar)));
                if (blockIdx.x == 0) {
                    hav_layer_trace* tr = d.tr + (static_cast<long long>(j) * S + tid) * kMaxLayers + l;
                    tr->k_star = st.kstar[tid];
                    tr->accepted = (st.flags[tid] & F_ACCEPT) ? 1 : 0;
                    tr->s_star = (st.flags[tid] & F_ACTIVE) ? st.s_star[tid] : 0.0f;
                }
            }
            if (tid == 0) st.cut_seg = -1;
            __syncthreads();
            {
                int li = 0;
                for (int it = blockIdx.x; it < st.items_total; it += nb, ++li) {
                    int a, b;
                    const int s = item_range(st, S, it, &a, &b);
                    if (!(st.flags[s] & F_ACTIVE)) continue;
                    const bool cut = st.kstar[s] > st.ml[s];
                    if (cut && st.cut_seg != s) {
                        // boundary bin: smallest b with (voxels in bins <= b) >= m_l
                        const uint32_t* h = hist + static_cast<long long>(s) * kHistBins;
                        constexpr int kPer = kHistBins / kThreads;
                        int mine[kPer];
                        int sum = 0;
#pragma unroll
                        for (int k = 0; k < kPer; ++k) {
                            mine[k] = static_cast<int>(h[kPer * tid + k]);
                            sum += mine[k];
                        }
                        int tot;
                        int before = block_excl_scan<int>(sum, &tot, st.scan_i);
                        const int need = st.ml[s];
#pragma unroll
                        for (int k = 0; k < kPer; ++k) {
                            if (before < need && before + mine[k] >= need) {
                                st.cut_bin = kPer * tid + k;
                                st.cut_below = before;
                            }
                            before += mine[k];
                        }
                        __syncthreads();
                        if (tid == 0) {
                            st.cut_seg = s;
                            ls[s].bin = st.cut_bin;
                            ls[s].below = static_cast<uint32_t>(st.cut_below);
                        }
                        __syncthreads();
                    }
                    const int sel = st.sel[s];
                    const int sc = st.sel_cand[s];
                    const int c = st.dcnt[sel][li][sc];
                    const uint32_t* lg = d.dirty[sel] + sc * dstride + a;
                    const long long voff = sc * tstride;
                    const long long C = 1ll << st.cap_log2[s];
                    const int bin = st.cut_bin;
                    for (int k = tid; k < c; k += kThreads) {
                        const uint32_t gs = lg[k];
                        const unsigned long long v = d.tv[gs - voff];
                        if (v == kEmptyVal) continue;
                        const int g = static_cast<int>(v & 0xffffffffull);
                        if (!cut) {
                            mark_taken(taken, ord, d.posof, g);
                            continue;
                        }
                        const unsigned long long h = priority(d.tk[sel][gs]);
                        const int hb = static_cast<int>(h >> (64 - kHistBits));
                        if (hb < bin) {
                            mark_taken(taken, ord, d.posof, g);
                        } else if (hb == bin) {
                            const uint32_t ci = atomicAdd(&ls[s].cand, 1u);
                            if (static_cast<long long>(ci) < (C >> 1)) {
                                Cand* cd = d.cand + st.cand_off[s] + ci;
                                cd->h = h;
                                cd->g = static_cast<uint32_t>(g);
                            } else {
                                seg_error(d, s, HAV_ERR_TABLE_FULL);
                            }
                        }
                    }
                    // the voxels the selection kept out of the table (owned whole)
                    const int oc = st.ocnt[li];
                    const Cand* ol = reinterpret_cast<const Cand*>(d.ord[(j + 1) & 1]) + a;
                    for (int k = tid; k < oc; k += kThreads) {
                        const unsigned long long h = ol[k].h;
                        const int g = static_cast<int>(ol[k].g);
                        const int hb = static_cast<int>(h >> (64 - kHistBits));
                        if (!cut || hb < bin) {
                            mark_taken(taken, ord, d.posof, g);
                        } else if (hb == bin) {
                            const uint32_t ci = atomicAdd(&ls[s].cand, 1u);
                            if (static_cast<long long>(ci) < (C >> 1)) {
                                Cand* cd = d.cand + st.cand_off[s] + ci;
                                cd->h = h;
                                cd->g = static_cast<uint32_t>(g);
                            } else {
                                seg_error(d, s, HAV_ERR_TABLE_FULL);
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            if (!grid_sync(d, nb, st, TAG(4, j, l, 0))) return;

            // --------------- cut-off: resolve; shortfall count; clean the tables
            {
                int c = 0;
                if (tid < S && (st.flags[tid] & F_ACTIVE) && st.kstar[tid] > st.ml[tid]) {
                    c = static_cast<int>(ld_volatile(reinterpret_cast<const int*>(&ls[tid].cand)));
                    // only the first C/2 were stored (the rest reported a full table)
                    const int cmax = 1 << (st.cap_log2[tid] - 1);
                    if (c > cmax) c = cmax;
                }
                int ctot;
                const int cpre = block_excl_scan<int>(tid < S ? c : 0, &ctot, st.scan_i);
                if (tid < S) st.cprefix[tid] = cpre;
                if (tid == 0) st.cprefix[S] = ctot;
                __syncthreads();
                for (long long w = gtid; w < ctot; w += gstride) {
                    const int s = find_seg(st.cprefix, S, w);
                    const int jdx = static_cast<int>(w) - st.cprefix[s];
                    const int cs = st.cprefix[s + 1] - st.cprefix[s];
                    const Cand* base = d.cand + st.cand_off[s];
                    const unsigned long long hj = base[jdx].h;
                    int rank = 0;
                    for (int k = 0; k < cs; ++k) rank += (base[k].h < hj) ? 1 : 0;
                    const int r = st.ml[s] - static_cast<int>(ls[s].below);
                    if (rank < r) mark_taken(taken, ord, d.posof, static_cast<int>(base[jdx].g));
                }
                int sf = 0;
                if (tid < S && (st.flags[tid] & F_ACTIVE) && st.kstar[tid] < st.ml[tid]) sf = 1;
                if (tid == 0) st.any = 0;
                __syncthreads();
                if (sf) st.any = 1;
                __syncthreads();
                if (st.any) {
                    for (int s = 0; s < S; ++s) {
                        if (!((st.flags[s] & F_ACTIVE) && st.kstar[s] < st.ml[s])) continue;
                        const int n = st.n[s];
                        const int a = static_cast<int>(st.off[s] + static_cast<long long>(n) * blockIdx.x / nb);
                        const int b = static_cast<int>(st.off[s] + static_cast<long long>(n) * (blockIdx.x + 1) / nb);
                        int cnt = 0;
                        for (int g = a + tid; g < b; g += kThreads) cnt += is_taken(taken, g) ? 0 : 1;
                        int tot;
                        block_excl_scan<int>(cnt, &tot, st.scan_i);
                        if (tid == 0) d.psf[static_cast<long long>(s) * kMaxBlocks + blockIdx.x] = tot;
                    }
                }
                // every candidate table of every set, and the value table, back to
                // empty, slot by slot
                int li = 0;
                for (int it = blockIdx.x; it < st.items_total; it += nb, ++li) {
                    int a, b;
                    const int s = item_range(st, S, it, &a, &b);
                    const bool act = (st.flags[s] & F_ACTIVE) != 0;
                    for (int t = 0; t < kTableSets; ++t) {
                        for (int cd = 0; cd < ncand; ++cd) {
                            const int c2 = st.dcnt[t][li][cd];
                            const bool v_too = act && st.sel[s] == t && st.sel_cand[s] == cd;
                            const uint32_t* lg = d.dirty[t] + cd * dstride + a;
                            const long long voff = cd * tstride;
                            for (int k = tid; k < c2; k += kThreads) {
                                const uint32_t gs = lg[k];
                                d.tk[t][gs] = kEmptyKey;
                                if (v_too) d.tv[gs - voff] = kEmptyVal;
                            }
                        }
                    }
                }
                __syncthreads();
                for (int k = tid; k < kTableSets * kLocalItems * kMaxCand; k += kThreads)
                    (&st.dcnt[0][0][0])[k] = 0;
                if (l + 1 < P.layers) clear_layer_state(d, S, q ^ 1, gtid, gstride);
                if (!grid_sync(d, nb, st, TAG(5, j, l, 0))) return;
                if (j + 1 == P.L && l + 1 == P.layers && blockIdx.x == 0 && tid == 0)
                    *(volatile unsigned*)d.clean = 1u;  // every table slot is empty again
            }
            // ------------------------------------------------ shortfall fill
            if (st.any) {
                for (int s = 0; s < S; ++s) {
                    if (!((st.flags[s] & F_ACTIVE) && st.kstar[s] < st.ml[s])) continue;
                    int pre = 0;
                    for (int b = tid; b < static_cast<int>(blockIdx.x); b += kThreads)
                        pre += d.psf[static_cast<long long>(s) * kMaxBlocks + b];
                    int tot;
                    block_excl_scan<int>(pre, &tot, st.scan_i);
                    int budget = (st.ml[s] - st.kstar[s]) - tot;
                    const int n = st.n[s];
                    const int a = static_cast<int>(st.off[s] + static_cast<long long>(n) * blockIdx.x / nb);
                    const int b = static_cast<int>(st.off[s] + static_cast<long long>(n) * (blockIdx.x + 1) / nb);
                    for (int g0 = a; g0 < b && budget > 0; g0 += kThreads) {
                        const int g = g0 + tid;
                        const int free_pt = (g < b && !is_taken(taken, g)) ? 1 : 0;
                        int chunk;
                        const int rank = block_excl_scan<int>(free_pt, &chunk, st.scan_i);
                        if (free_pt && rank < budget) mark_taken(taken, ord, d.posof, g);
                        budget -= chunk;
                    }
                }
                if (!grid_sync(d, nb, st, TAG(6, j, l, 0))) return;
            }
        }

        // ---------------------------------------------------- compaction
        // Segments in error take their first m points, so every other
        // segment's output positions stay exact.
        if (tid < S) st.err[tid] = ld_volatile(&d.sh[tid].status);
        if (tid == 0) st.any = 0;
        __syncthreads();
        if (tid < S && st.err[tid]) st.any = 1;
        __syncthreads();
        const bool any_err = st.any != 0;
        const bool last_level = (j + 1 == P.L);
        const long long W = (NL + 31) / 32;
        const long long wb = W * blockIdx.x / nb;
        const long long we = W * (blockIdx.x + 1) / nb;
        auto eff_word = [&](long long w) -> uint32_t {
            uint32_t bits = taken[w];
            const long long g0 = w * 32;
            if (g0 + 32 > NL) bits &= (NL - g0 >= 32) ? 0xffffffffu : ((1u << (NL - g0)) - 1u);
            if (any_err) {
                for (int k = 0; k < 32 && g0 + k < NL; ++k) {
                    const int s = find_seg(st.off, S, g0 + k);
                    if (st.err[s]) {
                        const bool on = (g0 + k - st.off[s]) < st.m[s];
                        bits = on ? (bits | (1u << k)) : (bits & ~(1u << k));
                    }
                }
            }
            return bits;
        };
        auto eff_taken = [&](int s, long long g) -> bool {
            if (st.err[s]) return (g - st.off[s]) < st.m[s];
            return is_taken(taken, g);
        };
        {
            // level j+1 accumulates its bounding box in the parity level j-1 used
            if (blockIdx.x == 0 && tid < S)
                for (int a = 0; a < 6; ++a) d.sh[tid].bbox[(j + 1) & 1][a] = 0u;
            // ascending order: per-word block-local prefixes and the block total
            unsigned run = 0;
            for (long long w0 = wb; w0 < we; w0 += kThreads) {
                const long long w = w0 + tid;
                const unsigned c = (w < we) ? __popc(eff_word(w)) : 0u;
                unsigned tot;
                const unsigned before = block_excl_scan<unsigned>(c, &tot, st.scan_u);
                if (w < we) d.wpre[w] = run + before;
                run += tot;
            }
            if (tid == 0) d.pcmp[blockIdx.x] = static_cast<int32_t>(run);
            // processing order: kept points per owned item
            if (!last_level) {
                for (int it = blockIdx.x; it < st.items_total; it += nb) {
                    int a, b;
                    const int s = item_range(st, S, it, &a, &b);
                    unsigned c = 0;
                    for (int i = a + tid; i < b; i += kThreads)
                        c += eff_taken(s, level_index(ord[i].w)) ? 1u : 0u;
                    const unsigned tot = block_sum(c, st.scan_u);
                    if (tid == 0) d.pitem[it] = static_cast<int32_t>(tot);
                }
            }
            if (!grid_sync(d, nb, st, TAG(7, j, 0, 0))) return;
        }
        {
            // prefixes of every block's count and (next level) every item's count
            if (tid == 0) st.set_clean = 0;
            int* pre_blk = reinterpret_cast<int*>(dyn);
            int* pre_item = pre_blk + kMaxBlocks;
            {
                int run = 0;
                for (int b0 = 0; b0 < static_cast<int>(nb); b0 += kThreads) {
                    const int b = b0 + tid;
                    const int c = (b < static_cast<int>(nb)) ? d.pcmp[b] : 0;
                    int tot;
                    const int before = block_excl_scan<int>(c, &tot, st.scan_i);
                    if (b < static_cast<int>(nb)) pre_blk[b] = run + before;
                    run += tot;
                }
                if (!last_level) {
                    run = 0;
                    for (int i0 = 0; i0 < st.items_total; i0 += kThreads) {
                        const int it = i0 + tid;
                        const int c = (it < st.items_total) ? d.pitem[it] : 0;
                        int tot;
                        const int before = block_excl_scan<int>(c, &tot, st.scan_i);
                        if (it < st.items_total) pre_item[it] = run + before;
                        run += tot;
                    }
                }
                __syncthreads();
            }
            // ascending position of a kept level index
            auto pos_asc = [&](long long g) -> long long {
                const long long w = g >> 5;
                long long b = (w * static_cast<long long>(nb)) / W;
                while (b + 1 < static_cast<long long>(nb) && W * (b + 1) / nb <= w) ++b;
                while (b > 0 && W * b / nb > w) --b;
                const uint32_t below = eff_word(w) & ((1u << (g & 31)) - 1u);
                return static_cast<long long>(pre_blk[b]) + d.wpre[w] + __popc(below);
            };
            int32_t* out = P.out[j];
            int32_t* orig_out = d.orig[j & 1];
            for (long long w = wb + tid; w < we; w += kThreads) {
                uint32_t bits = eff_word(w);
                long long pos = static_cast<long long>(pre_blk[blockIdx.x]) + d.wpre[w];
                while (bits) {
                    const int k = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const long long g = w * 32 + k;
                    if (pos >= st.m_total) {  // cannot happen: every segment takes exactly m
                        atomicCAS(&d.gh->status, 0, static_cast<int>(HAV_ERR_TABLE_FULL));
                        break;
                    }
                    const int s = find_seg(st.off, S, g);
                    const int32_t oi = orig_in ? orig_in[g] : static_cast<int32_t>(g - st.off[s]);
                    out[pos] = oi;
                    if (!last_level || P.keep_orig) orig_out[pos] = oi;
                    ++pos;
                }
            }
            if (!last_level) {
                float4* ord_out = d.ord[(j + 1) & 1];
                const int npar = (j + 1) & 1;
                for (int it = blockIdx.x; it < st.items_total; it += nb) {
                    int a, b;
                    const int s = item_range(st, S, it, &a, &b);
                    long long base = pre_item[it];
                    // the next level's bounding box over the points kept here
                    float mnv[3] = {INFINITY, INFINITY, INFINITY}, mxv[3] = {-INFINITY, -INFINITY, -INFINITY};
                    for (int i0 = a; i0 < b; i0 += kThreads) {
                        const int i = i0 + tid;
                        float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        int keep = 0;
                        if (i < b) {
                            q4 = ord[i];
                            keep = eff_taken(s, level_index(q4.w)) ? 1 : 0;
                        }
                        int tot;
                        const int rank = block_excl_scan<int>(keep, &tot, st.scan_i);
                        if (keep) {
                            const long long pos2 = base + rank;
                            const long long ng = pos_asc(level_index(q4.w));
                            if (pos2 < st.m_total && ng < st.m_total) {
                                ord_out[pos2] = make_float4(q4.x, q4.y, q4.z, __int_as_float(static_cast<int>(ng)));
                                d.posof[ng] = static_cast<int32_t>(pos2);
                            }
                            mnv[0] = fminf(mnv[0], q4.x);
                            mnv[1] = fminf(mnv[1], q4.y);
                            mnv[2] = fminf(mnv[2], q4.z);
                            mxv[0] = fmaxf(mxv[0], q4.x);
                            mxv[1] = fmaxf(mxv[1], q4.y);
                            mxv[2] = fmaxf(mxv[2], q4.z);
                        }
                        base += tot;
                    }
#pragma unroll
                    for (int a3 = 0; a3 < 3; ++a3) {
                        for (int o = 16; o > 0; o >>= 1) {
                            mnv[a3] = fminf(mnv[a3], __shfl_xor_sync(0xffffffffu, mnv[a3], o));
                            mxv[a3] = fmaxf(mxv[a3], __shfl_xor_sync(0xffffffffu, mxv[a3], o));
                        }
                    }
                    if ((tid & 31) == 0) {
                        for (int a3 = 0; a3 < 3; ++a3) {
                            st.redf[a3][tid >> 5] = mnv[a3];
                            st.redf[3 + a3][tid >> 5] = mxv[a3];
                        }
                    }
                    __syncthreads();
                    if (tid < 6) {
                        float r = st.redf[tid][0];
                        for (int w = 1; w < kThreads / 32; ++w)
                            r = (tid < 3) ? fminf(r, st.redf[tid][w]) : fmaxf(r, st.redf[tid][w]);
                        if (isfinite(r)) {
                            if (tid < 3) atomicMax(&d.sh[s].bbox[npar][tid], ~enc_f(r));
                            else atomicMax(&d.sh[s].bbox[npar][tid], enc_f(r));
                        }
                    }
                    __syncthreads();
                }
                // the next level's taken mask, layer states and search prefix
                fill<uint32_t>(d.taken[npar], st.m_total / 32 + 1, 0u, gtid, gstride);
                fill<int32_t>(d.prefix, static_cast<long long>(S) * kMaxIters, -1, gtid, gstride);
                clear_layer_state(d, S, 0, gtid, gstride);
                clear_layer_state(d, S, 1, gtid, gstride);
                if (!grid_sync(d, nb, st, TAG(8, j, 0, 0))) return;
            }
        }
    }
}

// ------------------------------------------------------- Cnt test hook
namespace {

__global__ void bbox_kernel(const float* pts, long long n, uint32_t* enc6) {
    float mnv[3] = {INFINITY, INFINITY, INFINITY}, mxv[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long long g = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; g < n;
         g += static_cast<long long>(gridDim.x) * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            const float x = pts[3 * g + a];
            if (!isfinite(x)) {
                enc6[6] = 1;
                continue;
            }
            mnv[a] = fminf(mnv[a], x);
            mxv[a] = fmaxf(mxv[a], x);
        }
    }
    for (int a = 0; a < 3; ++a) {
        if (isfinite(mnv[a])) atomicMax(&enc6[a], ~enc_f(mnv[a]));
        if (isfinite(mxv[a])) atomicMax(&enc6[3 + a], enc_f(mxv[a]));
    }
}

__global__ void count_kernel(const float* pts, long long n, float s, float r0, float r1, float r2,
                             const uint32_t* enc6, unsigned long long* T, int cap_log2,
                             unsigned long long* K, int* err) {
    __shared__ Grid g;
    __shared__ int ok;
    if (threadIdx.x == 0) {
        float mn[3], r[3] = {r0, r1, r2};
        for (int a = 0; a < 3; ++a) mn[a] = dec_f(~enc6[a]);
        ok = make_grid(s, r, mn, &g);
        if (!ok) atomicExch(err, static_cast<int>(HAV_ERR_RANGE));
    }
    __syncthreads();
    if (!ok) return;
    unsigned long long local = 0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        float p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]}, f[3];
        unsigned long long key;
        if (!cell_key(p, g, &key, f)) {
            atomicExch(err, static_cast<int>(HAV_ERR_RANGE));
            continue;
        }
        bool fr;
        if (find_or_insert(T, cap_log2, key, &fr) < 0) atomicExch(err, static_cast<int>(HAV_ERR_TABLE_FULL));
        local += fr ? 1 : 0;
    }
    if (local) atomicAdd(K, local);
}

__global__ void fill_u64(unsigned long long* p, long long n, unsigned long long v) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        p[i] = v;
}

}  // namespace

namespace {
// The instantiations, by pass shape: (points loaded ahead, probes in flight).
using ChainFn = void (*)(const Plan);
const ChainFn kChain[kPassShapes] = {hav_chain_kernel<2, 1>, hav_chain_kernel<1, 1>, hav_chain_kernel<2, 2>,
                                     hav_chain_kernel<4, 1>};
}  // namespace

int max_coresident_blocks(int device) {
    int sms = 0, per_sm = 0, least = 1 << 30;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    for (int k = 0; k < kPassShapes; ++k) {  // every shape must fit the same grid
        if (cudaFuncSetAttribute(kChain[k], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kDynSmem)) != cudaSuccess)
            return -1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kChain[k], kThreads, kDynSmem) != cudaSuccess)
            return -1;
        if (per_sm < least) least = per_sm;
    }
    long long nb = static_cast<long long>(sms) * least;
    if (nb > kMaxBlocks) nb = kMaxBlocks;
    return static_cast<int>(nb);
}

int launch_chain(const Plan& plan, cudaStream_t stream) {
    if (plan.pass_shape < 0 || plan.pass_shape >= kPassShapes) return -1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(plan.nblocks));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kDynSmem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kChain[plan.pass_shape], plan) == cudaSuccess ? 1 : -1;
}

int count_voxels(const float* points, int64_t n, float s, const float aspect[3], unsigned char* ws,
                 const Layout& lay, int64_t* K, int* launched, cudaStream_t stream) {
    // scratch: the level-0 key table; it is left dirty, so the next sampler
    // call on this workspace starts with a full clear
    int cap_log2 = kMinCapLog2;
    while ((1ll << cap_log2) < 2 * n) ++cap_log2;
    if ((1ll << cap_log2) > lay.tab_slots) return HAV_ERR_NOMEM;
    unsigned long long* T = reinterpret_cast<unsigned long long*>(ws + lay.tabk[0]);
    unsigned char* scratch = ws + lay.partial_cmp;  // 8 KB: bbox codes, K, error
    uint32_t* enc6 = reinterpret_cast<uint32_t*>(scratch);
    unsigned long long* dK = reinterpret_cast<unsigned long long*>(scratch + 64);
    int* derr = reinterpret_cast<int*>(scratch + 128);
    if (cudaMemsetAsync(ws + lay.clean, 0, sizeof(unsigned), stream) != cudaSuccess) return HAV_ERR_CUDA;
    if (cudaMemsetAsync(scratch, 0, 256, stream) != cudaSuccess) return HAV_ERR_CUDA;
    fill_u64<<<1024, 256, 0, stream>>>(T, 1ll << cap_log2, kEmptyKey);
    bbox_kernel<<<1024, 256, 0, stream>>>(points, n, enc6);
    count_kernel<<<1024, 256, 0, stream>>>(points, n, s, aspect[0], aspect[1], aspect[2], enc6, T, cap_log2, dK,
                                           derr);
    if (cudaGetLastError() != cudaSuccess) return HAV_ERR_CUDA;
    *launched = 3;
    unsigned long long hK = 0;
    int herr = 0;
    uint32_t henc[7];
    if (cudaMemcpyAsync(&hK, dK, 8, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return HAV_ERR_CUDA;
    if (cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return HAV_ERR_CUDA;
    if (cudaMemcpyAsync(henc, enc6, 28, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return HAV_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return HAV_ERR_CUDA;
    if (henc[6]) return HAV_ERR_NONFINITE;
    if (herr) return herr;
    *K = static_cast<int64_t>(hK);
    return HAV_OK;
}

}  // namespace havk
