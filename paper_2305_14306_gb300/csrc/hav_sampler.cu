// HAVSampler hot path for sm_103a: one persistent cooperative kernel runs a
// whole batched level chain.
//
// Per level j, for every segment (cloud) of the batch at once:
//   bbox   : per-axis min/max and finiteness (bracket of the Section 3.3 search)
//   layer l = 1..k (Section 3.4, Eq. 3):
//     pass p : Cnt(P_l, s_p) by open-addressed insertion of Eq. 2 voxel keys
//              (atomicCAS), counted per work tile; the bisection of Section 3.3
//              is decided redundantly and identically by every block from the
//              pass counts, so no block waits for a leader
//     select : centre-closest representative per voxel at s* by a packed 64-bit
//              atomicMin of (squared distance bits, point index) (Section 3.2);
//              first touch of a slot feeds the cut-off histogram
//     cut    : voxels below the boundary priority bin are taken, the boundary
//              bin's voxels are ranked exactly (or the shortfall is filled)
//   compact: taken bitmask -> ascending indices, composed to the segment's
//            original cloud, plus the gather that feeds level j+1
// Phases are separated by a grid barrier whose wait is bounded in time; a
// timeout sets an abort flag that every block honours, and the host reads
// HAV_ERR_TIMEOUT.  Every loop in this file has a fixed bound.
//
// Arithmetic: voxel keys and distances use explicitly rounded binary32
// intrinsics (__fdiv_rn, __fmul_rn, __fadd_rn, __fsub_rn), so the compiler
// cannot contract or reassociate them.

#include <cuda_runtime.h>

#include "hav_internal.h"

namespace havk {
namespace {

#define TAG(phase, level, layer, pass) \
    ((static_cast<unsigned>(phase) << 24) | (static_cast<unsigned>(level) << 16) | \
     (static_cast<unsigned>(layer) << 8) | static_cast<unsigned>(pass))

constexpr unsigned long long kSpinNs = 2000000000ull;  // 2 s per barrier wait
constexpr unsigned int kSpinIters = 1u << 26;
static_assert(kHistBins % kThreads == 0, "the cut-off scan gives each thread whole bins");

// ------------------------------------------------------------------ memory ops
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_strong64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Monotone map of binary32 onto uint32 (larger float -> larger code).
__device__ __forceinline__ uint32_t enc_f(float x) {
    uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float dec_f(uint32_t e) {
    return __uint_as_float((e & 0x80000000u) ? (e & 0x7fffffffu) : ~e);
}

// -------------------------------------------------------------------- hashing
// Slot hash: a 64-bit mixer (xor-shift / multiply rounds), top bits index the table.
__device__ __forceinline__ unsigned long long slot_mix(unsigned long long k) {
    k ^= k >> 32;
    k *= 0xd6e8feb86659fd93ull;
    k ^= k >> 32;
    k *= 0xd6e8feb86659fd93ull;
    k ^= k >> 32;
    return k;
}
// Cut-off priority: the SplitMix64 output finaliser (Steele, Lea, Flood 2014).
__device__ __forceinline__ unsigned long long priority(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------ Eq. 2 voxel keys
struct Grid {
    float v[3];
    long long fmin[3];
};

__device__ __forceinline__ bool floor_div(float x, float v, long long* F, float* f) {
    float q = __fdiv_rn(x, v);
    float fl = floorf(q);
    if (!(fabsf(fl) < 4.6e18f)) return false;
    *F = static_cast<long long>(fl);
    *f = fl;
    return true;
}

__device__ bool make_grid(float s, const float r[3], const float mn[3], Grid* g) {
    for (int a = 0; a < 3; ++a) {
        float v = __fmul_rn(s, r[a]);
        if (!(v > 0.0f) || !isfinite(v)) return false;
        g->v[a] = v;
        float f;
        if (!floor_div(mn[a], v, &g->fmin[a], &f)) return false;
    }
    return true;
}

// key = u_x | u_y << 21 | u_z << 42 with u = floor(x / v) - floor(min / v).
__device__ __forceinline__ bool cell_key(const float p[3], const Grid& g,
                                         unsigned long long* key, float f[3]) {
    unsigned long long k = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        long long F;
        if (!floor_div(p[a], g.v[a], &F, &f[a])) return false;
        long long u = F - g.fmin[a];
        if (u < 0 || u >= (1ll << 21)) return false;
        k |= static_cast<unsigned long long>(u) << (21 * a);
    }
    *key = k;
    return true;
}

// Section 3.2: squared distance to the voxel centre v * (g + 0.5).
__device__ __forceinline__ float centre_d2(const float p[3], const Grid& g, const float f[3]) {
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float c = __fmul_rn(g.v[a], __fadd_rn(f[a], 0.5f));
        d[a] = __fsub_rn(p[a], c);
    }
    float xy = __fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1]));
    return __fadd_rn(xy, __fmul_rn(d[2], d[2]));
}

// Find or insert `key` by linear probing; *fresh tells whether this call
// inserted it.  Returns the slot, or -1 after a full sweep (table full).
__device__ __forceinline__ long long find_or_insert(unsigned long long* T, int cap_log2,
                                                    unsigned long long key, bool* fresh) {
    const unsigned long long mask = (1ull << cap_log2) - 1;
    unsigned long long slot = slot_mix(key) >> (64 - cap_log2);
    *fresh = false;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        unsigned long long cur = ld_strong64(T + slot);
        if (cur == key) return static_cast<long long>(slot);
        if (cur == kEmptyKey) {
            unsigned long long prev = atomicCAS(T + slot, kEmptyKey, key);
            if (prev == kEmptyKey) {
                *fresh = true;
                return static_cast<long long>(slot);
            }
            if (prev == key) return static_cast<long long>(slot);
        }
        slot = (slot + 1) & mask;
    }
    return -1;
}

// Eq. 3 budget of layer l (0-based).
__device__ __forceinline__ long long layer_budget(long long m, int layers, int ratio, int l) {
    long long S = 0, pw = 1;
    for (int i = 0; i < layers; ++i) {
        S += pw;
        pw *= ratio;
    }
    long long used = 0;
    pw = 1;
    for (int i = 0; i < layers - 1; ++i) {
        long long mi = m * pw / S;
        if (i == l) return mi;
        used += mi;
        pw *= ratio;
    }
    return m - used;
}

// ------------------------------------------------------------ block helpers
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan over the block; *total receives the sum.  All threads call it.
template <typename T>
__device__ T block_excl_scan(T v, T* total, T* scratch /* >= 32 */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int kWarps = kThreads / 32;
    T x = warp_incl_scan(v);
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T w = (lane < kWarps) ? scratch[lane] : T(0);
        w = warp_incl_scan(w);
        scratch[lane] = w;
    }
    __syncthreads();
    T before = wid ? scratch[wid - 1] : T(0);
    *total = scratch[kWarps - 1];
    __syncthreads();
    return before + x - v;
}

// Grid barrier with a bounded wait.  Arrival is a release reduction on a
// counter that only grows within a launch (zeroed by the host before it);
// barrier number e of the launch completes when the counter reaches
// e * nblocks, so no block has to act as the last arriver.  Returns false
// (for the whole block) when this or another block gave up; the caller then
// leaves the kernel.
__device__ bool grid_sync_impl(Barrier* bar, GlobalHdr* gh, unsigned nblocks, unsigned* epoch,
                               int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int fail = 0;
        const unsigned target = (*epoch + 1u) * nblocks;
        *epoch += 1u;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->count) : "memory");
        const unsigned long long t0 = globaltimer();
        for (unsigned it = 0;; ++it) {
            if (ld_acquire(&bar->count) >= target) break;
            if ((it & 31) == 31) {
                if (ld_volatile(&gh->abort) || it > kSpinIters || globaltimer() - t0 > kSpinNs) {
                    fail = 1;
                    break;
                }
            }
            if (it > 64) __nanosleep(32);
        }
        if (fail) {
            atomicExch(&gh->abort, 1);
            atomicCAS(&gh->status, 0, static_cast<int>(HAV_ERR_TIMEOUT));
        }
        __threadfence();
        *s_flag = fail | ld_volatile(&gh->abort);
    }
    __syncthreads();
    return *s_flag == 0;
}

// ------------------------------------------------------------------ state
enum : int { F_ACTIVE = 1, F_SEARCH = 2, F_ACCEPT = 4 };

struct Smem {
    // level layout
    long long off[kMaxSegments + 1];
    long long tab_off[kMaxSegments];
    long long cand_off[kMaxSegments];
    int n[kMaxSegments];
    int m[kMaxSegments];
    int cap_log2[kMaxSegments];
    int tile0[kMaxSegments + 1];
    int stile0[kMaxSegments + 1];
    int err[kMaxSegments];
    // bracket
    float mn[kMaxSegments][3];
    float s_hi[kMaxSegments];
    // controller of the current layer
    float lo[kMaxSegments], hi[kMaxSegments], s_cur[kMaxSegments], s_star[kMaxSegments];
    Grid grid[kMaxSegments];
    int ml[kMaxSegments];
    int kmax[kMaxSegments];
    int iters[kMaxSegments];
    int flags[kMaxSegments];
    int sel[kMaxSegments];
    int kstar[kMaxSegments];
    int cprefix[kMaxSegments + 1];
    // scratch
    long long scan_ll[32];
    int scan_i[32];
    float redf[6][32];
    unsigned epoch;
    int ntimes;
    int cut_seg;
    int cut_bin;
    int cut_below;
    int flag;
    int any;
    int tiles_total;
    int stiles_total;
    long long n_level;
    long long m_total;
};

struct Dev {
    Barrier* bar;
    GlobalHdr* gh;
    SegHdr* sh;
    LayerState* ls;       // [2][S]
    uint32_t* hist;       // [2][S][kHistBins]
    int32_t* psf;         // [S][kMaxBlocks]
    int32_t* pcmp;        // [kMaxBlocks]
    hav_layer_trace* tr;  // [L][S][kMaxLayers]
    float* pts[2];
    int32_t* orig[2];
    uint32_t* taken[2];
    unsigned long long* tk[2];
    unsigned long long* tv;
    Cand* cand;
    unsigned long long* ptimes;  // [2 * cap] (globaltimer ns, tag) pairs, or null
    int ptimes_cap;
};

// Barrier plus, when phase timing is on, a (time, tag) record from block 0.
// tag = phase << 24 | level << 16 | layer << 8 | pass.
__device__ __forceinline__ bool grid_sync(Dev& d, unsigned nblocks, Smem& st, unsigned tag) {
    const bool ok = grid_sync_impl(d.bar, d.gh, nblocks, &st.epoch, &st.flag);
    if (d.ptimes && blockIdx.x == 0 && threadIdx.x == 0 && st.ntimes < d.ptimes_cap) {
        d.ptimes[2 * st.ntimes] = globaltimer();
        d.ptimes[2 * st.ntimes + 1] = tag;
        st.ntimes += 1;
    }
    return ok;
}

__device__ __forceinline__ void seg_error(Dev& d, int s, int code) {
    atomicCAS(&d.sh[s].status, 0, code);
    atomicCAS(&d.gh->status, 0, code);
}

__device__ __forceinline__ int find_seg(const int* prefix, int S, int t) {
    // largest s with prefix[s] <= t (prefix has S+1 entries, prefix[0] = 0)
    int lo = 0, hi = S;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (prefix[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int find_seg_ll(const long long* prefix, int S, long long g) {
    int lo = 0, hi = S;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (prefix[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool is_taken(const uint32_t* tk, long long g) {
    return (tk[g >> 5] >> (g & 31)) & 1u;
}
__device__ __forceinline__ void set_taken(uint32_t* tk, long long g) {
    atomicOr(&tk[g >> 5], 1u << (g & 31));
}

__device__ __forceinline__ void load_point(const float* pts, long long g, float p[3]) {
    const float* q = pts + 3 * g;
    p[0] = q[0];
    p[1] = q[1];
    p[2] = q[2];
}

// Level layout of every segment, computed identically by every block.
__device__ void level_setup(const Plan& P, int j, Smem& st) {
    const int S = P.S;
    const int s = threadIdx.x;
    long long n = 0, C = 0, tiles = 0, stiles = 0;
    int lg = kMinCapLog2;
    if (s < S) {
        n = (j == 0) ? (P.off0[s + 1] - P.off0[s]) : P.m[j - 1][s];
        while ((1ll << lg) < 2 * n) ++lg;
        C = 1ll << lg;
        tiles = (n + kTile - 1) / kTile;
        stiles = (C + kSlotTile - 1) / kSlotTile;
        st.n[s] = static_cast<int>(n);
        st.m[s] = P.m[j][s];
        st.cap_log2[s] = lg;
    }
    long long tot;
    long long o = block_excl_scan<long long>(n, &tot, st.scan_ll);
    if (s < S) st.off[s] = o;
    if (s == 0) {
        st.off[S] = tot;
        st.n_level = tot;
    }
    o = block_excl_scan<long long>(s < S ? static_cast<long long>(P.m[j][s]) : 0ll, &tot, st.scan_ll);
    if (s == 0) st.m_total = tot;
    o = block_excl_scan<long long>(C, &tot, st.scan_ll);
    if (s < S) {
        st.tab_off[s] = o;
        st.cand_off[s] = o / 2;
    }
    o = block_excl_scan<long long>(tiles, &tot, st.scan_ll);
    if (s < S) st.tile0[s] = static_cast<int>(o);
    if (s == 0) {
        st.tile0[S] = static_cast<int>(tot);
        st.tiles_total = static_cast<int>(tot);
    }
    o = block_excl_scan<long long>(stiles, &tot, st.scan_ll);
    if (s < S) st.stile0[s] = static_cast<int>(o);
    if (s == 0) {
        st.stile0[S] = static_cast<int>(tot);
        st.stiles_total = static_cast<int>(tot);
    }
    __syncthreads();
}

// Grid-strided fill of [0, count) with a value.
template <typename T>
__device__ __forceinline__ void fill(T* p, long long count, T v, long long gtid, long long gstride) {
    for (long long i = gtid; i < count; i += gstride) p[i] = v;
}

// Table region of one segment (slots [tab_off, tab_off + C)).
__device__ __forceinline__ void clear_tables(Dev& d, const Smem& st, int S, bool k0, bool k1, bool v,
                                             long long gtid, long long gstride) {
    const long long total = st.tab_off[S - 1] + (1ll << st.cap_log2[S - 1]);
    if (k0) fill<unsigned long long>(d.tk[0], total, kEmptyKey, gtid, gstride);
    if (k1) fill<unsigned long long>(d.tk[1], total, kEmptyKey, gtid, gstride);
    if (v) fill<unsigned long long>(d.tv, total, kEmptyVal, gtid, gstride);
}

__device__ __forceinline__ void clear_layer_state(Dev& d, int S, int q, long long gtid, long long gstride) {
    LayerState* ls = d.ls + q * S;
    fill<uint32_t>(reinterpret_cast<uint32_t*>(ls), static_cast<long long>(S) * (sizeof(LayerState) / 4),
                   0u, gtid, gstride);
    fill<uint32_t>(d.hist + static_cast<long long>(q) * S * kHistBins,
                   static_cast<long long>(S) * kHistBins, 0u, gtid, gstride);
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) hav_chain_kernel(const __grid_constant__ Plan P) {
    __shared__ Smem st;
    const int S = P.S;
    const int tid = threadIdx.x;
    const long long gtid = static_cast<long long>(blockIdx.x) * kThreads + tid;
    const long long gstride = static_cast<long long>(P.nblocks) * kThreads;

    Dev d;
    unsigned char* ws = P.ws;
    d.bar = reinterpret_cast<Barrier*>(ws + P.lay.barrier);
    d.gh = reinterpret_cast<GlobalHdr*>(ws + P.lay.ghdr);
    d.sh = reinterpret_cast<SegHdr*>(ws + P.lay.seghdr);
    d.ls = reinterpret_cast<LayerState*>(ws + P.lay.lstate);
    d.hist = reinterpret_cast<uint32_t*>(ws + P.lay.hist);
    d.psf = reinterpret_cast<int32_t*>(ws + P.lay.partial_sf);
    d.pcmp = reinterpret_cast<int32_t*>(ws + P.lay.partial_cmp);
    d.tr = reinterpret_cast<hav_layer_trace*>(ws + P.lay.trace);
    for (int b = 0; b < 2; ++b) {
        d.pts[b] = reinterpret_cast<float*>(ws + P.lay.pts[b]);
        d.orig[b] = reinterpret_cast<int32_t*>(ws + P.lay.orig[b]);
        d.taken[b] = reinterpret_cast<uint32_t*>(ws + P.lay.taken[b]);
        d.tk[b] = reinterpret_cast<unsigned long long*>(ws + P.lay.tabk[b]);
    }
    d.tv = reinterpret_cast<unsigned long long*>(ws + P.lay.tabv);
    d.cand = reinterpret_cast<Cand*>(ws + P.lay.cand);
    d.ptimes = P.ptimes;
    d.ptimes_cap = P.ptimes_cap;
    if (tid == 0) {
        st.epoch = 0u;
        st.ntimes = 0;
        if (d.ptimes && blockIdx.x == 0) {
            d.ptimes[0] = globaltimer();
            d.ptimes[1] = 0;
            st.ntimes = 1;
        }
    }
    __syncthreads();

    for (int j = 0; j < P.L; ++j) {
        level_setup(P, j, st);
        const float* pts = (j == 0) ? P.points : d.pts[(j - 1) & 1];
        const int32_t* orig_in = (j == 0) ? nullptr : d.orig[(j - 1) & 1];
        uint32_t* taken = d.taken[j & 1];
        const long long NL = st.n_level;

        // ---------------------------------------------------- bbox + clears
        {
            const int par = j & 1;
            for (int t = blockIdx.x; t < st.tiles_total; t += P.nblocks) {
                const int s = find_seg(st.tile0, S, t);
                const long long g = st.off[s] + static_cast<long long>(t - st.tile0[s]) * kTile + tid;
                const bool in = g < st.off[s] + st.n[s];
                float mnv[3] = {INFINITY, INFINITY, INFINITY}, mxv[3] = {-INFINITY, -INFINITY, -INFINITY};
                int bad = 0;
                if (in) {
                    float p[3];
                    load_point(pts, g, p);
                    for (int a = 0; a < 3; ++a) {
                        if (!isfinite(p[a])) bad = 1;
                        mnv[a] = p[a];
                        mxv[a] = p[a];
                    }
                }
                for (int a = 0; a < 3; ++a) {
                    for (int o = 16; o > 0; o >>= 1) {
                        mnv[a] = fminf(mnv[a], __shfl_xor_sync(0xffffffffu, mnv[a], o));
                        mxv[a] = fmaxf(mxv[a], __shfl_xor_sync(0xffffffffu, mxv[a], o));
                    }
                }
                if ((tid & 31) == 0) {
                    for (int a = 0; a < 3; ++a) {
                        st.redf[a][tid >> 5] = mnv[a];
                        st.redf[3 + a][tid >> 5] = mxv[a];
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
            clear_tables(d, st, S, true, true, true, gtid, gstride);
            clear_layer_state(d, S, 0, gtid, gstride);
            clear_layer_state(d, S, 1, gtid, gstride);
            if (!grid_sync(d, P.nblocks, st, TAG(1, j, 0, 0))) return;
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
                if (st.n[tid] == 0) mn = mx = 0.0f;
                st.mn[tid][a] = mn;
                float e = __fsub_rn(mx, mn);
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

        // ------------------------------------------------------------ layers
        long long taken_before = 0;  // per-thread copy for thread s (budget sum of earlier layers)
        for (int l = 0; l < P.layers; ++l) {
            const int q = l & 1;
            LayerState* ls = d.ls + q * S;
            uint32_t* hist = d.hist + static_cast<long long>(q) * S * kHistBins;
            const bool use_mask = l > 0;

            if (tid < S) {
                const long long ml = layer_budget(st.m[tid], P.layers, P.ratio, l);
                const long long kmax = ml + ml * P.sigma_num / P.sigma_den;
                const bool active = ml > 0 && st.err[tid] == 0;
                st.ml[tid] = static_cast<int>(ml);
                st.kmax[tid] = static_cast<int>(kmax);
                st.lo[tid] = 0.0f;
                st.hi[tid] = st.s_hi[tid];
                st.iters[tid] = 0;
                st.sel[tid] = 0;
                st.kstar[tid] = 0;
                int fl = active ? F_ACTIVE : 0;
                if (active && P.t_max > 0) fl |= F_SEARCH;
                if (active && P.t_max == 0) {
                    st.s_star[tid] = st.s_hi[tid];
                    if (!make_grid(st.s_star[tid], P.aspect, st.mn[tid], &st.grid[tid])) {
                        seg_error(d, tid, HAV_ERR_RANGE);
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
                    tr->s_star = 0.0f;
                }
                taken_before += ml;
            }
            __syncthreads();

            // --------------------------------------- Section 3.3 bisection
            for (int p = 0; p < P.t_max; ++p) {
                int searching = 0;
                if (tid < S && (st.flags[tid] & F_SEARCH)) {
                    const float s = __fmul_rn(__fadd_rn(st.lo[tid], st.hi[tid]), 0.5f);
                    st.s_cur[tid] = s;
                    if (make_grid(s, P.aspect, st.mn[tid], &st.grid[tid])) {
                        searching = 1;
                    } else {
                        seg_error(d, tid, HAV_ERR_RANGE);
                        st.flags[tid] = 0;
                        st.err[tid] = HAV_ERR_RANGE;
                    }
                }
                if (!__syncthreads_or(searching)) break;

                unsigned long long* T = d.tk[p & 1];
                for (int t = blockIdx.x; t < st.tiles_total; t += P.nblocks) {
                    const int s = find_seg(st.tile0, S, t);
                    if (!(st.flags[s] & F_SEARCH)) continue;  // uniform across the block
                    const long long g = st.off[s] + static_cast<long long>(t - st.tile0[s]) * kTile + tid;
                    int fresh = 0;
                    if (g < st.off[s] + st.n[s] && !(use_mask && is_taken(taken, g))) {
                        float p3[3], f[3];
                        unsigned long long key;
                        load_point(pts, g, p3);
                        if (cell_key(p3, st.grid[s], &key, f)) {
                            bool fr;
                            long long slot = find_or_insert(T + st.tab_off[s], st.cap_log2[s], key, &fr);
                            if (slot < 0) seg_error(d, s, HAV_ERR_TABLE_FULL);
                            fresh = fr;
                        } else {
                            seg_error(d, s, HAV_ERR_RANGE);
                        }
                    }
                    const int cnt = __syncthreads_count(fresh);
                    if (tid == 0 && cnt) atomicAdd(&ls[s].count[p % 3], static_cast<uint32_t>(cnt));
                }
                // the other table is the next pass's: clear it (it is clean before pass 1)
                if (p >= 1) {
                    unsigned long long* T2 = d.tk[(p + 1) & 1];
                    for (int t = blockIdx.x; t < st.stiles_total; t += P.nblocks) {
                        const int s = find_seg(st.stile0, S, t);
                        if (!(st.flags[s] & F_SEARCH)) continue;
                        const long long a0 = static_cast<long long>(t - st.stile0[s]) * kSlotTile;
                        const long long C = 1ll << st.cap_log2[s];
                        for (long long i = a0 + tid; i < a0 + kSlotTile && i < C; i += kThreads)
                            T2[st.tab_off[s] + i] = kEmptyKey;
                    }
                    if (blockIdx.x == 0 && tid < S) ls[tid].count[(p + 1) % 3] = 0;
                }
                if (!grid_sync(d, P.nblocks, st, TAG(2, j, l, p))) return;

                // decide (identically in every block)
                if (tid < S && (st.flags[tid] & F_SEARCH)) {
                    const long long K = ld_volatile(reinterpret_cast<const int*>(&ls[tid].count[p % 3]));
                    const float s = st.s_cur[tid];
                    if (blockIdx.x == 0) {
                        hav_layer_trace* tr = d.tr + (static_cast<long long>(j) * S + tid) * kMaxLayers + l;
                        tr->s[p] = s;
                        tr->K[p] = K;
                        tr->iters = p + 1;
                    }
                    st.iters[tid] = p + 1;
                    if (K > st.kmax[tid]) {
                        st.lo[tid] = s;
                    } else if (K < st.ml[tid]) {
                        st.hi[tid] = s;
                    } else {
                        st.s_star[tid] = s;
                        st.sel[tid] = p & 1;
                        st.flags[tid] = F_ACTIVE | F_ACCEPT;
                    }
                }
                __syncthreads();
            }
            // no acceptance within t_max steps
            if (tid < S && (st.flags[tid] & F_SEARCH)) {
                const float s = (st.lo[tid] > 0.0f) ? st.lo[tid] : st.hi[tid];
                st.s_star[tid] = s;
                st.sel[tid] = P.t_max & 1;
                st.flags[tid] = F_ACTIVE;
                if (!make_grid(s, P.aspect, st.mn[tid], &st.grid[tid])) {
                    seg_error(d, tid, HAV_ERR_RANGE);
                    st.flags[tid] = 0;
                    st.err[tid] = HAV_ERR_RANGE;
                }
            } else if (tid < S && (st.flags[tid] & F_ACCEPT)) {
                make_grid(st.s_star[tid], P.aspect, st.mn[tid], &st.grid[tid]);  // succeeded at that s
            }
            __syncthreads();

            // ------------------------------------- Section 3.2 selection at s*
            for (int t = blockIdx.x; t < st.tiles_total; t += P.nblocks) {
                const int s = find_seg(st.tile0, S, t);
                if (!(st.flags[s] & F_ACTIVE)) continue;
                const long long g = st.off[s] + static_cast<long long>(t - st.tile0[s]) * kTile + tid;
                int first = 0;
                if (g < st.off[s] + st.n[s] && !(use_mask && is_taken(taken, g))) {
                    float p3[3], f[3];
                    unsigned long long key;
                    load_point(pts, g, p3);
                    if (cell_key(p3, st.grid[s], &key, f)) {
                        bool fr;
                        const long long slot =
                            find_or_insert(d.tk[st.sel[s]] + st.tab_off[s], st.cap_log2[s], key, &fr);
                        if (slot >= 0) {
                            const float d2 = centre_d2(p3, st.grid[s], f);
                            const unsigned long long packed =
                                (static_cast<unsigned long long>(__float_as_uint(d2)) << 32) |
                                static_cast<unsigned long long>(g);
                            const unsigned long long old = atomicMin(d.tv + st.tab_off[s] + slot, packed);
                            if (old == kEmptyVal) {
                                first = 1;
                                atomicAdd(&hist[static_cast<long long>(s) * kHistBins +
                                                (priority(key) >> (64 - kHistBits))],
                                          1u);
                            }
                        } else {
                            seg_error(d, s, HAV_ERR_TABLE_FULL);
                        }
                    } else {
                        seg_error(d, s, HAV_ERR_RANGE);
                    }
                }
                const int cnt = __syncthreads_count(first);
                if (tid == 0 && cnt) atomicAdd(&ls[s].kstar, static_cast<uint32_t>(cnt));
            }
            if (!grid_sync(d, P.nblocks, st, TAG(3, j, l, 0))) return;

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
            for (int t = blockIdx.x; t < st.stiles_total; t += P.nblocks) {
                const int s = find_seg(st.stile0, S, t);
                if (!(st.flags[s] & F_ACTIVE)) continue;
                const bool cut = st.kstar[s] > st.ml[s];
                if (cut && st.cut_seg != s) {
                    // boundary bin: smallest b with (voxels in bins <= b) >= m_l
                    const uint32_t* h = hist + static_cast<long long>(s) * kHistBins;
                    constexpr int kPer = kHistBins / kThreads;  // bins owned by each thread
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
                const long long a0 = static_cast<long long>(t - st.stile0[s]) * kSlotTile;
                const long long C = 1ll << st.cap_log2[s];
                const unsigned long long* TK = d.tk[st.sel[s]] + st.tab_off[s];
                const unsigned long long* TV = d.tv + st.tab_off[s];
                const int bin = st.cut_bin;
                for (long long i = a0 + tid; i < a0 + kSlotTile && i < C; i += kThreads) {
                    const unsigned long long v = TV[i];
                    if (v == kEmptyVal) continue;
                    const long long g = static_cast<long long>(v & 0xffffffffull);
                    if (!cut) {
                        set_taken(taken, g);
                        continue;
                    }
                    const unsigned long long h = priority(TK[i]);
                    const int b = static_cast<int>(h >> (64 - kHistBits));
                    if (b < bin) {
                        set_taken(taken, g);
                    } else if (b == bin) {
                        const uint32_t c = atomicAdd(&ls[s].cand, 1u);
                        if (static_cast<long long>(c) < (C >> 1)) {
                            Cand* cd = d.cand + st.cand_off[s] + c;
                            cd->h = h;
                            cd->g = static_cast<uint32_t>(g);
                        } else {
                            seg_error(d, s, HAV_ERR_TABLE_FULL);
                        }
                    }
                }
                __syncthreads();
            }
            if (!grid_sync(d, P.nblocks, st, TAG(4, j, l, 0))) return;

            // ------------------------------- cut-off: resolve; shortfall count
            {
                int c = 0;
                if (tid < S && (st.flags[tid] & F_ACTIVE) && st.kstar[tid] > st.ml[tid])
                    c = static_cast<int>(ld_volatile(reinterpret_cast<const int*>(&ls[tid].cand)));
                int ctot;
                const int cpre = block_excl_scan<int>(tid < S ? c : 0, &ctot, st.scan_i);
                if (tid < S) st.cprefix[tid] = cpre;
                if (tid == 0) st.cprefix[S] = ctot;
                __syncthreads();
                for (long long w = gtid; w < ctot; w += gstride) {
                    const int s = find_seg(st.cprefix, S, static_cast<int>(w));
                    const int jdx = static_cast<int>(w) - st.cprefix[s];
                    const int cs = st.cprefix[s + 1] - st.cprefix[s];
                    const Cand* base = d.cand + st.cand_off[s];
                    const unsigned long long hj = base[jdx].h;
                    int rank = 0;
                    for (int k = 0; k < cs; ++k) rank += (base[k].h < hj) ? 1 : 0;
                    const int r = st.ml[s] - static_cast<int>(ls[s].below);
                    if (rank < r) set_taken(taken, base[jdx].g);
                }
                // shortfall: count the untaken points in this block's slice of each such segment
                int sf = 0;
                if (tid < S && (st.flags[tid] & F_ACTIVE) && st.kstar[tid] < st.ml[tid]) sf = 1;
                st.any = 0;
                __syncthreads();
                if (sf) st.any = 1;
                __syncthreads();
                if (st.any) {
                    for (int s = 0; s < S; ++s) {
                        if (!((st.flags[s] & F_ACTIVE) && st.kstar[s] < st.ml[s])) continue;
                        const long long n = st.n[s];
                        const long long a = st.off[s] + n * blockIdx.x / P.nblocks;
                        const long long b = st.off[s] + n * (blockIdx.x + 1) / P.nblocks;
                        int cnt = 0;
                        for (long long g = a + tid; g < b; g += kThreads) cnt += is_taken(taken, g) ? 0 : 1;
                        int tot;
                        block_excl_scan<int>(cnt, &tot, st.scan_i);
                        if (tid == 0) d.psf[static_cast<long long>(s) * kMaxBlocks + blockIdx.x] = tot;
                    }
                }
                if (l + 1 < P.layers) {
                    clear_tables(d, st, S, true, true, true, gtid, gstride);
                    clear_layer_state(d, S, q ^ 1, gtid, gstride);
                }
                if (!grid_sync(d, P.nblocks, st, TAG(5, j, l, 0))) return;
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
                    const long long n = st.n[s];
                    const long long a = st.off[s] + n * blockIdx.x / P.nblocks;
                    const long long b = st.off[s] + n * (blockIdx.x + 1) / P.nblocks;
                    for (long long g0 = a; g0 < b && budget > 0; g0 += kThreads) {
                        const long long g = g0 + tid;
                        const int free_pt = (g < b && !is_taken(taken, g)) ? 1 : 0;
                        int chunk;
                        const int rank = block_excl_scan<int>(free_pt, &chunk, st.scan_i);
                        if (free_pt && rank < budget) set_taken(taken, g);
                        budget -= chunk;
                        __syncthreads();
                    }
                }
                if (!grid_sync(d, P.nblocks, st, TAG(6, j, l, 0))) return;
            }
        }

        // ---------------------------------------------------- compaction
        // Segments in error take their first m points so every other
        // segment's output positions stay exact.
        if (tid < S) st.err[tid] = ld_volatile(&d.sh[tid].status);
        if (tid == 0) st.any = 0;
        __syncthreads();
        if (tid < S && st.err[tid]) st.any = 1;
        __syncthreads();
        const bool any_err = st.any != 0;
        const long long W = (NL + 31) / 32;
        const long long wb = W * blockIdx.x / P.nblocks;
        const long long we = W * (blockIdx.x + 1) / P.nblocks;
        auto eff_word = [&](long long w) -> uint32_t {
            uint32_t bits = taken[w];
            const long long g0 = w * 32;
            if (g0 + 32 > NL) bits &= (NL - g0 >= 32) ? 0xffffffffu : ((1u << (NL - g0)) - 1u);
            if (any_err) {
                for (int k = 0; k < 32 && g0 + k < NL; ++k) {
                    const int s = find_seg_ll(st.off, S, g0 + k);
                    if (st.err[s]) {
                        const bool on = (g0 + k - st.off[s]) < st.m[s];
                        bits = on ? (bits | (1u << k)) : (bits & ~(1u << k));
                    }
                }
            }
            return bits;
        };
        {
            // level j+1 accumulates its bounding box in the parity level j-1 used
            if (blockIdx.x == 0 && tid < S)
                for (int a = 0; a < 6; ++a) d.sh[tid].bbox[(j + 1) & 1][a] = 0u;
            int cnt = 0;
            for (long long w = wb + tid; w < we; w += kThreads) cnt += __popc(eff_word(w));
            int tot;
            block_excl_scan<int>(cnt, &tot, st.scan_i);
            if (tid == 0) d.pcmp[blockIdx.x] = tot;
            if (!grid_sync(d, P.nblocks, st, TAG(7, j, 0, 0))) return;
        }
        {
            int pre = 0;
            for (int b = tid; b < static_cast<int>(blockIdx.x); b += kThreads) pre += d.pcmp[b];
            int base;
            block_excl_scan<int>(pre, &base, st.scan_i);
            const bool last_level = (j + 1 == P.L);
            float* pts_out = d.pts[j & 1];
            int32_t* orig_out = d.orig[j & 1];
            int32_t* out = P.out[j];
            for (long long w0 = wb; w0 < we; w0 += kThreads) {
                const long long w = w0 + tid;
                const uint32_t bits = (w < we) ? eff_word(w) : 0u;
                int chunk;
                const int rank = block_excl_scan<int>(__popc(bits), &chunk, st.scan_i);
                long long pos = static_cast<long long>(base) + rank;
                uint32_t b = bits;
                while (b) {
                    const int k = __ffs(b) - 1;
                    b &= b - 1;
                    const long long g = w * 32 + k;
                    if (pos >= st.m_total) {  // cannot happen: every segment takes exactly m
                        atomicCAS(&d.gh->status, 0, static_cast<int>(HAV_ERR_TABLE_FULL));
                        break;
                    }
                    const int s = find_seg_ll(st.off, S, g);
                    const int32_t oi = orig_in ? orig_in[g] : static_cast<int32_t>(g - st.off[s]);
                    out[pos] = oi;
                    if (!last_level) {
                        pts_out[3 * pos + 0] = pts[3 * g + 0];
                        pts_out[3 * pos + 1] = pts[3 * g + 1];
                        pts_out[3 * pos + 2] = pts[3 * g + 2];
                        orig_out[pos] = oi;
                    }
                    ++pos;
                }
                base += chunk;
            }
            if (!last_level) {
                if (!grid_sync(d, P.nblocks, st, TAG(8, j, 0, 0))) return;
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

int max_coresident_blocks(int device) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hav_chain_kernel, kThreads, 0) != cudaSuccess)
        return -1;
    long long nb = static_cast<long long>(sms) * per_sm;
    if (nb > kMaxBlocks) nb = kMaxBlocks;
    return static_cast<int>(nb);
}

int launch_chain(const Plan& plan, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(plan.nblocks));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, hav_chain_kernel, plan) == cudaSuccess ? 0 : -1;
}

int count_voxels(const float* points, int64_t n, float s, const float aspect[3], unsigned char* ws,
                 const Layout& lay, int64_t* K, cudaStream_t stream) {
    // scratch: reuse the level-0 table region and the segment header area
    int cap_log2 = kMinCapLog2;
    while ((1ll << cap_log2) < 2 * n) ++cap_log2;
    if ((1ll << cap_log2) > lay.tab_slots) return HAV_ERR_NOMEM;
    unsigned long long* T = reinterpret_cast<unsigned long long*>(ws + lay.tabk[0]);
    unsigned char* scratch = ws + lay.partial_cmp;  // 8 KB: bbox codes, K, error
    uint32_t* enc6 = reinterpret_cast<uint32_t*>(scratch);
    unsigned long long* dK = reinterpret_cast<unsigned long long*>(scratch + 64);
    int* derr = reinterpret_cast<int*>(scratch + 128);
    if (cudaMemsetAsync(scratch, 0, 256, stream) != cudaSuccess) return HAV_ERR_CUDA;
    fill_u64<<<1024, 256, 0, stream>>>(T, 1ll << cap_log2, kEmptyKey);
    bbox_kernel<<<1024, 256, 0, stream>>>(points, n, enc6);
    count_kernel<<<1024, 256, 0, stream>>>(points, n, s, aspect[0], aspect[1], aspect[2], enc6, T,
                                           cap_log2, dK, derr);
    if (cudaGetLastError() != cudaSuccess) return HAV_ERR_CUDA;
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
