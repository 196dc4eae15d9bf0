// Device helpers of the HAVSampler kernels: memory-order primitives, the
// Eq. 2 voxel key, the Section 3.2 centre distance, hashing, block scans and
// the bounded grid barrier.
#pragma once

#include <cuda_runtime.h>

#include "hav_internal.h"

namespace havk {

constexpr unsigned long long kSpinNs = 2000000000ull;  // 2 s per barrier wait
constexpr unsigned int kSpinIters = 1u << 26;

// ------------------------------------------------------------------ memory ops
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_strong64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned ld_volatile_u(const unsigned* p) { return *(const volatile unsigned*)p; }
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
// Slot hash: a 64-bit mixer (xor-shift / multiply rounds).  The global table
// indexes by its top bits, the block-local sets by its low bits.
__device__ __forceinline__ unsigned long long slot_mix(unsigned long long k) {
    k ^= k >> 32;
    k *= 0xd6e8feb86659fd93ull;
    k ^= k >> 32;
    k *= 0xd6e8feb86659fd93ull;
    k ^= k >> 32;
    return k;
}
// Slot hash of the block-local sets (any mixing works there): multiplicative
// hashing of the two 32-bit halves, top bits.
__device__ __forceinline__ unsigned smem_hash(unsigned long long k, int log2) {
    const unsigned h = static_cast<unsigned>(k) * 0x9E3779B1u + static_cast<unsigned>(k >> 32) * 0x85EBCA77u;
    return h >> (32 - log2);
}
// Cut-off priority: the SplitMix64 output finaliser (Steele, Lea, Flood 2014).
__device__ __forceinline__ unsigned long long priority(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Draw `counter` of the SplitMix64 generator (Steele, Lea, Flood 2014)
// started at `seed`: the state advances by the golden-ratio step before each
// output, so draw c finalises seed + (c + 1) * step.
__device__ __forceinline__ unsigned long long random_draw(unsigned seed, unsigned long long counter) {
    return priority(static_cast<unsigned long long>(seed) + (counter + 1ull) * 0x9E3779B97F4A7C15ull);
}

// ------------------------------------------------------------ Eq. 2 voxel keys
// The cell indices are kept as integral binary32 values: floor(x / v) and
// floor(min / v) are exact floats, and their difference u is exact whenever
// the true u is below 2^21 (Sterbenz's lemma when both exceed 2^21 in size,
// small exact integers otherwise); a true u >= 2^21 rounds to a value >= 2^21,
// so the range test below is exact as well.
struct Grid {
    float v[3];
    float fmin[3];
    float r[3];  // RN(1 / v) where it is a normal number, else 0 (floor_div_r)
};

__device__ __forceinline__ bool floor_div(float x, float v, float* f) {
    const float q = __fdiv_rn(x, v);
    const float fl = floorf(q);
    if (!(fabsf(fl) < 4.6e18f)) return false;  // |floor| < 2^62 and finite, as the key range requires
    *f = fl;
    return true;
}

// floor(RN(x / v)), the Eq. 2 cell, through the reciprocal r = RN(1 / v) (a
// normal number): q = RN(x * r) equals x / v up to a relative 2^-23 (two
// roundings), and RN(x / v) is within a relative 2^-24 of x / v, so
// |RN(x / v) - q| < (|q| + 1) 2^-22.  If q lies farther than
// b = (|q| + 1) 2^-21 from both integers around it (b < d = q - floor(q) <
// RN(1 - b)), RN(x / v) lies strictly between them and both floors agree.
// Near an integer (or with |q| >= 2^21, where b exceeds 1, a quotient below
// the normal range, which leaves d within b of 0 or 1, r = 0, or x not
// finite) the quotient is taken correctly rounded and floored.  Either way
// the result is the floor of the correctly rounded quotient.
__device__ __forceinline__ bool floor_div_r(float x, const Grid& g, int a, float* f) {
    const float q = __fmul_rn(x, g.r[a]);
    const float n = floorf(q);
    const float d = __fsub_rn(q, n);
    const float b = __fmul_rn(__fadd_rn(fabsf(q), 1.0f), 4.76837158203125e-07f);  // (|q| + 1) 2^-21
    if (d > b && d < __fsub_rn(1.0f, b)) {
        *f = n;
        return true;
    }
    return floor_div(x, g.v[a], f);
}

// The grid of voxel size v = s * aspect; mn is the bounding box's minimum.
__device__ inline bool make_grid(float s, const float r[3], const float mn[3], Grid* g) {
    for (int a = 0; a < 3; ++a) {
        const float v = __fmul_rn(s, r[a]);
        if (!(v > 0.0f) || !isfinite(v)) return false;
        g->v[a] = v;
        const float rv = __fdiv_rn(1.0f, v);
        g->r[a] = (rv >= 1.17549435e-38f && rv <= 3.40282347e+38f) ? rv : 0.0f;
        if (!floor_div(mn[a], v, &g->fmin[a])) return false;
    }
    return true;
}

// One axis of make_grid (its three axes may be computed by three threads;
// the grid is valid when every axis is).
__device__ __forceinline__ bool make_grid_axis(float s, float r, float mn, Grid* g, int a) {
    const float v = __fmul_rn(s, r);
    if (!(v > 0.0f) || !isfinite(v)) return false;
    g->v[a] = v;
    const float rv = __fdiv_rn(1.0f, v);
    g->r[a] = (rv >= 1.17549435e-38f && rv <= 3.40282347e+38f) ? rv : 0.0f;
    return floor_div(mn, v, &g->fmin[a]);
}

// key = u_x | u_y << 21 | u_z << 42 with u = floor(x / v) - floor(min / v).
__device__ __forceinline__ bool cell_key(const float p[3], const Grid& g, unsigned long long* key,
                                         float f[3]) {
    unsigned long long k = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!floor_div_r(p[a], g, a, &f[a])) return false;
        const float u = __fsub_rn(f[a], g.fmin[a]);
        if (!(u >= 0.0f && u < 2097152.0f)) return false;
        k |= static_cast<unsigned long long>(static_cast<unsigned>(u)) << (21 * a);
    }
    *key = k;
    return true;
}

// At most this many voxels are occupied at size s: the grid cells the
// bounding box [mn, mx] spans, floor(mx / v) - floor(mn / v) + 1 per axis (the
// floor of Eq. 2 is monotone in the coordinate).  LLONG_MAX when the grid is
// not representable.
__device__ __forceinline__ long long cell_bound(float s, const float r[3], const float mn[3], const float mx[3]) {
    long long b = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float v = __fmul_rn(s, r[a]);
        float f0, f1;
        if (!(v > 0.0f) || !isfinite(v) || !floor_div(mn[a], v, &f0) || !floor_div(mx[a], v, &f1)) return LLONG_MAX;
        const float u = __fsub_rn(f1, f0);
        if (!(u >= 0.0f && u < 1048576.0f)) return LLONG_MAX;
        b *= static_cast<long long>(u) + 1;
    }
    return b;
}

// Section 3.2: squared distance to the voxel centre v * (g + 0.5).
__device__ __forceinline__ float centre_d2(const float p[3], const Grid& g, const float f[3]) {
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float c = __fmul_rn(g.v[a], __fadd_rn(f[a], 0.5f));
        d[a] = __fsub_rn(p[a], c);
    }
    const float xy = __fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1]));
    return __fadd_rn(xy, __fmul_rn(d[2], d[2]));
}

// Find or insert `key` in a global open-addressed table by linear probing;
// *fresh tells whether this call inserted it.  Returns the slot, or -1 after
// a full sweep (table full).
__device__ __forceinline__ long long find_or_insert(unsigned long long* T, int cap_log2,
                                                    unsigned long long key, bool* fresh) {
    const unsigned long long mask = (1ull << cap_log2) - 1;
    unsigned long long slot = slot_mix(key) >> (64 - cap_log2);
    *fresh = false;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long cur = ld_strong64(T + slot);
        if (cur == key) return static_cast<long long>(slot);
        if (cur == kEmptyKey) {
            const unsigned long long prev = atomicCAS(T + slot, kEmptyKey, key);
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

// find_or_insert for U keys at once: the first probe of every key is issued
// before any result is used (memory-level parallelism); keys equal to
// kEmptyKey are skipped.  slot[u] = -1 after a full sweep (table full).
template <int U>
__device__ __forceinline__ void find_or_insert_batch(unsigned long long* const (&T)[U], int cap_log2,
                                                     const unsigned long long (&key)[U],
                                                     long long (&slot)[U], bool (&fresh)[U]) {
    const unsigned mask = static_cast<unsigned>((1ull << cap_log2) - 1);
    unsigned sl[U];
    unsigned long long cur[U];
    // every probe is a compare-and-swap (it returns the slot's key whether or
    // not it swaps: one round trip per probe), and the probes of all U keys
    // are in flight together
#pragma unroll
    for (int u = 0; u < U; ++u) {
        sl[u] = static_cast<unsigned>(slot_mix(key[u]) >> (64 - cap_log2));
        cur[u] = (key[u] != kEmptyKey) ? atomicCAS(T[u] + sl[u], kEmptyKey, key[u]) : kEmptyKey;
    }
    bool open[U];
    bool any = false;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        fresh[u] = false;
        slot[u] = -1;
        open[u] = false;
        if (key[u] == kEmptyKey) continue;
        if (cur[u] == kEmptyKey || cur[u] == key[u]) {
            slot[u] = sl[u];
            fresh[u] = (cur[u] == kEmptyKey);
        } else {
            open[u] = true;
            any = true;
        }
    }
    // collisions: linear probing from the next slot
    for (unsigned probe = 1; any && probe <= mask; ++probe) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!open[u]) continue;
            sl[u] = (sl[u] + 1) & mask;
            cur[u] = atomicCAS(T[u] + sl[u], kEmptyKey, key[u]);
        }
        any = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!open[u]) continue;
            if (cur[u] == kEmptyKey || cur[u] == key[u]) {
                slot[u] = sl[u];
                fresh[u] = (cur[u] == kEmptyKey);
                open[u] = false;
            } else {
                any = true;
            }
        }
    }
}

// Warp-aggregated append to a shared-memory list: every lane of the warp
// calls it (flag false for lanes with nothing to add); returns the lane's
// position, or -1.
template <typename T>
__device__ __forceinline__ int warp_append(bool flag, T* counter) {
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (!m) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    T base = 0;
    if (lane == leader) base = atomicAdd(counter, static_cast<T>(__popc(m)));
    base = __shfl_sync(0xffffffffu, base, leader);
    return flag ? static_cast<int>(base) + __popc(m & ((1u << lane) - 1u)) : -1;
}

// As warp_append with one counter per key (key indexes counters): the lanes
// of each key share one atomic add.  Whole warp calls, converged.
template <typename T>
__device__ __forceinline__ int warp_append_keyed(bool flag, int key, T* counters) {
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (!m) return -1;
    int pos = -1;
    if (flag) {
        const int lane = threadIdx.x & 31;
        const unsigned grp = __match_any_sync(m, key);
        const int leader = __ffs(grp) - 1;
        T base = 0;
        if (lane == leader) base = atomicAdd(counters + key, static_cast<T>(__popc(grp)));
        base = __shfl_sync(m, base, leader);
        pos = static_cast<int>(base) + __popc(grp & ((1u << lane) - 1u));
    }
    return pos;
}

// Block-local set in shared memory (a filter in front of the global table):
// returns the slot holding `key` and whether this call inserted it, or -1
// when the probe limit is reached (the caller then goes to the global table).
template <int kSlots>
__device__ __forceinline__ int smem_insert(unsigned long long* set, unsigned long long key, bool* fresh) {
    static_assert(kSlots > 1 && (kSlots & (kSlots - 1)) == 0, "power of two");
    unsigned slot = smem_hash(key, __builtin_ctz(kSlots));
    *fresh = false;
#pragma unroll 1
    for (int probe = 0; probe < 32; ++probe) {
        const unsigned long long cur = set[slot];
        if (cur == key) return static_cast<int>(slot);
        if (cur == kEmptyKey) {
            const unsigned long long prev = atomicCAS(set + slot, kEmptyKey, key);
            if (prev == kEmptyKey) {
                *fresh = true;
                return static_cast<int>(slot);
            }
            if (prev == key) return static_cast<int>(slot);
        }
        slot = (slot + 1) & (kSlots - 1);
    }
    return -1;
}

// smem_insert on a set of (1 << log2) slots starting at set (runtime size).
__device__ __forceinline__ int smem_insert_n(unsigned long long* set, int log2, unsigned long long key, bool* fresh) {
    const unsigned m = (1u << log2) - 1u;
    unsigned slot = smem_hash(key, log2);
    *fresh = false;
#pragma unroll 1
    for (int probe = 0; probe < 32; ++probe) {
        const unsigned long long cur = set[slot];
        if (cur == key) return static_cast<int>(slot);
        if (cur == kEmptyKey) {
            const unsigned long long prev = atomicCAS(set + slot, kEmptyKey, key);
            if (prev == kEmptyKey) {
                *fresh = true;
                return static_cast<int>(slot);
            }
            if (prev == key) return static_cast<int>(slot);
        }
        slot = (slot + 1) & m;
    }
    return -1;
}

// ------------------------------------------------ Section 3.3 search steps
// The next size of a search with bracket (lo, hi): a pending first guess,
// 2 lo while doubling up (the guided start), else the bisection midpoint in
// binary32.
__device__ __forceinline__ float next_size(float lo, float hi, bool up, float first) {
    if (first > 0.0f) return first;
    const float d = __fmul_rn(lo, 2.0f);
    if (up && d < hi) return d;
    return __fmul_rn(__fadd_rn(lo, hi), 0.5f);
}

// Size at node c of the search subtree below the current state (heap order:
// child 2c + 1 follows a count below m_l, 2c + 2 a count above k_max): the
// path from the root follows the bits of c + 1 below its leading one (0: too
// few voxels, hi = s; 1: too many, lo = s), each step as next_size takes it.
__device__ __forceinline__ float cand_size(float lo, float hi, bool up, float first, int c) {
    const int x = c + 1;
    const int depth = 31 - __clz(x);
    float s = next_size(lo, hi, up, first);
    for (int b = depth - 1; b >= 0; --b) {
        if ((x >> b) & 1) {
            lo = s;
        } else {
            hi = s;
            up = false;
        }
        s = next_size(lo, hi, up, 0.0f);
    }
    return s;
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
        const long long mi = m * pw / S;
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
        const T y = __shfl_up_sync(0xffffffffu, x, o);
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
    const T before = wid ? scratch[wid - 1] : T(0);
    *total = scratch[kWarps - 1];
    __syncthreads();
    return before + x - v;
}

// Sum over the block (every thread receives it).
__device__ __forceinline__ unsigned block_sum(unsigned v, unsigned* scratch /* >= 32 */) {
    const unsigned w = __reduce_add_sync(0xffffffffu, v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) scratch[wid] = w;
    __syncthreads();
    unsigned t = 0;
#pragma unroll
    for (int k = 0; k < kThreads / 32; ++k) t += scratch[k];
    __syncthreads();
    return t;
}

// Grid barrier with a bounded wait.  Arrival is a release reduction on a
// counter that only grows within a launch (zeroed by the host before it);
// barrier number e of the launch completes when the counter reaches
// e * nblocks, so no block has to act as the last arriver.  Returns false
// (for the whole block) when this or another block gave up; the caller then
// leaves the kernel.
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier that also sums one count over the blocks.  Each block adds
// 2^48 + add to `word`; the barrier is complete when the arrival field (bits
// 48..63, mod 2^16) reaches uses * nblocks.  Between two uses of the same
// word every block has passed a barrier on the other word, so no block adds
// to it again before all have read it: the change of the low 48 bits since
// this block's last reading is exactly this barrier's sum.  The caller keeps
// the low field below 2^48.  Bounded like grid_wait_impl.
//
// Both barriers come in two halves.  The arrival orders every write the block
// made before it; work between the arrival and the wait (writes that only the
// block's next arrival has to publish) overlaps the wait for the other blocks.
__device__ inline void fused_arrive_impl(unsigned long long* word, unsigned* uses, unsigned long long add) {
    __syncthreads();
    if (threadIdx.x == 0) {
        *uses += 1u;
        const unsigned long long inc = (1ull << 48) | add;
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(word), "l"(inc) : "memory");
    }
}

__device__ inline bool fused_wait_impl(unsigned long long* word, GlobalHdr* gh, unsigned nblocks,
                                       const unsigned* uses, unsigned long long* last,
                                       unsigned long long* delta, int* s_flag) {
    if (threadIdx.x == 0) {
        int fail = 0;
        const unsigned target = (*uses * nblocks) & 0xffffu;
        const unsigned long long t0 = globaltimer();
        unsigned long long v = 0;
        int ab = 0;
        for (unsigned it = 0;; ++it) {
            ab = ld_volatile(&gh->abort);  // in flight together with the poll
            v = ld_acquire64(word);
            if ((static_cast<unsigned>(v >> 48) & 0xffffu) == target) break;
            if ((it & 31) == 31) {
                if (ab || it > kSpinIters || globaltimer() - t0 > kSpinNs) {
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
        const unsigned long long c = v & ((1ull << 48) - 1ull);
        *delta = c - *last;
        *last = c;
        *s_flag = fail | ab;
    }
    __syncthreads();
    return *s_flag == 0;
}

__device__ inline void grid_arrive_impl(Barrier* bar, unsigned* epoch) {
    __syncthreads();
    if (threadIdx.x == 0) {
        *epoch += 1u;
        // The block barrier above orders every thread's writes before this
        // release; the acquire load in the wait orders them before every
        // thread's reads after its closing block barrier.  No further fence
        // is needed.
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->count) : "memory");
    }
}

__device__ inline bool grid_wait_impl(Barrier* bar, GlobalHdr* gh, unsigned nblocks, const unsigned* epoch,
                                      int* s_flag) {
    if (threadIdx.x == 0) {
        int fail = 0;
        const unsigned target = *epoch * nblocks;
        const unsigned long long t0 = globaltimer();
        int ab = 0;
        for (unsigned it = 0;; ++it) {
            // the abort flag is read in the same round trip as the poll (a
            // relaxed load ahead of the acquire), not after the barrier
            ab = ld_volatile(&gh->abort);
            if (ld_acquire(&bar->count) >= target) break;
            if ((it & 31) == 31) {
                if (ab || it > kSpinIters || globaltimer() - t0 > kSpinNs) {
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
        *s_flag = fail | ab;
    }
    __syncthreads();
    return *s_flag == 0;
}

__device__ inline bool grid_sync_impl(Barrier* bar, GlobalHdr* gh, unsigned nblocks, unsigned* epoch,
                                      int* s_flag) {
    grid_arrive_impl(bar, epoch);
    return grid_wait_impl(bar, gh, nblocks, epoch, s_flag);
}

}  // namespace havk
