// Small levels on thread-block clusters, and on single CTAs.
//
// The same sampler as hav_chain_kernel (Sections 3.2-3.4 and Eq. 3, with the
// same readings), for levels of at most 32,768 points: one cluster of Q = 8
// or 16 CTAs per segment (16 where every segment's cluster runs at once: more
// SMs share each pass; 16 is above the portable cluster size and is used
// where the device schedules it), the voxel table spread over the CTAs' shared memory and
// reached through distributed shared memory, phases separated by the cluster
// barrier.  With Q = 1 a segment's level lives in one CTA: every exchange is
// a shared-memory access and every phase ends with a block barrier.  An
// exchange between SMs then costs a few hundred cycles instead
// of an L2 round trip across the chip, and a phase ends with a hardware
// cluster barrier instead of a grid barrier: on levels of tens of thousands
// of points the grid-wide kernel pays for that latency, not for work.  The
// search takes one size per pass (several sizes per pass were measured
// slower here: a pass is bound by its remote inserts, not by the cluster
// barrier), from either search start, so every evaluated size and count is
// the paper's.
//
// Inside a cluster, CTA r holds the level's points [n r / Q, n (r + 1) / Q)
// (level indices, ascending) in shared memory with their taken flags.  The
// voxel table has max(nextpow2(2 n), 64 Q) slots: key k lives in CTA
// owner(k) (the top bits of slot_mix(k)), at the next bits inside that CTA's
// part, with linear probing inside the part.  A level's points are read from
// the original cloud through the ascending original indices of the level
// (orig), so a chain can start here at any level.

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "hav.h"
#include "hav_device.cuh"
#include "hav_internal.h"

namespace cg = cooperative_groups;

namespace havk {
namespace {

constexpr int kST = 1024;         // threads per CTA
constexpr int kPtsPerCta = 4096;  // level points one CTA holds
constexpr int kPartMax = 2 * kPtsPerCta;  // table slots per CTA at most
constexpr int kPartMaxLog2 = 13;
static_assert(kPartMax == 1 << kPartMaxLog2, "kPartMaxLog2");
static_assert(kSmallMax == 8 * kPtsPerCta, "the 8-CTA cluster takes kSmallMax points");
constexpr int kMaxQ = 16;  // largest cluster
template <int Q>
__host__ __device__ constexpr int qlog2() {
    return Q == 16 ? 4 : (Q == 8 ? 3 : (Q == 4 ? 2 : (Q == 2 ? 1 : 0)));
}
constexpr size_t kSmallDyn = static_cast<size_t>(kPartMax) * 16 + static_cast<size_t>(kPtsPerCta) * 16 +
                             static_cast<size_t>(kPtsPerCta) + 4 * kHistBins;
static_assert(kHistBins == kST, "one histogram bin per thread");

struct SmallSmem {
    // pass counts, three-way rotation, and pass errors (1: range, 2: table
    // full), same rotation: every CTA's own copy, which every CTA adds into
    unsigned long long cnt[3];
    unsigned perr[3];
    // CTA 0's copy is the cluster's: written by every CTA through distributed shared memory
    unsigned long long kstar;   // occupied voxels at s*
    unsigned errbits;           // selection errors
    unsigned ncand;             // boundary-bin candidates appended
    uint32_t box[6];            // bounding box codes of the level
    int nonfinite;
    int part_cnt[kMaxQ];  // per-CTA counts for prefixes (shortfall, compaction)
    // this CTA's
    float mn[3], mx[3], s_hi;
    int pre[kMaxIters];         // counts at s_hi / 2^(k+1) of this level's earlier layers (-1: none)
    float st_s[kMaxIters];      // a layer's sizes s_hi / 2^(k+1) and their bounds (settled steps)
    long long st_b[kMaxIters];
    unsigned acc_cnt, acc_err;  // this CTA's pass totals
    int cut_bin, cut_below;
    int red_i[32];
    float redf[6][32];
    int flag;
    // the search's two possible next sizes and grids (0: the count was above
    // K_max, 1: below m_l), prepared while the cluster barrier completes
    float nx_s[2];
    int nx_ok[2][3];  // per axis
    Grid nx_g[2];
};

template <int Q>
__device__ __forceinline__ int part_start(long long n, int r) {
    return static_cast<int>((n * r) / Q);
}

template <int Q>
__device__ __forceinline__ int point_owner(long long n, int g) {
    int r = (n > 0) ? static_cast<int>((static_cast<long long>(g) * Q) / n) : 0;
    if (r > Q - 1) r = Q - 1;
    while (r > 0 && part_start<Q>(n, r) > g) --r;
    while (r + 1 < Q && part_start<Q>(n, r + 1) <= g) ++r;
    return r;
}

// CTA r's copy of a shared-memory variable (this CTA's own when Q = 1).
template <int Q, typename T>
__device__ __forceinline__ T* at_rank(cg::cluster_group& cl, T* p, int r) {
    if constexpr (Q == 1) {
        (void)cl;
        (void)r;
        return p;
    } else {
        return cl.map_shared_rank(p, r);
    }
}

template <int Q>
__device__ __forceinline__ void csync(cg::cluster_group& cl) {
    if constexpr (Q == 1) {
        (void)cl;
        __syncthreads();
    } else {
        cl.sync();
    }
}

// The cluster barrier in two halves (arrival releases this thread's earlier
// writes, the wait acquires everyone's); with Q = 1 the block barrier that
// the caller places between them stands for it.
template <int Q>
__device__ __forceinline__ void carrive(cg::cluster_group& cl) {
    if constexpr (Q > 1) (void)cl.barrier_arrive();
    (void)cl;
}
template <int Q>
__device__ __forceinline__ void cwait(cg::cluster_group& cl) {
    if constexpr (Q > 1) cl.barrier_wait();
    (void)cl;
}

// Insert `key` into the cluster table: the slot inside the owner's part, or
// -1 when the part is full; *fresh when this call inserted it.
template <int Q>
__device__ __forceinline__ int dsm_insert(cg::cluster_group& cl, unsigned long long* keys_local, int part_log2,
                                          unsigned long long key, int* owner_out, bool* fresh) {
    const unsigned long long h = slot_mix(key);
    const int owner = (Q == 1) ? 0 : static_cast<int>(h >> (64 - qlog2<Q>()));
    unsigned long long* part = at_rank<Q>(cl, keys_local, owner);
    const unsigned mask = (1u << part_log2) - 1u;
    unsigned slot = static_cast<unsigned>(h >> (64 - qlog2<Q>() - part_log2)) & mask;
    *owner_out = owner;
    *fresh = false;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(part + slot, kEmptyKey, key);
        if (prev == kEmptyKey) {
            *fresh = true;
            return static_cast<int>(slot);
        }
        if (prev == key) return static_cast<int>(slot);
        slot = (slot + 1) & mask;
    }
    return -1;
}

// 64-bit minimum in another CTA's shared memory with compare-and-swap (the
// operation the table inserts use).  The first attempt expects the empty
// value (v is always below it), so a slot nobody has written yet takes one
// round trip; every failed attempt returns the slot's current value, and
// the next one expects it, so the loop ends after at most as many attempts
// as writers.  In the CTA's own shared memory (Q = 1) the atomic minimum.
template <int Q>
__device__ __forceinline__ void dsm_min(unsigned long long* p, unsigned long long v) {
    if constexpr (Q == 1) {
        if (v < *reinterpret_cast<volatile unsigned long long*>(p)) atomicMin(p, v);
    } else {
        unsigned long long cur = kEmptyVal;
        while (v < cur) {
            const unsigned long long prev = atomicCAS(p, cur, v);
            if (prev == cur) break;
            cur = prev;
        }
    }
}

// This CTA's total of `local` and OR of `ebits` into acc_cnt / acc_err
// (cleared before the pass): one atomic per warp, one block barrier.
__device__ __forceinline__ void block_count(unsigned local, unsigned ebits, unsigned* acc_cnt, unsigned* acc_err) {
    const unsigned c = __reduce_add_sync(0xffffffffu, local);
    const unsigned e = __reduce_or_sync(0xffffffffu, ebits);
    if ((threadIdx.x & 31) == 0) {
        if (c) atomicAdd(acc_cnt, c);
        if (e) atomicOr(acc_err, e);
    }
    __syncthreads();
}

__device__ __forceinline__ void seg_fail(SegHdr* sh, GlobalHdr* gh, int seg, int code) {
    atomicCAS(&sh[seg].status, 0, code);
    atomicCAS(&gh->status, 0, code);
}

// Phase timer (HAV_FLAG_PHASE_TIMES): thread 0 of the first cluster's CTA 0
// appends (time, tag) records after the grid kernel's, tag = phase << 24 |
// level << 16 | layer << 8 | pass with the grid kernel's phase numbers.  The
// records of a call are a prefix of the zeroed buffer, so the first free one
// is found by bisection.
struct SmallTimer {
    unsigned long long* rec;
    int cap, n;
    __device__ void open(const Plan& P, bool on) {
        rec = on ? P.ptimes : nullptr;
        cap = P.ptimes_cap;
        n = 0;
        if (!rec) return;
        int lo = 0, hi = cap;  // rec[2k] != 0 exactly for k < n
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rec[2 * mid] != 0ull) lo = mid + 1;
            else hi = mid;
        }
        n = lo;
        if (n == 0) mark(0u);  // no earlier kernel in this call: the start record
    }
    __device__ __forceinline__ void mark(unsigned tag) {
        if (rec && n < cap) {
            rec[2 * n] = globaltimer();
            rec[2 * n + 1] = tag;
            ++n;
        }
    }
    __device__ __forceinline__ void mark(int phase, int level, int layer, int pass) {
        if (rec)
            mark((static_cast<unsigned>(phase) << 24) | (static_cast<unsigned>(level) << 16) |
                 (static_cast<unsigned>(layer) << 8) | static_cast<unsigned>(pass));
    }
};

// Levels [first_level, P.L) of every segment; level first_level > 0 reads its
// input through orig[(first_level - 1) & 1].
template <int Q>
__global__ void __cluster_dims__(Q, 1, 1) __launch_bounds__(kST, 1)
    hav_small_kernel(const __grid_constant__ Plan P, int first_level) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ SmallSmem sm;
    extern __shared__ __align__(16) unsigned char dyn[];
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(dyn);
    unsigned long long* vals = keys + kPartMax;
    float4* pts = reinterpret_cast<float4*>(vals + kPartMax);  // x, y, z, original index
    unsigned char* taken = reinterpret_cast<unsigned char*>(pts + kPtsPerCta);
    uint32_t* hist = reinterpret_cast<uint32_t*>(taken + kPtsPerCta);

    const int tid = threadIdx.x;
    const int rank = static_cast<int>(cl.block_rank());
    const int cluster_id = blockIdx.x / Q;
    const int nclusters = gridDim.x / Q;
    SmallSmem* sm0 = at_rank<Q>(cl, &sm, 0);
    unsigned char* ws = P.ws;
    SegHdr* sh = reinterpret_cast<SegHdr*>(ws + P.lay.seghdr);
    GlobalHdr* gh = reinterpret_cast<GlobalHdr*>(ws + P.lay.ghdr);
    hav_layer_trace* trace = reinterpret_cast<hav_layer_trace*>(ws + P.lay.trace);
    int32_t* orig[2] = {reinterpret_cast<int32_t*>(ws + P.lay.orig[0]), reinterpret_cast<int32_t*>(ws + P.lay.orig[1])};
    Cand* cand_all = reinterpret_cast<Cand*>(ws + P.lay.cand);
    const int S = P.S;
    const bool write_tr = (rank == 0 && tid == 0);
    SmallTimer tm;
    tm.open(P, write_tr && cluster_id == 0);

    for (int seg = cluster_id; seg < S; seg += nclusters) {
        // an error from earlier levels (another kernel) carries on: first m points
        int err = ld_volatile(&sh[seg].status);
        // the segment's last search of the call so far (guided start), from the
        // kernel that ran the earlier levels
        float gs = (first_level > 0) ? sh[seg].guide_s : 0.0f;
        int gm = (first_level > 0) ? sh[seg].guide_m : 0;
        for (int j = first_level; j < P.L; ++j) {
            const long long n = (j == 0) ? (P.off0[seg + 1] - P.off0[seg]) : P.m[j - 1][seg];
            const long long m = P.m[j][seg];
            long long obase = 0, ibase = 0;  // this segment's first output / input position in the level arrays
            for (int s2 = 0; s2 < seg; ++s2) {
                obase += P.m[j][s2];
                ibase += (j == 0) ? 0 : P.m[j - 1][s2];
            }
            const int a = part_start<Q>(n, rank), b = part_start<Q>(n, rank + 1);
            const int L = b - a;

            // --------------------------------------------- points and bbox
            if (tid == 0) {
                for (int k = 0; k < 3; ++k) {
                    sm.box[k] = 0u;
                    sm.box[3 + k] = 0u;
                }
                sm.nonfinite = 0;
            }
            csync<Q>(cl);
            float mnv[3] = {INFINITY, INFINITY, INFINITY}, mxv[3] = {-INFINITY, -INFINITY, -INFINITY};
            int bad = 0;
            for (int i = tid; i < L; i += kST) {
                const int o = (j == 0) ? (a + i) : orig[(j - 1) & 1][ibase + a + i];
                const float* p = P.points + 3 * (P.off0[seg] + o);
                const float4 q = make_float4(p[0], p[1], p[2], __int_as_float(o));
                pts[i] = q;
                taken[i] = 0;
                const float c3[3] = {q.x, q.y, q.z};
                for (int k = 0; k < 3; ++k) {
                    if (!isfinite(c3[k])) bad = 1;
                    mnv[k] = fminf(mnv[k], c3[k]);
                    mxv[k] = fmaxf(mxv[k], c3[k]);
                }
            }
            for (int k = 0; k < 3; ++k)
                for (int o = 16; o > 0; o >>= 1) {
                    mnv[k] = fminf(mnv[k], __shfl_xor_sync(0xffffffffu, mnv[k], o));
                    mxv[k] = fmaxf(mxv[k], __shfl_xor_sync(0xffffffffu, mxv[k], o));
                }
            if ((tid & 31) == 0)
                for (int k = 0; k < 3; ++k) {
                    sm.redf[k][tid >> 5] = mnv[k];
                    sm.redf[3 + k][tid >> 5] = mxv[k];
                }
            bad = __syncthreads_or(bad);
            if (tid < 6) {
                float r = sm.redf[tid][0];
                for (int w = 1; w < kST / 32; ++w) r = (tid < 3) ? fminf(r, sm.redf[tid][w]) : fmaxf(r, sm.redf[tid][w]);
                if (isfinite(r)) atomicMax(&sm0->box[tid], (tid < 3) ? ~enc_f(r) : enc_f(r));
            }
            if (tid == 0 && bad) atomicExch(&sm0->nonfinite, 1);
            csync<Q>(cl);
            tm.mark(1, j, 0, 0);
            // the bracket (0, s_hi] of Section 3.3 from CTA 0's box, in every CTA
            if (tid == 0) {
                const int nf = sm0->nonfinite;
                float s_hi = 0.0f;
                for (int k = 0; k < 3; ++k) {
                    float lo = dec_f(~sm0->box[k]), hi = dec_f(sm0->box[3 + k]);
                    if (n == 0 || nf || err) lo = hi = 0.0f;
                    sm.mn[k] = lo;
                    sm.mx[k] = hi;
                    if (j == 0 && rank == 0) {
                        sh[seg].bbox[0][k] = sm0->box[k];
                        sh[seg].bbox[0][3 + k] = sm0->box[3 + k];
                    }
                    s_hi = fmaxf(s_hi, __fdiv_rn(__fsub_rn(hi, lo), P.aspect[k]));
                }
                if (s_hi == 0.0f) s_hi = 1.0f;
                sm.s_hi = s_hi;
                sm.flag = nf;
            }
            if (tid < kMaxIters) sm.pre[tid] = -1;
            __syncthreads();
            if (!err && sm.flag) {
                err = HAV_ERR_NONFINITE;
                if (write_tr) seg_fail(sh, gh, seg, err);
            }
            if (!err && !isfinite(sm.s_hi)) {
                err = HAV_ERR_RANGE;
                if (write_tr) seg_fail(sh, gh, seg, err);
            }

            int part_log2 = kMinCapLog2;
            while ((1ll << part_log2) < 2 * n) ++part_log2;
            part_log2 -= qlog2<Q>();
            if (part_log2 < kMinCapLog2) part_log2 = kMinCapLog2;
            const int part = 1 << part_log2;

            // ----------------------------------------------------- layers
            long long taken_before = 0;
            unsigned pass_no = 0;
            for (int l = 0; l < P.layers; ++l) {
                const long long ml = layer_budget(m, P.layers, P.ratio, l);
                const long long kmax = ml + ml * P.sigma_num / P.sigma_den;
                hav_layer_trace* tr = trace + (static_cast<long long>(j) * S + seg) * kMaxLayers + l;
                if (write_tr) {
                    tr->m_l = ml;
                    tr->k_max = kmax;
                    tr->k_star = 0;
                    tr->n_in = n - taken_before;
                    tr->iters = 0;
                    tr->accepted = 0;
                    tr->bounded = 0u;
                    tr->s_hi = sm.s_hi;
                    tr->s_star = 0.0f;
                }
                taken_before += ml;
                if (ml == 0 || err) continue;
                const bool fixed = P.fixed_s > 0.0f;
                float lo = 0.0f, hi = sm.s_hi;
                float s_star = fixed ? P.fixed_s : sm.s_hi;
                bool accepted = false;
                const int steps = fixed ? 0 : P.t_max;
                const bool guided = (P.search == HAV_SEARCH_GUIDED);
                // guided start: the first size from the segment's previous search in
                // this call (or from s_hi), doubling up from it while the counts stay
                // too high; the same reading as the grid kernel's
                bool up = false;
                float first = 0.0f;
                if (guided && steps > 0) {
                    const float g = (gm > 0) ? __fmul_rn(gs, __fsqrt_rn(__fdiv_rn(__int2float_rn(gm), __ll2float_rn(ml))))
                                             : __fdiv_rn(sm.s_hi, __fsqrt_rn(__ll2float_rn(ml)));
                    if (g > 0.0f && g < sm.s_hi) {
                        first = g;
                        up = true;
                    }
                }

                // The leading steps settled by an exact bound below m_l are taken
                // without a pass, as in the grid kernel: the grid cells the
                // bounding box spans, or an earlier layer's count at the same size
                // s_hi / 2^(t+1) on a superset of the points; the trace keeps the
                // smaller bound
                // (the sizes s_hi / 2^(k+1) are known in advance: lane k of warp 0
                // takes step k by the same k + 1 halvings, and every thread then
                // walks the bounds in order)
                int t0 = 0;
                if (!guided && steps > 0) {
                    for (int k = tid; k < steps; k += kST) {  // (warp 0 for steps <= 32)
                        float sv = hi;
                        for (int h = 0; h <= k; ++h) sv = __fmul_rn(__fadd_rn(0.0f, sv), 0.5f);
                        long long bd = cell_bound(sv, P.aspect, sm.mn, sm.mx);
                        if (sm.pre[k] >= 0 && sm.pre[k] < bd) bd = sm.pre[k];
                        sm.st_s[k] = sv;
                        sm.st_b[k] = bd;
                    }
                    __syncthreads();
                    while (t0 < steps && sm.st_b[t0] < ml) {
                        const float sv = sm.st_s[t0];
                        if (write_tr) {
                            tr->s[t0] = sv;
                            tr->K[t0] = sm.st_b[t0];
                            tr->iters = t0 + 1;
                            tr->bounded |= 1u << t0;
                        }
                        hi = sv;
                        ++t0;
                    }
                    __syncthreads();  // (st_s, st_b are rewritten by the next layer)
                }
                bool pre = !guided;  // every step so far had too few voxels (plain bisection)

                // Section 3.3 search, one size per pass.  Two key tables alternate
                // (the value array holds keys during the search), each with up to
                // four times the selection's slots (emptier tables, shorter probe
                // chains): pass p inserts into table p & 1 while every CTA empties
                // its part of the other, whose inserts ended at the previous
                // pass's barrier.  Every CTA adds its totals into every CTA's copy
                // of the pass's count slot, so each reads the count locally; the
                // slots rotate over three, and slot (p + 1) % 3, emptied during
                // pass p, was last read right after the barrier of pass p - 2.
                // The barrier is split: between its arrival and its wait two
                // threads prepare the grids of both possible next sizes.
                int pass_log2 = part_log2 + 2;
                if (pass_log2 > kPartMaxLog2) pass_log2 = kPartMaxLog2;
                const int pass_part = 1 << pass_log2;
                unsigned long long* const tabs[2] = {keys, vals};
                float sv = 0.0f;
                Grid Gp;
                bool gok = false;
                if (t0 < steps) {
                    for (int k = tid; k < pass_part; k += kST) {
                        keys[k] = kEmptyKey;
                        vals[k] = kEmptyKey;
                    }
                    if (tid < 3) {
                        sm.cnt[tid] = 0ull;
                        sm.perr[tid] = 0u;
                    }
                    if (tid == 0) {
                        sm.acc_cnt = 0u;
                        sm.acc_err = 0u;
                    }
                    sv = next_size(lo, hi, up, first);
                    first = 0.0f;
                    if constexpr (Q > 1) {  // the first grid while the barrier completes
                        carrive<Q>(cl);
                        gok = make_grid(sv, P.aspect, sm.mn, &Gp);
                        cwait<Q>(cl);
                    } else {
                        gok = make_grid(sv, P.aspect, sm.mn, &Gp);
                        __syncthreads();
                    }
                }
                for (int t = t0; t < steps; ++t) {
                    unsigned long long* const tab = tabs[pass_no & 1];
                    unsigned long long* const other = tabs[(pass_no + 1) & 1];
                    for (int k = tid; k < pass_part; k += kST) other[k] = kEmptyKey;
                    if (tid == 0) {
                        sm.cnt[(pass_no + 1) % 3] = 0ull;
                        sm.perr[(pass_no + 1) % 3] = 0u;
                    }
                    unsigned local = 0;
                    unsigned ebits = gok ? 0u : 1u;
                    if (gok) {
                        for (int i = tid; i < L; i += kST) {
                            if (taken[i]) continue;
                            const float4 q = pts[i];
                            const float p3[3] = {q.x, q.y, q.z};
                            unsigned long long key;
                            float f[3];
                            if (!cell_key(p3, Gp, &key, f)) {
                                ebits |= 1u;
                                continue;
                            }
                            int owner;
                            bool fr;
                            if (dsm_insert<Q>(cl, tab, pass_log2, key, &owner, &fr) < 0) ebits |= 2u;
                            else if (fr) ++local;
                        }
                    }
                    block_count(local, ebits, &sm.acc_cnt, &sm.acc_err);
                    if (tid < 32) {  // this CTA's totals into every CTA's copy; emptied for the next pass
                        const unsigned c = sm.acc_cnt, e = sm.acc_err;
                        __syncwarp();
                        if (tid == 0) {
                            sm.acc_cnt = 0u;
                            sm.acc_err = 0u;
                        }
                        if (tid < Q) {
                            if (c) atomicAdd(at_rank<Q>(cl, &sm.cnt[pass_no % 3], tid), static_cast<unsigned long long>(c));
                            if (e) atomicOr(at_rank<Q>(cl, &sm.perr[pass_no % 3], tid), e);
                        }
                    }
                    carrive<Q>(cl);
                    if (tid < 64 && (tid & 31) < 3) {  // one axis of one outcome's grid per thread
                        const int w = tid >> 5, ax = tid & 31;
                        const float nsv = (w == 0) ? next_size(sv, hi, up, 0.0f) : next_size(lo, sv, false, 0.0f);
                        if (ax == 0) sm.nx_s[w] = nsv;
                        sm.nx_ok[w][ax] = make_grid_axis(nsv, P.aspect[ax], sm.mn[ax], &sm.nx_g[w], ax) ? 1 : 0;
                    }
                    __syncthreads();
                    cwait<Q>(cl);
                    tm.mark(2, j, l, t);
                    const long long K = static_cast<long long>(sm.cnt[pass_no % 3]);
                    const unsigned eb = sm.perr[pass_no % 3];
                    ++pass_no;
                    if (write_tr) {
                        tr->s[t] = sv;
                        tr->K[t] = K;
                        tr->iters = t + 1;
                    }
                    if (pre) {  // sv = s_hi / 2^(t+1): later layers of the level may reuse K
                        if (tid == 0) sm.pre[t] = static_cast<int>(K);
                        if (K >= ml) pre = false;
                    }
                    if (eb) {
                        err = (eb & 1u) ? HAV_ERR_RANGE : HAV_ERR_TABLE_FULL;
                        if (write_tr) seg_fail(sh, gh, seg, err);
                        break;
                    }
                    if (K > kmax) {  // the next pass takes the grid prepared for this outcome
                        lo = sv;
                        sv = sm.nx_s[0];
                        gok = sm.nx_ok[0][0] && sm.nx_ok[0][1] && sm.nx_ok[0][2];
                        Gp = sm.nx_g[0];
                    } else if (K < ml) {
                        hi = sv;
                        up = false;
                        sv = sm.nx_s[1];
                        gok = sm.nx_ok[1][0] && sm.nx_ok[1][1] && sm.nx_ok[1][2];
                        Gp = sm.nx_g[1];
                    } else {
                        s_star = sv;
                        accepted = true;
                        break;
                    }
                }
                if (err) continue;
                if (!accepted && !fixed && P.t_max > 0) s_star = (lo > 0.0f) ? lo : hi;
                if (guided && P.t_max > 0 && !fixed) {  // the next search's guided start follows this one
                    gs = s_star;
                    gm = static_cast<int>(ml);
                }
                Grid G = Gp;  // an accepted s* is the last pass's size: its grid is Gp
                if (!(accepted && gok) && !make_grid(s_star, P.aspect, sm.mn, &G)) {
                    err = HAV_ERR_RANGE;
                    if (write_tr) seg_fail(sh, gh, seg, err);
                    continue;
                }

                // ------------------------------ Section 3.2 selection at s*
                for (int k = tid; k < part; k += kST) {
                    keys[k] = kEmptyKey;
                    vals[k] = kEmptyVal;
                }
                hist[tid] = 0u;
                if (rank == 0 && tid == 0) {
                    sm.kstar = 0ull;
                    sm.errbits = 0u;
                    sm.ncand = 0u;
                }
                if (tid == 0) {
                    sm.acc_cnt = 0u;
                    sm.acc_err = 0u;
                }
                csync<Q>(cl);
                {
                    unsigned local = 0;
                    unsigned ebits = 0;
                    uint32_t* hist0 = at_rank<Q>(cl, hist, 0);
                    for (int i = tid; i < L; i += kST) {
                        if (taken[i]) continue;
                        const float4 q = pts[i];
                        const float p3[3] = {q.x, q.y, q.z};
                        unsigned long long key;
                        float f[3];
                        if (!cell_key(p3, G, &key, f)) {
                            ebits |= 1u;
                            continue;
                        }
                        const int g = a + i;  // the point's level index
                        const unsigned word =
                            (P.select == HAV_SELECT_RANDOM)
                                ? static_cast<unsigned>(random_draw(P.seed, static_cast<unsigned long long>(g)) >> 32)
                                : __float_as_uint(centre_d2(p3, G, f));
                        const unsigned long long packed =
                            (static_cast<unsigned long long>(word) << 32) | static_cast<unsigned>(g);
                        int owner;
                        bool fr;
                        const int slot = dsm_insert<Q>(cl, keys, part_log2, key, &owner, &fr);
                        if (slot < 0) {
                            ebits |= 2u;
                            continue;
                        }
                        dsm_min<Q>(at_rank<Q>(cl, vals, owner) + slot, packed);
                        if (fr) {
                            ++local;
                            atomicAdd(hist0 + static_cast<int>(priority(key) >> (64 - kHistBits)), 1u);
                        }
                    }
                    block_count(local, ebits, &sm.acc_cnt, &sm.acc_err);
                    if (tid == 0) {
                        if (sm.acc_cnt) atomicAdd(&sm0->kstar, static_cast<unsigned long long>(sm.acc_cnt));
                        if (sm.acc_err) atomicOr(&sm0->errbits, sm.acc_err);
                    }
                }
                csync<Q>(cl);
                tm.mark(3, j, l, 0);
                const long long kstar = static_cast<long long>(sm0->kstar);
                {
                    const unsigned eb = sm0->errbits;
                    if (write_tr) {
                        tr->k_star = kstar;
                        tr->accepted = accepted ? 1 : 0;
                        tr->s_star = s_star;
                    }
                    if (eb) {
                        err = (eb & 1u) ? HAV_ERR_RANGE : HAV_ERR_TABLE_FULL;
                        if (write_tr) seg_fail(sh, gh, seg, err);
                        continue;
                    }
                }

                // ----------------------------------- cut-off and taken marks
                const bool cut = kstar > ml;
                Cand* cand = cand_all + 2 * P.off0[seg];  // room for 2 n entries of this segment
                if (cut) {
                    // boundary bin: smallest b with (voxels in bins <= b) >= m_l
                    const int v = static_cast<int>(at_rank<Q>(cl, hist, 0)[tid]);
                    int total;
                    const int before = block_excl_scan<int>(v, &total, sm.red_i);
                    if (before < ml && before + v >= ml) {
                        sm.cut_bin = tid;
                        sm.cut_below = before;
                    }
                    __syncthreads();
                }
                for (int k = tid; k < part; k += kST) {
                    const unsigned long long key = keys[k];
                    if (key == kEmptyKey) continue;
                    const int g = static_cast<int>(vals[k] & 0xffffffffull);
                    bool take = !cut;
                    if (cut) {
                        const unsigned long long h = priority(key);
                        const int hb = static_cast<int>(h >> (64 - kHistBits));
                        if (hb < sm.cut_bin) {
                            take = true;
                        } else if (hb == sm.cut_bin) {
                            const unsigned ci = atomicAdd(&sm0->ncand, 1u);
                            if (ci < static_cast<unsigned>(2 * n)) {
                                cand[ci].h = h;
                                cand[ci].g = static_cast<uint32_t>(g);
                            }
                        }
                    }
                    if (take) {
                        const int r = point_owner<Q>(n, g);
                        at_rank<Q>(cl, taken, r)[g - part_start<Q>(n, r)] = 1;
                    }
                }
                csync<Q>(cl);
                tm.mark(4, j, l, 0);
                if (cut) {
                    // the boundary bin's candidates ranked exactly; the r smallest priorities are taken
                    const int c = static_cast<int>(sm0->ncand);
                    const int r = static_cast<int>(ml) - sm.cut_below;
                    for (int f = rank * kST + tid; f < c; f += Q * kST) {
                        const unsigned long long hf = cand[f].h;
                        int rk = 0;
                        for (int k = 0; k < c; ++k) rk += (cand[k].h < hf) ? 1 : 0;
                        if (rk < r) {
                            const int g = static_cast<int>(cand[f].g);
                            const int owner = point_owner<Q>(n, g);
                            at_rank<Q>(cl, taken, owner)[g - part_start<Q>(n, owner)] = 1;
                        }
                    }
                    csync<Q>(cl);
                    tm.mark(5, j, l, 0);
                } else if (kstar < ml) {
                    // shortfall: untaken points in ascending level index until m_l
                    int cnt = 0;
                    for (int i = tid; i < L; i += kST) cnt += taken[i] ? 0 : 1;
                    int tot;
                    block_excl_scan<int>(cnt, &tot, sm.red_i);
                    if (tid == 0) sm0->part_cnt[rank] = tot;
                    csync<Q>(cl);
                    long long before = 0;
                    for (int r2 = 0; r2 < rank; ++r2) before += sm0->part_cnt[r2];
                    long long budget = (ml - kstar) - before;
                    for (int i0 = 0; i0 < L && budget > 0; i0 += kST) {
                        const int i = i0 + tid;
                        const int free_pt = (i < L && !taken[i]) ? 1 : 0;
                        int chunk;
                        const int rk = block_excl_scan<int>(free_pt, &chunk, sm.red_i);
                        if (free_pt && rk < budget) taken[i] = 1;
                        budget -= chunk;
                    }
                    csync<Q>(cl);
                    tm.mark(6, j, l, 0);
                }
            }

            // ----------------------------------------------------- compaction
            // Segments in error take their first m points, as in the grid kernel.
            {
                int cnt = 0;
                for (int i = tid; i < L; i += kST) cnt += (err ? (a + i < m) : (taken[i] != 0)) ? 1 : 0;
                int tot;
                block_excl_scan<int>(cnt, &tot, sm.red_i);
                if (tid == 0) sm0->part_cnt[rank] = tot;
                csync<Q>(cl);
                tm.mark(7, j, 0, 0);
                long long pos = obase;
                for (int r2 = 0; r2 < rank; ++r2) pos += sm0->part_cnt[r2];
                int32_t* out = P.out[j];
                int32_t* orig_out = orig[j & 1];
                const bool more = (j + 1 < P.L) || P.keep_orig;
                for (int i0 = 0; i0 < L; i0 += kST) {
                    const int i = i0 + tid;
                    const int keep = (i < L && (err ? (a + i < m) : (taken[i] != 0))) ? 1 : 0;
                    int chunk;
                    const int rk = block_excl_scan<int>(keep, &chunk, sm.red_i);
                    if (keep) {
                        if (pos + rk < obase + m) {
                            const int o = __float_as_int(pts[i].w);
                            out[pos + rk] = o;
                            if (more) orig_out[pos + rk] = o;
                        } else {
                            seg_fail(sh, gh, seg, HAV_ERR_TABLE_FULL);  // cannot happen: every layer takes m_l
                        }
                    }
                    pos += chunk;
                }
                csync<Q>(cl);  // the next level reads orig_out; part_cnt is reused
                tm.mark(8, j, 0, 0);
            }
        }
        if (write_tr) {  // for a single-CTA launch that continues the chain
            sh[seg].guide_s = gs;
            sh[seg].guide_m = gm;
        }
    }
}

}  // namespace

int small_clusters(int device, int q) {
    (void)device;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(q * 16));
    cfg.blockDim = dim3(kST);
    cfg.dynamicSmemBytes = kSmallDyn;
    int nc = 0;
    if (q == 1) {
        if (cudaFuncSetAttribute(hav_small_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kSmallDyn)) != cudaSuccess)
            return -1;
        return 1;
    }
    if (q == 8) {
        if (cudaFuncSetAttribute(hav_small_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kSmallDyn)) != cudaSuccess ||
            cudaOccupancyMaxActiveClusters(&nc, hav_small_kernel<8>, &cfg) != cudaSuccess)
            return -1;
        return nc;
    }
    if (q == 16) {
        if (cudaFuncSetAttribute(hav_small_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kSmallDyn)) != cudaSuccess ||
            cudaFuncSetAttribute(hav_small_kernel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveClusters(&nc, hav_small_kernel<16>, &cfg) != cudaSuccess)
            return -1;
        return nc;
    }
    return -1;
}

int launch_small(const Plan& plan, int first_level, int q, int nclusters, cudaStream_t stream) {
    if (q != 8 && q != 16) return -1;
    // every level of the launch must fit its cluster's shared memory
    for (int j = first_level; j < plan.L; ++j)
        for (int s = 0; s < plan.S; ++s) {
            const long long n = (j == 0) ? plan.off0[s + 1] - plan.off0[s] : plan.m[j - 1][s];
            if (n > static_cast<long long>(kSmallMax)) return -1;
        }
    int nc = nclusters < plan.S ? nclusters : plan.S;
    if (nc < 1) nc = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(q * nc));
    cfg.blockDim = dim3(kST);
    cfg.dynamicSmemBytes = kSmallDyn;
    cfg.stream = stream;
    const cudaError_t e = (q == 16) ? cudaLaunchKernelEx(&cfg, hav_small_kernel<16>, plan, first_level)
                                    : cudaLaunchKernelEx(&cfg, hav_small_kernel<8>, plan, first_level);
    return e == cudaSuccess ? 1 : -1;
}

int launch_solo(const Plan& plan, int first_level, int nblocks, cudaStream_t stream) {
    for (int j = first_level; j < plan.L; ++j)  // every level must fit one CTA
        for (int s = 0; s < plan.S; ++s) {
            const long long n = (j == 0) ? plan.off0[s + 1] - plan.off0[s] : plan.m[j - 1][s];
            if (n > static_cast<long long>(kSoloMax)) return -1;
        }
    int nc = nblocks < plan.S ? nblocks : plan.S;
    if (nc < 1) nc = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(nc));
    cfg.blockDim = dim3(kST);
    cfg.dynamicSmemBytes = kSmallDyn;
    cfg.stream = stream;
    return cudaLaunchKernelEx(&cfg, hav_small_kernel<1>, plan, first_level) == cudaSuccess ? 1 : -1;
}

}  // namespace havk
