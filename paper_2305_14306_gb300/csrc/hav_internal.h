// Internal definitions shared by the HAVSampler kernels and the C ABI layer.
// Not part of the public interface (include/hav.h is).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "hav.h"

namespace havk {

constexpr int kThreads = 1024;             // threads per block of the persistent kernel (one block per SM)
constexpr int kMaxSegments = 256;          // segments per launch (plan lives in kernel params)
constexpr int kMaxLevels = 8;
constexpr int kMaxLayers = 8;
constexpr int kMaxIters = HAV_MAX_ITERS;
constexpr int kTile = kThreads;            // points per work tile (one per thread)
constexpr int kSlotTile = 4 * kThreads;    // hash slots per work tile
constexpr int kHistBits = 10;              // cut-off histogram over the top priority bits
constexpr int kHistBins = 1 << kHistBits;
constexpr int kMaxBlocks = 2048;
constexpr int kMinCapLog2 = 6;             // smallest per-segment table: 64 slots
constexpr int kPhaseTimes = 4096;          // (time, tag) records of the phase timer
constexpr int kMaxSpecDepth = 4;           // bisection steps one pass may evaluate ahead
constexpr int kMaxCand = (1 << kMaxSpecDepth) - 1;  // candidate sizes per pass (a full subtree)
// Key-table sets of the bisection passes, used in rotation: pass p inserts
// into set p % 3 and, once it has arrived at its closing grid barrier, empties
// set (p - 1) % 3 while it waits, ready for pass p + 2.
constexpr int kTableSets = 3;
// default level sizes (points) up to which a pass evaluates 4, 3 or 2 steps
// ahead (measured on GB300: 15 candidates per pass never paid off; with the
// coarse steps settled without a pass, the passes left are near the target,
// where 7 candidates pay up to about 4k points and 3 up to 64k)
constexpr int64_t kSpecN4 = 0;
constexpr int64_t kSpecN3 = 4096;
constexpr int64_t kSpecN2 = 65536;
constexpr int kChunkMin = 64;              // default smallest work item (points)
constexpr int kSmallMax = 32768;           // largest level the cluster kernel takes (points)
constexpr int kLocalItems = 8;             // work items one block can own in a level
// Pass shapes of the grid kernel (template instantiations): points each thread
// loads ahead in a bisection or selection pass, and first probes of the
// global flush it keeps in flight.  Shape 0 is the default.
constexpr int kPassShapes = 4;

constexpr unsigned long long kEmptyKey = ~0ull;  // valid keys use 63 bits
constexpr unsigned long long kEmptyVal = ~0ull;  // packed (d^2 bits, index) never reaches it

// Zeroed by the host (one memset) before every launch.
struct alignas(128) Barrier {
    unsigned int count;
    unsigned int pad0[31];
    unsigned int gen;
    unsigned int pad1[31];
    // counting barriers of single-cloud passes, alternating by pass parity:
    // arrivals (mod 2^16) in bits 48..63, summed counts in bits 0..47
    unsigned long long fused[2];
    unsigned long long pad2[14];
};

struct GlobalHdr {
    int32_t status;  // first error of the call (hav_status)
    int32_t abort;   // set when a bounded wait gave up; every block leaves
    int32_t pad[30];
};

struct SegHdr {
    int32_t status;         // first error of this segment
    int32_t nonfinite;      // set only in the bounding-box phase
    uint32_t bbox[2][6];    // per level parity: ~enc(min xyz) then enc(max xyz), atomicMax'ed
    // the segment's last search of the call so far (guided start): its s*
    // and budget m_l (0: none); handed from the grid kernel to the small-level one
    float guide_s;
    int32_t guide_m;
    // a batch segment sorted by Morton cell at level 0: that level's box (min
    // xyz, max xyz), for the ownership test of its later levels (b0_on = 1)
    float b0[6];
    int32_t b0_on;
    int32_t pad;
};

// Per segment, per layer parity: zeroed inside the kernel before use.
struct LayerState {
    uint32_t count[3][kMaxCand];  // Cnt per candidate of a bisection pass, three-way rotation
    uint32_t cerr[3];   // candidates with a voxel key out of range, same rotation
    uint32_t kstar;     // occupied voxels at s*
    uint32_t cand;      // cut-off candidates in the boundary bin
    int32_t bin;        // boundary bin of the cut-off
    uint32_t below;     // voxels in bins below the boundary
    uint32_t pad;
};

struct Cand {
    unsigned long long h;  // cut-off priority
    uint32_t g;            // point index (level-global)
    uint32_t pad;
};

// Byte offsets of every region inside one workspace allocation.
struct Layout {
    int64_t max_points;
    int32_t max_segments;
    int32_t table_log2;    // key tables sized for capacities nextpow2(2^table_log2 n)
    int64_t tab_slots;     // slots of one key-table array (all segments, all candidates of a pass)
    int64_t cand_slots;
    int64_t taken_words;
    int64_t dirty_slots;   // entries of one fresh-insert log array
    size_t barrier, ghdr, seghdr, zero_bytes;  // [barrier, barrier+zero_bytes) zeroed per call
    size_t clean;          // 1 when every hash-table slot is empty (kept across calls)
    size_t lstate, hist, partial_sf, partial_cmp, pitem, trace, ptimes;
    size_t ord[2], orig[2], taken[2], wpre, posof, dirty[kTableSets], bkt, prefix;
    size_t tabk[kTableSets], tabv, cand;
    size_t total;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int kMaxItems = kMaxBlocks + kMaxSegments;  // work items of one level

// Largest table load factor setting: capacity nextpow2(2^3 n), at most 1/8 full.
constexpr int kMaxTableLog2 = 3;
constexpr long long kSpacingGridMin = 32768;  // subsets from this size search their spacing on a grid

inline Layout make_layout(int64_t N, int32_t S, bool spec_room = true, int table_log2 = 1) {
    Layout L{};
    L.max_points = N;
    L.max_segments = S;
    L.table_log2 = table_log2;
    // Per-segment capacity C = max(nextpow2(2^f n), 64) < max(2^(f+1) n, 128)
    // for f = table_log2; small levels (at most 32,768 points) also get room
    // for kMaxCand tables per pass.
    const int64_t plain = (2ll << table_log2) * N + 128 * static_cast<int64_t>(S);
    const int64_t spec = spec_room ? static_cast<int64_t>(kMaxCand) * (65536 + 128 * static_cast<int64_t>(S)) : 0;
    L.tab_slots = plain > spec ? plain : spec;
    L.cand_slots = plain / 2;
    const int64_t dspec = spec_room ? static_cast<int64_t>(kMaxCand) * 32768 : 0;
    L.dirty_slots = N > dspec ? N : dspec;
    L.taken_words = N / 32 + 2;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = align_up(o, 256);
        o = at + bytes;
        return at;
    };
    L.barrier = take(sizeof(Barrier));
    L.ghdr = take(sizeof(GlobalHdr));
    L.seghdr = take(sizeof(SegHdr) * S);
    L.zero_bytes = o - L.barrier;
    L.clean = take(sizeof(uint32_t));
    L.lstate = take(sizeof(LayerState) * 2 * S);
    L.hist = take(sizeof(uint32_t) * 2 * S * kHistBins);
    L.partial_sf = take(sizeof(int32_t) * S * kMaxBlocks);
    L.partial_cmp = take(sizeof(int32_t) * kMaxBlocks);
    L.pitem = take(sizeof(int32_t) * kMaxItems);
    L.trace = take(sizeof(hav_layer_trace) * kMaxLevels * S * kMaxLayers);
    L.ptimes = take(sizeof(unsigned long long) * 2 * kPhaseTimes);
    for (int b = 0; b < 2; ++b) {
        L.ord[b] = take(16 * static_cast<size_t>(N) + 16);
        L.orig[b] = take(sizeof(int32_t) * N + 16);
        L.taken[b] = take(sizeof(uint32_t) * L.taken_words);
    }
    for (int b = 0; b < kTableSets; ++b) L.dirty[b] = take(sizeof(uint32_t) * L.dirty_slots + 16);
    L.wpre = take(sizeof(uint32_t) * L.taken_words);
    L.posof = take(sizeof(int32_t) * N + 16);
    L.bkt = take(sizeof(uint32_t) * 2 * 4096 * static_cast<size_t>(S));  // counts and cursors per segment
    L.prefix = take(sizeof(int32_t) * HAV_MAX_ITERS * S);
    for (int b = 0; b < kTableSets; ++b) L.tabk[b] = take(sizeof(unsigned long long) * L.tab_slots);
    L.tabv = take(sizeof(unsigned long long) * L.tab_slots);
    L.cand = take(sizeof(Cand) * L.cand_slots);
    L.total = align_up(o, 256);
    return L;
}

// Everything one launch needs, passed by value as the kernel's parameter
// block (about 10 KB), so a captured CUDA graph replays exactly this plan.
struct Plan {
    const float* points;      // level-0 input (device)
    unsigned char* ws;        // workspace base (device)
    Layout lay;
    int32_t* out[kMaxLevels]; // per-level outputs (device)
    unsigned long long* ptimes;  // phase timer records, or null (HAV_FLAG_PHASE_TIMES)
    int32_t ptimes_cap;
    int32_t chunk_min;           // smallest work item (points)
    int64_t spec_n[3];           // level sizes up to which a pass looks 4, 3, 2 steps ahead
    int32_t S, L, layers, ratio, t_max, sigma_num, sigma_den, nblocks;
    float aspect[3];
    int32_t select;              // HAV_SELECT_*
    uint32_t seed;               // draws of HAV_SELECT_RANDOM
    float fixed_s;               // > 0: fixed voxel size, no search
    int32_t keep_orig;           // write the last level's original indices (a cluster launch follows)
    int32_t search;              // HAV_SEARCH_*
    int32_t test_timeout;        // HAV_FLAG_TEST_TIMEOUT: the first barrier waits for a missing block
    int32_t test_table_full;     // HAV_FLAG_TEST_TABLE_FULL: segment 0's tables keep 64 slots
    int32_t table_log2;          // per-segment table capacity nextpow2(2^table_log2 n) (<= lay.table_log2)
    int32_t pass_shape;          // points loaded ahead / probes in flight per thread: kPassShapes[pass_shape]
    int64_t off0[kMaxSegments + 1];       // level-0 segment offsets
    int32_t m[kMaxLevels][kMaxSegments];  // budgets per level and segment
};

// The Table 6 fields of hav_params: a representative rule, its seed, a fixed
// voxel size; the variants that report other coordinates or skip the search
// run one layer.
inline hav_status check_variant_params(const hav_params* p) {
    if (p->select < HAV_SELECT_CENTRE_CLOSEST || p->select > HAV_SELECT_CENTRE) return HAV_ERR_INVALID;
    if (p->search != HAV_SEARCH_BISECT && p->search != HAV_SEARCH_GUIDED) return HAV_ERR_INVALID;
    if (!(p->fixed_s >= 0.0f) || !std::isfinite(p->fixed_s)) return HAV_ERR_INVALID;
    if ((p->fixed_s > 0.0f || p->select == HAV_SELECT_MEAN || p->select == HAV_SELECT_CENTRE) && p->layers != 1)
        return HAV_ERR_INVALID;
    return HAV_OK;
}

// Launchers: each launch_* returns the number of kernels it enqueued on
// `stream`, or -1 if a launch failed.  Grid-wide sampler (hav_sampler.cu).
int max_coresident_blocks(int device);
int launch_chain(const Plan& plan, cudaStream_t stream);
// Voxel count at one size: a hav_status; *launched receives the kernels enqueued.
int count_voxels(const float* points, int64_t n, float s, const float aspect[3],
                 unsigned char* ws, const Layout& lay, int64_t* K, int* launched, cudaStream_t stream);
int fps_coresident_blocks(int device);
// Small levels on thread-block clusters (hav_small.cu).
// small_clusters(device, q): clusters of q CTAs (8 or 16) that run at once
// (<= 0: none), after setting the kernel's launch attributes; q = 1 sets the
// single-CTA kernel's (1, or -1 on failure).  launch_small runs levels
// [first_level, plan.L) on nclusters clusters of q CTAs.
int small_clusters(int device, int q);
int launch_small(const Plan& plan, int first_level, int q, int nclusters, cudaStream_t stream);
// The same on single CTAs (one per segment), for levels of at most kSoloMax points.
constexpr int kSoloMax = 4096;
constexpr int kSoloAlone = 1024;  // a single segment this small goes to one CTA, not a cluster
int launch_solo(const Plan& plan, int first_level, int nblocks, cudaStream_t stream);
// Grouping around centres (hav_group.cu); the blocks of its cooperative grid build.
int group_coresident_blocks(int device);
int launch_ball_query(const float* points, long long n, const int32_t* centres, long long m, float radius,
                      int nsample, int32_t* out_idx, float* out_xyz, unsigned char* ws, const Layout& lay,
                      int32_t* status, int nblocks, cudaStream_t stream);
// Subset point spacing (hav_spacing.cu), and its histogram over bin edges.
// the spacing of a subset of 2 to max_points points on a grid (3 launches)
int launch_spacing_grid(const float* points, long long n, const int32_t* idx, long long m, float* out_d2,
                        unsigned char* ws, const Layout& lay, int32_t* status, int nblocks, cudaStream_t stream);
int launch_spacing(const float* points, long long n, const int32_t* idx, long long m, float* out_d2,
                   int32_t* status, int sms, cudaStream_t stream);
constexpr int kHistEdgesMax = HAV_SPACING_MAX_BINS + 1;
struct HistEdges {
    float e[kHistEdgesMax];
    int32_t nbins;
};
int launch_spacing_hist(const float* d2, long long m, const HistEdges& edges, unsigned long long* counts,
                        cudaStream_t stream);
// Representative coordinates after a one-layer call (hav_repr.cu).
int launch_repr(const float* points, long long n, long long m, const int32_t* idx, float* xyz, int select,
                const float aspect[3], unsigned char* ws, const Layout& lay, cudaStream_t stream);
int launch_fps(const float* points, int n, int m, int32_t* out, unsigned char* ws, const Layout& lay, int nblocks,
               cudaStream_t stream);

}  // namespace havk
