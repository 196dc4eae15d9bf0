/*
 * hav.h -- C ABI of the GB300 (sm_103a) HAVSampler library, libhav.so.
 *
 * HAVSampler (arXiv 2305.14306) picks m of n xyz points: it voxelises the
 * cloud (Section 3.2, Eq. 2), keeps the point closest to each occupied
 * voxel's centre (Section 3.2, "Center-closest Point Sampling"), searches the
 * voxel size by bisection until the occupied-voxel count K lies in
 * [m, (1 + sigma) m] (Section 3.3, "AVS"), and does so over k coarse-to-fine
 * layers whose budgets grow 4x per layer and sum to m (Section 3.4, Eq. 3).
 *
 * Conventions shared by every entry point:
 *   - points are float32 x/y/z interleaved (array of structs, 12 bytes per
 *     point), in DEVICE memory, owned by the caller, never modified;
 *   - output indices are int32, ascending within each cloud, written to
 *     caller-owned DEVICE memory;
 *   - calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream); argument errors are returned synchronously and nothing
 *     is enqueued; data-dependent errors (non-finite input, key range,
 *     timeouts) are recorded on the device and read with hav_status_get();
 *   - the context owns all scratch memory (hash tables, masks, traces), is
 *     bound to the device current at creation, and must not be used by two
 *     streams at once (calls on one context serialise on its workspace);
 *   - the arithmetic is plain IEEE binary32 rounded to nearest without fused
 *     multiply-add, so results are bit-identical to any conforming restatement
 *     of the same procedure.
 *
 * Readings of the paper fixed by this library (the text leaves them open):
 *   - v = s * aspect, with the scalar s bisected over (0, s_hi], s_hi the
 *     largest bounding-box extent divided by its aspect component (Section 3.3);
 *   - acceptance when m_l <= K <= m_l + floor(m_l * sigma); after t_max steps
 *     without acceptance, s* = lo if lo > 0 (too many voxels: cut off), else
 *     s* = hi (too few: shortfall fill) (Section 3.3);
 *   - the centre-closest rule compares squared distances; ties go to the
 *     lowest point index (Section 3.2);
 *   - "cut off" keeps the m_l voxels whose SplitMix64-finalised packed key is
 *     smallest; a shortfall adds untaken points in ascending index order;
 *   - layer budgets m_l = floor(m * r^(l-1) / sum_j r^(j-1)), the last layer
 *     takes the remainder (Eq. 3, r = 4);
 *   - voxel keys pack the three cell indices, made relative to the bounding
 *     box's minimum cell, into 21 bits each (t_max <= 20 keeps them in range).
 */
#ifndef HAV_H
#define HAV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HAV_OK = 0,
    HAV_ERR_INVALID = 1,     /* bad argument; nothing was enqueued */
    HAV_ERR_NONFINITE = 2,   /* a coordinate is NaN or infinite */
    HAV_ERR_TABLE_FULL = 3,  /* a hash probe ran through a whole table (cannot happen
                                with the library's sizing; reported, never trapped) */
    HAV_ERR_TIMEOUT = 4,     /* a bounded device wait gave up; the call's output is void */
    HAV_ERR_NOMEM = 5,       /* the context's workspace is too small for this call */
    HAV_ERR_CUDA = 6,        /* a CUDA runtime call failed */
    HAV_ERR_RANGE = 7        /* a voxel cell index does not fit 21 bits, or a quotient
                                is not a finite integer (extreme coordinates) */
} hav_status;

/* Sampler parameters.  hav_params_default() gives the paper's settings
 * (Section 4.1): sigma = 0.05, t_max = 20, k = 2 layers, ratio 4. */
typedef struct {
    int32_t sigma_num;    /* tolerance sigma = sigma_num / sigma_den, >= 0 */
    int32_t sigma_den;    /* > 0 */
    int32_t t_max;        /* bisection steps, 0..20 */
    int32_t layers;       /* k, 1..8 */
    int32_t layer_ratio;  /* budget ratio between consecutive layers, 1..64 */
    float aspect[3];      /* r: the voxel is v = s * r; each component finite, > 0 */
    uint32_t flags;       /* 0, or HAV_FLAG_PHASE_TIMES / HAV_FLAG_TEST_TIMEOUT /
                             HAV_FLAG_TEST_TABLE_FULL (context calls only) */
    int32_t select;       /* representative of a voxel (Table 6 of Section 4.5):
                             HAV_SELECT_CENTRE_CLOSEST (the method, default),
                             HAV_SELECT_RANDOM, HAV_SELECT_MEAN, HAV_SELECT_CENTRE */
    uint32_t seed;        /* draws of HAV_SELECT_RANDOM */
    float fixed_s;        /* 0: adaptive voxel (Section 3.3); > 0: fixed voxel
                             v = fixed_s * aspect, no search (Table 6 "Fix") */
    int32_t search;       /* HAV_SEARCH_BISECT (default) or HAV_SEARCH_GUIDED */
} hav_params;

/* Voxel representatives (hav_params.select).  CENTRE_CLOSEST keeps the point
 * nearest the voxel centre (Section 3.2).  RANDOM keeps, per voxel, the point
 * with the smallest draw of the counter-based SplitMix64 generator (Steele,
 * Lea, Flood 2014) started at `seed`, counter = the point's index in the
 * call's input (per segment); the high 32 bits of the draw decide, ties go to
 * the lowest index.  MEAN and CENTRE are not points of the cloud: they keep the
 * centre-closest indices, and hav_sample_xyz reports the voxel mean or the
 * voxel centre as their coordinates.  MEAN, CENTRE and fixed_s > 0 need
 * layers == 1, as in Table 6. */
#define HAV_SELECT_CENTRE_CLOSEST 0
#define HAV_SELECT_RANDOM 1
#define HAV_SELECT_MEAN 2
#define HAV_SELECT_CENTRE 3

/* Start of the Section 3.3 search (hav_params.search).  BISECT bisects over
 * (0, s_hi], s_hi the largest bounding-box extent over the aspect.  GUIDED
 * starts each search at a guess g and doubles up from it while the counts
 * stay above (1 + sigma) m_l; after the first count below m_l, or once
 * 2 * lo would reach hi, it bisects as BISECT does.  g = s_hi / sqrt(m_l) for
 * a cloud's first search in the call; then g = s_prev * sqrt(m_prev / m_l)
 * from the cloud's previous search (layers and levels of one call; s_prev
 * its chosen size, m_prev its budget), the surface law K ~ s^-2.  Products,
 * quotients and square roots are binary32, rounded to nearest; g >= s_hi
 * gives the plain bisection.  The paper bounds the search by
 * ceil(log 1/sigma) steps, which needs a start near s*; it does not say how
 * to start, and both modes stop by its rule. */
#define HAV_SEARCH_BISECT 0
#define HAV_SEARCH_GUIDED 1
/* Under BISECT every layer of a level starts with the same sizes s_hi / 2,
 * s_hi / 4, ... while its counts stay below m_l.  Two bounds settle such a
 * step without a pass (hav_layer_trace.bounded): a later layer's points are a
 * subset of an earlier layer's, so its count is at most the earlier layer's
 * count at the same size; and no count exceeds the number of grid cells the
 * bounding box spans, the product over the axes of
 * floor(max / v) - floor(min / v) + 1.  Where the smaller bound is below m_l
 * the step has too few voxels.  The sizes, decisions and output are those of
 * the plain bisection. */

/* Record a device timestamp after every grid-wide phase of the call (for
 * profiling; read back with hav_phase_times_get). */
#define HAV_FLAG_PHASE_TIMES 1u

/* Test hook for the failure path of the bounded device waits: the call's
 * first grid-wide barrier waits for one block more than the launch has, so
 * every block gives up after the bounded wait (about 2 s), the call's output
 * is void and its status is HAV_ERR_TIMEOUT.  Nothing faults or hangs; the
 * context stays usable and its next call empties the tables first.  The
 * levels run on the grid kernel whatever the context's cluster setting. */
#define HAV_FLAG_TEST_TIMEOUT 2u

/* Test hook for the full-table path: the hash tables of segment 0 keep the
 * smallest capacity (64 slots), so a first segment with more than 64
 * occupied voxels reports HAV_ERR_TABLE_FULL (its probes end after one sweep
 * of the table) and receives indices 0..m-1 like any segment in error; the
 * other segments of the call are unaffected.  Grid kernel only. */
#define HAV_FLAG_TEST_TABLE_FULL 4u

/* One layer of one call, as the device evaluated it (for tests and the
 * roofline's algorithmic-byte count). */
#define HAV_MAX_ITERS 20
typedef struct {
    int64_t m_l;                /* the layer's budget */
    int64_t k_max;              /* m_l + floor(m_l * sigma) */
    int64_t k_star;             /* occupied voxels at s* among the layer's points */
    int64_t n_in;               /* points entering the layer (untaken so far) */
    int32_t iters;              /* bisection steps evaluated */
    int32_t accepted;           /* 1 if a step landed in [m_l, k_max] */
    float s_hi;                 /* top of the bisection bracket */
    float s_star;               /* chosen scalar voxel size */
    float s[HAV_MAX_ITERS];     /* s evaluated at each step */
    int64_t K[HAV_MAX_ITERS];   /* occupied-voxel count at that s: exact, except
                                   for the steps in `bounded` */
    uint32_t bounded;           /* bit t: step t was decided without a count.  K[t]
                                   is then an upper bound below m_l (an earlier
                                   layer's count at the same s on a superset of
                                   the points, or the grid cells the bounding box
                                   spans): the step has too few voxels */
    int32_t reserved;
} hav_layer_trace;

typedef struct hav_ctx hav_ctx;
typedef struct CUstream_st* hav_stream;  /* same type as cudaStream_t */

/* Fill *p with the paper's defaults (centre-closest, adaptive voxel).  p must
 * not be NULL. */
void hav_params_default(hav_params* p);

/* Create a context on the CURRENT device with workspace for calls of up to
 * max_points points in total (all segments of a call, < 2^30) and up to
 * max_segments segments (1..256).  Allocates device memory once; no call
 * allocates afterwards.  Returns HAV_ERR_NOMEM if cudaMalloc fails,
 * HAV_ERR_CUDA if the device cannot run the kernels (e.g. not sm_103). */
hav_status hav_context_create(hav_ctx** out, int64_t max_points, int32_t max_segments);

/* Number of thread blocks (one per SM) the context's sampler launches use:
 * 1..the device's co-resident maximum, or 0 for that maximum (the default).
 * Contexts limited to disjoint shares of the SMs can run their calls
 * concurrently on different streams (the serving loop does this).  A call
 * with S segments uses at least ceil(S / 7) blocks whatever the setting
 * (HAV_ERR_INVALID if that exceeds the co-resident maximum). */
hav_status hav_context_set_blocks(hav_ctx* ctx, int32_t nblocks);

/* Launch-shape knobs of a context (the autotuner sets them; the paper has no
 * counterpart).  No setting changes a result: every call returns the same
 * indices, status and trace for every tuning, because the bisection's
 * decisions (Section 3.3) and the per-voxel choices (Section 3.2) depend only
 * on the points, never on how the work is cut. */
typedef struct {
    int64_t spec_points[3];  /* level sizes (points, all segments) up to which one
                                pass evaluates 4, 3 or 2 bisection steps at once
                                (larger levels: one step per pass); 0 <= [0] <= [1]
                                <= [2] <= 2^31 */
    int32_t chunk_min;       /* smallest work item in points, 1..65536 */
    int32_t nblocks;         /* as in hav_context_set_blocks (0: all co-resident) */
    int32_t small_points;    /* levels whose every segment has at most this many
                                points (0..32768; 0: none; default 32768 where
                                the device launches 8-CTA clusters) run on
                                thread-block clusters, one cluster of 8 SMs per
                                segment, the voxel table in distributed shared
                                memory (same results; one size per pass, settled
                                steps as in the grid kernel; same conditions as
                                solo_points) */
    int32_t solo_points;     /* levels whose every segment has at most this many
                                points (0..4096; 0: none; default 4096) run on
                                single CTAs, one per segment, its points and
                                voxel table in the CTA's shared memory and each
                                phase ended by a block barrier (same results;
                                used when select is CENTRE_CLOSEST or RANDOM
                                and no flag is set, either search start).  Levels run on the grid-wide kernel until
                                the first level within small_points, then on
                                clusters until the first level within
                                solo_points that has more segments than the
                                device runs clusters at once, or at most 1,024
                                points per segment */
    int32_t cluster_ctas;    /* CTAs per cluster of the small_points levels:
                                0 (default) = 16 where the call's segments all
                                get a 16-CTA cluster at once within the
                                context's blocks, else 8; or 8, or 16 (a
                                cluster size above the portable 8; only where
                                the device schedules it) */
    int32_t table_log2;      /* load factor of the grid-wide kernel's voxel
                                tables: a segment's table has nextpow2(2^f n)
                                slots for its n points, f = table_log2 in 1..3
                                (default 1: at most half full).  A value above the
                                context's current workspace makes this call
                                allocate a larger one (it first waits for the
                                device); no sampling call allocates */
    int32_t pass_shape;      /* the grid-wide kernel's instantiation: points each
                                thread loads ahead in a pass and global probes it
                                keeps in flight, 0: (2, 1) (default), 1: (1, 1),
                                2: (2, 2), 3: (4, 1) */
} hav_tuning;

/* Copy the context's tuning into *out (the defaults after creation:
 * {0, 4096, 65536}, 64, the co-resident maximum, 32768, 4096, 0, 1, 0). */
hav_status hav_context_get_tuning(const hav_ctx* ctx, hav_tuning* out);

/* Replace the context's tuning.  HAV_ERR_INVALID (and no change) on a value
 * outside the ranges above; HAV_ERR_NOMEM (and no change) when a larger
 * table_log2 needs a workspace that cannot be allocated.  Takes effect from
 * the next call. */
hav_status hav_context_set_tuning(hav_ctx* ctx, const hav_tuning* t);

/* Number of device kernels the context's calls have launched since it was
 * created (memsets and copies excluded), in *out (HOST).  A level chain
 * launches one to three kernels (hav_tuning), hav_sample_xyz one more, the
 * spacing call two (three for a subset searched on a grid), its histogram
 * one more, the farthest-point call one, the ball query two.
 * HAV_ERR_INVALID on a NULL argument. */
hav_status hav_context_launches(const hav_ctx* ctx, uint64_t* out);

/* Release the context and its device memory.  Waits for the device.  NULL is ignored. */
void hav_context_destroy(hav_ctx* ctx);

/* Device bytes a context of this size holds. */
size_t hav_workspace_bytes(int64_t max_points, int32_t max_segments);

/* Sample m of n points (one cloud, one level).  points: device, n*3 floats;
 * out_idx: device, m int32, receives ascending indices into points.
 * 0 <= m <= n < 2^31; m == 0 enqueues nothing.  Section 3, Eq. 3. */
hav_status hav_sample(hav_ctx* ctx, const float* points, int64_t n, int64_t m,
                      const hav_params* params, int32_t* out_idx, hav_stream stream);

/* hav_sample, plus the coordinates that stand for each selected index
 * (Table 6 point-selection strategies): out_xyz (device, 3m floats) receives,
 * for an index that represents its voxel at the chosen size, the point itself
 * (CENTRE_CLOSEST, RANDOM), the voxel centre v * (g + 0.5) in binary32
 * (CENTRE) or the voxel mean (MEAN); for an index added by the shortfall fill,
 * the point itself.  The mean is order-independent: with 2^(k-1) <= M < 2^k
 * for M the largest |coordinate| of the cloud (k = 0 when M = 0), each
 * coordinate x is taken as X = round-half-even(x * 2^(30-k)) and a voxel's
 * mean is RN32(RN64(RN64(sum X) / count) * 2^(k-30)).  Needs layers == 1.
 * Runs after the sampler on the same stream; the context's workspace is the
 * scratch. */
hav_status hav_sample_xyz(hav_ctx* ctx, const float* points, int64_t n, int64_t m,
                          const hav_params* params, int32_t* out_idx, float* out_xyz,
                          hav_stream stream);

/* Level chain on one cloud: level j+1 samples the points kept by level j (in
 * ascending order), the way successive set-abstraction stages of a point
 * network down-sample (Section 4.1).  m_levels: HOST array of num_levels
 * budgets, non-increasing, m_levels[0] <= n.  out_idx: HOST array of
 * num_levels DEVICE pointers; out_idx[j] receives m_levels[j] ascending
 * indices into the ORIGINAL cloud.  The levels run in at most three
 * launches on `stream`: the grid-wide kernel for the large levels, then the
 * cluster and single-CTA kernels for the small ones (hav_tuning). */
hav_status hav_sample_levels(hav_ctx* ctx, const float* points, int64_t n,
                             const int64_t* m_levels, int32_t num_levels,
                             const hav_params* params, int32_t* const* out_idx,
                             hav_stream stream);

/* Batched, segmented form: num_segments clouds stored back to back in
 * points.  seg_offsets: HOST array of num_segments+1 point offsets (first 0,
 * non-decreasing).  seg_m: HOST array [num_levels][num_segments] of budgets,
 * each level's budget <= the previous level's for that segment.  out_idx:
 * HOST array of num_levels DEVICE pointers; out_idx[j] receives, for each
 * segment s in order, seg_m[j][s] ascending indices LOCAL to segment s (into
 * the segment's original points).  Persistent launches (as in
 * hav_sample_levels) run every level of every segment; each segment's result
 * equals the single-cloud call's. */
hav_status hav_sample_batched(hav_ctx* ctx, const float* points, const int64_t* seg_offsets,
                              const int64_t* seg_m, int32_t num_segments, int32_t num_levels,
                              const hav_params* params, int32_t* const* out_idx,
                              hav_stream stream);

/* Synchronise `stream` and return the status of the last call enqueued on
 * this context: HAV_OK, or the first error any segment hit.  per_segment
 * (HOST, nullable) receives each segment's status: one entry per segment of
 * the last call, so it must hold at least that call's num_segments entries
 * (the context's max_segments always suffices).
 * A segment in error still gets seg_m indices (0..m-1) so that the other
 * segments' output positions stay valid. */
hav_status hav_status_get(hav_ctx* ctx, hav_stream stream, int32_t* per_segment);

/* Synchronise `stream` and copy the last call's per-layer traces to `out`
 * (HOST), ordered [level][segment][layer]; returns the number of records
 * written (<= max_records), or -1 on error. */
int32_t hav_trace_get(hav_ctx* ctx, hav_stream stream, hav_layer_trace* out, int32_t max_records);

/* Synchronise `stream` and copy the phase timer of the last call made with
 * HAV_FLAG_PHASE_TIMES: t_ns[k] is the device %globaltimer (ns) when phase k
 * ended, tag[k] = phase << 24 | level << 16 | layer << 8 | pass, with phase
 * 0 kernel start, 1 bbox, 2 bisection pass, 3 selection, 4 cut-off classify,
 * 5 cut-off resolve, 6 shortfall, 7 compaction count, 8 compaction scatter,
 * 9 / 10 Morton bucketing count / scatter.  The grid kernel records block 0's
 * phases, and the small-level kernels that continue the call append those of
 * their first cluster (or CTA); the timer does not change which kernel runs
 * a level.
 * HOST buffers of max_records entries; returns the number written, or -1.
 * Records of an earlier call may follow the last valid one if this call
 * recorded fewer. */
int32_t hav_phase_times_get(hav_ctx* ctx, hav_stream stream, uint64_t* t_ns, uint32_t* tag,
                            int32_t max_records);

/* Test hook for Cnt(P, v) of Section 3.3: exact number of occupied voxels at
 * v = s * aspect over all n points (bounding box from the same points).
 * Synchronous: *K (HOST) is valid on return. */
hav_status hav_count(hav_ctx* ctx, const float* points, int64_t n, float s,
                     const float aspect[3], int64_t* K, hav_stream stream);

/* Farthest point sampling, the comparator of Section 3.1 (Eq. 1): start at
 * index 0, repeatedly take the point farthest (squared binary32 distance,
 * ties to the lowest index) from the points taken so far.  points: device,
 * n*3 floats; out_idx: device, m int32 in selection order.  0 <= m <= n <=
 * the context's max_points.  One launch: up to 32,768 points one cluster of
 * 8 CTAs with one cluster barrier per selected point, above that a
 * cooperative grid with one grid barrier per selected point (each block's
 * share of the points and their distances held in its shared memory where 16
 * bytes a point fit, about 1.9 M points on 152 SMs); asynchronous on
 * `stream`; a grid barrier timeout is read with hav_status_get. */
hav_status hav_fps(hav_ctx* ctx, const float* points, int64_t n, int64_t m, int32_t* out_idx,
                   hav_stream stream);

/* Point spacing of a sampled subset, the quantity whose distributions Fig. 3
 * (Section 3.1) compares across samplers: out_d2[r] = the smallest squared
 * distance from subset point r to any other subset point, binary32
 * (dx*dx + dy*dy) + dz*dz without fusion (+inf when m == 1).  points: device,
 * n*3 floats; idx: device, m int32 indices into points (any order, repeats
 * allowed: a repeated point has spacing 0); out_d2: device, m floats.  An
 * index outside [0, n) is skipped and reported as HAV_ERR_INVALID by
 * hav_status_get.  Exact nearest-neighbour search: all pairs below 32,768
 * subset points (two launches); from there, when the subset fits the
 * context's max_points, on a grid built over the subset (three launches;
 * cells of 1/256 of the largest extent searched shell by shell with an exact
 * stopping bound: 0.2 ms for m = 262,144 on GB300, against 31 ms for all
 * pairs).  A measurement, not part of the sampler. */
hav_status hav_spacing(hav_ctx* ctx, const float* points, int64_t n, const int32_t* idx, int64_t m,
                       float* out_d2, hav_stream stream);

/* hav_spacing plus the histogram of the spacings that Fig. 3 (Section 3.1)
 * plots, over bin edges the caller chooses.  edges: HOST, nbins + 1 finite
 * binary32 squared distances, strictly ascending; 1 <= nbins <=
 * HAV_SPACING_MAX_BINS.  out_d2: device, m floats (as hav_spacing writes
 * them).  out_counts: device, nbins + 2 uint64: out_counts[0] counts the
 * spacings below edges[0], out_counts[nbins + 1] those above edges[nbins],
 * and out_counts[1 + i] those with edges[i] <= d2 < edges[i + 1], the last
 * bin also taking d2 == edges[nbins] (the bins of numpy.histogram).  Integer
 * counts, exact.  Three launches on `stream`. */
#define HAV_SPACING_MAX_BINS 1024
hav_status hav_spacing_histogram(hav_ctx* ctx, const float* points, int64_t n, const int32_t* idx, int64_t m,
                                 const float* edges, int32_t nbins, float* out_d2, uint64_t* out_counts,
                                 hav_stream stream);

/* Grouping around sampled centres, the step that follows sampling in the
 * sample-group-aggregate block of point networks (Section 3.1; the ball query
 * of PointNet++): for centre j (the point centres[j]), the nsample smallest
 * point indices k with (dx*dx + dy*dy) + dz*dz < radius*radius (binary32, no
 * fusion), ascending; if fewer qualify, the remaining slots repeat the
 * smallest (the centre itself always qualifies).  out_xyz, when not NULL,
 * receives p_k - c_j for every slot (the block's gather, fused).
 * points: device, n*3 floats, n <= the context's max_points; centres: device,
 * m int32 (e.g. the indices hav_sample returned); out_idx: device,
 * m*nsample int32; out_xyz: device, m*nsample*3 floats or NULL.
 * radius finite and > 0; 1 <= nsample <= 256.  A centre outside [0, n) gets
 * zeros and HAV_ERR_INVALID in hav_status_get.  Two launches on `stream`:
 * a cooperative one that builds a uniform grid of cells at least the radius
 * wide over the points (grid barriers with bounded waits; a wait that gives
 * up is read as HAV_ERR_TIMEOUT), and the query, one warp per centre.  Uses
 * the context's workspace (the phase-timer records of an earlier call are
 * overwritten). */
hav_status hav_ball_query(hav_ctx* ctx, const float* points, int64_t n, const int32_t* centres, int64_t m,
                          float radius, int32_t nsample, int32_t* out_idx, float* out_xyz, hav_stream stream);

/* Static description of a status code. */
const char* hav_status_string(hav_status s);

/* hav_sample without a context and without any allocation.  The paper has no
 * counterpart: this entry point serves callers that may not call cudaMalloc
 * (code running inside another framework's memory pool or a fixed memory
 * budget, plugin hosts that forbid allocation after start-up, real-time loops
 * where an allocation and the synchronisation it can imply are not allowed).
 * It computes exactly what hav_sample computes for one cloud, one level.
 *
 * Scratch: a static __device__ array of 8 MiB inside libhav.so, enough for
 * one cloud of at most 32,768 points; every GPU that loads the library holds
 * it until the process exits.  n > 32,768 returns HAV_ERR_NOMEM and enqueues
 * nothing.  Every call looks up the array's device address (no allocation).
 * The first call on a device, and the first after the library's module is
 * loaded again in a new context (after cudaDeviceReset), also sets the
 * sampler kernel's launch attribute and sizes its grid; make that first call
 * before any stream capture.  All calls on a device share the one array:
 * calls that overlap on the GPU (different streams, or host threads without
 * ordering) race and corrupt each other's results; serialise them.
 *
 * The call runs the grid-wide sampler without speculative look-ahead (one
 * bisection step per pass; the scratch holds no room for extra candidate
 * tables): the indices, status and search are those of hav_sample, but a
 * level takes more passes, so a call is slower than hav_sample's.
 *
 * points: device, n*3 floats; out_idx: device, m int32 (ascending indices);
 * status_out: device int32 or NULL, receives the call's hav_status when the
 * work completes on `stream`.  Argument errors are returned synchronously. */
hav_status hav_sample_noalloc(const float* points, int64_t n, int64_t m,
                              const hav_params* params, int32_t* out_idx,
                              int32_t* status_out, hav_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* HAV_H */
