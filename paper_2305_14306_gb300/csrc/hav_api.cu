// C ABI of libhav.so (declared in include/hav.h): argument validation, the
// launch plan, and status / trace read-back.  Every step of the sampler runs
// in the kernels of hav_sampler.cu; this file only marshals.

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "hav.h"
#include "hav_internal.h"

struct hav_ctx {
    int device;
    int nblocks;
    int max_blocks;
    int chunk_min;
    int64_t spec_n[3];
    int small_nc;      // 8-CTA clusters of the small-level kernel that fit at once (0: none)
    int big_nc;        // 16-CTA clusters that fit at once (0: none)
    int cluster_ctas;  // CTAs per cluster: 0 (by the call's segment count), 8 or 16
    int small_points;  // largest level run on clusters (0: never)
    int solo_ok;       // the single-CTA kernel can be launched
    int solo_points;   // largest level run on single CTAs (0: never)
    int table_log2;    // grid-kernel tables of capacity nextpow2(2^table_log2 n)
    int pass_shape;    // grid-kernel instantiation (points loaded ahead, probes in flight)
    int fps_nblocks;
    int group_nblocks;  // co-resident blocks of the ball query's cooperative grid build
    havk::Layout lay;
    unsigned char* ws;
    int32_t last_S;
    int32_t last_L;
    int32_t last_layers;
    uint64_t launches;  // kernels enqueued by this context's calls
};

namespace {

// Adds the kernels a launcher enqueued to the context's count; false on a failed launch.
bool counted(hav_ctx* ctx, int launched) {
    if (launched < 0) return false;
    ctx->launches += static_cast<uint64_t>(launched);
    return true;
}

hav_status check_params(const hav_params* p) {
    if (!p) return HAV_ERR_INVALID;
    if (p->sigma_num < 0 || p->sigma_den <= 0) return HAV_ERR_INVALID;
    if (p->t_max < 0 || p->t_max > HAV_MAX_ITERS) return HAV_ERR_INVALID;
    if (p->layers < 1 || p->layers > havk::kMaxLayers) return HAV_ERR_INVALID;
    if (p->layer_ratio < 1 || p->layer_ratio > 64) return HAV_ERR_INVALID;
    // budgets m * ratio^(layers-1) must fit int64 for m < 2^31
    long long w = 1;
    for (int i = 1; i < p->layers; ++i) {
        w *= p->layer_ratio;
        if (w > (1ll << 31)) return HAV_ERR_INVALID;
    }
    // sigma * m must stay below 2^31 in the tolerance bound
    if (static_cast<long long>(p->sigma_num) > 64ll * p->sigma_den) return HAV_ERR_INVALID;
    for (int a = 0; a < 3; ++a)
        if (!(p->aspect[a] > 0.0f) || !std::isfinite(p->aspect[a])) return HAV_ERR_INVALID;
    if ((p->flags & ~static_cast<uint32_t>(HAV_FLAG_PHASE_TIMES | HAV_FLAG_TEST_TIMEOUT |
                                           HAV_FLAG_TEST_TABLE_FULL)) != 0)
        return HAV_ERR_INVALID;
    return havk::check_variant_params(p);
}

}  // namespace

extern "C" {

void hav_params_default(hav_params* p) {
    if (!p) return;
    p->sigma_num = 5;
    p->sigma_den = 100;
    p->t_max = 20;
    p->layers = 2;
    p->layer_ratio = 4;
    p->aspect[0] = p->aspect[1] = p->aspect[2] = 1.0f;
    p->flags = 0;
    p->select = HAV_SELECT_CENTRE_CLOSEST;
    p->seed = 0;
    p->fixed_s = 0.0f;
    p->search = HAV_SEARCH_BISECT;
}

const char* hav_status_string(hav_status s) {
    switch (s) {
        case HAV_OK: return "ok";
        case HAV_ERR_INVALID: return "invalid argument";
        case HAV_ERR_NONFINITE: return "non-finite coordinate";
        case HAV_ERR_TABLE_FULL: return "hash table full";
        case HAV_ERR_TIMEOUT: return "bounded device wait timed out";
        case HAV_ERR_NOMEM: return "workspace too small or allocation failed";
        case HAV_ERR_CUDA: return "CUDA runtime error";
        case HAV_ERR_RANGE: return "voxel cell index out of range";
    }
    return "unknown status";
}

size_t hav_workspace_bytes(int64_t max_points, int32_t max_segments) {
    if (max_points < 1 || max_segments < 1) return 0;
    return havk::make_layout(max_points, max_segments).total;
}

hav_status hav_context_create(hav_ctx** out, int64_t max_points, int32_t max_segments) {
    if (!out) return HAV_ERR_INVALID;
    *out = nullptr;
    if (max_points < 1 || max_points >= (1ll << 30)) return HAV_ERR_INVALID;  // table slots index in 32 bits
    if (max_segments < 1 || max_segments > havk::kMaxSegments) return HAV_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HAV_ERR_CUDA;
    int major = 0, minor = 0, coop = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (major != 10 || minor != 3 || !coop) return HAV_ERR_CUDA;  // built for sm_103a only
    const int nb = havk::max_coresident_blocks(dev);
    const int fnb = havk::fps_coresident_blocks(dev);
    if (nb < 1 || fnb < 1) return HAV_ERR_CUDA;
    hav_ctx* c = new hav_ctx();
    c->device = dev;
    c->nblocks = nb;
    c->max_blocks = nb;
    c->fps_nblocks = fnb;
    c->group_nblocks = havk::group_coresident_blocks(dev);
    if (c->group_nblocks < 1) {
        delete c;
        return HAV_ERR_CUDA;
    }
    c->chunk_min = havk::kChunkMin;
    c->table_log2 = 1;
    c->pass_shape = 0;
    {
        const int snc = havk::small_clusters(dev, 8);
        cudaGetLastError();
        const int bnc = havk::small_clusters(dev, 16);
        cudaGetLastError();
        const int solo = havk::small_clusters(dev, 1);
        cudaGetLastError();
        c->small_nc = snc > 0 ? snc : 0;
        c->big_nc = (snc > 0 && bnc > 0) ? bnc : 0;
        c->cluster_ctas = 0;
        c->small_points = c->small_nc > 0 ? havk::kSmallMax : 0;
        c->solo_ok = (solo > 0) ? 1 : 0;
        c->solo_points = c->solo_ok ? havk::kSoloMax : 0;
    }
    c->spec_n[0] = havk::kSpecN4;
    c->spec_n[1] = havk::kSpecN3;
    c->spec_n[2] = havk::kSpecN2;
    c->lay = havk::make_layout(max_points, max_segments);
    if (cudaMalloc(&c->ws, c->lay.total) != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return HAV_ERR_NOMEM;
    }
    if (cudaMemset(c->ws, 0, c->lay.total) != cudaSuccess) {
        cudaFree(c->ws);
        delete c;
        return HAV_ERR_CUDA;
    }
    *out = c;
    return HAV_OK;
}

hav_status hav_context_set_blocks(hav_ctx* ctx, int32_t nblocks) {
    if (!ctx || nblocks < 0 || nblocks > ctx->max_blocks) return HAV_ERR_INVALID;
    ctx->nblocks = nblocks == 0 ? ctx->max_blocks : nblocks;
    return HAV_OK;
}

hav_status hav_context_get_tuning(const hav_ctx* ctx, hav_tuning* out) {
    if (!ctx || !out) return HAV_ERR_INVALID;
    for (int k = 0; k < 3; ++k) out->spec_points[k] = ctx->spec_n[k];
    out->chunk_min = ctx->chunk_min;
    out->nblocks = ctx->nblocks;
    out->small_points = ctx->small_points;
    out->solo_points = ctx->solo_points;
    out->cluster_ctas = ctx->cluster_ctas;
    out->table_log2 = ctx->table_log2;
    out->pass_shape = ctx->pass_shape;
    return HAV_OK;
}

hav_status hav_context_set_tuning(hav_ctx* ctx, const hav_tuning* t) {
    if (!ctx || !t) return HAV_ERR_INVALID;
    for (int k = 0; k < 3; ++k)
        if (t->spec_points[k] < 0 || t->spec_points[k] > (1ll << 31)) return HAV_ERR_INVALID;
    if (t->spec_points[0] > t->spec_points[1] || t->spec_points[1] > t->spec_points[2]) return HAV_ERR_INVALID;
    if (t->chunk_min < 1 || t->chunk_min > 65536) return HAV_ERR_INVALID;
    if (t->nblocks < 0 || t->nblocks > ctx->max_blocks) return HAV_ERR_INVALID;
    if (t->small_points < 0 || t->small_points > havk::kSmallMax) return HAV_ERR_INVALID;
    if (t->solo_points < 0 || t->solo_points > havk::kSoloMax) return HAV_ERR_INVALID;
    if (t->solo_points > 0 && !ctx->solo_ok) return HAV_ERR_INVALID;
    if (t->small_points > 0 && ctx->small_nc == 0) return HAV_ERR_INVALID;  // no cluster launch on this device
    if (t->cluster_ctas != 0 && t->cluster_ctas != 8 && t->cluster_ctas != 16) return HAV_ERR_INVALID;
    if (t->cluster_ctas == 16 && ctx->big_nc == 0) return HAV_ERR_INVALID;
    if (t->table_log2 < 1 || t->table_log2 > havk::kMaxTableLog2) return HAV_ERR_INVALID;
    if (t->pass_shape < 0 || t->pass_shape >= havk::kPassShapes) return HAV_ERR_INVALID;
    if (t->table_log2 > ctx->lay.table_log2) {
        // larger tables than the workspace holds: a new workspace (the only
        // allocation outside hav_context_create); the old one once the device is idle
        const havk::Layout lay = havk::make_layout(ctx->lay.max_points, ctx->lay.max_segments, true, t->table_log2);
        unsigned char* ws = nullptr;
        if (cudaDeviceSynchronize() != cudaSuccess) return HAV_ERR_CUDA;
        if (cudaMalloc(&ws, lay.total) != cudaSuccess) {
            cudaGetLastError();
            return HAV_ERR_NOMEM;
        }
        if (cudaMemset(ws, 0, lay.total) != cudaSuccess) {
            cudaFree(ws);
            return HAV_ERR_CUDA;
        }
        cudaFree(ctx->ws);
        ctx->ws = ws;
        ctx->lay = lay;
    }
    ctx->table_log2 = t->table_log2;
    ctx->pass_shape = t->pass_shape;
    ctx->small_points = t->small_points;
    ctx->solo_points = t->solo_points;
    ctx->cluster_ctas = t->cluster_ctas;
    for (int k = 0; k < 3; ++k) ctx->spec_n[k] = t->spec_points[k];
    ctx->chunk_min = t->chunk_min;
    ctx->nblocks = t->nblocks == 0 ? ctx->max_blocks : t->nblocks;
    return HAV_OK;
}

hav_status hav_context_launches(const hav_ctx* ctx, uint64_t* out) {
    if (!ctx || !out) return HAV_ERR_INVALID;
    *out = ctx->launches;
    return HAV_OK;
}

void hav_context_destroy(hav_ctx* ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    cudaFree(ctx->ws);
    delete ctx;
}

hav_status hav_sample_batched(hav_ctx* ctx, const float* points, const int64_t* seg_offsets,
                              const int64_t* seg_m, int32_t num_segments, int32_t num_levels,
                              const hav_params* params, int32_t* const* out_idx, hav_stream stream) {
    if (!ctx || !seg_offsets || !seg_m || !out_idx) return HAV_ERR_INVALID;
    hav_status st = check_params(params);
    if (st != HAV_OK) return st;
    if (num_segments < 1 || num_segments > ctx->lay.max_segments) return HAV_ERR_INVALID;
    if (num_levels < 1 || num_levels > havk::kMaxLevels) return HAV_ERR_INVALID;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != ctx->device) return HAV_ERR_INVALID;
    if (seg_offsets[0] != 0) return HAV_ERR_INVALID;
    for (int s = 0; s < num_segments; ++s)
        if (seg_offsets[s + 1] < seg_offsets[s]) return HAV_ERR_INVALID;
    const int64_t total = seg_offsets[num_segments];
    if (total > ctx->lay.max_points) return HAV_ERR_NOMEM;
    if (total > 0 && !points) return HAV_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(points) % 4 != 0) return HAV_ERR_INVALID;
    int64_t any_m = 0;
    for (int j = 0; j < num_levels; ++j) {
        int64_t level_sum = 0;
        for (int s = 0; s < num_segments; ++s) {
            const int64_t prev = (j == 0) ? (seg_offsets[s + 1] - seg_offsets[s])
                                          : seg_m[static_cast<int64_t>(j - 1) * num_segments + s];
            const int64_t m = seg_m[static_cast<int64_t>(j) * num_segments + s];
            if (m < 0 || m > prev) return HAV_ERR_INVALID;
            level_sum += m;
        }
        if (level_sum > 0 && !out_idx[j]) return HAV_ERR_INVALID;
        any_m += level_sum;
    }

    havk::Plan* plan = new havk::Plan();
    std::memset(plan, 0, sizeof(havk::Plan));
    plan->points = points;
    plan->ws = ctx->ws;
    plan->lay = ctx->lay;
    plan->S = num_segments;
    plan->L = num_levels;
    plan->layers = params->layers;
    plan->ratio = params->layer_ratio;
    plan->t_max = params->t_max;
    plan->sigma_num = params->sigma_num;
    plan->sigma_den = params->sigma_den;
    // a block tracks at most kLocalItems work items of a level, and a level
    // has at most nblocks + S of them at the smallest speculation depth
    const int min_blocks = (num_segments + havk::kLocalItems - 2) / (havk::kLocalItems - 1);
    plan->nblocks = ctx->nblocks < min_blocks ? min_blocks : ctx->nblocks;
    if (plan->nblocks > ctx->max_blocks) {
        delete plan;
        return HAV_ERR_INVALID;
    }
    plan->chunk_min = ctx->chunk_min;
    plan->table_log2 = ctx->table_log2;
    plan->pass_shape = ctx->pass_shape;
    for (int k = 0; k < 3; ++k) plan->spec_n[k] = ctx->spec_n[k];
    for (int a = 0; a < 3; ++a) plan->aspect[a] = params->aspect[a];
    plan->select = params->select;
    plan->seed = params->seed;
    plan->fixed_s = params->fixed_s;
    plan->search = params->search;
    plan->test_timeout = (params->flags & HAV_FLAG_TEST_TIMEOUT) ? 1 : 0;
    plan->test_table_full = (params->flags & HAV_FLAG_TEST_TABLE_FULL) ? 1 : 0;
    for (int j = 0; j < num_levels; ++j) plan->out[j] = out_idx[j];
    if (params->flags & HAV_FLAG_PHASE_TIMES) {
        plan->ptimes = reinterpret_cast<unsigned long long*>(ctx->ws + ctx->lay.ptimes);
        plan->ptimes_cap = havk::kPhaseTimes;
    }
    for (int s = 0; s <= num_segments; ++s) plan->off0[s] = seg_offsets[s];
    for (int j = 0; j < num_levels; ++j)
        for (int s = 0; s < num_segments; ++s)
            plan->m[j][s] = static_cast<int32_t>(seg_m[static_cast<int64_t>(j) * num_segments + s]);

    cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
    ctx->last_S = num_segments;
    ctx->last_L = num_levels;
    ctx->last_layers = params->layers;
    hav_status ret = HAV_OK;
    if (cudaMemsetAsync(ctx->ws + ctx->lay.barrier, 0, ctx->lay.zero_bytes, strm) != cudaSuccess) {
        ret = HAV_ERR_CUDA;
    } else if (plan->ptimes &&
               cudaMemsetAsync(plan->ptimes, 0, sizeof(unsigned long long) * 2 * havk::kPhaseTimes, strm) !=
                   cudaSuccess) {
        ret = HAV_ERR_CUDA;
    } else if (any_m > 0) {
        // levels from j0 on, where every segment has at most small_points points,
        // run on thread-block clusters, or else, where every segment has at most
        // solo_points points, on single CTAs (either search start, phase timer
        // on or off); the test hooks stay with the grid kernel, and so do the
        // calls whose representatives need the grid kernel's tables.
        const bool small_ok =
            (params->flags & ~static_cast<uint32_t>(HAV_FLAG_PHASE_TIMES)) == 0 &&
            (params->select == HAV_SELECT_CENTRE_CLOSEST || params->select == HAV_SELECT_RANDOM);
        // grid kernel for [0, j0), clusters for [j0, j1), single CTAs for [j1, L).
        // A level goes to single CTAs when it also has more segments than
        // 8-CTA clusters fit at once, or only tiny segments (measured on GB300:
        // one CTA per segment wins for many segments, a cluster for a few
        // above kSoloAlone points); later levels are no larger, so they follow.
        int j0 = num_levels, j1 = num_levels;
        for (int j = 0; j < num_levels; ++j) {
            int64_t mx = 0;
            for (int s = 0; s < num_segments; ++s) {
                const int64_t nj = (j == 0) ? seg_offsets[s + 1] - seg_offsets[s]
                                            : seg_m[static_cast<int64_t>(j - 1) * num_segments + s];
                if (nj > mx) mx = nj;
            }
            const bool clusters = small_ok && ctx->small_points > 0 && mx <= ctx->small_points;
            const bool solo = small_ok && ctx->solo_points > 0 && mx <= ctx->solo_points &&
                              (ctx->small_points == 0 || num_segments > ctx->small_nc || mx <= havk::kSoloAlone);
            if (j0 == num_levels && (clusters || solo)) j0 = j;
            if (j1 == num_levels && solo) j1 = j;
        }
        if (j0 > 0) {
            plan->L = j0;
            plan->keep_orig = (j0 < num_levels) ? 1 : 0;
            if (!counted(ctx, havk::launch_chain(*plan, strm))) ret = HAV_ERR_CUDA;
            plan->L = num_levels;
            plan->keep_orig = 0;
        }
        if (ret == HAV_OK && j0 < j1) {
            // 16-CTA clusters where every segment's cluster runs at once within
            // the context's SMs (more SMs per pass; measured on GB300: 10-13 %
            // faster than 8 on single clouds), else 8
            int q = ctx->cluster_ctas;
            if (q == 0)
                q = (ctx->big_nc > 0 && num_segments <= ctx->big_nc && 16 * num_segments <= plan->nblocks) ? 16 : 8;
            int nc = plan->nblocks / q;
            const int fit = (q == 16) ? ctx->big_nc : ctx->small_nc;
            if (nc > fit) nc = fit;
            if (nc < 1) nc = 1;
            plan->L = j1;
            plan->keep_orig = (j1 < num_levels) ? 1 : 0;
            if (!counted(ctx, havk::launch_small(*plan, j0, q, nc, strm))) ret = HAV_ERR_CUDA;
            plan->L = num_levels;
            plan->keep_orig = 0;
        }
        if (ret == HAV_OK && j1 < num_levels) {
            if (!counted(ctx, havk::launch_solo(*plan, j1, plan->nblocks, strm))) ret = HAV_ERR_CUDA;
        }
    }
    delete plan;
    return ret;
}

hav_status hav_sample_levels(hav_ctx* ctx, const float* points, int64_t n, const int64_t* m_levels,
                             int32_t num_levels, const hav_params* params, int32_t* const* out_idx,
                             hav_stream stream) {
    if (n < 0 || n >= (1ll << 31)) return HAV_ERR_INVALID;
    const int64_t offs[2] = {0, n};
    return hav_sample_batched(ctx, points, offs, m_levels, 1, num_levels, params, out_idx, stream);
}

hav_status hav_sample(hav_ctx* ctx, const float* points, int64_t n, int64_t m,
                      const hav_params* params, int32_t* out_idx, hav_stream stream) {
    if (n < 0 || n >= (1ll << 31)) return HAV_ERR_INVALID;
    const int64_t offs[2] = {0, n};
    int32_t* outs[1] = {out_idx};
    return hav_sample_batched(ctx, points, offs, &m, 1, 1, params, outs, stream);
}

hav_status hav_sample_xyz(hav_ctx* ctx, const float* points, int64_t n, int64_t m,
                          const hav_params* params, int32_t* out_idx, float* out_xyz, hav_stream stream) {
    if (!params || params->layers != 1) return HAV_ERR_INVALID;
    if (m > 0 && !out_xyz) return HAV_ERR_INVALID;
    hav_status st = hav_sample(ctx, points, n, m, params, out_idx, stream);
    if (st != HAV_OK || m == 0) return st;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return HAV_ERR_CUDA;
    if (!counted(ctx, havk::launch_repr(points, n, m, out_idx, out_xyz, params->select, params->aspect, ctx->ws,
                                        ctx->lay, reinterpret_cast<cudaStream_t>(stream))))
        return HAV_ERR_CUDA;
    return HAV_OK;
}

hav_status hav_spacing(hav_ctx* ctx, const float* points, int64_t n, const int32_t* idx, int64_t m,
                       float* out_d2, hav_stream stream) {
    if (!ctx || n < 0 || m < 0 || n >= (1ll << 31) || m >= (1ll << 31)) return HAV_ERR_INVALID;
    if (m > 0 && (!points || !idx || !out_d2)) return HAV_ERR_INVALID;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return HAV_ERR_CUDA;
    cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
    // the status words of this call start at zero
    if (cudaMemsetAsync(ctx->ws + ctx->lay.barrier, 0, ctx->lay.zero_bytes, strm) != cudaSuccess) return HAV_ERR_CUDA;
    ctx->last_S = 1;
    if (m == 0) return HAV_OK;
    havk::GlobalHdr* gh = reinterpret_cast<havk::GlobalHdr*>(ctx->ws + ctx->lay.ghdr);
    // large subsets that fit the workspace: the exact grid search; else all pairs
    if (m >= havk::kSpacingGridMin && m <= ctx->lay.max_points) {
        if (!counted(ctx, havk::launch_spacing_grid(points, n, idx, m, out_d2, ctx->ws, ctx->lay, &gh->status,
                                                    ctx->max_blocks, strm)))
            return HAV_ERR_CUDA;
        return HAV_OK;
    }
    if (!counted(ctx, havk::launch_spacing(points, n, idx, m, out_d2, &gh->status, ctx->max_blocks, strm)))
        return HAV_ERR_CUDA;
    return HAV_OK;
}

hav_status hav_spacing_histogram(hav_ctx* ctx, const float* points, int64_t n, const int32_t* idx, int64_t m,
                                 const float* edges, int32_t nbins, float* out_d2, uint64_t* out_counts,
                                 hav_stream stream) {
    if (!ctx || !edges || !out_counts || nbins < 1 || nbins > HAV_SPACING_MAX_BINS) return HAV_ERR_INVALID;
    havk::HistEdges E;
    std::memset(&E, 0, sizeof E);
    for (int i = 0; i <= nbins; ++i) {
        if (!std::isfinite(edges[i]) || (i > 0 && !(edges[i] > edges[i - 1]))) return HAV_ERR_INVALID;
        E.e[i] = edges[i];
    }
    E.nbins = nbins;
    hav_status st = hav_spacing(ctx, points, n, idx, m, out_d2, stream);
    if (st != HAV_OK) return st;
    cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(out_counts, 0, sizeof(uint64_t) * (nbins + 2), strm) != cudaSuccess) return HAV_ERR_CUDA;
    if (m == 0) return HAV_OK;
    if (!counted(ctx, havk::launch_spacing_hist(out_d2, m, E, reinterpret_cast<unsigned long long*>(out_counts),
                                                strm)))
        return HAV_ERR_CUDA;
    return HAV_OK;
}

hav_status hav_ball_query(hav_ctx* ctx, const float* points, int64_t n, const int32_t* centres, int64_t m,
                          float radius, int32_t nsample, int32_t* out_idx, float* out_xyz, hav_stream stream) {
    if (!ctx || n < 0 || m < 0 || n > ctx->lay.max_points || m >= (1ll << 31)) return HAV_ERR_INVALID;
    if (nsample < 1 || nsample > 256 || !(radius > 0.0f) || !std::isfinite(radius)) return HAV_ERR_INVALID;
    if (m > 0 && (!points || !centres || !out_idx)) return HAV_ERR_INVALID;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return HAV_ERR_CUDA;
    cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ctx->ws + ctx->lay.barrier, 0, ctx->lay.zero_bytes, strm) != cudaSuccess) return HAV_ERR_CUDA;
    ctx->last_S = 1;
    if (m == 0) return HAV_OK;
    havk::GlobalHdr* gh = reinterpret_cast<havk::GlobalHdr*>(ctx->ws + ctx->lay.ghdr);
    if (!counted(ctx, havk::launch_ball_query(points, n, centres, m, radius, nsample, out_idx, out_xyz, ctx->ws,
                                              ctx->lay, &gh->status, ctx->group_nblocks, strm)))
        return HAV_ERR_CUDA;
    return HAV_OK;
}

hav_status hav_status_get(hav_ctx* ctx, hav_stream stream, int32_t* per_segment) {
    if (!ctx) return HAV_ERR_INVALID;
    cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(strm) != cudaSuccess) return HAV_ERR_CUDA;
    havk::GlobalHdr gh;
    if (cudaMemcpy(&gh, ctx->ws + ctx->lay.ghdr, sizeof gh, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HAV_ERR_CUDA;
    if (per_segment && ctx->last_S > 0) {
        std::vector<havk::SegHdr> sh(ctx->last_S);
        if (cudaMemcpy(sh.data(), ctx->ws + ctx->lay.seghdr, sizeof(havk::SegHdr) * ctx->last_S,
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            return HAV_ERR_CUDA;
        for (int s = 0; s < ctx->last_S; ++s) per_segment[s] = sh[s].status;
    }
    return static_cast<hav_status>(gh.status);
}

int32_t hav_trace_get(hav_ctx* ctx, hav_stream stream, hav_layer_trace* out, int32_t max_records) {
    if (!ctx || !out || max_records < 0) return -1;
    cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(strm) != cudaSuccess) return -1;
    const int S = ctx->last_S, L = ctx->last_L, K = ctx->last_layers;
    std::vector<hav_layer_trace> all(static_cast<size_t>(L) * S * havk::kMaxLayers);
    if (all.empty()) return 0;
    if (cudaMemcpy(all.data(), ctx->ws + ctx->lay.trace, sizeof(hav_layer_trace) * all.size(),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    int32_t w = 0;
    for (int j = 0; j < L; ++j)
        for (int s = 0; s < S; ++s)
            for (int l = 0; l < K; ++l) {
                if (w >= max_records) return w;
                out[w++] = all[(static_cast<size_t>(j) * S + s) * havk::kMaxLayers + l];
            }
    return w;
}

int32_t hav_phase_times_get(hav_ctx* ctx, hav_stream stream, uint64_t* t_ns, uint32_t* tag,
                            int32_t max_records) {
    if (!ctx || !t_ns || !tag || max_records < 0) return -1;
    cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(strm) != cudaSuccess) return -1;
    std::vector<unsigned long long> buf(2 * havk::kPhaseTimes);
    if (cudaMemcpy(buf.data(), ctx->ws + ctx->lay.ptimes, sizeof(unsigned long long) * buf.size(),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    int32_t w = 0;
    for (int k = 0; k < havk::kPhaseTimes && w < max_records; ++k) {
        if (k > 0 && buf[2 * k] == 0) break;
        t_ns[w] = buf[2 * k];
        tag[w] = static_cast<uint32_t>(buf[2 * k + 1]);
        ++w;
    }
    return w;
}

hav_status hav_fps(hav_ctx* ctx, const float* points, int64_t n, int64_t m, int32_t* out_idx,
                   hav_stream stream) {
    if (!ctx || n < 0 || m < 0 || m > n || n > ctx->lay.max_points) return HAV_ERR_INVALID;
    if (m > 0 && (!points || !out_idx)) return HAV_ERR_INVALID;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != ctx->device) return HAV_ERR_INVALID;
    cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
    ctx->last_S = 1;
    ctx->last_L = 0;
    if (cudaMemsetAsync(ctx->ws + ctx->lay.barrier, 0, ctx->lay.zero_bytes, strm) != cudaSuccess) return HAV_ERR_CUDA;
    if (m == 0) return HAV_OK;
    if (!counted(ctx, havk::launch_fps(points, static_cast<int>(n), static_cast<int>(m), out_idx, ctx->ws, ctx->lay,
                                       ctx->fps_nblocks, strm)))
        return HAV_ERR_CUDA;
    return HAV_OK;
}

hav_status hav_count(hav_ctx* ctx, const float* points, int64_t n, float s, const float aspect[3],
                     int64_t* K, hav_stream stream) {
    if (!ctx || !points || !aspect || !K || n < 1 || n > ctx->lay.max_points) return HAV_ERR_INVALID;
    if (!(s > 0.0f) || !std::isfinite(s)) return HAV_ERR_INVALID;
    for (int a = 0; a < 3; ++a)
        if (!(aspect[a] > 0.0f) || !std::isfinite(aspect[a])) return HAV_ERR_INVALID;
    int launched = 0;
    const int st = havk::count_voxels(points, n, s, aspect, ctx->ws, ctx->lay, K, &launched,
                                      reinterpret_cast<cudaStream_t>(stream));
    ctx->launches += static_cast<uint64_t>(launched);
    return static_cast<hav_status>(st);
}

}  // extern "C"
