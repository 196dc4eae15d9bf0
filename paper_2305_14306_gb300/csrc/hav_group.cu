// Grouping around sampled centres: the step after sampling in the
// sample-group-aggregate block (Section 3.1), the ball query of PointNet++.
// For centre j (point centres[j]) the nsample smallest indices k with
// (dx*dx + dy*dy) + dz*dz < radius*radius (binary32, no fusion), ascending;
// missing slots repeat the smallest.  The offsets p_k - c_j of every slot are
// written beside them (the gather of the block, fused).
//
// A uniform grid with cells of at least the radius (so every ball lies in the
// 3 x 3 x 3 cells around its centre's cell) is built by a counting sort of the
// points by cell; one warp per centre then scans those cells, collects the
// qualifying indices in shared memory (sorted and cut to the nsample smallest
// whenever the buffer fills, the largest kept one then bounding the rest) and
// sorts them once at the end.  The result does not
// depend on the grid, only the work does.  Two kernels on the caller's
// stream: the grid build (one cooperative launch) and the query.

#include <cuda_runtime.h>

#include "hav.h"
#include "hav_device.cuh"
#include "hav_internal.h"

namespace havk {
namespace {

constexpr int kGrpMaxSample = 256;
constexpr int kScanItems = 4;                        // cells per thread in the scan
constexpr int kScanBlock = 1024 * kScanItems;       // cells per scan block
constexpr long long kMaxCells = 1ll << 24;

struct GroupGrid {
    uint32_t box[6];  // ~enc(min xyz), enc(max xyz), atomicMax'ed
    float mn[3];
    float inv_h;
    int dims[3];
    int pad;
    long long cells;
};

__device__ __forceinline__ int axis_cell(float x, float mn, float inv_h, int dim) {
    const float t = __fmul_rn(__fsub_rn(x, mn), inv_h);
    int c = (t > 0.0f) ? static_cast<int>(t) : 0;
    return c < dim ? c : dim - 1;
}

__device__ __forceinline__ long long cell_of(const float* p, const GroupGrid& g, int c[3]) {
    for (int a = 0; a < 3; ++a) c[a] = axis_cell(p[a], g.mn[a], g.inv_h, g.dims[a]);
    return (static_cast<long long>(c[2]) * g.dims[1] + c[1]) * g.dims[0] + c[0];
}

// Cell size h >= radius (1 + 2^-10) and at least 1/256 of the largest
// extent, grown by 2^(1/3) until the grid has at most `budget` cells.  With
// at most 257 cells per axis the cell map t = (x - mn) * RN(1/h) is off by
// under 2^-12 cells, so two points closer than the radius (under 1 - 2^-10
// cells apart) never land more than one cell apart.
__device__ void setup_grid(GroupGrid* g, float radius, long long budget) {
    float ext = 0.0f, e[3];
    for (int a = 0; a < 3; ++a) {
        g->mn[a] = dec_f(~g->box[a]);
        const float mx = dec_f(g->box[3 + a]);
        e[a] = (mx >= g->mn[a]) ? __fsub_rn(mx, g->mn[a]) : 0.0f;
        ext = fmaxf(ext, e[a]);
        if (!(mx >= g->mn[a])) g->mn[a] = 0.0f;  // no finite point
    }
    float h = fmaxf(__fmul_rn(radius, 1.0009765625f), __fmul_rn(ext, 0.00390625f));
    long long cells = 0;
    for (int guard = 0; guard < 200; ++guard) {
        cells = 1;
        for (int a = 0; a < 3; ++a) {
            const long long d = static_cast<long long>(__fdiv_rn(e[a], h)) + 1;
            g->dims[a] = static_cast<int>(d);
            cells *= d;
        }
        if (cells <= budget) break;
        h = __fmul_rn(h, 1.2599210739135742f);
    }
    g->inv_h = __fdiv_rn(1.0f, h);
    g->cells = cells;
}

// The grid in one cooperative launch, its phases separated by grid barriers
// (bounded waits; a wait that gives up sets the abort flag, which the query
// honours): bounding box and cleared counts; set-up (every block alike) and
// cell counts; a scan of each block's share of the cells; the shares'
// offsets; the scatter.  Afterwards end[c] holds the end of cell c in list
// (its start is end[c - 1]).
__global__ void __launch_bounds__(kThreads, 1)
    grp_build(const float* pts, long long n, float radius, long long budget, GroupGrid* g, uint32_t* end,
              uint32_t* block_sums, int32_t* list, Barrier* bar, GlobalHdr* gh) {
    __shared__ GroupGrid sg;
    __shared__ unsigned epoch;
    __shared__ int flag;
    __shared__ uint32_t scratch[32];
    __shared__ float redf[6][32];
    const int tid = threadIdx.x;
    const unsigned nb = gridDim.x;
    const long long gtid = blockIdx.x * static_cast<long long>(kThreads) + tid;
    const long long gstride = static_cast<long long>(nb) * kThreads;
    if (tid == 0) epoch = 0u;
    for (long long i = gtid; i < budget; i += gstride) end[i] = 0u;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long long i = gtid; i < n; i += gstride)
        for (int a = 0; a < 3; ++a) {
            const float x = pts[3 * i + a];
            if (isfinite(x)) {
                mn[a] = fminf(mn[a], x);
                mx[a] = fmaxf(mx[a], x);
            }
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if ((tid & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            redf[a][tid >> 5] = mn[a];
            redf[3 + a][tid >> 5] = mx[a];
        }
    __syncthreads();
    if (tid < 6) {
        float r = redf[tid][0];
        for (int w = 1; w < kThreads / 32; ++w) r = (tid < 3) ? fminf(r, redf[tid][w]) : fmaxf(r, redf[tid][w]);
        if (isfinite(r)) atomicMax(&g->box[tid], (tid < 3) ? ~enc_f(r) : enc_f(r));
    }
    if (!grid_sync_impl(bar, gh, nb, &epoch, &flag)) return;

    if (tid == 0) {
        for (int a = 0; a < 6; ++a) sg.box[a] = ld_volatile_u(&g->box[a]);
        setup_grid(&sg, radius, budget);
        if (blockIdx.x == 0) *g = sg;  // for the query
    }
    __syncthreads();
    for (long long i = gtid; i < n; i += gstride) {
        int c[3];
        atomicAdd(&end[cell_of(pts + 3 * i, sg, c)], 1u);
    }
    if (!grid_sync_impl(bar, gh, nb, &epoch, &flag)) return;

    // this block's share of the cells: an exclusive scan in place, the share's total aside
    const long long cells = sg.cells;
    const long long share = (cells + nb - 1) / nb;
    const long long cb = share * blockIdx.x;
    const long long ce = (cb + share < cells) ? cb + share : cells;
    uint32_t run = 0;
    for (long long t0 = cb; t0 < ce; t0 += static_cast<long long>(kThreads) * kScanItems) {
        uint32_t x[kScanItems], sum = 0;
        for (int k = 0; k < kScanItems; ++k) {
            const long long i = t0 + static_cast<long long>(tid) * kScanItems + k;
            x[k] = (i < ce) ? end[i] : 0u;
            sum += x[k];
        }
        uint32_t tot;
        uint32_t before = block_excl_scan<uint32_t>(sum, &tot, scratch);
        for (int k = 0; k < kScanItems; ++k) {
            const long long i = t0 + static_cast<long long>(tid) * kScanItems + k;
            if (i < ce) end[i] = run + before;
            before += x[k];
        }
        run += tot;
    }
    if (tid == 0) block_sums[blockIdx.x] = run;
    if (!grid_sync_impl(bar, gh, nb, &epoch, &flag)) return;

    // the shares before this one, then the offsets
    uint32_t pre = 0;
    for (unsigned b = tid; b < blockIdx.x; b += kThreads) pre += ld_volatile_u(&block_sums[b]);
    uint32_t tot;
    pre = block_excl_scan<uint32_t>(pre, &tot, scratch);  // (only the total matters)
    const uint32_t off = tot;
    for (long long i = cb + tid; i < ce; i += kThreads) end[i] += off;
    if (!grid_sync_impl(bar, gh, nb, &epoch, &flag)) return;

    for (long long i = gtid; i < n; i += gstride) {
        int c[3];
        const uint32_t pos = atomicAdd(&end[cell_of(pts + 3 * i, sg, c)], 1u);
        if (pos < static_cast<uint32_t>(n)) list[pos] = static_cast<int32_t>(i);
    }
}

// One warp per centre: the lanes test 32 candidates of the 27 cells at a
// time, and the warp collects the qualifying indices in shared memory; the
// nsample smallest do not depend on the order in which the candidates arrive.
constexpr int kQueryWarps = 4;  // warps per block of the query
constexpr int kCollect = 512;   // qualifying points a warp collects at most before it sorts and cuts them

// Ascending bitonic sort of buf[0, cnt) by one warp (cnt <= kCollect; the
// rest of the next power of two is padded with the largest index).
__device__ __forceinline__ void sort_prefix(int32_t* buf, int cnt, int lane) {
    int n2 = 32;
    while (n2 < cnt) n2 <<= 1;
    for (int e = cnt + lane; e < n2; e += 32) buf[e] = 0x7fffffff;
    __syncwarp();
    for (int k2 = 2; k2 <= n2; k2 <<= 1)
        for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
            for (int i = lane; i < n2; i += 32) {
                const int ixj = i ^ j2;
                if (ixj > i) {
                    const int32_t u = buf[i], w = buf[ixj];
                    if ((u > w) == ((i & k2) == 0)) {
                        buf[i] = w;
                        buf[ixj] = u;
                    }
                }
            }
            __syncwarp();
        }
}

__global__ void __launch_bounds__(32 * kQueryWarps)
    grp_query(const float* pts, long long n, const int32_t* centres, long long m, float radius, int nsample,
              const GroupGrid* g, const uint32_t* end, const int32_t* list, int32_t* out_idx, float* out_xyz,
              int32_t* status, const GlobalHdr* gh) {
    __shared__ int32_t sbuf[kQueryWarps][kCollect];
    if (ld_volatile(&gh->abort)) return;  // the build gave up (its status says so)
    const GroupGrid G = *g;
    const float r2 = __fmul_rn(radius, radius);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int32_t* buf = sbuf[wib];
    int cap = 64;
    while (cap < 2 * nsample && cap < kCollect) cap <<= 1;
    const long long warps = static_cast<long long>(gridDim.x) * kQueryWarps;
    for (long long j = blockIdx.x * static_cast<long long>(kQueryWarps) + wib; j < m; j += warps) {
        const int32_t ci = centres[j];
        int32_t* row = out_idx + j * nsample;
        if (ci < 0 || ci >= n) {
            if (lane == 0) atomicCAS(status, 0, static_cast<int>(HAV_ERR_INVALID));
            for (int s = lane; s < nsample; s += 32) row[s] = 0;
            if (out_xyz)
                for (int s = lane; s < 3 * nsample; s += 32) out_xyz[j * 3 * nsample + s] = 0.0f;
            continue;
        }
        const float cx = pts[3ll * ci], cy = pts[3ll * ci + 1], cz = pts[3ll * ci + 2];
        int c[3];
        const float cp[3] = {cx, cy, cz};
        cell_of(cp, G, c);
        // the 3 x 3 x 3 cells around the centre's, every point within the radius
        // visited once; visit(k, ok) is called by the whole warp per 32 points
        auto scan = [&](auto&& visit, const int32_t& top) {
            for (int dz = -1; dz <= 1; ++dz) {
                const int z = c[2] + dz;
                if (z < 0 || z >= G.dims[2]) continue;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int y = c[1] + dy;
                    if (y < 0 || y >= G.dims[1]) continue;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int x = c[0] + dx;
                        if (x < 0 || x >= G.dims[0]) continue;
                        const long long cell = (static_cast<long long>(z) * G.dims[1] + y) * G.dims[0] + x;
                        const uint32_t a = (cell > 0) ? end[cell - 1] : 0u;
                        uint32_t b = end[cell];
                        if (b > static_cast<uint32_t>(n)) b = static_cast<uint32_t>(n);
                        for (uint32_t q0 = a; q0 < b; q0 += 32) {  // warp-uniform
                            const uint32_t q = q0 + lane;
                            int32_t k = 0;
                            bool ok = false;
                            if (q < b) {
                                k = list[q];
                                if (k >= 0 && k < n && k < top) {
                                    const float ex = __fsub_rn(pts[3ll * k], cx), ey = __fsub_rn(pts[3ll * k + 1], cy),
                                                ez = __fsub_rn(pts[3ll * k + 2], cz);
                                    const float d2 =
                                        __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
                                    ok = d2 < r2;
                                }
                            }
                            visit(k, ok);
                        }
                    }
                }
            }
        };
        // the qualifying indices, unsorted, into the warp's buffer; when it is
        // full it is sorted and cut to the nsample smallest, whose largest then
        // bounds every later index (indices are distinct); one sort at the end.
        // The buffer holds 2 nsample rounded up to a power of two, 64 to
        // kCollect: a small one bounds the scan early where many points qualify
        int cnt = 0;
        int32_t top = 0x7fffffff;
        scan([&](int32_t k, bool ok) {
            unsigned mask = __ballot_sync(0xffffffffu, ok);
            if (cnt + __popc(mask) > cap) {  // (warp-uniform)
                sort_prefix(buf, cnt, lane);
                if (cnt > nsample) cnt = nsample;
                if (cnt == nsample) top = buf[nsample - 1];
                ok = ok && k < top;
                mask = __ballot_sync(0xffffffffu, ok);
            }
            if (ok) buf[cnt + __popc(mask & ((1u << lane) - 1u))] = k;
            cnt += __popc(mask);
        }, top);
        __syncwarp();
        sort_prefix(buf, cnt, lane);
        const int32_t* res = buf;
        if (cnt > nsample) cnt = nsample;
        if (cnt == 0) {  // unreachable: the centre is at distance 0
            if (lane == 0) buf[0] = ci;
            __syncwarp();
            cnt = 1;
        }
        for (int s = lane; s < nsample; s += 32) {
            const int32_t k = (s < cnt) ? res[s] : res[0];
            row[s] = k;
            if (out_xyz) {
                float* o = out_xyz + (j * nsample + s) * 3;
                o[0] = __fsub_rn(pts[3ll * k], cx);
                o[1] = __fsub_rn(pts[3ll * k + 1], cy);
                o[2] = __fsub_rn(pts[3ll * k + 2], cz);
            }
        }
        __syncwarp();  // the list is rewritten for the next centre
    }
}

// ------------------------------------------------------ spacing on the grid
// The Fig. 3 spacing of a large subset (hav_spacing): the subset's points are
// gathered (an invalid index or a non-finite coordinate as NaN: no distance
// involving such a point is ever below another, exactly as in the all-pairs
// search), the grid above is built over them (cells of 1/256 of the largest
// extent, grown within the budget), and one thread per point, in cell order,
// visits the shells of cells at Chebyshev distance r = 0, 1, ... around its
// own until no cell farther out can hold a nearer point.  A point of a cell r
// + 1 or more shells away lies at least (r - 0.01) h away (the cell map is
// exact to far less than 0.01 cells), and a computed squared distance is
// within a relative 2^-20 of the exact one, so the search stops once best <
// ((r - 0.01) h)^2 (1 - 2^-20), every bound rounded down.  A point still
// searching after kShellMax shells scans the whole subset instead.
constexpr int kShellMax = 32;

__global__ void spacing_gather(const float* pts, long long n, const int32_t* idx, long long m, float* sub,
                               int32_t* status) {
    for (long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; q < m;
         q += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int32_t i = idx[q];
        float x = NAN, y = NAN, z = NAN;
        if (i < 0 || i >= n) {
            atomicCAS(status, 0, static_cast<int>(HAV_ERR_INVALID));
        } else {
            x = pts[3ll * i];
            y = pts[3ll * i + 1];
            z = pts[3ll * i + 2];
            if (!(isfinite(x) && isfinite(y) && isfinite(z))) x = y = z = NAN;
        }
        sub[3 * q] = x;
        sub[3 * q + 1] = y;
        sub[3 * q + 2] = z;
    }
}

__device__ __forceinline__ float sq_dist(const float* p, float x, float y, float z) {
    const float ex = __fsub_rn(p[0], x), ey = __fsub_rn(p[1], y), ez = __fsub_rn(p[2], z);
    return __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
}

__global__ void spacing_grid_query(const float* sub, long long m, const GroupGrid* g, const uint32_t* end,
                                   const int32_t* list, float* out_d2, const GlobalHdr* gh) {
    if (ld_volatile(&gh->abort)) return;  // the build gave up (its status says so)
    const GroupGrid G = *g;
    // the cell width, rounded down and shrunk by 2^-20
    const float h = __fmul_rd(__fdiv_rd(1.0f, G.inv_h), 0.99999904632568359375f);
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < m;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = list[t];
        const float x = sub[3ll * i], y = sub[3ll * i + 1], z = sub[3ll * i + 2];
        float best = INFINITY;
        if (x == x) {  // (a gathered point is NaN on every axis or on none)
            int c[3];
            const float p3[3] = {x, y, z};
            cell_of(p3, G, c);
            bool done = false;
            int r = 0;
            for (; r <= kShellMax && !done; ++r) {
                for (int dz = -r; dz <= r; ++dz) {
                    const int zc = c[2] + dz;
                    if (zc < 0 || zc >= G.dims[2]) continue;
                    for (int dy = -r; dy <= r; ++dy) {
                        const int yc = c[1] + dy;
                        if (yc < 0 || yc >= G.dims[1]) continue;
                        const bool face = (dz == -r || dz == r || dy == -r || dy == r);
                        for (int dx = -r; dx <= r; dx += (face || r == 0) ? 1 : 2 * r) {
                            const int xc = c[0] + dx;
                            if (xc < 0 || xc >= G.dims[0]) continue;
                            const long long cell = (static_cast<long long>(zc) * G.dims[1] + yc) * G.dims[0] + xc;
                            const uint32_t a = (cell > 0) ? end[cell - 1] : 0u;
                            const uint32_t b = end[cell];
                            for (uint32_t q = a; q < b && q < static_cast<uint32_t>(m); ++q) {
                                const int j = list[q];
                                if (j == i) continue;
                                best = fminf(best, sq_dist(sub + 3ll * j, x, y, z));
                            }
                        }
                    }
                }
                // every cell visited, or none farther out can hold a nearer point
                bool all = true;
                for (int a3 = 0; a3 < 3; ++a3) all = all && c[a3] - r <= 0 && c[a3] + r >= G.dims[a3] - 1;
                if (all) {
                    done = true;
                } else if (r >= 1) {
                    const float bd = __fmul_rd(__fsub_rd(static_cast<float>(r), 0.01f), h);
                    const float bd2 = __fmul_rd(__fmul_rd(bd, bd), 0.99999904632568359375f);
                    if (best < bd2) done = true;
                }
            }
            if (!done) {  // an isolated point: the whole subset
                best = INFINITY;
                for (long long j = 0; j < m; ++j)
                    if (j != i) best = fminf(best, sq_dist(sub + 3 * j, x, y, z));
            }
        }
        out_d2[i] = best;
    }
}

}  // namespace

int group_coresident_blocks(int device) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grp_build, kThreads, 0) != cudaSuccess) return -1;
    if (per_sm < 1) return -1;
    return sms < kMaxBlocks ? sms : kMaxBlocks;  // one block per SM
}

int launch_ball_query(const float* points, long long n, const int32_t* centres, long long m, float radius,
                      int nsample, int32_t* out_idx, float* out_xyz, unsigned char* ws, const Layout& lay,
                      int32_t* status, int nblocks, cudaStream_t stream) {
    if (nsample < 1 || nsample > kGrpMaxSample) return -1;
    // scratch: grid parameters and scan block sums in the phase-timer area,
    // cell counts in the candidate area, the sorted point list in staged points
    GroupGrid* g = reinterpret_cast<GroupGrid*>(ws + lay.ptimes);
    uint32_t* block_sums = reinterpret_cast<uint32_t*>(ws + lay.ptimes + 256);
    uint32_t* counts = reinterpret_cast<uint32_t*>(ws + lay.cand);
    int32_t* list = reinterpret_cast<int32_t*>(ws + lay.ord[0]);
    long long budget = static_cast<long long>(sizeof(Cand)) * lay.cand_slots / 4;
    if (budget > kMaxCells) budget = kMaxCells;
    if (n > lay.max_points) return -1;
    static_assert(256 + 4 * (kMaxCells / kScanBlock) <= 2 * 8 * kPhaseTimes, "scan scratch fits");
    if (cudaMemsetAsync(g, 0, sizeof(GroupGrid), stream) != cudaSuccess) return -1;
    Barrier* bar = reinterpret_cast<Barrier*>(ws + lay.barrier);  // zeroed by the caller
    GlobalHdr* gh = reinterpret_cast<GlobalHdr*>(ws + lay.ghdr);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(nblocks));
    cfg.blockDim = dim3(kThreads);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, grp_build, points, static_cast<long long>(n), radius, budget, g, counts, block_sums,
                           list, bar, gh) != cudaSuccess)
        return -1;
    long long qb = (m + kQueryWarps - 1) / kQueryWarps;
    if (qb > 65536) qb = 65536;
    grp_query<<<static_cast<unsigned>(qb < 1 ? 1 : qb), 32 * kQueryWarps, 0, stream>>>(
        points, n, centres, m, radius, nsample, g, counts, list, out_idx, out_xyz, status, gh);
    return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

int launch_spacing_grid(const float* points, long long n, const int32_t* idx, long long m, float* out_d2,
                        unsigned char* ws, const Layout& lay, int32_t* status, int nblocks, cudaStream_t stream) {
    if (m < 2 || m > lay.max_points) return -1;
    // scratch as the ball query's, and the gathered subset in the second staged-point array
    GroupGrid* g = reinterpret_cast<GroupGrid*>(ws + lay.ptimes);
    uint32_t* block_sums = reinterpret_cast<uint32_t*>(ws + lay.ptimes + 256);
    uint32_t* counts = reinterpret_cast<uint32_t*>(ws + lay.cand);
    int32_t* list = reinterpret_cast<int32_t*>(ws + lay.ord[0]);
    float* sub = reinterpret_cast<float*>(ws + lay.ord[1]);
    long long budget = static_cast<long long>(sizeof(Cand)) * lay.cand_slots / 4;
    if (budget > kMaxCells) budget = kMaxCells;
    if (cudaMemsetAsync(g, 0, sizeof(GroupGrid), stream) != cudaSuccess) return -1;
    long long gb = (m + 255) / 256;
    if (gb > 65536) gb = 65536;
    spacing_gather<<<static_cast<unsigned>(gb), 256, 0, stream>>>(points, n, idx, m, sub, status);
    Barrier* bar = reinterpret_cast<Barrier*>(ws + lay.barrier);  // zeroed by the caller
    GlobalHdr* gh = reinterpret_cast<GlobalHdr*>(ws + lay.ghdr);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(nblocks));
    cfg.blockDim = dim3(kThreads);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // (the smallest normal radius: the cells follow the extent alone)
    if (cudaLaunchKernelEx(&cfg, grp_build, static_cast<const float*>(sub), m, 1.17549435e-38f, budget, g, counts,
                           block_sums, list, bar, gh) != cudaSuccess)
        return -1;
    spacing_grid_query<<<static_cast<unsigned>(gb), 256, 0, stream>>>(sub, m, g, counts, list, out_d2, gh);
    return cudaGetLastError() == cudaSuccess ? 3 : -1;
}

}  // namespace havk
