// Farthest point sampling (Eq. 1 of Section 3.1), the comparator the paper
// measures HAVSampler against: one cooperative launch, one bounded grid
// barrier per selected point; clouds of up to 32,768 points on one cluster
// of 8 CTAs instead, one cluster barrier per selected point.
//
// Start at index 0; every point keeps its squared distance to the selected
// set (binary32, (dx*dx + dy*dy) + dz*dz without contraction); the next pick
// is the largest distance, ties to the lowest index; picked points are never
// picked again.

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "hav_device.cuh"
#include "hav_internal.h"

namespace cg = cooperative_groups;

namespace havk {
namespace {

constexpr int kFpsThreads = 1024;
constexpr size_t kFpsResidentBytes = 200 * 1024;  // shared memory for a block's resident points

// packed (distance bits, inverted index): the maximum is the farthest point,
// ties to the lowest index; picked points pack to 0 and never win
__device__ __forceinline__ unsigned long long fps_pack(float d2, int i) {
    return (static_cast<unsigned long long>(__float_as_uint(d2)) << 32) |
           static_cast<unsigned long long>(0xffffffffu - static_cast<unsigned>(i));
}

// kResident: the block's points and distances stay in shared memory (x, y,
// z, distance per point) for the whole run instead of being read from L2 in
// every round; the arithmetic and the picks are the same.
template <bool kResident>
__global__ void __launch_bounds__(kFpsThreads, 1)
    fps_kernel(const float* pts, int n, int m, int32_t* out, float* dist_g, unsigned long long* bmax, Barrier* bar,
               GlobalHdr* gh, int nblocks) {
    extern __shared__ float4 res[];
    __shared__ unsigned long long red[32];
    __shared__ int s_flag;
    __shared__ unsigned epoch;
    __shared__ int s_last;
    const int tid = threadIdx.x;
    if (tid == 0) epoch = 0u;
    const int chunk = (n + nblocks - 1) / nblocks;
    const int a = blockIdx.x * chunk;
    const int b = min(n, a + chunk);
    for (int i = a + tid; i < b; i += kFpsThreads) {
        if constexpr (kResident) res[i - a] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], INFINITY);
        else dist_g[i] = INFINITY;
    }
    int last = 0;
    if (blockIdx.x == 0 && tid == 0) out[0] = 0;
    __syncthreads();
    for (int j = 1; j < m; ++j) {
        const float qx = pts[3 * last], qy = pts[3 * last + 1], qz = pts[3 * last + 2];
        unsigned long long best = 0ull;
        for (int i = a + tid; i < b; i += kFpsThreads) {
            float px, py, pz, di;
            if constexpr (kResident) {
                const float4 r4 = res[i - a];
                px = r4.x;
                py = r4.y;
                pz = r4.z;
                di = r4.w;
            } else {
                di = dist_g[i];
            }
            if (i == last) {
                di = -1.0f;  // picked: never again
                if constexpr (kResident) res[i - a].w = di;
                else dist_g[i] = di;
            }
            if (di < 0.0f) continue;
            if constexpr (!kResident) {
                px = pts[3 * i];
                py = pts[3 * i + 1];
                pz = pts[3 * i + 2];
            }
            const float dx = __fsub_rn(px, qx);
            const float dy = __fsub_rn(py, qy);
            const float dz = __fsub_rn(pz, qz);
            const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            if (d2 < di) {
                di = d2;
                if constexpr (kResident) res[i - a].w = di;
                else dist_g[i] = di;
            }
            const unsigned long long k = fps_pack(di, i);
            best = k > best ? k : best;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
            best = v > best ? v : best;
        }
        if ((tid & 31) == 0) red[tid >> 5] = best;
        __syncthreads();
        if (tid == 0) {
            unsigned long long bb = red[0];
            for (int w = 1; w < kFpsThreads / 32; ++w) bb = red[w] > bb ? red[w] : bb;
            bmax[(j & 1) * kMaxBlocks + blockIdx.x] = bb;
        }
        if (!grid_sync_impl(bar, gh, static_cast<unsigned>(nblocks), &epoch, &s_flag)) return;
        // every block finds the same maximum over the block maxima
        unsigned long long bb = 0ull;
        for (int k = tid; k < nblocks; k += kFpsThreads) {
            const unsigned long long v = bmax[(j & 1) * kMaxBlocks + k];
            bb = v > bb ? v : bb;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, bb, o);
            bb = v > bb ? v : bb;
        }
        if ((tid & 31) == 0) red[tid >> 5] = bb;
        __syncthreads();
        if (tid == 0) {
            unsigned long long m2 = red[0];
            for (int w = 1; w < kFpsThreads / 32; ++w) m2 = red[w] > m2 ? red[w] : m2;
            const int pick = static_cast<int>(0xffffffffu - static_cast<unsigned>(m2 & 0xffffffffull));
            s_last = (m2 != 0ull && pick >= 0 && pick < n) ? pick : 0;  // m <= n: an unpicked point exists
            if (blockIdx.x == 0) out[j] = s_last;
        }
        __syncthreads();
        last = s_last;
    }
}

constexpr int kFpsQ = 8;                  // CTAs of the small-cloud cluster (portable size)
constexpr int kFpsQPoints = 4096;         // points one CTA of it holds
constexpr int kFpsClusterMax = kFpsQ * kFpsQPoints;

// a CTA's best candidate of a round with the point's coordinates
struct FpsCand {
    unsigned long long key;  // fps_pack of the CTA's farthest unpicked point
    float x, y, z, pad;
};

// Clouds of at most kFpsClusterMax points: CTA r of one cluster holds points
// [r c, (r + 1) c), c = ceil(n / kFpsQ), with their distances in its shared
// memory.  Each round every CTA writes its best candidate into its own slot
// (two slots alternate), the cluster barrier publishes them, and every CTA
// takes the same maximum over the kFpsQ slots read through distributed shared
// memory; round j + 2 rewrites a slot only after every CTA has passed round
// j + 1's barrier, so no read of round j can see it.  The same arithmetic,
// ties and picks as fps_kernel.
__global__ void __cluster_dims__(kFpsQ, 1, 1) __launch_bounds__(kFpsThreads, 1)
    fps_cluster_kernel(const float* pts, int n, int m, int32_t* out) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 res[];
    __shared__ unsigned long long red[32];
    __shared__ FpsCand cand[2];
    __shared__ float4 s_q;  // the last pick: x, y, z and its index bits
    const int tid = threadIdx.x;
    const int r = static_cast<int>(cl.block_rank());
    const int chunk = (n + kFpsQ - 1) / kFpsQ;
    const int a = r * chunk;
    const int b = min(n, a + chunk);
    for (int i = a + tid; i < b; i += kFpsThreads)
        res[i - a] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], INFINITY);
    if (r == 0 && tid == 0 && m > 0) out[0] = 0;
    float qx = 0.0f, qy = 0.0f, qz = 0.0f;
    if (n > 0) {
        qx = pts[0];
        qy = pts[1];
        qz = pts[2];
    }
    int last = 0;
    __syncthreads();
    for (int j = 1; j < m; ++j) {
        unsigned long long best = 0ull;
        for (int i = a + tid; i < b; i += kFpsThreads) {
            const float4 p4 = res[i - a];
            float di = p4.w;
            if (i == last) {
                di = -1.0f;  // picked: never again
                res[i - a].w = di;
            }
            if (di < 0.0f) continue;
            const float dx = __fsub_rn(p4.x, qx);
            const float dy = __fsub_rn(p4.y, qy);
            const float dz = __fsub_rn(p4.z, qz);
            const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            if (d2 < di) {
                di = d2;
                res[i - a].w = di;
            }
            const unsigned long long k = fps_pack(di, i);
            best = k > best ? k : best;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
            best = v > best ? v : best;
        }
        if ((tid & 31) == 0) red[tid >> 5] = best;
        __syncthreads();
        if (tid == 0) {
            unsigned long long bb = red[0];
            for (int w = 1; w < kFpsThreads / 32; ++w) bb = red[w] > bb ? red[w] : bb;
            FpsCand& c = cand[j & 1];
            c.key = bb;
            if (bb != 0ull) {  // this CTA's point: its coordinates travel with it
                const int g = static_cast<int>(0xffffffffu - static_cast<unsigned>(bb & 0xffffffffull));
                const float4 p4 = res[g - a];
                c.x = p4.x;
                c.y = p4.y;
                c.z = p4.z;
            }
        }
        cl.sync();
        if (tid == 0) {
            unsigned long long bk = 0ull;
            float bx = qx, by = qy, bz = qz;
            for (int q = 0; q < kFpsQ; ++q) {
                const FpsCand* c = cl.map_shared_rank(&cand[j & 1], q);
                const unsigned long long k = c->key;
                if (k > bk) {
                    bk = k;
                    bx = c->x;
                    by = c->y;
                    bz = c->z;
                }
            }
            const int pick = static_cast<int>(0xffffffffu - static_cast<unsigned>(bk & 0xffffffffull));
            const int s_last = (bk != 0ull && pick >= 0 && pick < n) ? pick : 0;  // m <= n: an unpicked point exists
            s_q = make_float4(bx, by, bz, __int_as_float(s_last));
            if (r == 0) out[j] = s_last;
        }
        __syncthreads();
        const float4 q4 = s_q;
        qx = q4.x;
        qy = q4.y;
        qz = q4.z;
        last = __float_as_int(q4.w);
    }
    cl.sync();  // no CTA leaves while another may still read its slots
}

}  // namespace

int fps_coresident_blocks(int device) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fps_kernel<false>, kFpsThreads, 0) != cudaSuccess)
        return -1;
    long long nb = static_cast<long long>(sms) * per_sm;
    if (nb > kMaxBlocks) nb = kMaxBlocks;
    return static_cast<int>(nb);
}

int launch_fps(const float* points, int n, int m, int32_t* out, unsigned char* ws, const Layout& lay, int nblocks,
               cudaStream_t stream) {
    // scratch: the distance array in the first log array, block maxima in the phase-timer region
    float* dist = reinterpret_cast<float*>(ws + lay.dirty[0]);
    unsigned long long* bmax = reinterpret_cast<unsigned long long*>(ws + lay.ptimes);
    Barrier* bar = reinterpret_cast<Barrier*>(ws + lay.barrier);
    GlobalHdr* gh = reinterpret_cast<GlobalHdr*>(ws + lay.ghdr);
    // up to 32,768 points: one cluster of 8 CTAs, a cluster barrier per pick
    // (where the device refuses the cluster, the grid form below)
    if (n <= kFpsClusterMax) {
        const int chunk = (n + kFpsQ - 1) / kFpsQ;
        const size_t bytes = static_cast<size_t>(chunk < 1 ? 1 : chunk) * sizeof(float4);
        if (cudaFuncSetAttribute(fps_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kFpsQPoints * sizeof(float4))) == cudaSuccess) {
            cudaLaunchConfig_t cc = {};
            cc.gridDim = dim3(kFpsQ);
            cc.blockDim = dim3(kFpsThreads);
            cc.dynamicSmemBytes = bytes;
            cc.stream = stream;
            if (cudaLaunchKernelEx(&cc, fps_cluster_kernel, points, n, m, out) == cudaSuccess) return 1;
            (void)cudaGetLastError();  // a refused launch configuration leaves no sticky error
        }
    }
    // fewer blocks than points per block of work would only add barrier arrivals
    int nb = nblocks;
    const int want = (n + kFpsThreads - 1) / kFpsThreads;
    if (want < nb) nb = want < 1 ? 1 : want;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(nb));
    cfg.blockDim = dim3(kFpsThreads);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the block's share resident in shared memory where it fits and the grid
    // stays co-resident with that much shared memory per block
    const long long chunk = (static_cast<long long>(n) + nb - 1) / nb;
    const size_t bytes = static_cast<size_t>(chunk) * sizeof(float4);
    bool resident = bytes <= kFpsResidentBytes &&
                    cudaFuncSetAttribute(fps_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kFpsResidentBytes)) == cudaSuccess;
    if (resident) {
        int dev = 0, sms = 0, per_sm = 0;
        resident = cudaGetDevice(&dev) == cudaSuccess &&
                   cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                   cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fps_kernel<true>, kFpsThreads, bytes) ==
                       cudaSuccess &&
                   static_cast<long long>(sms) * per_sm >= nb;
    }
    if (resident) {
        cfg.dynamicSmemBytes = bytes;
        return cudaLaunchKernelEx(&cfg, fps_kernel<true>, points, n, m, out, dist, bmax, bar, gh, nb) == cudaSuccess
                   ? 1
                   : -1;
    }
    return cudaLaunchKernelEx(&cfg, fps_kernel<false>, points, n, m, out, dist, bmax, bar, gh, nb) == cudaSuccess
               ? 1
               : -1;
}

}  // namespace havk
