// Point spacing of a sampled subset: the distributions of Fig. 3 (Section
// 3.1).  For each subset point, the smallest squared distance to any other
// subset point, binary32 (dx*dx + dy*dy) + dz*dz without fusion; +inf for a
// subset of one point.  The minimum does not depend on the order in which
// candidates are visited, so the result is exact.
//
// Exact all-pairs search, tiled: a block takes kSpQ x kSpThreads query points
// and one range of candidates, stages the candidates in shared memory tile by
// tile, and keeps kSpQ running minima per thread.  Ranges of candidates are
// split over a second grid dimension so that small subsets still fill the
// GPU; the partial minima meet in an atomicMin on the float bits (squared
// distances are non-negative, so their bit patterns order like the values).

#include <cuda_runtime.h>

#include "hav.h"
#include "hav_device.cuh"
#include "hav_internal.h"

namespace havk {
namespace {

constexpr int kSpThreads = 256;
constexpr int kSpQ = 4;        // query points per thread
constexpr int kSpTile = 1024;  // candidates per shared-memory tile
constexpr unsigned kInfBits = 0x7f800000u;

__global__ void spacing_init(unsigned* out, long long m) {
    for (long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; q < m;
         q += static_cast<long long>(gridDim.x) * blockDim.x)
        out[q] = kInfBits;
}

__global__ void __launch_bounds__(kSpThreads) spacing_kernel(const float* pts, long long n, const int32_t* idx,
                                                             long long m, long long chunk, unsigned* out,
                                                             int32_t* status) {
    __shared__ float4 tile[kSpTile];
    const int tid = threadIdx.x;
    const long long qbase = static_cast<long long>(blockIdx.x) * (kSpThreads * kSpQ);
    float qx[kSpQ], qy[kSpQ], qz[kSpQ], best[kSpQ];
    int qpos[kSpQ];
#pragma unroll
    for (int u = 0; u < kSpQ; ++u) {
        const long long q = qbase + tid + u * kSpThreads;
        qpos[u] = -1;
        best[u] = INFINITY;
        qx[u] = qy[u] = qz[u] = 0.0f;
        if (q < m) {
            const int32_t i = idx[q];
            if (i >= 0 && i < n) {
                qx[u] = pts[3ll * i];
                qy[u] = pts[3ll * i + 1];
                qz[u] = pts[3ll * i + 2];
                qpos[u] = static_cast<int>(q);
            } else {
                atomicCAS(status, 0, static_cast<int>(HAV_ERR_INVALID));
            }
        }
    }
    const long long c0 = static_cast<long long>(blockIdx.y) * chunk;
    const long long c1 = (c0 + chunk < m) ? c0 + chunk : m;
    for (long long t0 = c0; t0 < c1; t0 += kSpTile) {
        __syncthreads();
        for (int k = tid; k < kSpTile; k += kSpThreads) {
            const long long j = t0 + k;
            float4 b = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(-1));  // w: subset position, -1 = none
            if (j < c1) {
                const int32_t i = idx[j];
                if (i >= 0 && i < n)
                    b = make_float4(pts[3ll * i], pts[3ll * i + 1], pts[3ll * i + 2], __int_as_float(static_cast<int>(j)));
            }
            tile[k] = b;
        }
        __syncthreads();
        const int cnt = static_cast<int>((c1 - t0 < kSpTile) ? c1 - t0 : kSpTile);
        for (int k = 0; k < cnt; ++k) {
            const float4 b = tile[k];
            const int j = __float_as_int(b.w);
#pragma unroll
            for (int u = 0; u < kSpQ; ++u) {
                const float dx = __fsub_rn(qx[u], b.x), dy = __fsub_rn(qy[u], b.y), dz = __fsub_rn(qz[u], b.z);
                const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                if (j >= 0 && j != qpos[u] && d2 < best[u]) best[u] = d2;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kSpQ; ++u)
        if (qpos[u] >= 0 && best[u] < INFINITY) atomicMin(out + qpos[u], __float_as_uint(best[u]));
}

// Histogram of the spacings over caller-given bin edges e[0] < ... < e[B]
// (binary32 squared distances): bin i holds e[i] <= d2 < e[i + 1], the last
// bin also d2 == e[B] (numpy's convention); counts[0] holds the values below
// e[0] (or not ordered against it), counts[B + 1] those above e[B], bins at
// counts[1..B].  Integer counts, so the order of the additions does not matter.
__global__ void __launch_bounds__(kSpThreads) spacing_hist(const unsigned* d2bits, long long m, const HistEdges E,
                                                           unsigned long long* counts) {
    __shared__ float se[kHistEdgesMax];
    __shared__ unsigned sc[kHistEdgesMax + 1];
    const int nb = E.nbins;
    for (int k = threadIdx.x; k <= nb; k += kSpThreads) se[k] = E.e[k];
    for (int k = threadIdx.x; k <= nb + 1; k += kSpThreads) sc[k] = 0u;
    __syncthreads();
    for (long long r = blockIdx.x * static_cast<long long>(kSpThreads) + threadIdx.x; r < m;
         r += static_cast<long long>(gridDim.x) * kSpThreads) {
        const float x = __uint_as_float(d2bits[r]);
        int slot;
        if (!(x >= se[0])) {
            slot = 0;
        } else if (x > se[nb]) {
            slot = nb + 1;
        } else if (x == se[nb]) {
            slot = nb;
        } else {
            int lo = 0, hi = nb;  // largest i < nb with se[i] <= x
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (se[mid] <= x) lo = mid; else hi = mid;
            }
            slot = lo + 1;
        }
        atomicAdd(&sc[slot], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= nb + 1; k += kSpThreads)
        if (sc[k]) atomicAdd(counts + k, static_cast<unsigned long long>(sc[k]));
}

}  // namespace

int launch_spacing_hist(const float* d2, long long m, const HistEdges& edges, unsigned long long* counts,
                        cudaStream_t stream) {
    long long b = (m + kSpThreads - 1) / kSpThreads;
    if (b > 1024) b = 1024;
    spacing_hist<<<static_cast<unsigned>(b < 1 ? 1 : b), kSpThreads, 0, stream>>>(
        reinterpret_cast<const unsigned*>(d2), m, edges, counts);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_spacing(const float* points, long long n, const int32_t* idx, long long m, float* out_d2,
                   int32_t* status, int sms, cudaStream_t stream) {
    unsigned* out = reinterpret_cast<unsigned*>(out_d2);
    const long long qblocks = (m + kSpThreads * kSpQ - 1) / (kSpThreads * kSpQ);
    long long tiles = (m + kSpTile - 1) / kSpTile;
    long long want = (4ll * sms + qblocks - 1) / qblocks;  // candidate ranges per query block
    if (want > tiles) want = tiles;
    if (want > 65535) want = 65535;
    if (want < 1) want = 1;
    const long long chunk = ((tiles + want - 1) / want) * kSpTile;
    const long long splits = (m + chunk - 1) / chunk;
    long long ib = (m + 255) / 256;
    int launched = 1;
    spacing_init<<<static_cast<unsigned>(ib > 4096 ? 4096 : (ib < 1 ? 1 : ib)), 256, 0, stream>>>(out, m);
    if (qblocks > 0 && qblocks <= 0x7fffffffll) {
        spacing_kernel<<<dim3(static_cast<unsigned>(qblocks), static_cast<unsigned>(splits)), kSpThreads, 0, stream>>>(
            points, n, idx, m, chunk, out, status);
        ++launched;
    }
    return cudaGetLastError() == cudaSuccess ? launched : -1;
}

}  // namespace havk
