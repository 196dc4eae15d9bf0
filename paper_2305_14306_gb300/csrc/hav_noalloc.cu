// hav_sample_noalloc: the single-cloud sampler for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs inside another
// framework's memory pool or a strict memory budget, plugin hosts that forbid
// allocation after start-up, and real-time loops where an allocation (and the
// device-wide synchronisation it can imply) is not allowed.  They cannot
// create a hav_ctx, because the context allocates its workspace.  This entry
// point gives them the same sampler without a context: its scratch lives in a
// file-scope static __device__ array that the CUDA module reserves when the
// library is loaded, so no call allocates.
//
// The scratch holds the workspace of one cloud of up to
// kNoAllocMaxPoints = 32,768 points (7.25 MB of the 8.39 MB array).  Every GPU
// that loads libhav.so keeps this array until the process exits.

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "hav.h"
#include "hav_internal.h"

namespace {

constexpr int64_t kNoAllocMaxPoints = 32768;
constexpr size_t kNoAllocScratchBytes = 8u << 20;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceSetup {
    unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch at the last set-up
    int nblocks = 0;                   // co-resident blocks of the sampler kernel on this device
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Every call, with the device current: resolve the array's device address
// (in host code its name is only a stand-in).  The lookup allocates nothing.
// The launch set-up (the kernel's shared-memory attribute, the grid size) is
// kept per device and redone whenever the address changes, which is what
// happens when the module is loaded again in a new context (after
// cudaDeviceReset, or in another primary context).
hav_status setup_device(int dev, unsigned char** scratch, int* nblocks) {
    if (dev < 0 || dev >= kMaxDevices) return HAV_ERR_INVALID;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return HAV_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (s.scratch != ptr || s.nblocks < 1) {
        const int nb = havk::max_coresident_blocks(dev);
        if (nb < 1) {
            cudaGetLastError();
            return HAV_ERR_CUDA;
        }
        s.scratch = static_cast<unsigned char*>(ptr);
        s.nblocks = nb;
    }
    *scratch = s.scratch;
    *nblocks = s.nblocks;
    return HAV_OK;
}

hav_status check_noalloc_params(const hav_params* p) {
    if (!p) return HAV_ERR_INVALID;
    if (p->sigma_num < 0 || p->sigma_den <= 0) return HAV_ERR_INVALID;
    if (static_cast<long long>(p->sigma_num) > 64ll * p->sigma_den) return HAV_ERR_INVALID;
    if (p->t_max < 0 || p->t_max > HAV_MAX_ITERS) return HAV_ERR_INVALID;
    if (p->layers < 1 || p->layers > havk::kMaxLayers) return HAV_ERR_INVALID;
    if (p->layer_ratio < 1 || p->layer_ratio > 64) return HAV_ERR_INVALID;
    long long w = 1;
    for (int i = 1; i < p->layers; ++i) {
        w *= p->layer_ratio;
        if (w > (1ll << 31)) return HAV_ERR_INVALID;
    }
    for (int a = 0; a < 3; ++a)
        if (!(p->aspect[a] > 0.0f) || !std::isfinite(p->aspect[a])) return HAV_ERR_INVALID;
    if (p->flags != 0) return HAV_ERR_INVALID;
    return havk::check_variant_params(p);
}

}  // namespace

extern "C" hav_status hav_sample_noalloc(const float* points, int64_t n, int64_t m,
                                         const hav_params* params, int32_t* out_idx,
                                         int32_t* status_out, hav_stream stream) {
    hav_status st = check_noalloc_params(params);
    if (st != HAV_OK) return st;
    if (n < 0 || m < 0 || m > n) return HAV_ERR_INVALID;
    if (n > kNoAllocMaxPoints) return HAV_ERR_NOMEM;  // beyond the static scratch
    if (m > 0 && (!points || !out_idx)) return HAV_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(points) % 4 != 0) return HAV_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HAV_ERR_CUDA;
    unsigned char* scratch = nullptr;
    int nblocks = 0;
    st = setup_device(dev, &scratch, &nblocks);
    if (st != HAV_OK) return st;

    const havk::Layout lay = havk::make_layout(kNoAllocMaxPoints, 1, /*spec_room=*/false);
    if (lay.total > kNoAllocScratchBytes) return HAV_ERR_NOMEM;

    cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
    // The header (barrier, status words, bounding-box codes) must start at
    // zero; every other region is cleared by the kernel before it is read.
    if (cudaMemsetAsync(scratch + lay.barrier, 0, lay.zero_bytes, strm) != cudaSuccess)
        return HAV_ERR_CUDA;
    if (m > 0) {
        havk::Plan plan;
        std::memset(&plan, 0, sizeof plan);
        plan.points = points;
        plan.ws = scratch;
        plan.lay = lay;
        plan.S = 1;
        plan.L = 1;
        plan.layers = params->layers;
        plan.ratio = params->layer_ratio;
        plan.t_max = params->t_max;
        plan.sigma_num = params->sigma_num;
        plan.sigma_den = params->sigma_den;
        plan.nblocks = nblocks;
        plan.chunk_min = havk::kChunkMin;
        plan.table_log2 = 1;
        plan.pass_shape = 0;
        for (int a = 0; a < 3; ++a) plan.aspect[a] = params->aspect[a];
        plan.select = params->select;
        plan.seed = params->seed;
        plan.fixed_s = params->fixed_s;
        plan.search = params->search;
        plan.out[0] = out_idx;
        plan.off0[0] = 0;
        plan.off0[1] = n;
        plan.m[0][0] = static_cast<int32_t>(m);
        if (havk::launch_chain(plan, strm) < 0) return HAV_ERR_CUDA;
    }
    if (status_out) {
        const havk::GlobalHdr* gh = reinterpret_cast<const havk::GlobalHdr*>(scratch + lay.ghdr);
        if (cudaMemcpyAsync(status_out, &gh->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, strm) !=
            cudaSuccess)
            return HAV_ERR_CUDA;
    }
    return HAV_OK;
}
