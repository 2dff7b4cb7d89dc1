// pakr_static.cu -- pakr_nearest_static: the cost-pruned nearest-neighbour
// search for callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a nearest
// neighbour: real-time control loops that forbid allocation (and the device-wide
// synchronisation cudaFree can bring) after start-up, and plugins that live
// inside another framework's memory pool and may only use what it hands them.
// They own their inputs and outputs; what they cannot provide is the library's
// per-query scratch (the packed distance / index keys that the node chunks merge
// into, plus the two scalars the search kernel reads).  This file keeps that
// scratch in one file-scope device array instead, sized for kStaticMaxQueries
// queries; every GPU that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/pakr.h"
#include "pakr_internal.h"

namespace pakr {
namespace {

constexpr int kStaticMaxQueries = 65536;
// The array starts with a control block (tree size and bound for the search
// kernel), followed by one 64-bit key per query.
constexpr int kCtlWords = (int)((sizeof(Ctl) + 255) / 256 * 256 / sizeof(unsigned long long));
constexpr int kScratchWords = kCtlWords + kStaticMaxQueries;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_nn_scratch[kScratchWords];

std::mutex g_setup_mu;
bool g_ready[kMaxDevices];                        // per device: kernels loaded, sizes queried
int g_nn_occ[kMaxDevices][3];                     // occupancy of the three search variants, per device
int g_sms[kMaxDevices];
int g_occ_d[kMaxDevices];                         // state dimension the occupancy was taken for

pakr_status fail(pakr_status st, const char *msg)
{
    record_error(msg);
    return st;
}

__global__ void k_static_begin(unsigned long long *scratch, int n_queries, int n, float bound);
__global__ void k_static_finish(const unsigned long long *scratch, int n_queries, int32_t *nearest, float *dist2);

// Per call, with the device current: the device address of the scratch array (in host code
// its name is only a host-side stand-in).  Looked up on every call, so that a module that was
// reloaded (a device reset, a new context) is never reached through a stale address; once
// the module is loaded the lookup allocates nothing.  The first call on a device also loads
// the GPU code of every search variant and of the two helper kernels, and reads the SM count,
// so that no later call loads code.
pakr_status setup(int dev, unsigned long long **addr)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_nn_scratch);
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        return fail(PAKR_ERR_CUDA, buf);
    }
    *addr = (unsigned long long *)p;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_ready[dev]) {
        cudaFuncAttributes fa;
        e = nn_preload_all();
        if (e == cudaSuccess)
            e = cudaFuncGetAttributes(&fa, k_static_begin);
        if (e == cudaSuccess)
            e = cudaFuncGetAttributes(&fa, k_static_finish);
        if (e != cudaSuccess) {
            char buf[256];
            snprintf(buf, sizeof(buf), "loading the search kernels failed: %s", cudaGetErrorString(e));
            return fail(PAKR_ERR_CUDA, buf);
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return fail(PAKR_ERR_CUDA, "cudaDeviceGetAttribute failed");
        g_sms[dev] = sms;
        g_ready[dev] = true;
    }
    return PAKR_OK;
}

int dyn_for_dim(int d)
{
    switch (d) {
    case 3: return UNICYCLE1;
    case 4: return DI2;
    case 5: return UNICYCLE2;
    case 6: return DI3;
    case 12: return QUAD12;
    default: return -1;
    }
}

// Clears the keys the search merges into and writes the two scalars it reads.
__global__ void k_static_begin(unsigned long long *scratch, int n_queries, int n, float bound)
{
    Ctl *ctl = reinterpret_cast<Ctl *>(scratch);
    unsigned long long *keys = scratch + kCtlWords;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_queries)
        keys[i] = kNoKey;
    if (i == 0) {
        ctl->n_start = n;
        ctl->bound = bound;
    }
}

// Unpacks the merged keys into the caller's outputs.
__global__ void k_static_finish(const unsigned long long *scratch, int n_queries, int32_t *nearest, float *dist2)
{
    const unsigned long long *keys = scratch + kCtlWords;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_queries)
        return;
    const unsigned long long key = keys[i];
    nearest[i] = key == kNoKey ? -1 : (int32_t)(uint32_t)(key & 0xFFFFFFFFull);
    if (dist2)
        dist2[i] = key == kNoKey ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(key >> 32));
}

}  // namespace
}  // namespace pakr

using namespace pakr;

extern "C" pakr_status pakr_nearest_static(const float *states, int64_t ld, int64_t n, int32_t d, const float *fcost,
                                           float bound, const float *queries, int32_t n_queries, int32_t *nearest,
                                           float *dist2, void *cuda_stream)
{
    const int dyn = dyn_for_dim(d);
    if (dyn < 0)
        return fail(PAKR_ERR_INVALID_ARG, "pakr_nearest_static: d must be 3, 4, 5, 6 or 12");
    if (n_queries < 0 || n_queries > kStaticMaxQueries)
        return fail(PAKR_ERR_INVALID_ARG,
                    "pakr_nearest_static: n_queries must be in [0, 65536], the size of the static scratch");
    if (n < 0 || n > kMaxTreeNodes || ld < n || ld > 0x7FFFFFFFLL)
        return fail(PAKR_ERR_INVALID_ARG, "pakr_nearest_static: need 0 <= n <= 2^31 - 2^20 and n <= ld < 2^31");
    if (std::isnan(bound))
        return fail(PAKR_ERR_INVALID_ARG, "pakr_nearest_static: bound is NaN");
    if (n_queries == 0)
        return PAKR_OK;
    if (!nearest || !queries || (n > 0 && (!states || !fcost)))
        return fail(PAKR_ERR_INVALID_ARG, "pakr_nearest_static: NULL buffer");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(PAKR_ERR_CUDA, "pakr_nearest_static: no current CUDA device");
    unsigned long long *scratch = nullptr;
    pakr_status st = setup(dev, &scratch);
    if (st != PAKR_OK)
        return st;

    DevProblem P{};
    P.dyn = dyn;
    P.d = d;
    for (int a = 0; a < kMaxD; ++a)
        P.sw[a] = 1.f;
    P.K = n_queries;
    P.k = 1;
    P.cap = (int)ld;
    DevTree T{};
    T.X = const_cast<float *>(states);
    T.fcost = const_cast<float *>(fcost);
    DevWork W{};
    W.xr = const_cast<float *>(queries);
    W.nn_key = scratch + kCtlWords;
    LaunchCfg L{};
    if (n_queries >= 1024) {
        L.nn_variant = 2;
        L.nn_threads = 256;
        L.nn_qpt = 4;
    } else if (n_queries >= 256) {
        L.nn_variant = 1;
        L.nn_threads = 128;
        L.nn_qpt = 2;
    } else {
        L.nn_variant = 0;
        L.nn_threads = 64;
        L.nn_qpt = 2;
    }
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (g_occ_d[dev] != d) {
            for (int v = 0; v < 3; ++v)
                g_nn_occ[dev][v] = std::max(1, nn_blocks_per_sm(d, v));
            g_occ_d[dev] = d;
        }
        const int per_block = L.nn_threads * L.nn_qpt;
        L.nn_qgroups = (n_queries + per_block - 1) / per_block;
        L.nn_chunks = std::max(1, g_sms[dev] * g_nn_occ[dev][L.nn_variant] / L.nn_qgroups);
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int blocks = (n_queries + 255) / 256;
    k_static_begin<<<blocks, 256, 0, s>>>(scratch, n_queries, (int)n, bound);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_nn(P, reinterpret_cast<const Ctl *>(scratch), T, W, L, s);
    if (e == cudaSuccess) {
        k_static_finish<<<blocks, 256, 0, s>>>(scratch, n_queries, nearest, dist2);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "pakr_nearest_static: launch failed: %s", cudaGetErrorString(e));
        return fail(PAKR_ERR_CUDA, buf);
    }
    return PAKR_OK;
}
