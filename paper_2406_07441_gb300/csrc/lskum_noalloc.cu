// Density-residual norm for callers that cannot allocate device memory.
//
// Some callers of this library must not call cudaMalloc: hosts whose device
// memory is entirely handed to their own pool allocator, latency-critical
// loops where an allocation or a free could synchronise the device, and
// deployments whose policy forbids runtime allocation.  For them
// lskum_density_norm_noalloc computes the same norm as the solver's own
// two-stage reduction (block partial sums of squares, then one block adding
// the partials in a fixed order) with the partials kept in a fixed,
// file-scope device array instead of memory allocated per context.
//
// The array is kNoAllocMaxPartials doubles (64 KiB); every GPU that loads
// this library holds it until the process exits.  All calls share it:
// stage 1 writes every partial that stage 2 of the same call reads, so
// nothing needs clearing, but calls that overlap on the GPU (concurrent
// streams, or several host threads) race on it and must be serialised by the
// caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/lskum.h"

namespace {

constexpr int kNoAllocMaxPartials = 8192;          // stage-1 blocks (partials)
constexpr int kNoAllocThreads = 256;               // threads per stage-1 block
constexpr int kNoAllocMaxPerThread = 64;           // elements one thread may add
constexpr int64_t kNoAllocMaxN =
    (int64_t)kNoAllocMaxPartials * kNoAllocThreads * kNoAllocMaxPerThread;  // 134,217,728
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kNoAllocMaxPartials];

// Host-side device addresses of g_partials, one per device (the symbol's name
// in host code is only a stand-in, never a device address).  Valid while the
// device's primary context lives; a failed launch clears the entry.
double *g_partials_dev[kMaxDevices] = {};
std::mutex g_setup_mutex;

__global__ void __launch_bounds__(kNoAllocThreads) k_sumsq_partials(const double *__restrict__ r, int32_t n,
                                                                     double *__restrict__ partials)
{
    __shared__ double red[kNoAllocThreads / 32];
    double t = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        t += r[k] * r[k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < (kNoAllocThreads / 32) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(1024) k_sqrt_of_partials(const double *__restrict__ partials, int nparts,
                                                           double *__restrict__ out)
{
    __shared__ double red[32];
    double t = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) t += partials[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[0] = sqrt(s);
    }
}

}  // namespace

extern "C" lskum_status lskum_density_norm_noalloc(const double *r_rho_dev, int32_t n, double *norm_dev,
                                                   void *cuda_stream)
{
    if (!norm_dev || n < 0 || (n > 0 && !r_rho_dev)) return LSKUM_ERR_ARG;
    if ((int64_t)n > kNoAllocMaxN) return LSKUM_ERR_ARG;  // beyond the fixed scratch's reach
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LSKUM_ERR_CUDA;
    double *partials = nullptr;
    {
        // one-time set-up per device, with that device current
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_dev[dev]) {
            double *p = nullptr;
            if (cudaGetSymbolAddress((void **)&p, g_partials) != cudaSuccess || !p) return LSKUM_ERR_CUDA;
            g_partials_dev[dev] = p;
        }
        partials = g_partials_dev[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int blocks = (int)(((int64_t)n + kNoAllocThreads - 1) / kNoAllocThreads);
    if (blocks > kNoAllocMaxPartials) blocks = kNoAllocMaxPartials;
    if (blocks > 0) k_sumsq_partials<<<blocks, kNoAllocThreads, 0, s>>>(r_rho_dev, n, partials);
    k_sqrt_of_partials<<<1, 1024, 0, s>>>(partials, blocks, norm_dev);
    if (cudaGetLastError() == cudaSuccess) return LSKUM_OK;
    // the cached address may be stale (a reset device reloads the module):
    // forget it, so that the next call looks it up again
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    g_partials_dev[dev] = nullptr;
    return LSKUM_ERR_CUDA;
}
