// pn_dot_noalloc: an inner product that allocates nothing.
//
// pn_dot works through a pn_handle, and creating a handle allocates device
// memory (medium copies, reduction scratch).  Some callers cannot allocate at
// the point where they need a reduction: a host application that reserves
// the whole device-memory budget up front and forbids hidden allocations, a
// real-time loop that must not take the allocator's locks or risk an
// out-of-memory failure midway, or code that holds device vectors but no
// pn_handle.  For them this entry point keeps its scratch in a fixed,
// file-scope __device__ array that exists for as long as the library is
// loaded on a device.
//
// Scratch: g_noalloc_scratch holds one FP64 partial sum per block of 8192
// elements plus one result slot; PN_NOALLOC_MAX_ELEMS bounds n.  Each call
// overwrites every slot it reads (partials are stored, never accumulated, and
// the result slot is written by the final kernel), so nothing has to be
// cleared between calls.  All calls share the array: two calls whose kernels
// overlap on the GPU (different streams, or different host threads) race.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "pn_gb300.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 32;                                   // elements per thread
constexpr int64_t kPerBlock = int64_t(kThreads) * kItems;    // elements per block
constexpr int kMaxBlocks = PN_NOALLOC_MAX_ELEMS / kPerBlock;  // partial-sum slots
static_assert(int64_t(kMaxBlocks) * kPerBlock == PN_NOALLOC_MAX_ELEMS, "capacity must be whole blocks");

// kMaxBlocks partials, then the result slot (2 MiB + 256 B per device).
static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks + 32];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  The symbol's
// name in host code is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int scratch_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PN_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return PN_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_dev_ptr[dev] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return PN_ERR_CUDA;
        }
        g_dev_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_dev_ptr[dev];
    return PN_OK;
}

__device__ __forceinline__ double block_total(double v) {
    __shared__ double red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = 0.0;
    if (threadIdx.x < 32) {
        v = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Block b sums x_i * y_i over its own 8192 elements (products and sums in FP64).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot_blocks(const T* x, const T* y, int64_t n, double* partials) {
    const int64_t base = int64_t(blockIdx.x) * kPerBlock + threadIdx.x;
    double acc = 0.0;
#pragma unroll 8
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = base + int64_t(i) * kThreads;
        if (idx < n) acc = fma(double(x[idx]), double(y[idx]), acc);
    }
    const double t = block_total(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// result = sum of the nb partials, in a fixed order.
__global__ void __launch_bounds__(kThreads) k_dot_total(const double* partials, int nb, double* result) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) acc += partials[i];
    const double t = block_total(acc);
    if (threadIdx.x == 0) *result = t;
}

}  // namespace

extern "C" int pn_dot_noalloc(const void* x, const void* y, int64_t n, int dtype, double* out, void* stream) {
    if (!out || (n > 0 && (!x || !y))) return PN_ERR_ARG;
    if (dtype != PN_F32 && dtype != PN_F64) return PN_ERR_ARG;
    if (n < 0) return PN_ERR_ARG;
    if (n > PN_NOALLOC_MAX_ELEMS) return PN_ERR_TOO_LARGE;
    const uintptr_t esz = dtype == PN_F32 ? 4u : 8u;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & (esz - 1)) return PN_ERR_ARG;
    if (n == 0) {
        *out = 0.0;
        return PN_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the result comes back through a host copy and a stream synchronisation,
    // which a capturing stream cannot take
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return PN_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return PN_ERR_ARG;
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != PN_OK) return rc;
    const int nb = int((n + kPerBlock - 1) / kPerBlock);
    if (dtype == PN_F32)
        k_dot_blocks<float><<<nb, kThreads, 0, s>>>(static_cast<const float*>(x), static_cast<const float*>(y), n,
                                                    scratch);
    else
        k_dot_blocks<double><<<nb, kThreads, 0, s>>>(static_cast<const double*>(x), static_cast<const double*>(y),
                                                     n, scratch);
    k_dot_total<<<1, kThreads, 0, s>>>(scratch, nb, scratch + kMaxBlocks);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PN_ERR_CUDA;
    }
    return PN_OK;
}
