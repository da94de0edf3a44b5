// pn_wait_timeout_test: exercises the bounded mbarrier wait that every
// TMA-staged kernel of the library uses (pn_mbar.cuh), without any copy.
//
// One CTA initialises an mbarrier with one expected arrival.  With deliver = 1
// its thread 0 arrives expecting no bytes, which completes the phase; with
// deliver = 0 it arrives expecting 16 bytes that no copy ever brings, so the
// phase never completes and every thread's wait runs out after limit_ns of
// %globaltimer and sets the error flag -- the same flag (the handle's fault
// word) that the operator's and the vector kernels' waits set, which pn_solve
// reports as PN_ERR_TIMEOUT.  No copy is in flight when the CTA exits.
#include <cuda_runtime.h>

#include <cstdint>

#include "pn_internal.h"
#include "pn_mbar.cuh"

namespace {

__global__ void k_wait_timeout_test(int deliver, unsigned long long limit_ns, unsigned int* err) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = pn::mbar::smem_u32(&bar);
    if (threadIdx.x == 0) {
        pn::mbar::init(b, 1u);
        pn::mbar::fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) pn::mbar::arrive_expect_tx(b, deliver ? 0u : 16u);
    bool failed = false;
    pn::mbar::wait_ns(b, 0u, err, failed, limit_ns);
    __syncthreads();
}

}  // namespace

extern "C" int pn_wait_timeout_test(pn_handle* h, int deliver, long long limit_ns, int* timed_out, void* stream) {
    if (!timed_out || limit_ns <= 0 || limit_ns > 10000000000LL || (deliver != 0 && deliver != 1))
        return h ? pn_fail(h, PN_ERR_ARG, "pn_wait_timeout_test: bad argument") : PN_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned int* flag = nullptr;
    bool own = false;
    if (h) {
        flag = reinterpret_cast<unsigned int*>(h->d_scalars + PN_S_FAULT);
    } else {
        if (cudaMalloc(&flag, sizeof(unsigned int)) != cudaSuccess) {
            cudaGetLastError();
            return PN_ERR_ALLOC;
        }
        own = true;
        if (cudaMemsetAsync(flag, 0, sizeof(unsigned int), s) != cudaSuccess) {
            cudaFree(flag);
            return PN_ERR_CUDA;
        }
    }
    // the flag's state before the launch (a handle's earlier fault stays reported)
    unsigned int before = 0, after = 0;
    cudaError_t e = cudaMemcpyAsync(&before, flag, sizeof(before), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        k_wait_timeout_test<<<1, 64, 0, s>>>(deliver, static_cast<unsigned long long>(limit_ns), flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&after, flag, sizeof(after), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (own) cudaFree(flag);
    if (e != cudaSuccess) return h ? pn_cuda_fail(h, e, "pn_wait_timeout_test") : PN_ERR_CUDA;
    *timed_out = (after != 0u && before == 0u) ? 1 : 0;
    return *timed_out ? PN_ERR_TIMEOUT : PN_OK;
}

// ---- arithmetic peaks ---------------------------------------------------------
//
// pn_fma_peak: the FP64 (or FP32) FMA rate of this GPU, measured by a kernel of
// independent FMA chains (8 per thread, 2048 iterations each, every SM full),
// timed with CUDA events.  The denominator of the roofline of kernels bound
// by FP64 arithmetic (GB300's FP64 rate is a small fraction of its FP32 rate).

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T seed, int iters, T* sink) {
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + T(threadIdx.x + k);
    const T m = T(0.999999), c = T(1e-7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = a[k] * m + c;  // one FMA each
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == T(-1)) sink[0] = s;  // keeps the chains alive; never true for these inputs
}

template <typename T>
int fma_peak(double* gflops, cudaStream_t s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return PN_ERR_CUDA;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_chains<T>, 256, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return PN_ERR_CUDA;
    }
    const int blocks = occ * sms, iters = 2048;
    T* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (sink) cudaFree(sink);
        if (e0) cudaEventDestroy(e0);
        return PN_ERR_ALLOC;
    }
    k_fma_chains<T><<<blocks, 256, 0, s>>>(T(1), iters, sink);  // warm-up
    float best = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, s);
        k_fma_chains<T><<<blocks, 256, 0, s>>>(T(1), iters, sink);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) best = ms;
    }
    cudaFree(sink);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PN_ERR_CUDA;
    }
    const double flops = 2.0 * 8.0 * double(iters) * double(blocks) * 256.0;
    *gflops = flops / (double(best) * 1e-3) / 1e9;
    return PN_OK;
}

}  // namespace

extern "C" int pn_fma_peak(int dtype, double* gflops_out, void* stream) {
    if (!gflops_out || (dtype != PN_F32 && dtype != PN_F64)) return PN_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return dtype == PN_F64 ? fma_peak<double>(gflops_out, s) : fma_peak<float>(gflops_out, s);
}
