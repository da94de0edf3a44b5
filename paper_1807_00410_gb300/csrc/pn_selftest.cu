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

// ---- bandwidth of the operator's access pattern -------------------------------
//
// pn_access_probe: a copy of `planes` coefficient planes of a padded R^3 grid
// in the library's plane-major layout, marching column tiles through z the way
// the tiled operator does, with none of its arithmetic.  Each CTA of 512
// threads (four groups of 128, like the operator's) owns a tile of tile_x x
// (128 / tile_x) columns and a z chunk; thread (column, group g) copies planes
// g, g + 4, ... at its column, SL z-slices at a time, so that every thread
// has SL x planes / 4 loads in flight.  It measures what DRAM delivers to
// this pattern -- rows of tile_x floats scattered over `planes` planes whose
// starts lie (R + 1)^2 pitch_x floats apart -- as a function of the run
// length and of the bytes in flight per SM.

namespace {

constexpr int kProbeThreads = 512;

template <int SL, int WX>
__global__ void __launch_bounds__(kProbeThreads, 1)
    k_access_probe(const float* __restrict__ in, float* __restrict__ out, int R, int planes, int64_t pitch_x,
                   int64_t pitch_y, int64_t plane_stride, int zc) {
    constexpr int WY = 128 / WX;
    const int g = threadIdx.y, lin = threadIdx.x + 32 * threadIdx.z;  // group, position within the tile
    const int x = blockIdx.x * WX + lin % WX, y = blockIdx.y * WY + lin / WX;
    const int za = blockIdx.z * zc, zb = min(za + zc, R + 1);
    if (y > R) return;
    const int np = (planes - g + 3) / 4;  // planes g, g + 4, ... below `planes`
    for (int z = za; z < zb; z += SL) {
        float v[SL][16];
#pragma unroll
        for (int d = 0; d < SL; ++d)
#pragma unroll
            for (int j = 0; j < 16; ++j)
                v[d][j] = (j < np && z + d < zb)
                              ? __ldg(in + (g + 4 * j) * plane_stride + (z + d) * pitch_y + y * pitch_x + x)
                              : 0.0f;
#pragma unroll
        for (int d = 0; d < SL; ++d)
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < np && z + d < zb) out[(g + 4 * j) * plane_stride + (z + d) * pitch_y + y * pitch_x + x] = v[d][j];
    }
}

template <int SL, int WX>
cudaError_t launch_probe(const float* in, float* out, int R, int planes, int64_t px, int64_t py, int64_t ps, int zc,
                         cudaStream_t s) {
    constexpr int WY = 128 / WX;
    const dim3 grid(unsigned(R / WX), unsigned((R + 1 + WY - 1) / WY), unsigned((R + 1 + zc - 1) / zc));
    k_access_probe<SL, WX><<<grid, dim3(32, 4, 4), 0, s>>>(in, out, R, planes, px, py, ps, zc);
    return cudaGetLastError();
}

cudaError_t probe_once(int tile_x, int slices, const float* in, float* out, int R, int planes, int64_t px, int64_t py,
                       int64_t ps, int zc, cudaStream_t s) {
    switch (tile_x * 8 + slices) {
        case 32 * 8 + 1: return launch_probe<1, 32>(in, out, R, planes, px, py, ps, zc, s);
        case 32 * 8 + 2: return launch_probe<2, 32>(in, out, R, planes, px, py, ps, zc, s);
        case 32 * 8 + 4: return launch_probe<4, 32>(in, out, R, planes, px, py, ps, zc, s);
        case 64 * 8 + 1: return launch_probe<1, 64>(in, out, R, planes, px, py, ps, zc, s);
        case 64 * 8 + 2: return launch_probe<2, 64>(in, out, R, planes, px, py, ps, zc, s);
        case 64 * 8 + 4: return launch_probe<4, 64>(in, out, R, planes, px, py, ps, zc, s);
        case 128 * 8 + 1: return launch_probe<1, 128>(in, out, R, planes, px, py, ps, zc, s);
        case 128 * 8 + 2: return launch_probe<2, 128>(in, out, R, planes, px, py, ps, zc, s);
        default: return launch_probe<4, 128>(in, out, R, planes, px, py, ps, zc, s);
    }
}

}  // namespace

extern "C" int pn_access_probe(int R, int planes, int tile_x, int slices, double* gbs_out, void* stream) {
    if (!gbs_out || R < 128 || R > 512 || planes < 4 || planes > 64 || planes % 4 != 0 ||
        (tile_x != 32 && tile_x != 64 && tile_x != 128) || (slices != 1 && slices != 2 && slices != 4) ||
        R % tile_x != 0)
        return PN_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the plane-major layout of a handle of this size: rows padded to 16
    // bytes, planes padded to 256 bytes
    const int64_t px = (int64_t(R) + 1 + 3) / 4 * 4;
    const int64_t py = px * (R + 1);
    const int64_t ps = (py * (R + 1) + 63) / 64 * 64;
    const size_t n = size_t(planes) * size_t(ps);
    float* in = nullptr;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&in, n * sizeof(float)) != cudaSuccess || cudaMalloc(&out, n * sizeof(float)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (in) cudaFree(in);
        if (out) cudaFree(out);
        if (e0) cudaEventDestroy(e0);
        return PN_ERR_ALLOC;
    }
    const int zc = (R + 1 + 3) / 4;  // four z chunks
    cudaError_t e = cudaMemsetAsync(in, 0, n * sizeof(float), s);
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = probe_once(tile_x, slices, in, out, R, planes, px, py, ps, zc, s);
    float best = 1e30f;
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = probe_once(tile_x, slices, in, out, R, planes, px, py, ps, zc, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) best = ms;
    }
    cudaFree(in);
    cudaFree(out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PN_ERR_CUDA;
    }
    const double bytes = 2.0 * 4.0 * double(planes) * double(R) * double(R + 1) * double(R + 1);
    *gbs_out = bytes / (double(best) * 1e-3) / 1e9;
    return PN_OK;
}
