// Layer kernels of the learned preconditioner (3D convolutional
// encoder-decoder).  The paper has no network: this is the learned
// extension of the solver.  Activations are BF16, channels-last
// ([b][z][y][x][c], channel counts multiples of 16, layers may read and
// write channel slices of wider tensors); weights are BF16 for the tensor
// cores with FP32 master copies; every product accumulates in FP32.
//
// 3x3x3 convolutions (stride 1, zero padding) run as implicit GEMMs on the
// BF16 tensor cores (mma.sync m16n8k16, FP32 accumulators): M = voxels,
// N = output channels, K = 27 taps x input channels.  Each warp owns 16
// consecutive voxels and loads its fragments straight from global memory
// (zero outside the grid), so arbitrary (also tiny) grid sizes need no
// tiling logic.  The input gradient is the same kernel on tap-flipped,
// transposed weights; the weight gradient is a GEMM over voxels with one
// CTA per tap.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pn_cnn.h"

namespace pn {
namespace cnn {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return __ldg(reinterpret_cast<const unsigned int*>(p)); }

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}

struct Vox {
    int b, z, y, x;
    bool ok;
};

__device__ __forceinline__ Vox vox_of(int64_t v, const Grid& g) {
    Vox r;
    r.ok = v < g.nvox;
    if (!r.ok) v = 0;
    r.x = int(v % g.X);
    int64_t t = v / g.X;
    r.y = int(t % g.Y);
    t /= g.Y;
    r.z = int(t % g.Z);
    r.b = int(t / g.Z);
    return r;
}

__device__ __forceinline__ int64_t nb_index(const Vox& v, int dz, int dy, int dx, const Grid& g, bool& ok) {
    const int z = v.z + dz, y = v.y + dy, x = v.x + dx;
    ok = v.ok && z >= 0 && y >= 0 && x >= 0 && z < g.Z && y < g.Y && x < g.X;
    return ((int64_t(v.b) * g.Z + z) * g.Y + y) * g.X + x;
}

// out[v][o] = act(bias[o] + sum_{t,c} w[t][o][c] in[v + t][c])
// Warp: 16 consecutive voxels x NT*8 output channels (chunk blockIdx.y).
template <int NT>
__global__ void __launch_bounds__(256) k_conv3(ConvArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t v0 = (int64_t(blockIdx.x) * 8 + warp) * 16;
    const int co0 = blockIdx.y * NT * 8;
    const Vox va = vox_of(v0 + g, a.g), vb = vox_of(v0 + g + 8, a.g);
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.0f;
    for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        bool oka, okb;
        const int64_t na = nb_index(va, dz, dy, dx, a.g, oka), nb = nb_index(vb, dz, dy, dx, a.g, okb);
        const bf16* pa = a.in + na * a.in_cs + a.in_co + 2 * t;
        const bf16* pb = a.in + nb * a.in_cs + a.in_co + 2 * t;
        const bf16* wt = a.w + (int64_t(tap) * a.co_total + co0 + g) * a.ci + 2 * t;
        for (int k = 0; k < a.ci; k += 16) {
            uint32_t A[4];
            A[0] = oka ? ld32(pa + k) : 0u;
            A[1] = okb ? ld32(pb + k) : 0u;
            A[2] = oka ? ld32(pa + k + 8) : 0u;
            A[3] = okb ? ld32(pb + k + 8) : 0u;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const bf16* wn = wt + int64_t(n) * 8 * a.ci + k;
                mma_bf16(acc[n], A, ld32(wn), ld32(wn + 8));
            }
        }
    }
    // epilogue: rows g and g + 8, channels co0 + n*8 + 2t, +1
#pragma unroll
    for (int n = 0; n < NT; ++n) {
        const int co = co0 + n * 8 + 2 * t;
        const float b0 = a.bias ? a.bias[co] : 0.0f, b1 = a.bias ? a.bias[co + 1] : 0.0f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t v = v0 + g + 8 * h;
            if (v >= a.g.nvox) continue;
            float x0 = acc[n][2 * h] + b0, x1 = acc[n][2 * h + 1] + b1;
            if (a.relu) {
                x0 = fmaxf(x0, 0.0f);
                x1 = fmaxf(x1, 0.0f);
            }
            *reinterpret_cast<uint32_t*>(a.out + v * a.out_cs + a.out_co + co) =
                pack2(__float2bfloat16_rn(x0), __float2bfloat16_rn(x1));
        }
    }
}

// dW[tap][o][c] += sum_v gy[v][o] x[v + t][c]   (CTA: one tap, one voxel range)
// M = output channels (rows), N = input channels, K = voxels.  Warp w owns
// (m, n) tile pairs w, w+8, ...; fragments are gathered from global memory.
constexpr int kWPairs = 8;  // max (m, n) pairs per warp

__global__ void __launch_bounds__(256) k_conv3_wgrad(WgradArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int tap = blockIdx.x;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int mt = a.co / 16, ntiles = a.ci / 8;
    const int npairs = mt * ntiles;
    float acc[kWPairs][4];
#pragma unroll
    for (int p = 0; p < kWPairs; ++p) acc[p][0] = acc[p][1] = acc[p][2] = acc[p][3] = 0.0f;
    const int64_t per = (a.g.nvox + gridDim.y - 1) / gridDim.y;
    const int64_t vbeg = int64_t(blockIdx.y) * per, vend = min(a.g.nvox, vbeg + per);
    for (int64_t vk = vbeg; vk < vend; vk += 16) {
        // this thread's voxels for the k dimension: 2t, 2t+1, 2t+8, 2t+9
        int64_t vv[4] = {vk + 2 * t, vk + 2 * t + 1, vk + 2 * t + 8, vk + 2 * t + 9};
        bool in_ok[4];
        int64_t xi[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Vox vo = vox_of(vv[q] < vend ? vv[q] : a.g.nvox, a.g);
            xi[q] = nb_index(vo, dz, dy, dx, a.g, in_ok[q]);
            in_ok[q] = in_ok[q] && vv[q] < vend;
        }
#pragma unroll
        for (int p = 0; p < kWPairs; ++p) {
            const int pair = warp + 8 * p;
            if (pair >= npairs) break;
            const int m = pair / ntiles, n = pair % ntiles;
            // A (16 out-channels x 16 voxels, row-major): rows o = 16m + g (+8), cols v
            uint32_t A[4];
            const int o0 = 16 * m + g, o1 = o0 + 8;
            auto gyv = [&](int q, int o) -> bf16 {
                return vv[q] < vend ? a.gy[vv[q] * a.gy_cs + a.gy_co + o] : __float2bfloat16_rn(0.0f);
            };
            A[0] = pack2(gyv(0, o0), gyv(1, o0));
            A[1] = pack2(gyv(0, o1), gyv(1, o1));
            A[2] = pack2(gyv(2, o0), gyv(3, o0));
            A[3] = pack2(gyv(2, o1), gyv(3, o1));
            // B (16 voxels x 8 in-channels, col-major): col c = 8n + g
            const int c = 8 * n + g;
            auto xv = [&](int q) -> bf16 {
                return in_ok[q] ? a.x[xi[q] * a.x_cs + a.x_co + c] : __float2bfloat16_rn(0.0f);
            };
            mma_bf16(acc[p], A, pack2(xv(0), xv(1)), pack2(xv(2), xv(3)));
        }
    }
    // C fragment: rows o = 16m + g (+8), cols c = 8n + 2t, +1
#pragma unroll
    for (int p = 0; p < kWPairs; ++p) {
        const int pair = warp + 8 * p;
        if (pair >= npairs) break;
        const int m = pair / ntiles, n = pair % ntiles;
        const int o0 = 16 * m + g, c = 8 * n + 2 * t;
        float* d0 = a.dw + (int64_t(tap) * a.co + o0) * a.ci + c;
        float* d1 = a.dw + (int64_t(tap) * a.co + o0 + 8) * a.ci + c;
        atomicAdd(d0, acc[p][0]);
        atomicAdd(d0 + 1, acc[p][1]);
        atomicAdd(d1, acc[p][2]);
        atomicAdd(d1 + 1, acc[p][3]);
    }
}

// db[o] += sum_v gy[v][o]
__global__ void k_bias_grad(const bf16* gy, int cs, int co_off, int co, int64_t nvox, float* db) {
    const int o = blockIdx.y * 32 + (threadIdx.x & 31);
    if (o >= co) return;
    float acc = 0.0f;
    for (int64_t v = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5); v < nvox; v += int64_t(gridDim.x) * 8)
        acc += __bfloat162float(gy[v * cs + co_off + o]);
    atomicAdd(db + o, acc);
}

// wt[tap][c][o] = w[26 - tap][o][c]  (weights of the input-gradient convolution)
__global__ void k_flip_weights(const bf16* w, bf16* wt, int co, int ci) {
    const int64_t n = int64_t(27) * co * ci;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % ci);
        const int64_t r = i / ci;
        const int o = int(r % co);
        const int tap = int(r / co);
        wt[(int64_t(tap) * ci + c) * co + o] = w[(int64_t(26 - tap) * co + o) * ci + c];
    }
}

// FP32 master weights -> BF16 copies
__global__ void k_to_bf16(const float* src, bf16* dst, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

// The resampling and ReLU kernels move 8 channels (16 bytes) per thread:
// every channel count and slice offset of the network is a multiple of 16.
__device__ __forceinline__ void bf8_to_f(const uint4 u, float (&f)[8]) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 t = __bfloat1622float2(h[k]);
        f[2 * k] = t.x;
        f[2 * k + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 f_to_bf8(const float (&f)[8]) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    return u;
}

__device__ __forceinline__ const uint4* at8(const bf16* base, int64_t v, int cs, int co, int c8) {
    return reinterpret_cast<const uint4*>(base + v * cs + co + 8 * c8);
}

// fine voxel index of child q (0..7) of coarse voxel o
__device__ __forceinline__ int64_t child(const Vox& o, int q, const Grid& gi) {
    return ((int64_t(o.b) * gi.Z + 2 * o.z + (q >> 2)) * gi.Y + 2 * o.y + ((q >> 1) & 1)) * gi.X + 2 * o.x + (q & 1);
}

// out[v][c] = scale * sum of the 2x2x2 block of the input grid (channel
// slices); accumulate adds to out.  scale 1/8: mean pooling; 1: the backward
// of nearest upsampling.
__global__ void k_pool2(PoolArgs a, float scale) {
    const int g8 = a.c / 8;
    const int64_t n = a.g_out.nvox * g8;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int c8 = int(i % g8);
        const int64_t vo = i / g8;
        const Vox o = vox_of(vo, a.g_out);
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float f[8];
            bf8_to_f(*at8(a.in, child(o, q, a.g_in), a.in_cs, a.in_co, c8), f);
#pragma unroll
            for (int k = 0; k < 8; ++k) s[k] += f[k];
        }
        uint4* dst = reinterpret_cast<uint4*>(a.out + vo * a.out_cs + a.out_co + 8 * c8);
        float r[8];
        if (a.accumulate) bf8_to_f(*dst, r);
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = (a.accumulate ? r[k] : 0.0f) + s[k] * scale;
        *dst = f_to_bf8(r);
    }
}

// Backward of pooling / forward of nearest upsampling: out[v] (fine grid) =
// scale * in[parent(v)]; accumulate adds to out.
__global__ void k_up2(PoolArgs a, float scale) {
    const int g8 = a.c / 8;
    const int64_t n = a.g_out.nvox * g8;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int c8 = int(i % g8);
        const int64_t vo = i / g8;
        const Vox o = vox_of(vo, a.g_out);
        const int64_t vi = ((int64_t(o.b) * a.g_in.Z + o.z / 2) * a.g_in.Y + o.y / 2) * a.g_in.X + o.x / 2;
        float f[8], r[8];
        bf8_to_f(*at8(a.in, vi, a.in_cs, a.in_co, c8), f);
        uint4* dst = reinterpret_cast<uint4*>(a.out + vo * a.out_cs + a.out_co + 8 * c8);
        if (a.accumulate) bf8_to_f(*dst, r);
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = (a.accumulate ? r[k] : 0.0f) + scale * f[k];
        *dst = f_to_bf8(r);
    }
}

// g[v][c] *= (y[v][c] > 0)   (ReLU backward; y is the layer's output)
__global__ void k_relu_bwd(bf16* gr, int g_cs, int g_co, const bf16* y, int y_cs, int y_co, int c, int64_t nvox) {
    const int g8 = c / 8;
    const int64_t n = nvox * g8;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int c8 = int(i % g8);
        const int64_t v = i / g8;
        float yv[8], gv[8];
        bf8_to_f(*at8(y, v, y_cs, y_co, c8), yv);
        uint4* dst = reinterpret_cast<uint4*>(gr + v * g_cs + g_co + 8 * c8);
        bf8_to_f(*dst, gv);
#pragma unroll
        for (int k = 0; k < 8; ++k) gv[k] = yv[k] > 0.0f ? gv[k] : 0.0f;
        *dst = f_to_bf8(gv);
    }
}

// Adam on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* w, const float* gr, float* m, float* v, bf16* wbf, int64_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2, float gscale) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float gg = gr[i] * gscale;
        const float mi = b1 * m[i] + (1.0f - b1) * gg;
        const float vi = b2 * v[i] + (1.0f - b2) * gg * gg;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        w[i] = wi;
        if (wbf) wbf[i] = __float2bfloat16_rn(wi);
    }
}

}  // namespace cnn
}  // namespace pn

// ---- launchers -----------------------------------------------------------------

namespace pn {
namespace cnn {

static int grid1d(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 16384) b = 16384;
    return int(b < 1 ? 1 : b);
}

cudaError_t conv3(const ConvArgs& a, cudaStream_t s) {
    if (a.use_tc && conv3_tc_serves(a)) return conv3_tc(a, a.err, s);
    // mma.sync: output-channel chunk of 32 (NT = 4) or 16 (NT = 2)
    const int64_t blocks = (a.g.nvox + 127) / 128;
    if (a.co % 32 == 0) k_conv3<4><<<dim3(unsigned(blocks), a.co / 32), 256, 0, s>>>(a);
    else k_conv3<2><<<dim3(unsigned(blocks), a.co / 16), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t conv3_wgrad(const WgradArgs& a, cudaStream_t s) {
    cudaError_t e;
    if (a.use_tc && conv3_wgrad_tc_serves(a)) {
        e = conv3_wgrad_tc(a, a.err, s);
    } else {
        const int chunks = int(std::min<int64_t>(64, std::max<int64_t>(1, a.g.nvox / 4096)));
        k_conv3_wgrad<<<dim3(27, chunks), 256, 0, s>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess || !a.db) return e;
    k_bias_grad<<<dim3(unsigned(std::min<int64_t>(1024, (a.g.nvox + 7) / 8)), (a.co + 31) / 32), 256, 0, s>>>(
        a.gy, a.gy_cs, a.gy_co, a.co, a.g.nvox, a.db);
    return cudaGetLastError();
}

cudaError_t flip_weights(const bf16* w, bf16* wt, int co, int ci, cudaStream_t s) {
    k_flip_weights<<<grid1d(int64_t(27) * co * ci), 256, 0, s>>>(w, wt, co, ci);
    return cudaGetLastError();
}

cudaError_t to_bf16(const float* src, bf16* dst, int64_t n, cudaStream_t s) {
    k_to_bf16<<<grid1d(n), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t pool2(const PoolArgs& a, cudaStream_t s) {
    k_pool2<<<grid1d(a.g_out.nvox * (a.c / 8)), 256, 0, s>>>(a, 0.125f);
    return cudaGetLastError();
}

cudaError_t up2(const PoolArgs& a, float scale, cudaStream_t s) {
    k_up2<<<grid1d(a.g_out.nvox * (a.c / 8)), 256, 0, s>>>(a, scale);
    return cudaGetLastError();
}

cudaError_t up2_bwd(const PoolArgs& a, cudaStream_t s) {
    if (a.accumulate) return cudaErrorInvalidValue;  // the backward of upsampling overwrites
    k_pool2<<<grid1d(a.g_out.nvox * (a.c / 8)), 256, 0, s>>>(a, 1.0f);
    return cudaGetLastError();
}

cudaError_t relu_bwd(bf16* gr, int g_cs, int g_co, const bf16* y, int y_cs, int y_co, int c, int64_t nvox,
                     cudaStream_t s) {
    k_relu_bwd<<<grid1d(nvox * (c / 8)), 256, 0, s>>>(gr, g_cs, g_co, y, y_cs, y_co, c, nvox);
    return cudaGetLastError();
}

cudaError_t adam(float* w, const float* gr, float* m, float* v, bf16* wbf, int64_t n, float lr, float b1, float b2,
                 float eps, int step, float gscale, cudaStream_t s) {
    const float c1 = 1.0f / (1.0f - std::pow(b1, float(step)));
    const float c2 = 1.0f / (1.0f - std::pow(b2, float(step)));
    k_adam<<<grid1d(n), 256, 0, s>>>(w, gr, m, v, wbf, n, lr, b1, b2, eps, c1, c2, gscale);
    return cudaGetLastError();
}

}  // namespace cnn
}  // namespace pn
