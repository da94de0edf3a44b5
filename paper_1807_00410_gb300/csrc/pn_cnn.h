// Internal declarations of the learned-preconditioner network kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

namespace pn {
namespace cnn {

using bf16 = __nv_bfloat16;

// B samples of Z x Y x X voxels, channels-last.
struct Grid {
    int B, Z, Y, X;
    int64_t nvox;  // B * Z * Y * X
};

inline Grid make_grid(int B, int Z, int Y, int X) { return Grid{B, Z, Y, X, int64_t(B) * Z * Y * X}; }

// 3x3x3 convolution: channel slices [in_co, in_co + ci) of an in_cs-wide
// input and [out_co, out_co + co) of an out_cs-wide output; ci, co multiples
// of 16; weights [27][co_total][ci] (co_total = co).
struct ConvArgs {
    const bf16* in;
    int in_cs, in_co, ci;
    const bf16* w;
    int co_total;
    const float* bias;  // or null
    bf16* out;
    int out_cs, out_co, co;
    int relu;
    Grid g;
    int use_tc = 1;               // 1: the tcgen05 kernel (pn_cnn_tc.cu); 0: the mma.sync kernel
    unsigned int* err = nullptr;  // error word of the tcgen05 kernel's bounded waits
};

// dW[tap][co][ci] += sum_v gy[v][o] x[v + t][c]; db[o] += sum_v gy[v][o] (if db).
struct WgradArgs {
    const bf16* x;
    int x_cs, x_co, ci;
    const bf16* gy;
    int gy_cs, gy_co, co;
    float* dw;
    float* db;
    Grid g;
    int use_tc = 1;               // 1: the tcgen05 kernel (pn_cnn_tc.cu); 0: the mma.sync kernel
    unsigned int* err = nullptr;  // error word of the tcgen05 kernel's bounded waits
};

// Resampling between a fine grid and the grid of half its size.
struct PoolArgs {
    const bf16* in;
    int in_cs, in_co;
    bf16* out;
    int out_cs, out_co;
    int c;
    Grid g_in, g_out;
    int accumulate;
};

cudaError_t conv3(const ConvArgs& a, cudaStream_t s);
// the same convolution on the tcgen05 tensor cores (pn_cnn_tc.cu); err: the
// network's error word (set where a bounded wait ran out)
bool conv3_tc_serves(const ConvArgs& a);
cudaError_t conv3_tc(const ConvArgs& a, unsigned int* err, cudaStream_t s);
cudaError_t conv3_wgrad(const WgradArgs& a, cudaStream_t s);
bool conv3_wgrad_tc_serves(const WgradArgs& a);
cudaError_t conv3_wgrad_tc(const WgradArgs& a, unsigned int* err, cudaStream_t s);
cudaError_t flip_weights(const bf16* w, bf16* wt, int co, int ci, cudaStream_t s);
cudaError_t to_bf16(const float* src, bf16* dst, int64_t n, cudaStream_t s);
cudaError_t pool2(const PoolArgs& a, cudaStream_t s);               // fine -> coarse mean
cudaError_t up2(const PoolArgs& a, float scale, cudaStream_t s);    // coarse -> fine copy * scale
cudaError_t up2_bwd(const PoolArgs& a, cudaStream_t s);             // fine -> coarse sum
cudaError_t relu_bwd(bf16* gr, int g_cs, int g_co, const bf16* y, int y_cs, int y_co, int c, int64_t nvox,
                     cudaStream_t s);
cudaError_t adam(float* w, const float* gr, float* m, float* v, bf16* wbf, int64_t n, float lr, float b1, float b2,
                 float eps, int step, float gscale, cudaStream_t s);

}  // namespace cnn
}  // namespace pn
