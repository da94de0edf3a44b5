// The learned preconditioner's network: a 3D convolutional encoder-decoder
// (four resolution levels, widths w0..w3, 3x3x3 convolutions with ReLU,
// 2x average pooling down, nearest 2x upsampling up, skip connections by
// channel concatenation, a linear 3x3x3 output layer), with training
// (backward passes and Adam) on the GPU.  The paper has no network; this is
// the learned extension of its solver.
//
//   e0a,e0b (w0) -> pool -> e1a,e1b (w1) -> pool -> e2a,e2b (w2) -> pool ->
//   e3a,e3b (w3) -> up ++ s2 -> d2 (w2) -> up ++ s1 -> d1 (w1) -> up ++ s0 ->
//   d0 (w0) -> out (c_out, linear)
//
// Parameters live as FP32 master copies (Adam) with BF16 copies for the
// tensor-core kernels.  Host-visible parameter order (pn_cnn_get_params):
// per layer, W[o][c][tap] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)) then b[o],
// unpadded channel counts; the device layout pads channels to multiples of 16
// and stores W as [tap][o][c].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "pn_cnn.h"
#include "pn_gb300.h"

using pn::cnn::bf16;

namespace {

int pad16(int c) { return (c + 15) / 16 * 16; }

struct Layer {
    const char* name;
    int ci, co;      // real channel counts
    int cip, cop;    // padded
    size_t w_off;    // offset (floats) of W in the device parameter array ([tap][cop][cip])
    size_t b_off;    // offset of b ([cop])
};

struct Buf {
    bf16* p = nullptr;
    int cs = 0;      // channels (stride)
    int level = 0;
};

}  // namespace

struct pn_cnn {
    int c_in = 0, c_out = 0, cinp = 0, coutp = 0;
    int w[4] = {16, 32, 48, 64};
    int wp[4] = {16, 32, 48, 64};
    std::vector<Layer> layers;
    size_t nparams_dev = 0;   // padded device parameter count
    int64_t nparams_host = 0; // unpadded host parameter count
    float* d_w32 = nullptr;
    float* d_g = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    bf16* d_wbf = nullptr;    // BF16 copy, same offsets
    bf16* d_wflip = nullptr;  // flipped weights for the input gradients, same offsets
    int step = 0;
    // activations for the current (B, Z, Y, X)
    int B = 0, Z = 0, Y = 0, X = 0;
    void* act_mem = nullptr;
    size_t act_bytes = 0;
    Buf xin, a0, cat0, d0, yout, p0, a1, cat1, d1, p1, a2, cat2, d2, p2, a3, bt;
    Buf gy, g_d0, g_cat0, g_d1, g_cat1, g_d2, g_cat2, g_bt, g_a3, g_p2, g_a2, g_p1, g_a1, g_p0, g_a0;
    float* d_loss = nullptr;  // per-sample sums (2 * B floats) and the total, then the error word
    unsigned int* d_err = nullptr;  // set by a tcgen05 convolution whose bounded wait ran out (in d_loss's tail)
    int conv_kernel = PN_CNN_CONV_TCGEN05;
    std::string err;
};

namespace {

const Layer* find(const pn_cnn* n, const char* name) {
    for (const Layer& L : n->layers)
        if (std::strcmp(L.name, name) == 0) return &L;
    return nullptr;
}

pn::cnn::Grid grid_at(const pn_cnn* n, int level) {
    return pn::cnn::make_grid(n->B, n->Z >> level, n->Y >> level, n->X >> level);
}

int fail(pn_cnn* n, int code, const std::string& msg) {
    if (n) n->err = msg;
    return code;
}

#define CK(expr)                                                   \
    do {                                                           \
        cudaError_t e_ = (expr);                                   \
        if (e_ != cudaSuccess) return fail(n, PN_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int conv(pn_cnn* n, const char* name, const Buf& in, int in_co, const Buf& out, int out_co, bool relu,
         cudaStream_t s) {
    const Layer* L = find(n, name);
    pn::cnn::ConvArgs a;
    a.in = in.p;
    a.in_cs = in.cs;
    a.in_co = in_co;
    a.ci = L->cip;
    a.w = n->d_wbf + L->w_off;
    a.co_total = L->cop;
    a.bias = n->d_w32 + L->b_off;
    a.out = out.p;
    a.out_cs = out.cs;
    a.out_co = out_co;
    a.co = L->cop;
    a.relu = relu ? 1 : 0;
    a.g = grid_at(n, in.level);
    a.use_tc = n->conv_kernel == PN_CNN_CONV_TCGEN05 ? 1 : 0;
    a.err = n->d_err;
    CK(pn::cnn::conv3(a, s));
    return PN_OK;
}

// grad wrt the layer's input (into gin slice) and parameter gradients, given
// the gradient wrt its pre-activation output (gout slice).
int conv_back(pn_cnn* n, const char* name, const Buf& in, int in_co, const Buf& gout, int gout_co, const Buf* gin,
              int gin_co, cudaStream_t s) {
    const Layer* L = find(n, name);
    pn::cnn::WgradArgs w;
    w.x = in.p;
    w.x_cs = in.cs;
    w.x_co = in_co;
    w.ci = L->cip;
    w.gy = gout.p;
    w.gy_cs = gout.cs;
    w.gy_co = gout_co;
    w.co = L->cop;
    w.dw = n->d_g + L->w_off;
    w.db = n->d_g + L->b_off;
    w.g = grid_at(n, in.level);
    w.use_tc = n->conv_kernel == PN_CNN_CONV_TCGEN05 ? 1 : 0;
    w.err = n->d_err;
    CK(pn::cnn::conv3_wgrad(w, s));
    if (gin) {
        pn::cnn::ConvArgs a;
        a.in = gout.p;
        a.in_cs = gout.cs;
        a.in_co = gout_co;
        a.ci = L->cop;
        a.w = n->d_wflip + L->w_off;
        a.co_total = L->cip;
        a.bias = nullptr;
        a.out = gin->p;
        a.out_cs = gin->cs;
        a.out_co = gin_co;
        a.co = L->cip;
        a.relu = 0;
        a.g = grid_at(n, in.level);
        a.use_tc = n->conv_kernel == PN_CNN_CONV_TCGEN05 ? 1 : 0;
        a.err = n->d_err;
        CK(pn::cnn::conv3(a, s));
    }
    return PN_OK;
}

int relu_b(pn_cnn* n, const Buf& g, int g_co, const Buf& y, int y_co, int c, cudaStream_t s) {
    CK(pn::cnn::relu_bwd(g.p, g.cs, g_co, y.p, y.cs, y_co, c, grid_at(n, y.level).nvox, s));
    return PN_OK;
}

pn::cnn::PoolArgs pargs(const Buf& in, int in_co, const Buf& out, int out_co, int c, pn::cnn::Grid gi,
                        pn::cnn::Grid go, int acc) {
    pn::cnn::PoolArgs a;
    a.in = in.p;
    a.in_cs = in.cs;
    a.in_co = in_co;
    a.out = out.p;
    a.out_cs = out.cs;
    a.out_co = out_co;
    a.c = c;
    a.g_in = gi;
    a.g_out = go;
    a.accumulate = acc;
    return a;
}

int ensure_acts(pn_cnn* n, int B, int Z, int Y, int X) {
    if (n->B == B && n->Z == Z && n->Y == Y && n->X == X && n->act_mem) return PN_OK;
    if (n->act_mem) cudaFree(n->act_mem);
    n->act_mem = nullptr;
    n->B = B;
    n->Z = Z;
    n->Y = Y;
    n->X = X;
    const int* c = n->wp;
    struct Spec {
        Buf* b;
        int ch;
        int level;
    };
    std::vector<Spec> specs = {
        {&n->xin, n->cinp, 0},          {&n->a0, c[0], 0},          {&n->cat0, c[1] + c[0], 0},
        {&n->d0, c[0], 0},              {&n->yout, n->coutp, 0},    {&n->p0, c[0], 1},
        {&n->a1, c[1], 1},              {&n->cat1, c[2] + c[1], 1}, {&n->d1, c[1], 1},
        {&n->p1, c[1], 2},              {&n->a2, c[2], 2},          {&n->cat2, c[3] + c[2], 2},
        {&n->d2, c[2], 2},              {&n->p2, c[2], 3},          {&n->a3, c[3], 3},
        {&n->bt, c[3], 3},              {&n->gy, n->coutp, 0},      {&n->g_d0, c[0], 0},
        {&n->g_cat0, c[1] + c[0], 0},   {&n->g_d1, c[1], 1},        {&n->g_cat1, c[2] + c[1], 1},
        {&n->g_d2, c[2], 2},            {&n->g_cat2, c[3] + c[2], 2}, {&n->g_bt, c[3], 3},
        {&n->g_a3, c[3], 3},            {&n->g_p2, c[2], 3},        {&n->g_a2, c[2], 2},
        {&n->g_p1, c[1], 2},            {&n->g_a1, c[1], 1},        {&n->g_p0, c[0], 1},
        {&n->g_a0, c[0], 0}};
    size_t total = 0;
    for (const Spec& sp : specs) total += size_t(grid_at(n, sp.level).nvox) * sp.ch * sizeof(bf16) + 256;
    if (cudaMalloc(&n->act_mem, total) != cudaSuccess) {
        cudaGetLastError();
        n->B = 0;
        return fail(n, PN_ERR_ALLOC, "pn_cnn: cannot allocate activations");
    }
    n->act_bytes = total;
    char* p = static_cast<char*>(n->act_mem);
    for (const Spec& sp : specs) {
        sp.b->p = reinterpret_cast<bf16*>(p);
        sp.b->cs = sp.ch;
        sp.b->level = sp.level;
        p += (size_t(grid_at(n, sp.level).nvox) * sp.ch * sizeof(bf16) + 255) / 256 * 256;
    }
    return PN_OK;
}

// FP32 [v][c] -> BF16 [v][cp] (zero padded; cp a multiple of 8): one thread
// per (voxel, group of 8 padded channels), one 16-byte store.  Also the
// gradient of the output (same layouts).
__global__ void k_pack(const float* in, int c, bf16* out, int cp, int64_t nvox) {
    const int g8 = cp / 8;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nvox * g8; i += int64_t(gridDim.x) * blockDim.x) {
        const int k0 = int(i % g8) * 8;
        const int64_t v = i / g8;
        const float* src = in + v * c;
        uint4 u;
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + 2 * q;
            h[q] = __floats2bfloat162_rn(k < c ? src[k] : 0.0f, k + 1 < c ? src[k + 1] : 0.0f);
        }
        *reinterpret_cast<uint4*>(out + v * cp + k0) = u;
    }
}

// BF16 [v][cp] -> FP32 [v][c]: one thread per (voxel, group of 8 channels),
// one 16-byte load.
__global__ void k_unpack(const bf16* in, int cp, float* out, int c, int64_t nvox) {
    const int g8 = (c + 7) / 8;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nvox * g8; i += int64_t(gridDim.x) * blockDim.x) {
        const int k0 = int(i % g8) * 8;
        const int64_t v = i / g8;
        const uint4 u = *reinterpret_cast<const uint4*>(in + v * cp + k0);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
        float* dst = out + v * c;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(h[q]);
            const int k = k0 + 2 * q;
            if (k < c) dst[k] = f.x;
            if (k + 1 < c) dst[k + 1] = f.y;
        }
    }
}

// per-sample sums: acc[2b] += |y - t|^2, acc[2b+1] += |t|^2
__global__ void k_loss_sums(const bf16* y, int cp, const float* t, int c, int64_t vox_per_sample, int B, float* acc) {
    const int b = blockIdx.y;
    float e = 0.0f, q = 0.0f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < vox_per_sample * c;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t v = b * vox_per_sample + i / c;
        const int k = int(i % c);
        const float tv = t[v * c + k];
        const float d = __bfloat162float(y[v * cp + k]) - tv;
        e += d * d;
        q += tv * tv;
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        q += __shfl_down_sync(0xffffffffu, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc + 2 * b, e);
        atomicAdd(acc + 2 * b + 1, q);
    }
}

// loss = (1/B) sum_b |y_b - t_b|^2 / |t_b|^2 ; gy = dloss/dy
__global__ void k_loss_grad(const bf16* y, int cp, const float* t, int c, int64_t vox_per_sample, int B,
                            const float* acc, bf16* gy) {
    const int64_t n = int64_t(B) * vox_per_sample * cp;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int k = int(i % cp);
        const int64_t v = i / cp;
        const int b = int(v / vox_per_sample);
        float gval = 0.0f;
        if (k < c) {
            const float tn = fmaxf(acc[2 * b + 1], 1e-30f);
            gval = 2.0f * (__bfloat162float(y[i]) - t[v * c + k]) / (float(B) * tn);
        }
        gy[i] = __float2bfloat16_rn(gval);
    }
}

int grid1(int64_t n) { return int(std::min<int64_t>(16384, std::max<int64_t>(1, (n + 255) / 256))); }

int forward(pn_cnn* n, cudaStream_t s) {
    using pn::cnn::Grid;
    const int* c = n->wp;
    const Grid g0 = grid_at(n, 0), g1 = grid_at(n, 1), g2 = grid_at(n, 2), g3 = grid_at(n, 3);
    int rc;
#define RC(x)                     \
    do {                          \
        rc = (x);                 \
        if (rc != PN_OK) return rc; \
    } while (0)
    RC(conv(n, "e0a", n->xin, 0, n->a0, 0, true, s));
    RC(conv(n, "e0b", n->a0, 0, n->cat0, c[1], true, s));  // s0 into cat0[c1:]
    CK(pn::cnn::pool2(pargs(n->cat0, c[1], n->p0, 0, c[0], g0, g1, 0), s));
    RC(conv(n, "e1a", n->p0, 0, n->a1, 0, true, s));
    RC(conv(n, "e1b", n->a1, 0, n->cat1, c[2], true, s));  // s1
    CK(pn::cnn::pool2(pargs(n->cat1, c[2], n->p1, 0, c[1], g1, g2, 0), s));
    RC(conv(n, "e2a", n->p1, 0, n->a2, 0, true, s));
    RC(conv(n, "e2b", n->a2, 0, n->cat2, c[3], true, s));  // s2
    CK(pn::cnn::pool2(pargs(n->cat2, c[3], n->p2, 0, c[2], g2, g3, 0), s));
    RC(conv(n, "e3a", n->p2, 0, n->a3, 0, true, s));
    RC(conv(n, "e3b", n->a3, 0, n->bt, 0, true, s));
    CK(pn::cnn::up2(pargs(n->bt, 0, n->cat2, 0, c[3], g3, g2, 0), 1.0f, s));
    RC(conv(n, "d2", n->cat2, 0, n->d2, 0, true, s));
    CK(pn::cnn::up2(pargs(n->d2, 0, n->cat1, 0, c[2], g2, g1, 0), 1.0f, s));
    RC(conv(n, "d1", n->cat1, 0, n->d1, 0, true, s));
    CK(pn::cnn::up2(pargs(n->d1, 0, n->cat0, 0, c[1], g1, g0, 0), 1.0f, s));
    RC(conv(n, "d0", n->cat0, 0, n->d0, 0, true, s));
    RC(conv(n, "out", n->d0, 0, n->yout, 0, false, s));
    return PN_OK;
}

// parameter gradients from n->gy (gradient wrt the output)
int backward(pn_cnn* n, cudaStream_t s) {
    using pn::cnn::Grid;
    const int* c = n->wp;
    const Grid g0 = grid_at(n, 0), g1 = grid_at(n, 1), g2 = grid_at(n, 2), g3 = grid_at(n, 3);
    int rc;
    CK(cudaMemsetAsync(n->d_g, 0, n->nparams_dev * sizeof(float), s));
    RC(conv_back(n, "out", n->d0, 0, n->gy, 0, &n->g_d0, 0, s));
    RC(relu_b(n, n->g_d0, 0, n->d0, 0, c[0], s));
    RC(conv_back(n, "d0", n->cat0, 0, n->g_d0, 0, &n->g_cat0, 0, s));
    CK(pn::cnn::up2_bwd(pargs(n->g_cat0, 0, n->g_d1, 0, c[1], g0, g1, 0), s));
    RC(relu_b(n, n->g_d1, 0, n->d1, 0, c[1], s));
    RC(conv_back(n, "d1", n->cat1, 0, n->g_d1, 0, &n->g_cat1, 0, s));
    CK(pn::cnn::up2_bwd(pargs(n->g_cat1, 0, n->g_d2, 0, c[2], g1, g2, 0), s));
    RC(relu_b(n, n->g_d2, 0, n->d2, 0, c[2], s));
    RC(conv_back(n, "d2", n->cat2, 0, n->g_d2, 0, &n->g_cat2, 0, s));
    CK(pn::cnn::up2_bwd(pargs(n->g_cat2, 0, n->g_bt, 0, c[3], g2, g3, 0), s));
    RC(relu_b(n, n->g_bt, 0, n->bt, 0, c[3], s));
    RC(conv_back(n, "e3b", n->a3, 0, n->g_bt, 0, &n->g_a3, 0, s));
    RC(relu_b(n, n->g_a3, 0, n->a3, 0, c[3], s));
    RC(conv_back(n, "e3a", n->p2, 0, n->g_a3, 0, &n->g_p2, 0, s));
    // s2 gradient: skip part (g_cat2[c3:]) + pooling path
    CK(pn::cnn::up2(pargs(n->g_p2, 0, n->g_cat2, c[3], c[2], g3, g2, 1), 0.125f, s));
    RC(relu_b(n, n->g_cat2, c[3], n->cat2, c[3], c[2], s));
    RC(conv_back(n, "e2b", n->a2, 0, n->g_cat2, c[3], &n->g_a2, 0, s));
    RC(relu_b(n, n->g_a2, 0, n->a2, 0, c[2], s));
    RC(conv_back(n, "e2a", n->p1, 0, n->g_a2, 0, &n->g_p1, 0, s));
    CK(pn::cnn::up2(pargs(n->g_p1, 0, n->g_cat1, c[2], c[1], g2, g1, 1), 0.125f, s));
    RC(relu_b(n, n->g_cat1, c[2], n->cat1, c[2], c[1], s));
    RC(conv_back(n, "e1b", n->a1, 0, n->g_cat1, c[2], &n->g_a1, 0, s));
    RC(relu_b(n, n->g_a1, 0, n->a1, 0, c[1], s));
    RC(conv_back(n, "e1a", n->p0, 0, n->g_a1, 0, &n->g_p0, 0, s));
    CK(pn::cnn::up2(pargs(n->g_p0, 0, n->g_cat0, c[1], c[0], g1, g0, 1), 0.125f, s));
    RC(relu_b(n, n->g_cat0, c[1], n->cat0, c[1], c[0], s));
    RC(conv_back(n, "e0b", n->a0, 0, n->g_cat0, c[1], &n->g_a0, 0, s));
    RC(relu_b(n, n->g_a0, 0, n->a0, 0, c[0], s));
    RC(conv_back(n, "e0a", n->xin, 0, n->g_a0, 0, nullptr, 0, s));
    return PN_OK;
#undef RC
}

int refresh_weights(pn_cnn* n, cudaStream_t s) {
    CK(pn::cnn::to_bf16(n->d_w32, n->d_wbf, int64_t(n->nparams_dev), s));
    for (const Layer& L : n->layers) CK(pn::cnn::flip_weights(n->d_wbf + L.w_off, n->d_wflip + L.w_off, L.cop, L.cip, s));
    return PN_OK;
}

int check_dims(pn_cnn* n, int B, int Z, int Y, int X) {
    if (B < 1 || Z < 8 || Y < 8 || X < 8 || Z % 8 || Y % 8 || X % 8)
        return fail(n, PN_ERR_ARG, "pn_cnn: grid sizes must be multiples of 8 (three 2x poolings)");
    return PN_OK;
}

}  // namespace

extern "C" {

int pn_cnn_create(pn_cnn** out, int c_in, int c_out, const int widths[4]) {
    if (!out || c_in < 1 || c_out < 1 || c_in > 256 || c_out > 256) return PN_ERR_ARG;
    *out = nullptr;
    pn_cnn* n = new (std::nothrow) pn_cnn();
    if (!n) return PN_ERR_ALLOC;
    n->c_in = c_in;
    n->c_out = c_out;
    n->cinp = pad16(c_in);
    n->coutp = pad16(c_out);
    for (int i = 0; i < 4; ++i) {
        if (widths && (widths[i] < 1 || widths[i] > 256)) {
            delete n;
            return PN_ERR_ARG;
        }
        n->w[i] = widths ? widths[i] : n->w[i];
        n->wp[i] = pad16(n->w[i]);
    }
    const int* c = n->w;
    const int* cp = n->wp;
    struct Def {
        const char* name;
        int ci, co, cip, cop;
    };
    const Def defs[] = {{"e0a", c_in, c[0], n->cinp, cp[0]},
                        {"e0b", c[0], c[0], cp[0], cp[0]},
                        {"e1a", c[0], c[1], cp[0], cp[1]},
                        {"e1b", c[1], c[1], cp[1], cp[1]},
                        {"e2a", c[1], c[2], cp[1], cp[2]},
                        {"e2b", c[2], c[2], cp[2], cp[2]},
                        {"e3a", c[2], c[3], cp[2], cp[3]},
                        {"e3b", c[3], c[3], cp[3], cp[3]},
                        {"d2", c[3] + c[2], c[2], cp[3] + cp[2], cp[2]},
                        {"d1", c[2] + c[1], c[1], cp[2] + cp[1], cp[1]},
                        {"d0", c[1] + c[0], c[0], cp[1] + cp[0], cp[0]},
                        {"out", c[0], c_out, cp[0], n->coutp}};
    size_t off = 0;
    int64_t hostn = 0;
    for (const Def& d : defs) {
        Layer L{d.name, d.ci, d.co, d.cip, d.cop, 0, 0};
        L.w_off = off;
        off += size_t(27) * d.cop * d.cip;
        L.b_off = off;
        off += size_t(d.cop);
        off = (off + 63) / 64 * 64;
        n->layers.push_back(L);
        hostn += int64_t(d.co) * d.ci * 27 + d.co;
        if ((d.cop / 16) * (d.cip / 8) > 64) {  // weight-gradient kernel: at most 8 tile pairs per warp
            delete n;
            return PN_ERR_UNSUPPORTED;
        }
    }
    n->nparams_dev = off;
    n->nparams_host = hostn;
    const size_t bytes = off * sizeof(float);
    if (cudaMalloc(&n->d_w32, bytes) != cudaSuccess || cudaMalloc(&n->d_g, bytes) != cudaSuccess ||
        cudaMalloc(&n->d_m, bytes) != cudaSuccess || cudaMalloc(&n->d_v, bytes) != cudaSuccess ||
        cudaMalloc(&n->d_wbf, off * sizeof(bf16)) != cudaSuccess ||
        cudaMalloc(&n->d_wflip, off * sizeof(bf16)) != cudaSuccess ||
        cudaMalloc(&n->d_loss, (2 * 4096 + 64) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        pn_cnn_destroy(n);
        return PN_ERR_ALLOC;
    }
    n->d_err = reinterpret_cast<unsigned int*>(n->d_loss + 2 * 4096 + 32);
    cudaMemset(n->d_err, 0, sizeof(unsigned int));
    cudaMemset(n->d_w32, 0, bytes);
    cudaMemset(n->d_g, 0, bytes);
    cudaMemset(n->d_m, 0, bytes);
    cudaMemset(n->d_v, 0, bytes);
    *out = n;
    return PN_OK;
}

int pn_cnn_destroy(pn_cnn* n) {
    if (!n) return PN_OK;
    void* ptrs[] = {n->d_w32, n->d_g, n->d_m, n->d_v, n->d_wbf, n->d_wflip, n->act_mem, n->d_loss};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete n;
    return PN_OK;
}

const char* pn_cnn_last_error(const pn_cnn* n) { return n ? n->err.c_str() : ""; }

int64_t pn_cnn_num_params(const pn_cnn* n) { return n ? n->nparams_host : 0; }

// host layout: per layer W[o][c][tap] (real channels) then b[o]
static int copy_params(pn_cnn* n, float* host, int64_t count, const float* dev, bool to_device) {
    if (!host || count != n->nparams_host) return fail(n, PN_ERR_ARG, "pn_cnn: parameter count mismatch");
    std::vector<float> d(n->nparams_dev, 0.0f);
    if (!to_device) CK(cudaMemcpy(d.data(), dev, d.size() * sizeof(float), cudaMemcpyDeviceToHost));
    int64_t h = 0;
    for (const Layer& L : n->layers) {
        for (int o = 0; o < L.co; ++o)
            for (int c = 0; c < L.ci; ++c) {
                // map real input channel c to its padded position (concatenated inputs
                // keep each part's padding)
                int cpos = c;
                if (std::strcmp(L.name, "d2") == 0) cpos = c < n->w[3] ? c : n->wp[3] + (c - n->w[3]);
                if (std::strcmp(L.name, "d1") == 0) cpos = c < n->w[2] ? c : n->wp[2] + (c - n->w[2]);
                if (std::strcmp(L.name, "d0") == 0) cpos = c < n->w[1] ? c : n->wp[1] + (c - n->w[1]);
                for (int t = 0; t < 27; ++t) {
                    const size_t di = L.w_off + (size_t(t) * L.cop + o) * L.cip + cpos;
                    if (to_device) d[di] = host[h];
                    else host[h] = d[di];
                    ++h;
                }
            }
        for (int o = 0; o < L.co; ++o) {
            if (to_device) d[L.b_off + o] = host[h];
            else host[h] = d[L.b_off + o];
            ++h;
        }
    }
    if (to_device) CK(cudaMemcpy(const_cast<float*>(dev), d.data(), d.size() * sizeof(float), cudaMemcpyHostToDevice));
    return PN_OK;
}

int pn_cnn_set_params(pn_cnn* n, const float* host, int64_t count) {
    if (!n) return PN_ERR_ARG;
    int rc = copy_params(n, const_cast<float*>(host), count, n->d_w32, true);
    if (rc != PN_OK) return rc;
    CK(cudaMemset(n->d_m, 0, n->nparams_dev * sizeof(float)));
    CK(cudaMemset(n->d_v, 0, n->nparams_dev * sizeof(float)));
    n->step = 0;
    rc = refresh_weights(n, nullptr);
    if (rc != PN_OK) return rc;
    CK(cudaDeviceSynchronize());
    return PN_OK;
}

int pn_cnn_get_params(pn_cnn* n, float* host, int64_t count) {
    if (!n) return PN_ERR_ARG;
    return copy_params(n, host, count, n->d_w32, false);
}

int pn_cnn_get_grads(pn_cnn* n, float* host, int64_t count) {
    if (!n) return PN_ERR_ARG;
    return copy_params(n, host, count, n->d_g, false);
}

int pn_cnn_set_conv_kernel(pn_cnn* n, int kernel) {
    if (!n) return PN_ERR_ARG;
    if (kernel != PN_CNN_CONV_TCGEN05 && kernel != PN_CNN_CONV_MMA_SYNC)
        return fail(n, PN_ERR_ARG, "pn_cnn_set_conv_kernel: bad kernel");
    n->conv_kernel = kernel;
    return PN_OK;
}

int pn_cnn_take_error(pn_cnn* n) {
    if (!n) return PN_ERR_ARG;
    unsigned int e = 0;
    CK(cudaMemcpy(&e, n->d_err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e == 0) return PN_OK;
    CK(cudaMemset(n->d_err, 0, sizeof(e)));
    return fail(n, PN_ERR_TIMEOUT, "pn_cnn: a bounded wait of the tcgen05 convolution ran out");
}

int pn_cnn_forward(pn_cnn* n, const float* in, float* out, int B, int Z, int Y, int X, void* stream) {
    if (!n || !in) return PN_ERR_ARG;
    int rc = check_dims(n, B, Z, Y, X);
    if (rc != PN_OK) return rc;
    rc = ensure_acts(n, B, Z, Y, X);
    if (rc != PN_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nv = int64_t(B) * Z * Y * X;
    k_pack<<<grid1(nv * (n->cinp / 8)), 256, 0, s>>>(in, n->c_in, n->xin.p, n->cinp, nv);
    CK(cudaGetLastError());
    rc = forward(n, s);
    if (rc != PN_OK) return rc;
    if (out) {
        k_unpack<<<grid1(nv * ((n->c_out + 7) / 8)), 256, 0, s>>>(n->yout.p, n->coutp, out, n->c_out, nv);
        CK(cudaGetLastError());
    }
    return PN_OK;
}

int pn_cnn_backward(pn_cnn* n, const float* grad_out, void* stream) {
    if (!n || !grad_out || !n->act_mem) return PN_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nv = int64_t(n->B) * n->Z * n->Y * n->X;
    k_pack<<<grid1(nv * (n->coutp / 8)), 256, 0, s>>>(grad_out, n->c_out, n->gy.p, n->coutp, nv);
    CK(cudaGetLastError());
    return backward(n, s);
}

int pn_cnn_adam_step(pn_cnn* n, double lr, void* stream) {
    if (!n) return PN_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    n->step += 1;
    CK(pn::cnn::adam(n->d_w32, n->d_g, n->d_m, n->d_v, nullptr, int64_t(n->nparams_dev), float(lr), 0.9f, 0.999f,
                     1e-8f, n->step, 1.0f, s));
    return refresh_weights(n, s);
}

int pn_cnn_train_step(pn_cnn* n, const float* in, const float* target, int B, int Z, int Y, int X, double lr,
                      double* loss_out, void* stream) {
    if (!n || !in || !target || B > 4096) return PN_ERR_ARG;
    int rc = pn_cnn_forward(n, in, nullptr, B, Z, Y, X, stream);
    if (rc != PN_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t vps = int64_t(Z) * Y * X;
    CK(cudaMemsetAsync(n->d_loss, 0, 2 * B * sizeof(float), s));
    k_loss_sums<<<dim3(unsigned(std::min<int64_t>(256, (vps * n->c_out + 255) / 256)), B), 256, 0, s>>>(
        n->yout.p, n->coutp, target, n->c_out, vps, B, n->d_loss);
    CK(cudaGetLastError());
    k_loss_grad<<<grid1(B * vps * n->coutp), 256, 0, s>>>(n->yout.p, n->coutp, target, n->c_out, vps, B, n->d_loss,
                                                          n->gy.p);
    CK(cudaGetLastError());
    rc = backward(n, s);
    if (rc != PN_OK) return rc;
    rc = pn_cnn_adam_step(n, lr, stream);
    if (rc != PN_OK) return rc;
    if (loss_out) {
        std::vector<float> acc(2 * B);
        CK(cudaMemcpyAsync(acc.data(), n->d_loss, 2 * B * sizeof(float), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        rc = pn_cnn_take_error(n);
        if (rc != PN_OK) return rc;
        double l = 0.0;
        for (int b = 0; b < B; ++b) l += acc[2 * b] / std::max(acc[2 * b + 1], 1e-30f);
        *loss_out = l / B;
    }
    return PN_OK;
}

}  // extern "C"
