// Operator and vector kernels of the GB300 P_N library.
//
// k_op_naive is the plain, one-thread-per-output form of the staggered P_N
// operator (appendix "Final equation"; central differences between
// staggered grids, section "Precomputation"; Dirichlet dropping, section
// "Runtime").  It serves FP64 and every order N through the per-handle term
// table, and is the correctness baseline for the tiled FP32 kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "pn_internal.h"
#include "pn_op.cuh"

namespace pn {

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = 0.0;
    if (wid == 0) {
        for (int i = lane; i < nw; i += 32) v += red[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;  // valid in thread 0
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_op_naive(OpArgs<T> a) {
    const int p = blockIdx.y;
    const Plane P = a.planes[p];
    const int R = a.R;
    const int ny = R + 1;
    const int64_t box = a.pitch_y * int64_t(a.nzb);
    const int64_t pbase = int64_t(p) * a.plane_stride;
    double racc = 0.0;
    T rrun = T(0);  // residual squares summed in T per thread, flushed to FP64 every 16
    int rcnt = 0;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < a.plane_stride;
         s += int64_t(gridDim.x) * blockDim.x) {
        const int x = int(s % a.pitch_x);
        const int64_t t = s / a.pitch_x;
        const int y = int(t % ny);
        const int z = int(t / ny);
        const int ext = a.periodic ? 0 : 1;  // periodic: R slots per axis for every class
        const bool active = s < box && x < R + ext * P.px && y < R + ext * P.py && z < R + ext * P.pz;
        T out = T(0);
        if (active) {
            out = op_point<T, MODE>(a, p, P, x, y, z, s);
            if (MODE == OP_RESIDUAL) {
                rrun += out * out;
                if (++rcnt == 16) {
                    racc += double(rrun);
                    rrun = T(0);
                    rcnt = 0;
                }
            }
        }
        a.y[pbase + s] = out;
    }
    if (MODE == OP_RESIDUAL && a.partials != nullptr) {
        const double bs = block_sum(racc + double(rrun));
        if (threadIdx.x == 0) a.partials[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = bs;
    }
}

// The slots a tiled launch does not cover: columns x >= x_lo of every plane
// box, and each plane's tail beyond its box.  Thread t of plane p handles
// slot t of the list [(z, y, x) for x in [x_lo, pitch_x)] + tail.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_op_slab(OpArgs<T> a, int x_lo) {
    const int p = blockIdx.y;
    const Plane P = a.planes[p];
    const int R = a.R;
    const int w = int(a.pitch_x) - x_lo;
    const int64_t box = a.pitch_y * int64_t(R + 1);
    const int64_t ncol = int64_t(w) * (R + 1) * (R + 1);
    const int64_t ntail = a.plane_stride - box;
    const int64_t pbase = int64_t(p) * a.plane_stride;
    double racc = 0.0;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < ncol + ntail;
         t += int64_t(gridDim.x) * blockDim.x) {
        if (t >= ncol) {
            a.y[pbase + box + (t - ncol)] = T(0);
            continue;
        }
        const int x = x_lo + int(t % w);
        const int64_t u = t / w;
        const int y = int(u % (R + 1));
        const int z = int(u / (R + 1));
        const int64_t s = int64_t(z) * a.pitch_y + int64_t(y) * a.pitch_x + x;
        T out = T(0);
        if (!a.periodic && x < R + P.px && y < R + P.py && z < R + P.pz) {  // the slab path is never periodic
            out = op_point<T, MODE>(a, p, P, x, y, z, s);
            if (MODE == OP_RESIDUAL) racc += double(out) * double(out);
        }
        a.y[pbase + s] = out;
    }
    if (MODE == OP_RESIDUAL && a.partials != nullptr) {
        const double bs = block_sum(racc);
        if (threadIdx.x == 0) a.partials[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = bs;
    }
}

// ---- FP64 operator of 3D vacuum-boundary handles ---------------------------------
//
// The refinement residual of the mixed-precision solvers runs in FP64, which
// GB300 executes at a small fraction of its FP32 rate: the kernel keeps the
// FP64 work per output to the operator's own arithmetic.  The mean of sigma_t
// and of sigma_s over the voxel centres adjacent to each slot (section
// "Precomputation": parameters interpolated to the staggered locations)
// depends only on the slot's parity class, so it is computed once per handle
// (cmean_build: 8 classes x 2 fields, the slot layout of a plane) and read as
// two values per output.  Work items are (plane, z slice, 8-row band); block b
// of G takes items b, b + G, ... (the residual's per-block FP64 partials are
// then summed in a fixed order); a plane's term list goes to shared memory
// once per item.

// the class means: cm[(2 c + f) * plane_stride + slot], f = 0 (sigma_t), 1 (sigma_s)
__global__ void __launch_bounds__(256) k_cmean_build(double* cm, const double* st, const double* ss, int R,
                                                     int64_t pitch_x, int64_t pitch_y, int64_t plane_stride) {
    const int c = blockIdx.y;
    const int px = c & 1, py = (c >> 1) & 1, pz = c >> 2;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < plane_stride;
         s += int64_t(gridDim.x) * blockDim.x) {
        const int x = int(s % pitch_x);
        const int64_t t = s / pitch_x;
        const int y = int(t % (R + 1));
        const int z = int(t / (R + 1));
        double mt = 0.0, ms = 0.0;
        if (x < R + px && y < R + py && z < R + pz && z <= R) {
            mt = centre_mean(st, R, x, y, z, px, py, pz);
            ms = centre_mean(ss, R, x, y, z, px, py, pz);
        }
        cm[int64_t(2 * c) * plane_stride + s] = mt;
        cm[int64_t(2 * c + 1) * plane_stride + s] = ms;
    }
}

constexpr int kF64MaxTerms = 16;

template <int MODE>
__global__ void __launch_bounds__(256) k_op_f64(OpArgs<double> a, const double* cm, int nyb, int64_t items) {
    __shared__ Term ts[kF64MaxTerms];
    __shared__ Plane ps;
    const int R = a.R;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    double racc = 0.0;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int yb = int(it % nyb);
        const int64_t u = it / nyb;
        const int z = int(u % (R + 1));
        const int p = int(u / (R + 1));
        __syncthreads();  // the previous item's reads of ps and ts are done
        if (threadIdx.x == 0) ps = a.planes[p];
        __syncthreads();
        const int nt = ps.t1 - ps.t0;
        if (int(threadIdx.x) < nt) ts[threadIdx.x] = a.terms[ps.t0 + threadIdx.x];
        __syncthreads();
        const int px = ps.px, py = ps.py, pz = ps.pz;
        const double fl = ps.fl_d;
        const int cls = px + 2 * py + 4 * pz;
        const double* cmt = cm + int64_t(2 * cls) * a.plane_stride;
        const double* cms = cmt + a.plane_stride;
        const int64_t pbase = int64_t(p) * a.plane_stride;
        const int y = yb * 8 + ly;
        if (y > R) continue;  // (no barrier follows before the next item's first)
        const int64_t row = int64_t(z) * a.pitch_y + int64_t(y) * a.pitch_x;
        const bool rowact = y < R + py && z < R + pz;
        for (int x = lx; x < a.pitch_x; x += 32) {
            const int64_t s = row + x;
            double out = 0.0;
            if (rowact && x < R + px) {
                const double diag = fma_rn(-fl, cms[s], cmt[s]);  // op_point's rounding, step for step
                double tr = 0.0;
                for (int ti = 0; ti < nt; ++ti) {
                    const Term tm = ts[ti];
                    int i, b;
                    int64_t stride;
                    if (tm.axis == 0) { i = x; b = px; stride = 1; }
                    else if (tm.axis == 1) { i = y; b = py; stride = a.pitch_x; }
                    else { i = z; b = pz; stride = a.pitch_y; }
                    const int64_t qb = int64_t(tm.q) * a.plane_stride + s;
                    const double vp = (i + 1 - b < R + 1 - b) ? a.x[qb + (1 - b) * stride] : 0.0;
                    const double vm = (i - b >= 0) ? a.x[qb - b * stride] : 0.0;
                    tr = fma_rn(tm.cd, sub_rn(vp, vm), tr);
                }
                const double own = mul_rn(diag, a.x[pbase + s]);
                out = MODE == OP_APPLY_T ? sub_rn(own, tr) : add_rn(own, tr);
                if (MODE == OP_RESIDUAL) {
                    const double bq = a.bvec ? a.bvec[pbase + s] : ((p < a.n_q) ? a.q[pbase + s] : 0.0);
                    out = sub_rn(bq, out);
                    racc = fma(out, out, racc);
                }
            }
            a.y[pbase + s] = out;
        }
    }
    if (MODE == OP_RESIDUAL && a.partials != nullptr) {
        const double bs = block_sum(racc);
        if (threadIdx.x == 0) a.partials[blockIdx.x] = bs;
    }
}

// plane tails (slots beyond each plane's box) are written 0 by this kernel
__global__ void __launch_bounds__(256) k_zero_tails(double* y, int K, int64_t box, int64_t plane_stride) {
    const int64_t tail = plane_stride - box;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < int64_t(K) * tail;
         i += int64_t(gridDim.x) * blockDim.x)
        y[(i / tail) * plane_stride + box + i % tail] = 0.0;
}

static bool use_f64_tiled(const pn_handle* h, int dtype) {
    if (dtype != PN_F64 || h->dims != 3 || h->periodic) return false;
    for (const Plane& P : h->planes)
        if (P.t1 - P.t0 > kF64MaxTerms) return false;
    return true;
}

static int64_t f64_items(const pn_handle* h) { return int64_t(h->K) * (h->R + 1) * ((h->R + 1 + 7) / 8); }

static int f64_grid(const pn_handle* h) {
    return int(std::min<int64_t>(f64_items(h), 8 * int64_t(pn_sm_count())));
}

// the class means of the handle (built on the first FP64 operator launch and
// kept until pn_destroy)
static cudaError_t ensure_cmean(const pn_handle* h, cudaStream_t s) {
    pn_handle* hm = const_cast<pn_handle*>(h);
    if (hm->d_cmean) return cudaSuccess;
    cudaError_t e = cudaMalloc(&hm->d_cmean, size_t(16) * size_t(h->plane_stride) * sizeof(double));
    if (e != cudaSuccess) {
        hm->d_cmean = nullptr;
        return e;
    }
    const int gx = int(std::min<int64_t>(4096, (h->plane_stride + 255) / 256));
    k_cmean_build<<<dim3(gx, 8), 256, 0, s>>>(hm->d_cmean, h->d_st_d, h->d_ss_d, h->R, h->pitch_x, h->pitch_y,
                                             h->plane_stride);
    return cudaGetLastError();
}

static int naive_grid_x(const pn_handle* h) {
    int64_t want = (h->plane_stride + 1023) / 1024;
    if (want > 4096) want = 4096;
    if (want < 1) want = 1;
    return int(want);
}

static int slab_grid_x(const pn_handle* h) {
    const int64_t w = h->pitch_x - tiled_x_end(h);
    const int64_t n = w * (h->R + 1) * (h->R + 1) + (h->plane_stride - h->pitch_y * (h->R + 1));
    int64_t g = (n + 255) / 256;
    if (g > 1024) g = 1024;
    return int(g < 1 ? 1 : g);
}

static bool use_tiled(const pn_handle* h, int dtype) {
    // the tiled kernel (3D only) forms addresses with 32-bit element offsets
    // of up to 16 planes: it needs plane_stride * 16 < 2^32 (R <= 1000 or so)
    return dtype == PN_F32 && h->dims == 3 && !h->periodic && h->plane_stride * 16 < (int64_t(1) << 32);
}

bool tiled_serves(const pn_handle* h) { return use_tiled(h, PN_F32); }

int op_launch_count(const pn_handle* h, int dtype) { return (use_tiled(h, dtype) || use_f64_tiled(h, dtype)) ? 2 : 1; }

int op_partial_count(const pn_handle* h, int dtype) {
    if (use_tiled(h, dtype)) return tiled_partial_count(h);
    if (use_f64_tiled(h, dtype)) return f64_grid(h);
    return naive_grid_x(h) * h->K;
}

template <typename T>
static cudaError_t op_t(const pn_handle* h, int mode, const T* x, T* y, const T* st, const T* ss,
                        const T* q, const T* bvec, double* partials, cudaStream_t s) {
    OpArgs<T> a;
    a.x = x; a.y = y; a.q = q; a.n_q = h->n_q_planes; a.bvec = bvec;
    a.st = st; a.ss = ss;
    a.planes = h->d_planes; a.terms = h->d_terms;
    a.R = h->R; a.nzb = int(h->nz_box); a.periodic = h->periodic;
    a.pitch_x = h->pitch_x; a.pitch_y = h->pitch_y; a.plane_stride = h->plane_stride;
    a.partials = partials;
    dim3 grid(naive_grid_x(h), h->K);
    if (mode == OP_APPLY) k_op_naive<T, OP_APPLY><<<grid, 256, 0, s>>>(a);
    else if (mode == OP_APPLY_T) k_op_naive<T, OP_APPLY_T><<<grid, 256, 0, s>>>(a);
    else k_op_naive<T, OP_RESIDUAL><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_op(const pn_handle* h, int mode, const void* x, void* y, int dtype,
                      double* partials, cudaStream_t s, const void* bvec) {
    if (use_tiled(h, dtype)) {
        // tiled kernel for x < x_end, face-column kernel for the rest
        return launch_tiled(h, mode, (const float*)x, (float*)y, (const float*)bvec, partials, s);
    }
    if (dtype == PN_F32)
        return op_t<float>(h, mode, (const float*)x, (float*)y, h->d_st_f, h->d_ss_f, h->d_q_f, (const float*)bvec,
                           partials, s);
    if (use_f64_tiled(h, dtype)) {
        cudaError_t e = ensure_cmean(h, s);
        if (e != cudaSuccess) return e;
        OpArgs<double> a;
        a.x = (const double*)x; a.y = (double*)y; a.q = h->d_q_d; a.n_q = h->n_q_planes; a.bvec = (const double*)bvec;
        a.st = h->d_st_d; a.ss = h->d_ss_d;
        a.planes = h->d_planes; a.terms = h->d_terms;
        a.R = h->R; a.nzb = int(h->nz_box); a.periodic = 0;
        a.pitch_x = h->pitch_x; a.pitch_y = h->pitch_y; a.plane_stride = h->plane_stride;
        a.partials = partials;
        const int nyb = (h->R + 1 + 7) / 8;
        const int G = f64_grid(h);
        if (mode == OP_APPLY) k_op_f64<OP_APPLY><<<G, 256, 0, s>>>(a, h->d_cmean, nyb, f64_items(h));
        else if (mode == OP_APPLY_T) k_op_f64<OP_APPLY_T><<<G, 256, 0, s>>>(a, h->d_cmean, nyb, f64_items(h));
        else k_op_f64<OP_RESIDUAL><<<G, 256, 0, s>>>(a, h->d_cmean, nyb, f64_items(h));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t box = h->pitch_y * (h->R + 1);
        const int64_t nt = int64_t(h->K) * (h->plane_stride - box);
        k_zero_tails<<<int(std::max<int64_t>(1, std::min<int64_t>(1024, (nt + 255) / 256))), 256, 0, s>>>(
            (double*)y, h->K, box, h->plane_stride);
        return cudaGetLastError();
    }
    return op_t<double>(h, mode, (const double*)x, (double*)y, h->d_st_d, h->d_ss_d, h->d_q_d,
                        (const double*)bvec, partials, s);
}

// ---- reductions -------------------------------------------------------------

// two blocks per SM of the current device (pn_sm_count caches per device)
int reduce_blocks() { return 2 * pn_sm_count(); }

// FP64 dot.  FP32 inputs: each thread sums runs of up to 32 products in FP32
// and accumulates each run's sum in FP64.
__global__ void __launch_bounds__(256) k_dot_f32(const float4* a, const float4* b, int64_t n4, double* partials) {
    double acc = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    while (i < n4) {
        float run = 0.0f;  // up to 8 float4 products in FP32, then into FP64
        for (int r = 0; r < 8 && i < n4; ++r, i += stride) {
            const float4 u = a[i], v = b[i];
            run = fmaf(u.w, v.w, fmaf(u.z, v.z, fmaf(u.y, v.y, fmaf(u.x, v.x, run))));
        }
        acc += double(run);
    }
    const double bs = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
}

__global__ void __launch_bounds__(256) k_dot_f64(const double* a, const double* b, int64_t n, double* partials) {
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        acc = fma(a[i], b[i], acc);
    const double bs = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
}

// out[v] = sum_b partials[v * nblocks + b], fixed order (deterministic).
__global__ void __launch_bounds__(256) k_reduce(const double* partials, int nblocks, double* out) {
    const double* p = partials + int64_t(blockIdx.x) * nblocks;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += p[i];
    const double bs = block_sum(acc);
    if (threadIdx.x == 0) out[blockIdx.x] = bs;
}

cudaError_t launch_reduce(const double* partials, int nblocks, int nvals, double* out_dev, cudaStream_t s) {
    k_reduce<<<nvals, 256, 0, s>>>(partials, nblocks, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_dot(const pn_handle* h, const void* a, const void* b, int64_t n, int dtype,
                       double* out_dev, cudaStream_t s) {
    const int nb = h->red_blocks;  // the handle's partials buffer is sized for it
    if (dtype == PN_F32) {
        k_dot_f32<<<nb, 256, 0, s>>>((const float4*)a, (const float4*)b, n / 4, h->d_partials);
    } else {
        k_dot_f64<<<nb, 256, 0, s>>>((const double*)a, (const double*)b, n, h->d_partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce(h->d_partials, nb, 1, out_dev, s);
}

template <typename T>
__global__ void __launch_bounds__(256) k_axpby(int64_t n, T alpha, const T* x, T beta, T* y) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = alpha * x[i] + beta * y[i];
}

cudaError_t launch_axpby(int64_t n, double alpha, const void* x, double beta, void* y, int dtype, cudaStream_t s) {
    const int nb = 8 * pn_sm_count();
    if (dtype == PN_F32)
        k_axpby<float><<<nb, 256, 0, s>>>(n, float(alpha), (const float*)x, float(beta), (float*)y);
    else
        k_axpby<double><<<nb, 256, 0, s>>>(n, alpha, (const double*)x, beta, (double*)y);
    return cudaGetLastError();
}

}  // namespace pn
