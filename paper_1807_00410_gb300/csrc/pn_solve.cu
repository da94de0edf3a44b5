// Krylov solvers of the GB300 P_N library (pn_solve).
//
//  * CGLS: CG on the normal equations A^T A u = A^T Q without forming A^T A,
//    the paper's solver (sections "Runtime" and "Results").  Scalars stay on
//    the device; the host reads ||r||^2 every `check_every` iterations.
//  * GMRES(m): restarted GMRES on A u = Q (A is nonsingular with a positive
//    definite symmetric part, so the normal equations are not needed).
//    Classical Gram-Schmidt applied twice, FP64 inner products, Hessenberg
//    matrix, Givens rotations and the triangular solve in FP64 on the device.
//  * IR: iterative refinement; the residual and the iterate are FP64, each
//    correction comes from an FP32 GMRES solve of A d = r / ||r||.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <string>

#include "pn_internal.h"
#include "pn_mbar.cuh"
#include "pn_pdl.cuh"

namespace {

// scalar slots in h->d_scalars
enum { S_RR = 0, S_QQ = 1, S_G0 = 2, S_G1 = 3, S_BETA2 = 4, S_RES = 5, S_SCALE = 6, S_NRM2 = 7, S_MAXPY = 64,
       S_PNRM = 65, S_TICKET = 66 };

int nb_vec() { return 4 * pn_sm_count(); }
// the fused CGS1 step: one full wave (its 42-46 registers allow 5 CTAs of 256
// threads per SM); partials: nb_mdot * (PN_MAX_MDOT + 1) doubles
int nb_mdot() { return 5 * pn_sm_count(); }

__device__ __forceinline__ double warp_block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = lane; i < nw; i += 32) v += red[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// x += alpha p ; r -= alpha q ; partial sums of r^2.   alpha = S[g] / S[qq].
template <typename T>
__global__ void __launch_bounds__(256) k_cgls_xr(int64_t n, T* x, T* r, const T* p, const T* q,
                                                 const double* S, int g, double* partials) {
    const double qq = S[S_QQ];
    const T alpha = qq > 0.0 ? T(S[g] / qq) : T(0);
    double acc = 0.0;
    T run = T(0);
    int cnt = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        x[i] += alpha * p[i];
        const T ri = r[i] - alpha * q[i];
        r[i] = ri;
        run += ri * ri;  // short runs in T, each run's sum added in FP64
        if (++cnt == 16) {
            acc += double(run);
            run = T(0);
            cnt = 0;
        }
    }
    acc += double(run);
    const double bs = warp_block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
}

// p = s + beta p,  beta = S[gnew] / S[gold]
template <typename T>
__global__ void __launch_bounds__(256) k_cgls_p(int64_t n, T* p, const T* s, const double* S, int gold, int gnew) {
    const double go = S[gold];
    const T beta = go > 0.0 ? T(S[gnew] / go) : T(0);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        p[i] = s[i] + beta * p[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_copy(int64_t n, T* dst, const T* src) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = src[i];
}

// v *= 1 / sqrt(S[idx])  (or v = 0 if S[idx] == 0)
template <typename T>
__global__ void __launch_bounds__(256) k_scale_invnorm(int64_t n, T* v, const double* S, int idx) {
    const double nn = S[idx];
    const T sc = nn > 0.0 ? T(1.0 / sqrt(nn)) : T(0);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        v[i] *= sc;
}

// Multi-dot: partials[j * gridDim.x + b] = block b's share of V_j . w, j < nv.
// FP32 vectors: float4 loads; each thread sums kRun float4 products in FP32,
// then adds the run's sum to its FP64 accumulator (FP64 work is 1/(4 kRun)
// of the elements; GB300's FP64 rate is far below its FP32 rate).
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_mdot(int64_t n, const T* V, int64_t vstride, int nv, const T* w,
                                              double* partials, int self_dot) {
    double acc[NV + 1];
#pragma unroll
    for (int j = 0; j <= NV; ++j) acc[j] = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T wi = w[i];
#pragma unroll
        for (int j = 0; j < NV; ++j)
            if (j < nv) acc[j] = fma(double(V[j * vstride + i]), double(wi), acc[j]);
        if (self_dot) acc[NV] = fma(double(wi), double(wi), acc[NV]);
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        if (j < nv) {
            const double bs = warp_block_sum(acc[j]);
            if (threadIdx.x == 0) partials[int64_t(j) * gridDim.x + blockIdx.x] = bs;
        }
    }
    if (self_dot) {
        const double bs = warp_block_sum(acc[NV]);
        if (threadIdx.x == 0) partials[int64_t(nv) * gridDim.x + blockIdx.x] = bs;
    }
}

constexpr int kRun = 16;

// Sums acc[0..nv) (and acc[NV] if self_dot) over the block: every thread
// stores its FP64 partials in shared memory, then warp w sums the values of
// vectors w, w + 8, ... (eight strided FP64 adds per lane, then a shuffle
// tree), so the FP64 work per block is a few hundred adds per vector.
template <int NV>
__device__ __forceinline__ void block_sum_multi(const double (&acc)[NV + 1], int nv, int self_dot, double* out,
                                                int64_t out_stride) {
    __shared__ double red[NV + 1][256];
#pragma unroll
    for (int j = 0; j <= NV; ++j) red[j][threadIdx.x] = acc[j];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nvals = nv + (self_dot ? 1 : 0);
    for (int v = warp; v < nvals; v += 8) {
        const int j = v < nv ? v : NV;  // the self-dot lives in slot NV
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[j][lane + 32 * q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) out[int64_t(v) * out_stride] = t;
    }
}

template <int NV>
__global__ void __launch_bounds__(256) k_mdot_f32(int64_t n4, const float4* V, int64_t vstride4, int nv,
                                                  const float4* w, double* partials, int self_dot) {
    double acc[NV + 1];
#pragma unroll
    for (int j = 0; j <= NV; ++j) acc[j] = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    while (i < n4) {
        float part[NV + 1];
#pragma unroll
        for (int j = 0; j <= NV; ++j) part[j] = 0.0f;
        for (int r = 0; r < kRun && i < n4; ++r, i += stride) {
            const float4 wi = w[i];
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                if (j < nv) {
                    const float4 v = V[j * vstride4 + i];
                    part[j] = fmaf(v.w, wi.w, fmaf(v.z, wi.z, fmaf(v.y, wi.y, fmaf(v.x, wi.x, part[j]))));
                }
            }
            if (self_dot) part[NV] = fmaf(wi.w, wi.w, fmaf(wi.z, wi.z, fmaf(wi.y, wi.y, fmaf(wi.x, wi.x, part[NV]))));
        }
#pragma unroll
        for (int j = 0; j <= NV; ++j) acc[j] += double(part[j]);
    }
    // partials[v * gridDim.x + block]; the self-dot goes to slot v = nv
    block_sum_multi<NV>(acc, nv, self_dot, partials + blockIdx.x, gridDim.x);
}

// w = (w + sign * sum_j c[j] V_j) * scale, scale = *scale_p (1 if null)
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_maxpy(int64_t n, T* w, const T* V, int64_t vstride, int nv,
                                               const double* c, double sign, const double* scale_p) {
    T cj[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) cj[j] = j < nv ? T(sign * c[j]) : T(0);
    const T sc = scale_p ? T(*scale_p) : T(1);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        T acc = w[i];
#pragma unroll
        for (int j = 0; j < NV; ++j)
            if (j < nv) acc += cj[j] * V[j * vstride + i];
        w[i] = acc * sc;
    }
}

template <int NV>
__global__ void __launch_bounds__(256) k_maxpy_f32(int64_t n4, float4* w, const float4* V, int64_t vstride4, int nv,
                                                   const double* c, double sign, const double* scale_p) {
    float cj[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) cj[j] = j < nv ? float(sign * c[j]) : 0.0f;
    const float sc = scale_p ? float(*scale_p) : 1.0f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x) {
        float4 acc = w[i];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            if (j < nv) {
                const float4 v = V[j * vstride4 + i];
                acc.x = fmaf(cj[j], v.x, acc.x);
                acc.y = fmaf(cj[j], v.y, acc.y);
                acc.z = fmaf(cj[j], v.z, acc.z);
                acc.w = fmaf(cj[j], v.w, acc.w);
            }
        }
        acc.x *= sc;
        acc.y *= sc;
        acc.z *= sc;
        acc.w *= sc;
        w[i] = acc;
    }
}

// Typed launchers: FP32 vectors take the float4 kernels (n is a multiple of 32).
template <typename T>
void launch_mdot(int nb, cudaStream_t s, int64_t n, const T* V, int64_t vstride, int nv, const T* w, double* part,
                 int self_dot = 0);
template <>
void launch_mdot<float>(int nb, cudaStream_t s, int64_t n, const float* V, int64_t vstride, int nv, const float* w,
                        double* part, int self_dot) {
    k_mdot_f32<PN_MAX_MDOT><<<nb, 256, 0, s>>>(n / 4, (const float4*)V, vstride / 4, nv, (const float4*)w, part,
                                               self_dot);
}
template <>
void launch_mdot<double>(int nb, cudaStream_t s, int64_t n, const double* V, int64_t vstride, int nv,
                         const double* w, double* part, int self_dot) {
    k_mdot<double, PN_MAX_MDOT><<<nb, 256, 0, s>>>(n, V, vstride, nv, w, part, self_dot);
}
template <typename T>
void launch_maxpy(int nb, cudaStream_t s, int64_t n, T* w, const T* V, int64_t vstride, int nv, const double* c,
                  double sign, const double* scale_p = nullptr);
template <>
void launch_maxpy<float>(int nb, cudaStream_t s, int64_t n, float* w, const float* V, int64_t vstride, int nv,
                         const double* c, double sign, const double* scale_p) {
    k_maxpy_f32<PN_MAX_MDOT><<<nb, 256, 0, s>>>(n / 4, (float4*)w, (const float4*)V, vstride / 4, nv, c, sign,
                                                scale_p);
}
template <>
void launch_maxpy<double>(int nb, cudaStream_t s, int64_t n, double* w, const double* V, int64_t vstride, int nv,
                          const double* c, double sign, const double* scale_p) {
    k_maxpy<double, PN_MAX_MDOT><<<nb, 256, 0, s>>>(n, w, V, vstride, nv, c, sign, scale_p);
}

// Arnoldi step bookkeeping, one thread, FP64.
//   col: H column j (rows 0..j from pass 1), add: pass-2 corrections (rows 0..j),
//   S[S_NRM2] = ||w||^2 after orthogonalisation.
// Applies the previous rotations, forms rotation j, updates g and writes
// |g[j+1]| to S[S_RES] and 1/||w|| to S[S_SCALE].
// sum_{b = lane, lane + 32, ...} p[b] in that order (the order of a plain
// loop), with eight loads issued before their adds: the last block's
// reduction is a chain of L2 reads otherwise.
__device__ __forceinline__ double lane_sum_partials(const double* p, int nb, int lane) {
    double t = 0.0;
    for (int b0 = lane; b0 < nb; b0 += 32 * 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = b0 + 32 * u < nb ? __ldcg(p + b0 + 32 * u) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (b0 + 32 * u < nb) t += v[u];
    }
    return t;
}

// The Givens update of Arnoldi column j, run by one whole warp.  On entry the
// shared array c[0..j] holds the column's projections h_{0..j} (the column of
// H after Gram-Schmidt); `scr` (shared, >= 2 (j + 1) doubles) is scratch.
//  * pythagoras != 0 (a single Gram-Schmidt pass): ||w - V h||^2 =
//    ||w||^2 - ||h||^2 for orthonormal V; a remainder at rounding level is a
//    breakdown (w lies in the span of V: the Krylov space is invariant and the
//    least-squares solution exact): h_{j+1,j} = 0, the next basis vector 0, the
//    residual estimate 0.  Otherwise nrm2_in is ||w||^2 after orthogonalisation.
//  * the previous rotations are applied to the column, rotation j is formed,
//    g is updated, |g[j+1]| goes to S[S_RES] and 1/h_{j+1,j} to S[S_SCALE].
// The lanes load the earlier rotations and store the column in parallel; lane
// 0 runs the sequential rotation chain in shared memory (on the global arrays,
// which may alias, every step of the chain was a dependent round trip to L2).
__device__ __forceinline__ void givens_warp(double* c, double* scr, double* H, int ldh, double* cs, double* sn, double* g, int j,
                            double* S, int pythagoras, double nrm2_in) {
    const int lane = threadIdx.x & 31;
    double* css = scr;
    double* sns = scr + (j + 1);
    for (int i = lane; i < j; i += 32) {
        css[i] = cs[i];
        sns[i] = sn[i];
    }
    __syncwarp();
    if (lane == 0) {
        double nrm2 = nrm2_in;
        if (pythagoras) {
            double hh = 0.0;
            for (int i = 0; i <= j; ++i) hh += c[i] * c[i];
            nrm2 = nrm2 - hh;
            // (rounding level: about 1e-14 of |w|^2 for FP32 vectors (pythagoras = 1),
            // 1e-30 for FP64 (2), 1e-6 for a basis stored in FP16 (3))
            const double tiny = pythagoras == 2 ? 1e-26 : (pythagoras == 3 ? 1e-5 : 1e-12);
            if (!(nrm2 > tiny * nrm2_in)) nrm2 = 0.0;
        }
        const double hn = sqrt(fmax(nrm2, 0.0));
        c[j + 1] = hn;
        S[S_SCALE] = hn > 0.0 ? 1.0 / hn : 0.0;
        for (int i = 0; i < j; ++i) {
            const double t = css[i] * c[i] + sns[i] * c[i + 1];
            c[i + 1] = -sns[i] * c[i] + css[i] * c[i + 1];
            c[i] = t;
        }
        const double a = c[j], b = c[j + 1];
        const double den = hypot(a, b);
        const double cr = den > 0.0 ? a / den : 1.0;
        const double sr = den > 0.0 ? b / den : 0.0;
        cs[j] = cr;
        sn[j] = sr;
        c[j] = den;
        c[j + 1] = 0.0;
        const double gj = g[j];
        g[j + 1] = -sr * gj;
        g[j] = cr * gj;
        S[S_RES] = fabs(-sr * gj);
    }
    __syncwarp();
    double* col = H + int64_t(j) * ldh;
    for (int i = lane; i <= j + 1; i += 32) col[i] = c[i];
}

// Givens update of column j after classical Gram-Schmidt (one warp): the
// column of H plus the second pass's corrections `add` (pythagoras = 0), or
// the column alone with ||w||^2 in S[S_NRM2] (pythagoras != 0).
__global__ void __launch_bounds__(32) k_givens(double* H, int ldh, const double* add, double* cs, double* sn,
                                               double* g, int j, double* S, int pythagoras) {
    __shared__ double c[202];
    __shared__ double scr[402];  // j <= 199 (restart <= 200)
    const double* col = H + int64_t(j) * ldh;
    for (int i = threadIdx.x; i <= j; i += 32) c[i] = pythagoras ? col[i] : col[i] + add[i];
    __syncwarp();
    givens_warp(c, scr, H, ldh, cs, sn, g, j, S, pythagoras, S[S_NRM2]);
}

// One fused CGS1 step for j + 1 <= PN_MAX_MDOT basis vectors (FP32):
//  * every block: V_i . w (i <= j) and w . w over its grid-stride share, each
//    thread summing its products in FP32, each warp's 32 sums added in FP32,
//    the block's 8 warp sums added in FP64, one FP64 partial per block;
//  * the last block to finish (ticket counter) adds the partials in block
//    order (deterministic), writes the projections to `add` and the
//    Hessenberg column, and runs the Givens update with |w - V h|^2 =
//    |w|^2 - |h|^2 (what k_reduce + k_cgs1_gather + k_givens do in three
//    launches), then resets the ticket.
__global__ void __launch_bounds__(256) k_mdot_givens_f32(int64_t n4, const float4* V, int64_t vstride4, int nv,
                                                         const float4* w, double* partials, unsigned int* ticket,
                                                         double* H, int ldh, double* add, double* cs, double* sn,
                                                         double* g, int j, double* S) {
    constexpr int NV = PN_MAX_MDOT;
    float part[NV + 1];
#pragma unroll
    for (int v = 0; v <= NV; ++v) part[v] = 0.0f;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 wi = w[i];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v < nv) {
                const float4 q = V[v * vstride4 + i];
                part[v] = fmaf(q.w, wi.w, fmaf(q.z, wi.z, fmaf(q.y, wi.y, fmaf(q.x, wi.x, part[v]))));
            }
        }
        part[NV] = fmaf(wi.w, wi.w, fmaf(wi.z, wi.z, fmaf(wi.y, wi.y, fmaf(wi.x, wi.x, part[NV]))));
    }
    __shared__ double red[NV + 1][8];
    __shared__ double tot[NV + 1];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v <= NV; ++v) {
        if (v < nv || v == NV) {
            float t = part[v];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) red[v][warp] = double(t);
        }
    }
    __syncthreads();
    const int nb = gridDim.x;
    if (threadIdx.x <= NV && (int(threadIdx.x) < nv || threadIdx.x == NV)) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[threadIdx.x][q];
        partials[int64_t(threadIdx.x) * nb + blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == unsigned(nb - 1)) ? 1 : 0;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int v = warp; v <= NV; v += 8) {
        if (v < nv || v == NV) {
            double t = lane_sum_partials(partials + int64_t(v) * nb, nb, lane);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) tot[v] = t;
        }
    }
    __syncthreads();
    if (warp == 0) {
        // red is free again: c[0..j+1] at red[0..], the rotations' scratch after it
        double* cc = &red[0][0];
        for (int i = lane; i <= j; i += 32) {
            cc[i] = tot[i];
            add[i] = tot[i];
        }
        if (lane == 0) S[S_NRM2] = tot[NV];
        __syncwarp();
        givens_warp(cc, cc + (NV + 2), H, ldh, cs, sn, g, j, S, 1, tot[NV]);
        if (lane == 0) *ticket = 0u;
    }
}

// CGS1 bookkeeping: the first chunk's reduction wrote nv0 projections and
// ||w||^2 into tmp0, later chunks wrote their projections into proj directly.
// Completes proj[0..j], copies it into the H column (which the Givens kernel
// then rotates) and puts ||w||^2 into S[S_NRM2].
__global__ void k_cgs1_gather(double* col, double* proj, const double* tmp0, int nv0, int j, double* S) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < nv0; ++i) proj[i] = tmp0[i];
    for (int i = 0; i <= j; ++i) col[i] = proj[i];
    S[S_NRM2] = tmp0[nv0];
}

__global__ void k_gm_init(double* g, int m, double* S) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double beta = sqrt(fmax(S[S_BETA2], 0.0));
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    S[S_RES] = beta;
}

// Solve the k x k upper-triangular system H y = g in FP64 (k <= 200).  One
// block: the threads copy the triangle and g into shared memory when it fits
// (k <= 64), then thread 0 substitutes from there (a one-thread solve
// straight from global memory waits on a dependent load chain).
__global__ void k_gm_backsolve(const double* H, int ldh, const double* g, double* y, int k) {
    constexpr int KS = 64;
    __shared__ double hs[KS * (KS + 1) / 2];
    __shared__ double gs[KS];
    __shared__ double ys[KS];
    if (k <= KS) {
        // column c of the triangle (rows 0..c) at hs[c (c + 1) / 2 + row]
        for (int e = threadIdx.x; e < k * (k + 1) / 2; e += blockDim.x) {
            int c = int((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
            while (c * (c + 1) / 2 > e) --c;
            while ((c + 1) * (c + 2) / 2 <= e) ++c;
            const int row = e - c * (c + 1) / 2;
            hs[e] = H[int64_t(c) * ldh + row];
        }
        for (int i = threadIdx.x; i < k; i += blockDim.x) gs[i] = g[i];
        __syncthreads();
        if (threadIdx.x != 0) return;
        for (int i = k - 1; i >= 0; --i) {
            double t = gs[i];
            for (int c = i + 1; c < k; ++c) t -= hs[c * (c + 1) / 2 + i] * ys[c];
            const double d = hs[i * (i + 1) / 2 + i];
            ys[i] = d != 0.0 ? t / d : 0.0;
        }
        for (int i = 0; i < k; ++i) y[i] = ys[i];
        return;
    }
    if (threadIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int c = i + 1; c < k; ++c) t -= H[int64_t(c) * ldh + i] * y[c];
        const double d = H[int64_t(i) * ldh + i];
        y[i] = d != 0.0 ? t / d : 0.0;
    }
}

// v *= S[S_SCALE]
template <typename T>
__global__ void __launch_bounds__(256) k_scale_by(int64_t n, T* v, const double* S, int idx) {
    const T sc = T(S[idx]);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        v[i] *= sc;
}

// r32 = r64 / sqrt(S[idx])
__global__ void __launch_bounds__(256) k_to_f32_scaled(int64_t n, float* dst, const double* src, const double* S, int idx) {
    const double nn = S[idx];
    const double sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = float(src[i] * sc);
}

// x64 += sqrt(S[idx]) * d32
__global__ void __launch_bounds__(256) k_add_f32_scaled(int64_t n, double* x, const float* d, const double* S, int idx) {
    const double sc = sqrt(fmax(S[idx], 0.0));
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] += sc * double(d[i]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_zero(int64_t n, T* v) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        v[i] = T(0);
}

struct Ctx {
    pn_handle* h;
    cudaStream_t s;
    int rc = PN_OK;
    void pb() { pn_prof_begin(h, s); }
    void pe(int kind, double bytes) { pn_prof_end(h, s, kind, bytes); }
    // algorithmic bytes of `nvec` unknown-sized vector passes of element size esz
    double vb(double nvec, double esz) const { return nvec * double(h->n_active) * esz; }
    // algorithmic bytes of one operator launch (x read, y written, sigma_t and
    // sigma_s read; residual also reads its right-hand side)
    double ob(int mode, double esz, bool bvec) const {
        const double V = double(h->R) * h->R * h->R;
        double b = (2.0 * h->n_active + 2.0 * V) * esz;
        if (mode == pn::OP_RESIDUAL) b += (bvec || h->n_q_planes > 1 ? double(h->n_active) : (h->n_q_planes ? V : 0.0)) * esz;
        return b;
    }
    bool ok(cudaError_t e, const char* where) {
        if (e != cudaSuccess && rc == PN_OK) rc = pn_cuda_fail(h, e, where);
        return rc == PN_OK;
    }
    int64_t launches = 0;  // kernels launched by this solve
    bool launched(const char* where, int count = 1) {
        launches += count;
        return ok(cudaGetLastError(), where);
    }
    bool lk(cudaError_t e, const char* where, int count = 1) {
        launches += count;
        return ok(e, where);
    }
    bool lk2(cudaError_t e, const char* where) { return lk(e, where, 2); }
    // read n doubles from d_scalars[idx..] (synchronises)
    bool read(int idx, int n, double* out) {
        if (!ok(cudaMemcpyAsync(h->h_pinned, h->d_scalars + idx, n * sizeof(double), cudaMemcpyDeviceToHost, s),
                "pn_solve: read scalar"))
            return false;
        if (!ok(cudaStreamSynchronize(s), "pn_solve: sync")) return false;
        pn_prof_drain(h);
        for (int i = 0; i < n; ++i) out[i] = h->h_pinned[i];
        return true;
    }
};

int ensure_work(pn_handle* h, size_t bytes) {
    if (h->work_bytes >= bytes) return PN_OK;
    if (h->d_work) cudaFree(h->d_work);
    h->d_work = nullptr;
    h->work_bytes = 0;
    ++h->work_allocs;
    if (cudaMalloc(&h->d_work, bytes) != cudaSuccess) {
        cudaGetLastError();
        h->d_work = nullptr;
        return pn_fail(h, PN_ERR_ALLOC, "pn_solve: cannot allocate Krylov workspace");
    }
    h->work_bytes = bytes;
    return PN_OK;
}

double rel_of(const pn_handle* h, double rr) {
    return h->q_norm2 > 0.0 ? std::sqrt(rr / h->q_norm2) : std::sqrt(rr);
}

template <typename T>
int cgls(Ctx& c, T* x, const pn_solve_opts& o, pn_solve_stats& st) {
    pn_handle* h = c.h;
    const int64_t n = h->n_elems;
    int rc = ensure_work(h, size_t(4) * n * sizeof(T));
    if (rc != PN_OK) return rc;
    T* r = (T*)h->d_work;
    T* s = r + n;
    T* p = s + n;
    T* q = p + n;
    const int dt = sizeof(T) == 4 ? PN_F32 : PN_F64;
    const double es = sizeof(T);
    const int nb = nb_vec();
    double* S = h->d_scalars;
    auto residual = [&]() {
        c.pb();
        c.lk(pn::launch_op(h, pn::OP_RESIDUAL, x, r, dt, h->d_partials, c.s), "cgls: residual",
             pn::op_launch_count(h, dt));
        c.pe(PN_PROF_RESIDUAL, c.ob(pn::OP_RESIDUAL, es, false));
        c.pb();
        c.lk(pn::launch_reduce(h->d_partials, pn::op_partial_count(h, dt), 1, S + S_RR, c.s), "cgls: reduce");
        c.pe(PN_PROF_SCALAR, 0.0);
    };
    auto op = [&](int mode, const T* in, T* out) {
        c.pb();
        c.lk(pn::launch_op(h, mode, in, out, dt, nullptr, c.s), "cgls: operator", pn::op_launch_count(h, dt));
        c.pe(PN_PROF_APPLY, c.ob(mode, es, false));
    };
    auto dot = [&](const T* a, double* out) {
        c.pb();
        c.lk2(pn::launch_dot(h, a, a, n, dt, out, c.s), "cgls: dot");
        c.pe(PN_PROF_DOT, c.vb(1, es));
    };
    // r = Q - A x ; s = A^T r ; p = s ; gamma = ||s||^2
    residual();
    op(pn::OP_APPLY_T, r, s);
    dot(s, S + S_G0);
    c.pb();
    k_copy<T><<<nb, 256, 0, c.s>>>(n, p, s);
    c.launched("cgls: copy");
    c.pe(PN_PROF_VECTOR, c.vb(2, es));
    double rr = 0.0;
    if (!c.read(S_RR, 1, &rr)) return c.rc;
    double rel = rel_of(h, rr);
    int it = 0, gcur = S_G0, gnew = S_G1;
    const int every = o.check_every > 0 ? o.check_every : 10;
    while (c.rc == PN_OK && std::isfinite(rel) && rel > o.tol && it < o.max_iter) {
        op(pn::OP_APPLY, p, q);
        dot(q, S + S_QQ);
        c.pb();
        k_cgls_xr<T><<<h->red_blocks, 256, 0, c.s>>>(n, x, r, p, q, S, gcur, h->d_partials);
        c.launched("cgls: update");
        c.pe(PN_PROF_VECTOR, c.vb(6, es));
        c.pb();
        c.lk(pn::launch_reduce(h->d_partials, h->red_blocks, 1, S + S_RR, c.s), "cgls: reduce");
        c.pe(PN_PROF_SCALAR, 0.0);
        op(pn::OP_APPLY_T, r, s);
        dot(s, S + gnew);
        c.pb();
        k_cgls_p<T><<<nb, 256, 0, c.s>>>(n, p, s, S, gcur, gnew);
        c.launched("cgls: direction");
        c.pe(PN_PROF_VECTOR, c.vb(3, es));
        std::swap(gcur, gnew);
        ++it;
        if (it % every == 0 || it >= o.max_iter) {
            double v[2];
            if (!c.read(S_RR, 2, v)) break;
            rel = rel_of(h, v[0]);
            if (v[1] == 0.0 && rel > o.tol) {
                st.iterations = it;
                st.rel_residual = rel;
                return pn_fail(h, PN_ERR_BREAKDOWN, "cgls: ||A p|| = 0");
            }
        }
    }
    if (c.rc != PN_OK) return c.rc;
    // final residual in the solve's own precision (FP64 accumulation)
    residual();
    if (!c.read(S_RR, 1, &rr)) return c.rc;
    st.iterations = it;
    st.rel_residual = rel_of(h, rr);
    if (!std::isfinite(st.rel_residual)) return pn_fail(h, PN_ERR_NONFINITE, "cgls: non-finite residual");
    if (st.rel_residual > o.tol) return pn_fail(h, PN_ERR_NOT_CONVERGED, "cgls: max_iter reached");
    return PN_OK;
}

// ---- GMRES with the Krylov basis stored in FP16 -----------------------------
//
// The basis vectors are stored as FP16 values of sigma * v (sigma = sqrt of the
// number of unknowns, so the entries of a unit vector are of order one and
// stay inside FP16's range); every product, sum and update is FP32, and the
// cross-block sums and the Arnoldi scalars FP64, as in the FP32 path.  The
// newest basis vector is also kept in FP32 for the operator.  The stored
// basis carries a relative rounding of about 5e-4 per entry, far below the
// inner solve's relative target (1e-2 by default): the refinement's FP64
// residual corrects what the inner solve leaves.  Per Arnoldi step the vector
// kernels move about (26 + 4 j) bytes per unknown instead of (28 + 8 j).

__device__ __forceinline__ void h8_to_f(const uint4 u, float (&f)[8]) {
    const __half2* h = reinterpret_cast<const __half2*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 t = __half22float2(h[k]);
        f[2 * k] = t.x;
        f[2 * k + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 f_to_h8(const float (&f)[8]) {
    uint4 u;
    __half2* h = reinterpret_cast<__half2*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(f[2 * k], f[2 * k + 1]);
    return u;
}

// The fused CGS1 step of the FP16-basis path: projections (V16_i . w) / sigma
// for i < nv, |w|^2, the deterministic last-block reduction and the Givens
// update (as k_mdot_givens_f32).  n8 = n / 8; w is FP32.
// The end of a fused CGS1 step over a 256-thread block: block sums of the
// per-thread FP32 partial products (warp sums in FP32, across warps in FP64)
// into partials[v * gridDim.x + block]; the last block to finish (ticket)
// adds them in block order (deterministic), writes the projections and the
// Hessenberg column and runs the Givens update.
__device__ __forceinline__ void mdot16_finish(const float (&part)[PN_MAX_MDOT + 1], int nv, float inv_sigma,
                                              double* partials, unsigned int* ticket, double* H, int ldh,
                                              double* add, double* cs, double* sn, double* g, int j, double* S) {
    constexpr int NV = PN_MAX_MDOT;
    __shared__ double red[NV + 1][8];
    __shared__ double tot[NV + 1];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v <= NV; ++v) {
        if (v < nv || v == NV) {
            float t = part[v];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) red[v][warp] = double(t);
        }
    }
    __syncthreads();
    const int nb = gridDim.x;
    if (threadIdx.x <= NV && (int(threadIdx.x) < nv || threadIdx.x == NV)) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[threadIdx.x][q];
        partials[int64_t(threadIdx.x) * nb + blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == unsigned(nb - 1)) ? 1 : 0;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int v = warp; v <= NV; v += 8) {
        if (v < nv || v == NV) {
            double t = lane_sum_partials(partials + int64_t(v) * nb, nb, lane);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) tot[v] = t;
        }
    }
    __syncthreads();
    if (warp == 0) {
        // red is free again: c[0..j+1] at red[0..], the rotations' scratch after it
        double* cc = &red[0][0];
        for (int i = lane; i <= j; i += 32) {
            const double hi = tot[i] * double(inv_sigma);
            cc[i] = hi;
            add[i] = hi;
        }
        if (lane == 0) S[S_NRM2] = tot[NV];
        __syncwarp();
        givens_warp(cc, cc + (NV + 2), H, ldh, cs, sn, g, j, S, 3, tot[NV]);
        if (lane == 0) *ticket = 0u;
    }
}

__global__ void __launch_bounds__(256) k_mdot16_givens(int64_t n8, const uint4* V16, int64_t vstride8, int nv,
                                                       const float4* w, float inv_sigma, double* partials,
                                                       unsigned int* ticket, double* H, int ldh, double* add,
                                                       double* cs, double* sn, double* g, int j, double* S) {
    constexpr int NV = PN_MAX_MDOT;
    pn::pdl_wait();  // w comes from the operator launched before (programmatic dependent launch)
    float part[NV + 1];
#pragma unroll
    for (int v = 0; v <= NV; ++v) part[v] = 0.0f;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n8; i += stride) {
        const float4 wa = w[2 * i], wb = w[2 * i + 1];
        const float wf[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v < nv) {
                float q[8];
                h8_to_f(V16[v * vstride8 + i], q);
                float t = part[v];
#pragma unroll
                for (int k = 0; k < 8; ++k) t = fmaf(q[k], wf[k], t);
                part[v] = t;
            }
        }
        float t = part[NV];
#pragma unroll
        for (int k = 0; k < 8; ++k) t = fmaf(wf[k], wf[k], t);
        part[NV] = t;
    }
    pn::pdl_trigger();  // the multi-axpy may start during the reduction tail
    mdot16_finish(part, nv, inv_sigma, partials, ticket, H, ldh, add, cs, sn, g, j, S);
}

// The same fused CGS1 step with the streams staged by bulk copies (TMA): each
// block walks every G-th MD_CH-element chunk (G blocks); one thread copies
// each chunk's w (FP32) and nv basis slices (FP16) into one of MD_ST shared
// slots, MD_ST - 1 chunks ahead of the arithmetic (mbarrier per slot, bounded
// waits that set *err).  n is a multiple of 32, so every chunk's byte counts
// are multiples of 16 and every address 16-byte aligned.
constexpr int MD_MIN_NV = 5;  // fewest basis vectors the staged kernels are used for
template <int MD_CH, int MD_ST>
constexpr size_t md_smem_bytes() {
    return size_t(MD_ST) * MD_CH * 4 + size_t(MD_ST) * PN_MAX_MDOT * MD_CH * 2 + MD_ST * 8 + 128;
}

template <int MD_CH, int MD_ST, int MINB>
__global__ void __launch_bounds__(256, MINB) k_mdot16_tma(int64_t n, const __half* V16, int64_t vstride, int nv,
                                                      const float* w, float inv_sigma, double* partials,
                                                      unsigned int* ticket, double* H, int ldh, double* add,
                                                      double* cs, double* sn, double* g, int j, double* S,
                                                      unsigned int* err) {
    constexpr int NV = PN_MAX_MDOT;
    extern __shared__ __align__(128) unsigned char md_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(md_raw) + 127) &
                                                           ~uintptr_t(127));
    float* sw = reinterpret_cast<float*>(base);                                  // [MD_ST][MD_CH]
    __half* sv = reinterpret_cast<__half*>(base + size_t(MD_ST) * MD_CH * 4);    // [MD_ST][NV][MD_CH]
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + size_t(MD_ST) * MD_CH * 4 + size_t(MD_ST) * NV * MD_CH * 2);
    const uint32_t bar_s = pn::mbar::smem_u32(bars);
    const int tid = threadIdx.x;
    // block b takes chunks b, b + G, b + 2G, ...: at any moment the blocks work
    // on neighbouring chunks, so each stream is read from one region of DRAM
    const int64_t nch = (n + MD_CH - 1) / MD_CH;
    const int64_t G = gridDim.x;
    const int64_t nk = nch > int64_t(blockIdx.x) ? (nch - blockIdx.x + G - 1) / G : 0;  // chunks of this block
    if (tid == 0) {
        for (int st = 0; st < MD_ST; ++st) pn::mbar::init(bar_s + 8u * st, 1u);
        pn::mbar::fence_init();
    }
    __syncthreads();
    // a chunk's copies: the basis slices (written by earlier launches) and w
    // (written by the operator just before this kernel), one mbarrier
    auto issue_v = [&](int64_t c, int st) {
        const int64_t e0 = c * MD_CH;
        const int64_t rem = n - e0;
        const uint32_t cnt = uint32_t(rem < MD_CH ? rem : MD_CH);
        const uint32_t bar = bar_s + 8u * st;
        pn::mbar::arrive_expect_tx(bar, cnt * 4u + uint32_t(nv) * cnt * 2u);
        for (int v = 0; v < nv; ++v)
            pn::mbar::bulk_g2s(pn::mbar::smem_u32(sv + (size_t(st) * NV + v) * MD_CH), V16 + v * vstride + e0, cnt * 2u,
                           bar);
    };
    auto issue_w = [&](int64_t c, int st) {
        const int64_t e0 = c * MD_CH;
        const int64_t rem = n - e0;
        const uint32_t cnt = uint32_t(rem < MD_CH ? rem : MD_CH);
        pn::mbar::bulk_g2s(pn::mbar::smem_u32(sw + st * MD_CH), w + e0, cnt * 4u, bar_s + 8u * st);
    };
    auto issue = [&](int64_t c, int st) {
        issue_v(c, st);
        issue_w(c, st);
    };
    // programmatic dependent launch: the basis copies of the first chunks go
    // out before the wait for the operator, w's after it
    if (tid == 0)
        for (int k = 0; k < MD_ST && k < nk; ++k) issue_v(blockIdx.x + k * G, k);
    pn::pdl_wait();
    if (tid == 0)
        for (int k = 0; k < MD_ST && k < nk; ++k) issue_w(blockIdx.x + k * G, k);
    float part[NV + 1];
#pragma unroll
    for (int v = 0; v <= NV; ++v) part[v] = 0.0f;
    bool failed = false;
    for (int64_t kk = 0; kk < nk; ++kk) {
        const int64_t c = blockIdx.x + kk * G;
        const int k = int(kk);
        const int st = k % MD_ST;
        pn::mbar::wait(bar_s + 8u * st, uint32_t(k / MD_ST) & 1u, err, failed);
        const int64_t rem = n - c * MD_CH;
        const int64_t cnt = rem < MD_CH ? rem : MD_CH;
        for (int gq = tid; 4 * gq < cnt; gq += 256) {
            const float4 wv = reinterpret_cast<const float4*>(sw + st * MD_CH)[gq];
            const float wf[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (v < nv) {
                    const uint2 hv = reinterpret_cast<const uint2*>(sv + (size_t(st) * NV + v) * MD_CH)[gq];
                    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&hv.x));
                    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hv.y));
                    float t = part[v];
                    t = fmaf(a.x, wf[0], t);
                    t = fmaf(a.y, wf[1], t);
                    t = fmaf(b.x, wf[2], t);
                    t = fmaf(b.y, wf[3], t);
                    part[v] = t;
                }
            }
            float t = part[NV];
#pragma unroll
            for (int q = 0; q < 4; ++q) t = fmaf(wf[q], wf[q], t);
            part[NV] = t;
        }
        __syncthreads();  // slot st is free again
        if (tid == 0 && kk + MD_ST < nk) issue(c + MD_ST * G, st);
    }
    pn::pdl_trigger();  // the multi-axpy may start during the reduction tail
    mdot16_finish(part, nv, inv_sigma, partials, ticket, H, ldh, add, cs, sn, g, j, S);
}

// w' = (w - sum_{i < nv} add[i] V16_i / sigma) * S[S_SCALE];
// V16_out = fp16(sigma w'), vcur = w'.  Each thread loads two 8-element groups
// before combining either (launched with 8 CTAs per SM).  V16_out is basis
// vector nv, which no thread reads here (the restrict qualifiers say so).
__global__ void __launch_bounds__(256) k_maxpy16(int64_t n8, const float4* __restrict__ w,
                                                 const uint4* __restrict__ V16, int64_t vstride8, int nv,
                                                 const double* add, float inv_sigma, float sigma, const double* S,
                                                 uint4* __restrict__ V16_out, float4* __restrict__ vcur) {
    constexpr int NV = PN_MAX_MDOT;
    pn::pdl_wait();  // the projections come from the multi-dot launched before
    float cj[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) cj[v] = v < nv ? -float(add[v]) * inv_sigma : 0.0f;
    const float sc = float(S[S_SCALE]);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n8; i += 2 * stride) {
        const int64_t i2 = i + stride;
        const bool two = i2 < n8;
        float acc[2][8];
        {
            const float4 a = w[2 * i], b = w[2 * i + 1];
            const float4 c = two ? w[2 * i2] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 d = two ? w[2 * i2 + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float t0[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            const float t1[8] = {c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                acc[0][k] = t0[k];
                acc[1][k] = t1[k];
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v < nv) {
                const uint4 u0 = V16[v * vstride8 + i];
                const uint4 u1 = two ? V16[v * vstride8 + i2] : make_uint4(0u, 0u, 0u, 0u);
                float q0[8], q1[8];
                h8_to_f(u0, q0);
                h8_to_f(u1, q1);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    acc[0][k] = fmaf(cj[v], q0[k], acc[0][k]);
                    acc[1][k] = fmaf(cj[v], q1[k], acc[1][k]);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            if (g == 1 && !two) break;
            const int64_t ii = g == 0 ? i : i2;
            float hs[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                acc[g][k] *= sc;
                hs[k] = acc[g][k] * sigma;
            }
            V16_out[ii] = f_to_h8(hs);
            vcur[2 * ii] = make_float4(acc[g][0], acc[g][1], acc[g][2], acc[g][3]);
            vcur[2 * ii + 1] = make_float4(acc[g][4], acc[g][5], acc[g][6], acc[g][7]);
        }
    }
    pn::pdl_trigger();
}

// The multi-axpy of k_maxpy16 with its streams (w and the nv basis slices)
// staged like k_mdot16_tma: bulk copies of MD_CH-element chunks (every G-th
// chunk per block) into MD_ST shared slots; each thread
// combines 4 elements per chunk and writes V16_out and vcur directly.
template <int MD_CH, int MD_ST, int MINB>
__global__ void __launch_bounds__(256, MINB) k_maxpy16_tma(int64_t n, const float* w, const __half* V16,
                                                       int64_t vstride, int nv, const double* add, float inv_sigma,
                                                       float sigma, const double* S, __half* __restrict__ V16_out,
                                                       float* __restrict__ vcur, unsigned int* err) {
    constexpr int NV = PN_MAX_MDOT;
    extern __shared__ __align__(128) unsigned char mx_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(mx_raw) + 127) &
                                                           ~uintptr_t(127));
    float* sw = reinterpret_cast<float*>(base);                                  // [MD_ST][MD_CH]
    __half* sv = reinterpret_cast<__half*>(base + size_t(MD_ST) * MD_CH * 4);    // [MD_ST][NV][MD_CH]
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + size_t(MD_ST) * MD_CH * 4 + size_t(MD_ST) * NV * MD_CH * 2);
    const uint32_t bar_s = pn::mbar::smem_u32(bars);
    const int tid = threadIdx.x;
    // block b takes chunks b, b + G, b + 2G, ...: at any moment the blocks work
    // on neighbouring chunks, so each stream is read from one region of DRAM
    const int64_t nch = (n + MD_CH - 1) / MD_CH;
    const int64_t G = gridDim.x;
    const int64_t nk = nch > int64_t(blockIdx.x) ? (nch - blockIdx.x + G - 1) / G : 0;  // chunks of this block
    if (tid == 0) {
        for (int st = 0; st < MD_ST; ++st) pn::mbar::init(bar_s + 8u * st, 1u);
        pn::mbar::fence_init();
    }
    __syncthreads();
    auto issue = [&](int64_t c, int st) {
        const int64_t e0 = c * MD_CH;
        const int64_t rem = n - e0;
        const uint32_t cnt = uint32_t(rem < MD_CH ? rem : MD_CH);
        const uint32_t bar = bar_s + 8u * st;
        pn::mbar::arrive_expect_tx(bar, cnt * 4u + uint32_t(nv) * cnt * 2u);
        pn::mbar::bulk_g2s(pn::mbar::smem_u32(sw + st * MD_CH), w + e0, cnt * 4u, bar);
        for (int v = 0; v < nv; ++v)
            pn::mbar::bulk_g2s(pn::mbar::smem_u32(sv + (size_t(st) * NV + v) * MD_CH), V16 + v * vstride + e0,
                               cnt * 2u, bar);
    };
    // programmatic dependent launch: w (from the operator two launches back,
    // complete once the multi-dot before this kernel passed its own wait) and
    // the basis are copied before the wait for the multi-dot's projections
    if (tid == 0)
        for (int k = 0; k < MD_ST && k < nk; ++k) issue(blockIdx.x + k * G, k);
    pn::pdl_wait();
    float cj[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) cj[v] = v < nv ? -float(add[v]) * inv_sigma : 0.0f;
    const float sc = float(S[S_SCALE]);
    bool failed = false;
    for (int64_t kk = 0; kk < nk; ++kk) {
        const int64_t c = blockIdx.x + kk * G;
        const int k = int(kk);
        const int st = k % MD_ST;
        pn::mbar::wait(bar_s + 8u * st, uint32_t(k / MD_ST) & 1u, err, failed);
        const int64_t rem = n - c * MD_CH;
        const int64_t cnt = rem < MD_CH ? rem : MD_CH;
        for (int gq = tid; 4 * gq < cnt; gq += 256) {
            const float4 wv = reinterpret_cast<const float4*>(sw + st * MD_CH)[gq];
            float acc[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (v < nv) {
                    const uint2 hv = reinterpret_cast<const uint2*>(sv + (size_t(st) * NV + v) * MD_CH)[gq];
                    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&hv.x));
                    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hv.y));
                    acc[0] = fmaf(cj[v], a.x, acc[0]);
                    acc[1] = fmaf(cj[v], a.y, acc[1]);
                    acc[2] = fmaf(cj[v], b.x, acc[2]);
                    acc[3] = fmaf(cj[v], b.y, acc[3]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] *= sc;
            const int64_t e = c * MD_CH + 4 * gq;
            reinterpret_cast<float4*>(vcur + e)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            __half2 h01 = __floats2half2_rn(acc[0] * sigma, acc[1] * sigma);
            __half2 h23 = __floats2half2_rn(acc[2] * sigma, acc[3] * sigma);
            uint2 o;
            o.x = *reinterpret_cast<uint32_t*>(&h01);
            o.y = *reinterpret_cast<uint32_t*>(&h23);
            reinterpret_cast<uint2*>(V16_out + e)[0] = o;
        }
        __syncthreads();  // slot st is free again
        if (tid == 0 && kk + MD_ST < nk) issue(c + MD_ST * G, st);
    }
    pn::pdl_trigger();
}

// Launchers of the staged vector kernels: chunk size, slots and blocks per SM.
template <int CH, int ST, int MINB>
cudaError_t launch_md(int64_t n, const __half* V16, int nv, const float* w, float inv_sigma, double* partials,
                      unsigned int* ticket, double* H, int ldh, double* add, double* cs, double* sn, double* g, int j,
                      double* S, unsigned int* err, cudaStream_t s, bool pdl) {
    static std::atomic<unsigned long long> configured{0};
    {
        cudaError_t e = pn_smem_attr_once(configured, reinterpret_cast<const void*>(k_mdot16_tma<CH, ST, MINB>),
                                          int(md_smem_bytes<CH, ST>()));
        if (e != cudaSuccess) return e;
    }
    return pn::launch_pdl(pdl, k_mdot16_tma<CH, ST, MINB>, dim3(MINB * pn_sm_count()), dim3(256),
                          md_smem_bytes<CH, ST>(), s, n, V16, int64_t(n), nv, w, inv_sigma, partials, ticket, H, ldh,
                          add, cs, sn, g, j, S, err);
}

template <int CH, int ST, int MINB>
cudaError_t launch_mx(int64_t n, const float* w, const __half* V16, int nv, const double* add, float inv_sigma,
                      float sigma, const double* S, __half* V16_out, float* vcur, unsigned int* err, cudaStream_t s,
                      bool pdl) {
    static std::atomic<unsigned long long> configured{0};
    {
        cudaError_t e = pn_smem_attr_once(configured, reinterpret_cast<const void*>(k_maxpy16_tma<CH, ST, MINB>),
                                          int(md_smem_bytes<CH, ST>()));
        if (e != cudaSuccess) return e;
    }
    return pn::launch_pdl(pdl, k_maxpy16_tma<CH, ST, MINB>, dim3(MINB * pn_sm_count()), dim3(256),
                          md_smem_bytes<CH, ST>(), s, n, w, V16, int64_t(n), nv, add, inv_sigma, sigma, S, V16_out,
                          vcur, err);
}

// 1024-element chunks, two slots, three blocks per SM: the best of
// {512, 4, 3}, {1024, 3, 2}, {1024, 2, 3}, {2048, 3, 1} (chunk elements,
// slots, blocks per SM) on the P5 64^3 solve.
cudaError_t launch_mdot16_tma(int64_t n, const __half* V16, int nv, const float* w, float inv_sigma,
                              double* partials, unsigned int* ticket, double* H, int ldh, double* add, double* cs,
                              double* sn, double* g, int j, double* S, unsigned int* err, cudaStream_t s, bool pdl) {
    return launch_md<1024, 2, 3>(n, V16, nv, w, inv_sigma, partials, ticket, H, ldh, add, cs, sn, g, j, S, err, s,
                                 pdl);
}

cudaError_t launch_maxpy16_tma(int64_t n, const float* w, const __half* V16, int nv, const double* add,
                               float inv_sigma, float sigma, const double* S, __half* V16_out, float* vcur,
                               unsigned int* err, cudaStream_t s, bool pdl) {
    return launch_mx<1024, 2, 3>(n, w, V16, nv, add, inv_sigma, sigma, S, V16_out, vcur, err, s, pdl);
}

// First basis vector: r / beta (beta^2 = S[S_BETA2]) into V16_0 (scaled) and vcur.
__global__ void __launch_bounds__(256) k_first16(int64_t n8, const float4* r, float sigma, const double* S,
                                                 uint4* V16_0, float4* vcur) {
    const double b2 = S[S_BETA2];
    const float inv = b2 > 0.0 ? float(1.0 / sqrt(b2)) : 0.0f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n8; i += int64_t(gridDim.x) * blockDim.x) {
        const float4 a = r[2 * i], b = r[2 * i + 1];
        const float f[8] = {a.x * inv, a.y * inv, a.z * inv, a.w * inv, b.x * inv, b.y * inv, b.z * inv, b.w * inv};
        float hs[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) hs[k] = f[k] * sigma;
        V16_0[i] = f_to_h8(hs);
        vcur[2 * i] = make_float4(f[0], f[1], f[2], f[3]);
        vcur[2 * i + 1] = make_float4(f[4], f[5], f[6], f[7]);
    }
}

// x += sum_{i < nv} y_i V16_i / sigma (two 8-element groups loaded per iteration).
__global__ void __launch_bounds__(256) k_update16(int64_t n8, float4* __restrict__ x, const uint4* __restrict__ V16,
                                                  int64_t vstride8, int nv, const double* y, float inv_sigma) {
    constexpr int NV = PN_MAX_MDOT;
    float yj[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) yj[v] = v < nv ? float(y[v]) * inv_sigma : 0.0f;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n8; i += 2 * stride) {
        const int64_t i2 = i + stride;
        const bool two = i2 < n8;
        float acc[2][8];
        {
            const float4 a = x[2 * i], b = x[2 * i + 1];
            const float4 c = two ? x[2 * i2] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 d = two ? x[2 * i2 + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float t0[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            const float t1[8] = {c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                acc[0][k] = t0[k];
                acc[1][k] = t1[k];
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v < nv) {
                const uint4 u0 = V16[v * vstride8 + i];
                const uint4 u1 = two ? V16[v * vstride8 + i2] : make_uint4(0u, 0u, 0u, 0u);
                float q0[8], q1[8];
                h8_to_f(u0, q0);
                h8_to_f(u1, q1);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    acc[0][k] = fmaf(yj[v], q0[k], acc[0][k]);
                    acc[1][k] = fmaf(yj[v], q1[k], acc[1][k]);
                }
            }
        }
        x[2 * i] = make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
        x[2 * i + 1] = make_float4(acc[0][4], acc[0][5], acc[0][6], acc[0][7]);
        if (two) {
            x[2 * i2] = make_float4(acc[1][0], acc[1][1], acc[1][2], acc[1][3]);
            x[2 * i2 + 1] = make_float4(acc[1][4], acc[1][5], acc[1][6], acc[1][7]);
        }
    }
}

// Error approximations appended to each restart cycle (LGMRES: the cycle's
// search space is the m Krylov vectors plus the corrections x_i - x_{i-1} of
// the last k cycles, which carry the directions restarting loses).
#define PN_MAX_AUG 8
struct Aug {
    float* z = nullptr;  // ring of k + 1 FP32 vectors (n elements each)
    int k = 0;           // corrections appended per cycle
    int count = 0;       // stored so far (at most k)
    int newest = -1;     // ring slot of the latest
};
struct AugIn {
    const float4* z[PN_MAX_AUG];
};

// c = sum_{i < nv} y_i V16_i / sigma + sum_{a < na} y_{nv + a} Z_a;
// x += c; cout = c (the cycle's correction, the next error approximation).
__global__ void __launch_bounds__(256) k_update16_aug(int64_t n8, float4* __restrict__ x,
                                                      const uint4* __restrict__ V16, int64_t vstride8, int nv,
                                                      const double* y, float inv_sigma, AugIn za, int na,
                                                      float4* __restrict__ cout) {
    constexpr int NV = PN_MAX_MDOT;
    float yj[NV], ya[PN_MAX_AUG];
#pragma unroll
    for (int v = 0; v < NV; ++v) yj[v] = v < nv ? float(y[v]) * inv_sigma : 0.0f;
#pragma unroll
    for (int q = 0; q < PN_MAX_AUG; ++q) ya[q] = q < na ? float(y[nv + q]) : 0.0f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n8; i += int64_t(gridDim.x) * blockDim.x) {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v < nv) {
                float q[8];
                h8_to_f(V16[v * vstride8 + i], q);
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] = fmaf(yj[v], q[k], acc[k]);
            }
        }
#pragma unroll
        for (int q = 0; q < PN_MAX_AUG; ++q) {
            if (q < na) {
                const float4 a = za.z[q][2 * i], b = za.z[q][2 * i + 1];
                const float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] = fmaf(ya[q], f[k], acc[k]);
            }
        }
        const float4 xa = x[2 * i], xb = x[2 * i + 1];
        x[2 * i] = make_float4(xa.x + acc[0], xa.y + acc[1], xa.z + acc[2], xa.w + acc[3]);
        x[2 * i + 1] = make_float4(xb.x + acc[4], xb.y + acc[5], xb.z + acc[6], xb.w + acc[7]);
        cout[2 * i] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        cout[2 * i + 1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
}

// Keeps [base, base + bytes) resident in L2 for the launches of stream s while
// it lives, if it fits in L2: a persisting access-policy window (at most the
// device's persisting capacity; the hit ratio covers the rest of the window
// proportionally).  The
// stream is the solver's own (the handle's solve stream).  On destruction the
// window is closed, the persisting lines are released and the context's
// persisting-lines limit is put back.
struct L2Resident {
    cudaStream_t s = nullptr;
    bool on = false;
    size_t old_limit = 0;
    L2Resident(cudaStream_t st, void* base, size_t bytes, bool enable) : s(st) {
        if (!enable || bytes == 0 || st == nullptr) return;
        int dev = 0, maxp = 0, maxw = 0, l2 = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || maxp <= 0 || maxw <= 0) {
            cudaGetLastError();
            return;
        }
        // only vectors that fit in L2: a window over a sliver of larger ones
        // takes L2 from every other access (P7 256^3: 20.8 against 12.0 ms
        // per iteration)
        if (bytes > size_t(l2)) return;
        const size_t win = std::min(bytes, size_t(maxw));
        const size_t lim = std::min(win, size_t(maxp));
        if (cudaDeviceGetLimit(&old_limit, cudaLimitPersistingL2CacheSize) != cudaSuccess ||
            cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, lim) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        cudaStreamAttrValue v{};
        v.accessPolicyWindow.base_ptr = base;
        v.accessPolicyWindow.num_bytes = win;
        v.accessPolicyWindow.hitRatio = float(double(lim) / double(win));
        v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        if (cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &v) != cudaSuccess) {
            cudaGetLastError();
            cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
            return;
        }
        on = true;
    }
    ~L2Resident() {
        if (!on) return;
        cudaStreamAttrValue v{};
        v.accessPolicyWindow.num_bytes = 0;
        v.accessPolicyWindow.hitRatio = 0.0f;
        v.accessPolicyWindow.hitProp = cudaAccessPropertyNormal;
        v.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
        cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &v);
        cudaStreamSynchronize(s);
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
        cudaGetLastError();
    }
};

// Restarted GMRES(m), CGS1, FP32 arithmetic with the basis in FP16 (m <= 16).
// Same contract as gmres<float>.  With aug (k > 0) each cycle that has stored
// corrections appends up to k of them (newest first) after its m Krylov
// steps, as the flexible Arnoldi process allows (A Z = V H for the cycle's
// search directions Z), with m + k <= 16.
int gmres_f16(Ctx& c, float* x, const float* bvec, double bnorm2, double tol, int m, int max_iter, int check_every,
              int* iters, double* rel_out, Aug* aug = nullptr) {
    pn_handle* h = c.h;
    const int64_t n = h->n_elems;  // a multiple of 32
    const int64_t n8 = n / 8;
    const int nb = 8 * pn_sm_count();  // the FP16-basis streaming kernels: 8 CTAs per SM
    double* S = h->d_scalars;
    const float sigma = float(std::sqrt(double(h->n_active)));
    const float inv_sigma = 1.0f / sigma;
    const int ka = aug ? aug->k : 0;
    const int ms = m + ka;  // Hessenberg columns
    const size_t v16bytes = size_t(ms + 1) * n * sizeof(__half);
    const size_t fbytes = 2 * size_t(n) * sizeof(float);  // w and vcur
    const size_t vbytes = ((v16bytes + 255) / 256) * 256 + fbytes;
    const int ldh = ms + 1;
    const size_t dcount = size_t(ldh) * ms + 4 * size_t(ms + 1) + 16 * size_t(ms + 1);
    int rc = ensure_work(h, vbytes + dcount * sizeof(double) + 256);
    if (rc != PN_OK) return rc;
    __half* V16 = (__half*)h->d_work;
    float* w = (float*)((char*)h->d_work + ((v16bytes + 255) / 256) * 256);
    float* vcur = w + n;
    double* H = (double*)((char*)h->d_work + ((vbytes + 255) / 256) * 256);
    double* cs = H + size_t(ldh) * ms;
    double* sn = cs + (ms + 1);
    double* g = sn + (ms + 1);
    double* y = g + (ms + 1);
    double* add = y + (ms + 1);
    // w and vcur (adjacent): written and read again within every Arnoldi step
    L2Resident l2(c.s, w, 2 * size_t(n) * sizeof(float), h->l2_resident != 0);
    c.ok(cudaMemsetAsync(S + S_TICKET, 0, sizeof(double), c.s), "gmres16: ticket");
    const double bnorm = std::sqrt(bnorm2);
    const double target = tol * (bnorm > 0.0 ? bnorm : 1.0);
    const double ob = c.ob(pn::OP_APPLY, 4.0, false);
    int total = 0;
    double res = 0.0;
    const int every = check_every > 0 ? check_every : 1;
    const int64_t vs8 = n / 8;
    for (;;) {
        c.pb();
        c.lk(pn::launch_op(h, pn::OP_RESIDUAL, x, w, PN_F32, h->d_partials, c.s, bvec), "gmres16: residual",
             pn::op_launch_count(h, PN_F32));
        c.pe(PN_PROF_RESIDUAL, c.ob(pn::OP_RESIDUAL, 4.0, bvec != nullptr));
        c.pb();
        c.lk(pn::launch_reduce(h->d_partials, pn::op_partial_count(h, PN_F32), 1, S + S_BETA2, c.s),
             "gmres16: reduce");
        c.pe(PN_PROF_SCALAR, 0.0);
        double b2 = 0.0;
        if (!c.read(S_BETA2, 1, &b2)) return c.rc;
        res = std::sqrt(b2);
        if (!std::isfinite(res)) return pn_fail(h, PN_ERR_NONFINITE, "gmres16: non-finite residual");
        if (res <= target || total >= max_iter) break;
        c.pb();
        k_gm_init<<<1, 32, 0, c.s>>>(g, ms, S);
        k_first16<<<nb, 256, 0, c.s>>>(n8, (const float4*)w, sigma, S, (uint4*)V16, (float4*)vcur);
        c.launched("gmres16: init", 2);
        c.pe(PN_PROF_VECTOR, double(h->n_active) * (4.0 + 2.0 + 4.0));
        const int na = aug ? std::min(aug->count, ka) : 0;  // corrections appended to this cycle
        const int s = m + na;
        auto zaug = [&](int q) {  // q-th newest stored correction
            return aug->z + size_t((aug->newest - q + 2 * (ka + 1)) % (ka + 1)) * size_t(n);
        };
        int j = 0;
        for (; j < s && total < max_iter; ++j) {
            c.pb();
            const float* zin = j < m ? vcur : zaug(j - m);
            // the Arnoldi step's kernels (operator, multi-dot, multi-axpy) are
            // chained by programmatic dependent launch (pn_pdl.cuh)
            const bool pdl = h->pdl_enabled != 0;
            h->pdl = pdl ? 1 : 0;
            c.lk(pn::launch_op(h, pn::OP_APPLY, zin, w, PN_F32, nullptr, c.s), "gmres16: A v",
                 pn::op_launch_count(h, PN_F32));
            h->pdl = 0;
            c.pe(PN_PROF_APPLY, ob);
            c.pb();
            // staged from MD_MIN_NV basis vectors on (ncu, P5 64^3, cold: the
            // direct kernel is faster below, e.g. 24.0 against 33.9 us at one
            // vector; 90.8 against 77.2 us at sixteen)
            if ((h->stream_tma & 1) && j + 1 >= MD_MIN_NV) {
                c.ok(launch_mdot16_tma(n, V16, j + 1, w, inv_sigma, h->d_partials,
                                       reinterpret_cast<unsigned int*>(S + S_TICKET), H, ldh, add, cs, sn, g, j, S,
                                       reinterpret_cast<unsigned int*>(S + PN_S_FAULT), c.s, pdl),
                     "gmres16: mdot");
            } else {
                c.ok(pn::launch_pdl(pdl, k_mdot16_givens, dim3(nb_mdot()), dim3(256), 0, c.s, n8, (const uint4*)V16,
                                    vs8, j + 1, (const float4*)w, inv_sigma, h->d_partials,
                                    reinterpret_cast<unsigned int*>(S + S_TICKET), H, ldh, add, cs, sn, g, j, S),
                     "gmres16: mdot");
            }
            c.launched("gmres16: mdot");
            c.pe(PN_PROF_MDOT, double(h->n_active) * (2.0 * (j + 1) + 4.0));
            c.pb();
            if ((h->stream_tma & 2) && j + 1 >= MD_MIN_NV) {  // (23.3 against 30.5 us at one vector)
                c.ok(launch_maxpy16_tma(n, w, V16, j + 1, add, inv_sigma, sigma, S, V16 + size_t(j + 1) * n, vcur,
                                        reinterpret_cast<unsigned int*>(S + PN_S_FAULT), c.s, pdl),
                     "gmres16: maxpy");
            } else {
                c.ok(pn::launch_pdl(pdl, k_maxpy16, dim3(nb), dim3(256), 0, c.s, n8, (const float4*)w,
                                    (const uint4*)V16, vs8, j + 1, (const double*)add, inv_sigma, sigma,
                                    (const double*)S, (uint4*)V16 + int64_t(j + 1) * vs8, (float4*)vcur),
                     "gmres16: maxpy");
            }
            c.launched("gmres16: maxpy");
            c.pe(PN_PROF_MAXPY, double(h->n_active) * (4.0 + 2.0 * (j + 1) + 2.0 + 4.0));
            ++total;
            if ((j + 1) % every == 0 || j + 1 == s || total >= max_iter) {
                double r1 = 0.0;
                if (!c.read(S_RES, 1, &r1)) return c.rc;
                if (!std::isfinite(r1)) return pn_fail(h, PN_ERR_NONFINITE, "gmres16: non-finite Hessenberg");
                if (r1 <= target) {
                    ++j;
                    break;
                }
            }
        }
        c.pb();
        k_gm_backsolve<<<1, 128, 0, c.s>>>(H, ldh, g, y, j);
        if (aug && j > 0) {
            // x += V y + Z y_aug; the correction becomes the newest stored one
            const int nk = std::min(j, m), nz = j - nk;
            AugIn za{};
            for (int q = 0; q < nz; ++q) za.z[q] = (const float4*)zaug(q);
            const int slot = (aug->newest + 1) % (ka + 1);  // the oldest: not among the nz <= k read here
            k_update16_aug<<<nb, 256, 0, c.s>>>(n8, (float4*)x, (const uint4*)V16, vs8, nk, y, inv_sigma, za, nz,
                                                (float4*)(aug->z + size_t(slot) * size_t(n)));
            aug->newest = slot;
            aug->count = std::min(aug->count + 1, ka);
            c.launched("gmres16: update", 2);
            c.pe(PN_PROF_MAXPY, double(h->n_active) * (12.0 + 2.0 * nk + 4.0 * nz));
        } else {
            k_update16<<<nb, 256, 0, c.s>>>(n8, (float4*)x, (const uint4*)V16, vs8, j, y, inv_sigma);
            c.launched("gmres16: update", 2);
            c.pe(PN_PROF_MAXPY, double(h->n_active) * (8.0 + 2.0 * j));
        }
        if (c.rc != PN_OK) return c.rc;
    }
    *iters += total;
    *rel_out = bnorm > 0.0 ? res / bnorm : res;
    return c.rc;
}

// Restarted GMRES(m) for A x = b (b = Q if bvec is null).  tol is relative to
// ||b|| (bnorm2 = ||b||^2).  Adds the inner iterations to *iters.
template <typename T>
int gmres(Ctx& c, T* x, const T* bvec, double bnorm2, double tol, int m, int max_iter, int check_every,
          int* iters, double* rel_out, int ortho = PN_ORTHO_CGS2, struct pn_cnn* net = nullptr,
          int* papps = nullptr, int* fell_back = nullptr) {
    pn_handle* h = c.h;
    const int64_t n = h->n_elems;
    const int dt = sizeof(T) == 4 ? PN_F32 : PN_F64;
    const double es = sizeof(T);
    const int nb = nb_vec();
    double* S = h->d_scalars;
    // workspace: V (m+1 vectors), [Z (m vectors), preconditioner scratch],
    // then FP64 H ((m+1) x m), cs, sn, g, y, add
    if (net && (sizeof(T) != 4 || h->R % 8 || h->dims != 3)) net = nullptr;  // the network runs on FP32, R % 8 == 0
    const int64_t V3 = int64_t(h->R) * h->R * h->R;
    const size_t zbytes = net ? size_t(m) * n * sizeof(T) + size_t(V3) * (2 * h->K + 3) * sizeof(float) + 256 : 0;
    const size_t vbytes = size_t(m + 1) * n * sizeof(T) + zbytes;
    const int ldh = m + 1;
    const size_t dcount = size_t(ldh) * m + 4 * size_t(m + 1) + 16 * size_t(m + 1);
    int rc = ensure_work(h, vbytes + dcount * sizeof(double) + 256);
    if (rc != PN_OK) return rc;
    T* V = (T*)h->d_work;
    T* Zb = V + int64_t(m + 1) * n;
    float* pscratch = (float*)(((uintptr_t)(Zb + int64_t(m) * n) + 255) / 256 * 256);
    double* H = (double*)((char*)h->d_work + ((vbytes + 255) / 256) * 256);
    double* cs = H + size_t(ldh) * m;
    double* sn = cs + (m + 1);
    double* g = sn + (m + 1);
    double* y = g + (m + 1);
    double* add = y + (m + 1);
    // the fused CGS1 kernel's ticket counter starts at zero
    c.ok(cudaMemsetAsync(S + S_TICKET, 0, sizeof(double), c.s), "gmres: ticket");
    const double bnorm = std::sqrt(bnorm2);
    const double target = tol * (bnorm > 0.0 ? bnorm : 1.0);
    int total = 0;
    double res = 0.0, res_cycle = -1.0;
    const int every = check_every > 0 ? check_every : 1;
    for (;;) {
        // r = b - A x into V_0, beta = ||r||
        c.pb();
        c.lk(pn::launch_op(h, pn::OP_RESIDUAL, x, V, dt, h->d_partials, c.s, bvec), "gmres: residual", pn::op_launch_count(h, dt));
        c.pe(PN_PROF_RESIDUAL, c.ob(pn::OP_RESIDUAL, es, bvec != nullptr));
        c.pb();
        c.lk(pn::launch_reduce(h->d_partials, pn::op_partial_count(h, dt), 1, S + S_BETA2, c.s), "gmres: reduce");
        c.pe(PN_PROF_SCALAR, 0.0);
        double b2 = 0.0;
        if (!c.read(S_BETA2, 1, &b2)) return c.rc;
        res = std::sqrt(b2);
        if (!std::isfinite(res)) return pn_fail(h, PN_ERR_NONFINITE, "gmres: non-finite residual");
        if (res <= target || total >= max_iter) break;
        // fallback: a learned cycle that removed less than 10 % of the residual
        // hands the rest of the solve to plain GMRES
        if (net && res_cycle > 0.0 && res > 0.9 * res_cycle) {
            net = nullptr;
            if (fell_back) *fell_back = 1;
        }
        res_cycle = res;
        c.pb();
        k_gm_init<<<1, 32, 0, c.s>>>(g, m, S);
        c.launched("gmres: init");
        c.pe(PN_PROF_SCALAR, 0.0);
        c.pb();
        k_scale_invnorm<T><<<nb, 256, 0, c.s>>>(n, V, S, S_BETA2);
        c.launched("gmres: init");
        c.pe(PN_PROF_VECTOR, c.vb(2, es));
        int j = 0;
        for (; j < m && total < max_iter; ++j) {
            T* w = V + int64_t(j + 1) * n;
            const T* av = V + int64_t(j) * n;
            if (net) {
                // z_j = M(v_j); w = A z_j
                T* zj = Zb + int64_t(j) * n;
                c.pb();
                const int prc = pn::precond_apply(h, net, (const float*)av, (float*)zj, pscratch, S + S_PNRM, c.s);
                if (prc != PN_OK) return prc;
                c.launches += 36;
                c.pe(PN_PROF_PRECOND, 0.0);
                if (papps) ++*papps;
                av = zj;
            }
            c.pb();
            c.lk(pn::launch_op(h, pn::OP_APPLY, av, w, dt, nullptr, c.s), "gmres: A v", pn::op_launch_count(h, dt));
            c.pe(PN_PROF_APPLY, c.ob(pn::OP_APPLY, es, false));
            if (ortho == PN_ORTHO_CGS1 && sizeof(T) == 4 && j + 1 <= PN_MAX_MDOT) {
                // classical Gram-Schmidt once, one fused launch for the
                // projections, |w|^2, their reduction and the Givens update;
                // the new vector is normalised by the maxpy below
                c.pb();
                k_mdot_givens_f32<<<nb_mdot(), 256, 0, c.s>>>(
                    n / 4, (const float4*)V, n / 4, j + 1, (const float4*)w, h->d_partials,
                    reinterpret_cast<unsigned int*>(S + S_TICKET), H, ldh, add, cs, sn, g, j, S);
                c.launched("gmres: mdot");
                c.pe(PN_PROF_MDOT, c.vb(j + 2, es));
                c.pb();
                launch_maxpy<T>(nb, c.s, n, w, V, n, j + 1, add, -1.0, S + S_SCALE);
                c.launched("gmres: maxpy");
                c.pe(PN_PROF_MAXPY, c.vb(j + 3, es));
            } else if (ortho == PN_ORTHO_CGS1) {
                // classical Gram-Schmidt once: all projections and ||w||^2 in one
                // pass over the basis; the new vector is normalised by the last
                // update.  The projections stay unrotated in `add` (the Givens
                // kernel rotates the H column in place before the updates run).
                double* tmp0 = add + (m + 1);  // chunk 0: nv projections + ||w||^2
                const int nv0 = std::min(PN_MAX_MDOT, j + 1);
                for (int i0 = 0; i0 <= j; i0 += PN_MAX_MDOT) {
                    const int nv = std::min(PN_MAX_MDOT, j + 1 - i0);
                    c.pb();
                    launch_mdot<T>(h->red_blocks, c.s, n, V + int64_t(i0) * n, n, nv, w, h->d_partials, i0 == 0);
                    c.launched("gmres: mdot");
                    c.pe(PN_PROF_MDOT, c.vb(nv + 1, es));
                    c.pb();
                    c.lk(pn::launch_reduce(h->d_partials, h->red_blocks, i0 == 0 ? nv + 1 : nv,
                                           i0 == 0 ? tmp0 : add + i0, c.s),
                         "gmres: reduce");
                    c.pe(PN_PROF_SCALAR, 0.0);
                }
                c.pb();
                k_cgs1_gather<<<1, 32, 0, c.s>>>(H + int64_t(j) * ldh, add, tmp0, nv0, j, S);
                k_givens<<<1, 32, 0, c.s>>>(H, ldh, add, cs, sn, g, j, S, sizeof(T) == 4 ? 1 : 2);
                c.launched("gmres: givens", 2);
                c.pe(PN_PROF_SCALAR, 0.0);
                for (int i0 = 0; i0 <= j; i0 += PN_MAX_MDOT) {
                    const int nv = std::min(PN_MAX_MDOT, j + 1 - i0);
                    const bool last = i0 + PN_MAX_MDOT > j;
                    c.pb();
                    launch_maxpy<T>(nb, c.s, n, w, V + int64_t(i0) * n, n, nv, add + i0, -1.0,
                                    last ? S + S_SCALE : nullptr);
                    c.launched("gmres: maxpy");
                    c.pe(PN_PROF_MAXPY, c.vb(nv + 2, es));
                }
            } else {
                // classical Gram-Schmidt, twice
                for (int pass = 0; pass < 2; ++pass) {
                    double* hc = pass == 0 ? H + int64_t(j) * ldh : add;
                    for (int i0 = 0; i0 <= j; i0 += PN_MAX_MDOT) {
                        const int nv = std::min(PN_MAX_MDOT, j + 1 - i0);
                        c.pb();
                        launch_mdot<T>(h->red_blocks, c.s, n, V + int64_t(i0) * n, n, nv, w, h->d_partials);
                        c.launched("gmres: mdot");
                        c.pe(PN_PROF_MDOT, c.vb(nv + 1, es));
                        c.pb();
                        c.lk(pn::launch_reduce(h->d_partials, h->red_blocks, nv, hc + i0, c.s), "gmres: reduce");
                        c.pe(PN_PROF_SCALAR, 0.0);
                        c.pb();
                        launch_maxpy<T>(nb, c.s, n, w, V + int64_t(i0) * n, n, nv, hc + i0, -1.0);
                        c.launched("gmres: maxpy");
                        c.pe(PN_PROF_MAXPY, c.vb(nv + 2, es));
                    }
                }
                c.pb();
                c.lk2(pn::launch_dot(h, w, w, n, dt, S + S_NRM2, c.s), "gmres: norm");
                c.pe(PN_PROF_DOT, c.vb(1, es));
                c.pb();
                k_givens<<<1, 32, 0, c.s>>>(H, ldh, add, cs, sn, g, j, S, 0);
                c.launched("gmres: givens");
                c.pe(PN_PROF_SCALAR, 0.0);
                c.pb();
                k_scale_by<T><<<nb, 256, 0, c.s>>>(n, w, S, S_SCALE);
                c.launched("gmres: scale");
                c.pe(PN_PROF_VECTOR, c.vb(2, es));
            }
            ++total;
            if ((j + 1) % every == 0 || j + 1 == m || total >= max_iter) {
                double r1 = 0.0;
                if (!c.read(S_RES, 1, &r1)) return c.rc;
                if (!std::isfinite(r1)) return pn_fail(h, PN_ERR_NONFINITE, "gmres: non-finite Hessenberg");
                if (r1 <= target) {
                    ++j;
                    break;
                }
            }
        }
        // x += V y
        c.pb();
        k_gm_backsolve<<<1, 128, 0, c.s>>>(H, ldh, g, y, j);
        c.launched("gmres: backsolve");
        c.pe(PN_PROF_SCALAR, 0.0);
        const T* basis = net ? Zb : V;  // x += Z y (flexible) or V y
        for (int i0 = 0; i0 < j; i0 += PN_MAX_MDOT) {
            const int nv = std::min(PN_MAX_MDOT, j - i0);
            c.pb();
            launch_maxpy<T>(nb, c.s, n, x, basis + int64_t(i0) * n, n, nv, y + i0, 1.0);
            c.launched("gmres: update");
            c.pe(PN_PROF_MAXPY, c.vb(nv + 2, es));
        }
        if (c.rc != PN_OK) return c.rc;
    }
    *iters += total;
    *rel_out = bnorm > 0.0 ? res / bnorm : res;
    return c.rc;
}

int ir_gmres(Ctx& c, double* x, const pn_solve_opts& o, pn_solve_stats& st, struct pn_cnn* net = nullptr) {
    pn_handle* h = c.h;
    int fell_back = 0;
    const int64_t n = h->n_elems;
    // r64, the FP32 rhs / correction and the LGMRES ring live in the handle's
    // refinement workspace (outside the GMRES workspace): [r64][r32][d32][z ring]
    const int ka = (o.augment > 0 && o.basis == PN_BASIS_F16 && !net) ? o.augment : 0;
    const size_t b64 = size_t(n) * sizeof(double), b32 = size_t(n) * sizeof(float);  // n: a multiple of 32
    const size_t need = b64 + 2 * b32 + size_t(ka ? ka + 1 : 0) * b32;
    if (h->ir_bytes < need) {
        if (h->d_ir) cudaFree(h->d_ir);
        h->d_ir = nullptr;
        h->ir_bytes = 0;
        ++h->work_allocs;
        if (cudaMalloc(&h->d_ir, need) != cudaSuccess) {
            cudaGetLastError();
            h->d_ir = nullptr;
            return pn_fail(h, PN_ERR_ALLOC, "ir: cannot allocate the refinement vectors");
        }
        h->ir_bytes = need;
    }
    double* r64 = static_cast<double*>(h->d_ir);
    float* r32 = reinterpret_cast<float*>(static_cast<char*>(h->d_ir) + b64);
    float* d32 = r32 + n;
    // LGMRES corrections (FP16-basis inner solver): kept across restarts and
    // refinement steps (the same operator throughout)
    Aug aug;
    if (ka > 0) {
        aug.k = ka;
        aug.z = d32 + n;
    }
    const int nb = nb_vec();
    double* S = h->d_scalars;
    int outer = 0, inner = 0;
    double rel = 0.0;
    int rc = PN_OK;
    for (;;) {
        c.pb();
        c.lk(pn::launch_op(h, pn::OP_RESIDUAL, x, r64, PN_F64, h->d_partials, c.s), "ir: residual", pn::op_launch_count(h, PN_F64));
        c.pe(PN_PROF_RESIDUAL, c.ob(pn::OP_RESIDUAL, 8.0, false));
        c.pb();
        c.lk(pn::launch_reduce(h->d_partials, pn::op_partial_count(h, PN_F64), 1, S + S_RR, c.s), "ir: reduce");
        c.pe(PN_PROF_SCALAR, 0.0);
        double rr = 0.0;
        if (!c.read(S_RR, 1, &rr)) break;
        rel = rel_of(h, rr);
        if (!std::isfinite(rel)) {
            rc = pn_fail(h, PN_ERR_NONFINITE, "ir: non-finite residual");
            break;
        }
        if (rel <= o.tol || outer >= o.max_outer || inner >= o.max_iter) break;
        c.pb();
        k_to_f32_scaled<<<nb, 256, 0, c.s>>>(n, r32, r64, S, S_RR);
        k_zero<float><<<nb, 256, 0, c.s>>>(n, d32);
        c.launched("ir: convert", 2);
        c.pe(PN_PROF_VECTOR, c.vb(8.0 / 4.0 + 1.0 + 1.0, 4.0));
        // keep ||r|| for the correction: copy S_RR aside (GMRES reuses slots)
        cudaMemcpyAsync(S + S_MAXPY, S + S_RR, sizeof(double), cudaMemcpyDeviceToDevice, c.s);
        double inner_rel = 0.0;
        // inner tolerance: relative reduction, but not beyond what the outer target needs
        double itol = o.inner_tol;
        if (rel > 0.0 && o.tol / rel > itol) itol = std::min(0.5, o.tol / rel);
        if (o.basis == PN_BASIS_F16 && !net)
            rc = gmres_f16(c, d32, r32, 1.0, itol, o.restart, o.max_iter - inner, o.check_every, &inner, &inner_rel,
                           aug.k > 0 ? &aug : nullptr);
        else
            rc = gmres<float>(c, d32, r32, 1.0, itol, o.restart, o.max_iter - inner, o.check_every, &inner,
                              &inner_rel, o.ortho, net, &st.precond_applications, &fell_back);
        if (fell_back) net = nullptr;
        if (rc != PN_OK) break;
        c.pb();
        k_add_f32_scaled<<<nb, 256, 0, c.s>>>(n, x, d32, S, S_MAXPY);
        c.launched("ir: update");
        c.pe(PN_PROF_VECTOR, c.vb(2.0 * 8.0 + 4.0, 1.0));
        ++outer;
    }
    if (rc == PN_OK) rc = c.rc;
    st.iterations = inner;
    st.outer_iterations = outer;
    st.rel_residual = rel;
    st.fallback = fell_back;
    if (rc == PN_OK && rel > o.tol) rc = pn_fail(h, PN_ERR_NOT_CONVERGED, "ir: iteration cap reached");
    return rc;
}

}  // namespace

extern "C" int pn_get_workspace(const pn_handle* h, int64_t* bytes, int64_t* allocations) {
    if (!h) return PN_ERR_ARG;
    if (bytes) *bytes = int64_t(h->work_bytes + h->ir_bytes);
    if (allocations) *allocations = h->work_allocs;
    return PN_OK;
}

extern "C" int pn_solve(pn_handle* h, void* u, const pn_solve_opts* opts, pn_solve_stats* stats, void* stream) {
    if (!h) return PN_ERR_ARG;
    if (!u || !opts) return pn_fail(h, PN_ERR_ARG, "pn_solve: NULL argument");
    if (reinterpret_cast<uintptr_t>(u) & 15u) return pn_fail(h, PN_ERR_ARG, "pn_solve: u must be 16-byte aligned");
    const pn_solve_opts& o = *opts;
    if (!(o.tol > 0.0) || o.max_iter < 0) return pn_fail(h, PN_ERR_ARG, "pn_solve: bad tol or max_iter");
    if (o.solver != PN_SOLVER_CGLS && o.solver != PN_SOLVER_GMRES && o.solver != PN_SOLVER_IR_GMRES &&
        o.solver != PN_SOLVER_IR_FGMRES)
        return pn_fail(h, PN_ERR_ARG, "pn_solve: unknown solver");
    if (o.solver == PN_SOLVER_IR_FGMRES && !o.precond)
        return pn_fail(h, PN_ERR_ARG, "pn_solve: PN_SOLVER_IR_FGMRES needs opts->precond");
    if (o.solver == PN_SOLVER_IR_FGMRES && (h->dims != 3 || h->periodic))
        return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_solve: the learned preconditioner is 3D, vacuum boundary only");
    if (o.solver == PN_SOLVER_IR_FGMRES && h->R % 8)
        return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_solve: the learned preconditioner needs R % 8 == 0");
    if (o.solver < PN_SOLVER_IR_GMRES && o.precision != PN_F32 && o.precision != PN_F64)
        return pn_fail(h, PN_ERR_ARG, "pn_solve: bad precision");
    if (o.solver != PN_SOLVER_CGLS && (o.restart < 1 || o.restart > 200))
        return pn_fail(h, PN_ERR_ARG, "pn_solve: restart must be in [1, 200]");
    if (o.ortho != PN_ORTHO_CGS2 && o.ortho != PN_ORTHO_CGS1) return pn_fail(h, PN_ERR_ARG, "pn_solve: bad ortho");
    if (o.basis != PN_BASIS_F32 && o.basis != PN_BASIS_F16) return pn_fail(h, PN_ERR_ARG, "pn_solve: bad basis");
    if (o.basis == PN_BASIS_F16 && (o.solver != PN_SOLVER_IR_GMRES || o.restart > PN_MAX_MDOT))
        return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_solve: the FP16 basis needs PN_SOLVER_IR_GMRES and restart <= 16");
    if (o.augment < 0 || o.augment > PN_MAX_AUG) return pn_fail(h, PN_ERR_ARG, "pn_solve: augment must be in [0, 8]");
    if (o.augment > 0 && (o.basis != PN_BASIS_F16 || o.restart + o.augment > PN_MAX_MDOT))
        return pn_fail(h, PN_ERR_UNSUPPORTED,
                       "pn_solve: augment needs the FP16 basis (PN_SOLVER_IR_GMRES) and restart + augment <= 16");
    pn_solve_stats st{};
    // the solve runs on the handle's own stream, ordered after the caller's
    // stream on entry and before it on exit
    cudaStream_t user = (cudaStream_t)stream;
    if (!h->solve_s) {
        if (cudaStreamCreateWithFlags(&h->solve_s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
            cudaError_t e = cudaGetLastError();
            return pn_cuda_fail(h, e != cudaSuccess ? e : cudaErrorUnknown, "pn_solve: solve stream");
        }
    }
    if (cudaEventRecord(h->ev_in, user) != cudaSuccess || cudaStreamWaitEvent(h->solve_s, h->ev_in, 0) != cudaSuccess)
        return pn_cuda_fail(h, cudaGetLastError(), "pn_solve: stream join");
    Ctx c{h, h->solve_s};
    pn_prof_reset(h, o.profile != 0);
    const auto t0 = std::chrono::steady_clock::now();
    int rc;
    if (o.solver == PN_SOLVER_CGLS) {
        rc = o.precision == PN_F32 ? cgls<float>(c, (float*)u, o, st) : cgls<double>(c, (double*)u, o, st);
    } else if (o.solver == PN_SOLVER_GMRES) {
        int it = 0;
        double rel = 0.0;
        if (o.precision == PN_F32)
            rc = gmres<float>(c, (float*)u, nullptr, h->q_norm2, o.tol, o.restart, o.max_iter, o.check_every, &it, &rel,
                              o.ortho);
        else
            rc = gmres<double>(c, (double*)u, nullptr, h->q_norm2, o.tol, o.restart, o.max_iter, o.check_every, &it,
                               &rel, o.ortho);
        st.iterations = it;
        st.rel_residual = rel;
        if (rc == PN_OK && rel > o.tol) rc = pn_fail(h, PN_ERR_NOT_CONVERGED, "gmres: max_iter reached");
    } else {
        rc = ir_gmres(c, (double*)u, o, st,
                      o.solver == PN_SOLVER_IR_FGMRES ? static_cast<struct pn_cnn*>(o.precond) : nullptr);
    }
    if (cudaStreamSynchronize(c.s) == cudaSuccess) pn_prof_drain(h);
    h->prof_on = false;
    if (cudaEventRecord(h->ev_out, c.s) != cudaSuccess || cudaStreamWaitEvent(user, h->ev_out, 0) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        if (rc == PN_OK) rc = pn_cuda_fail(h, e, "pn_solve: stream join");
    }
    {
        // a bounded wait of the TMA-staged operator that ran out
        unsigned int fault = 0;
        if (cudaMemcpy(&fault, h->d_scalars + PN_S_FAULT, sizeof(fault), cudaMemcpyDeviceToHost) == cudaSuccess &&
            fault != 0) {
            cudaMemset(h->d_scalars + PN_S_FAULT, 0, sizeof(double));
            rc = pn_fail(h, PN_ERR_TIMEOUT, "pn_solve: a wait of the TMA-staged operator ran out");
        }
    }
    const auto t1 = std::chrono::steady_clock::now();
    st.seconds = std::chrono::duration<double>(t1 - t0).count();
    st.status = rc;
    st.launches = c.launches;
    if (stats) *stats = st;
    return rc;
}
