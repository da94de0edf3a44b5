// Batched solver: many P_N systems of different grid sizes and orders solved
// together (an extension of the paper's one-system solver).
//
// Every phase of the solve is ONE kernel launch over a work list that covers
// all instances: the operator over (instance, plane, slot chunk) items with
// each instance's own coupling table (so uneven N and R share a launch), the
// vector kernels over (instance, element chunk) items.  Each kernel is a
// persistent grid-stride loop over its list, sized to a multiple of the SM
// count.  Instances converge independently: per-instance flags on the device
// gate every item, and an instance whose GMRES residual estimate reaches its
// target freezes itself inside the cycle.
//
// The inner solver is GMRES(m) in FP32 with one classical Gram-Schmidt pass
// (projections and |w|^2 in one sweep, the new norm by Pythagoras), FP64
// reductions, Hessenberg matrix, Givens rotations and back-substitution per
// instance on the device.  One restart cycle (residual, m Arnoldi steps,
// back-substitution, correction update: 4 m + 5 launches) has no host
// synchronisation and is captured once as a CUDA graph, then replayed.  An
// FP64 iterative refinement wraps it: the FP64 residual r of each instance,
// an inner solve of A d = r / |r| to a relative target, x += |r| d.  The host
// reads the per-instance state once per cycle and once per refinement step.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "pn_internal.h"
#include "pn_op.cuh"

namespace {

constexpr int BM_MAX = 16;         // restart length limit (projections + |w|^2 in one pass)
constexpr int NV1 = BM_MAX + 1;    // values per vector chunk partial (slot BM_MAX: |w|^2)

struct BInst {
    // operator (from the handle)
    int R, K, n_q, nzb;
    int generic;     // 1: the Arnoldi-step operator runs in the generic batched launch
    int periodic;    // the handle's periodic test mode
    int64_t pitch_x, pitch_y, plane_stride, n;
    const pn::Plane* planes;
    const pn::Term* terms;
    const float* st_f;
    const float* ss_f;
    const double* st_d;
    const double* ss_d;
    const float* q_f;
    const double* q_d;
    // solver vectors (batch-owned)
    double* r64;
    float* r32;
    float* d32;
    float* V;        // m + 1 vectors of n elements
    // per-instance FP64 scalars
    double* H;       // (m + 1) x m, column j at H + j (m + 1)
    double* cs;
    double* sn;
    double* g;
    double* y;
    double* proj;
};

// Per-instance state.  Never read through __restrict__ / read-only-cache
// pointers: inside the persistent kernel other CTAs rewrite it between grid
// barriers.
struct BState {
    int run;         // takes part in the current inner solve
    int live;        // still iterating in the current cycle
    int kdim;        // Krylov dimension reached in the current cycle
    int done;        // refinement finished
    double target;   // inner target (the inner system has |b| = 1)
    double res;      // |g[kdim]|: the inner residual estimate
    double scale;    // 1 / |w| of the last Arnoldi step (1 / beta at cycle start)
    double rr;       // FP64 outer residual |Q - A x|^2
    double rnorm;    // |r| of the current refinement step
};

struct OpChunk {
    int inst, plane;
    int64_t s0;
};
struct VecChunk {
    int inst;
    int pad;
    int64_t e0;      // first element (multiple of 4)
};

enum Gate { G_LIVE = 0, G_RUN = 1, G_NOT_DONE = 2, G_ALL = 3, G_LIVE_GENERIC = 4 };

__device__ __forceinline__ bool gate_ok(const BState& s, int gate) {
    return gate == G_ALL || ((gate == G_LIVE || gate == G_LIVE_GENERIC) && s.live) || (gate == G_RUN && s.run) ||
           (gate == G_NOT_DONE && !s.done);
}

__device__ __forceinline__ double bsum(double v) {
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
    return v;  // thread 0
}

// y_i = op(x_i) for every instance whose gate is open; one FP64 partial of
// |y|^2 per chunk in residual mode (0 for closed chunks).
template <typename T, int MODE>
__device__ __forceinline__ void ph_op(const BInst* __restrict__ I, const BState* st,
                                      const OpChunk* __restrict__ ch, int nch, int64_t cho, const T* const* X,
                                      T* const* Y, const T* const* Bv, int gate, double* partials, int cta,
                                      int ncta) {
    for (int c = cta; c < nch; c += ncta) {
        const OpChunk k = ch[c];
        // uniform over the block
        const bool go = gate_ok(st[k.inst], gate) && (gate != G_LIVE_GENERIC || I[k.inst].generic);
        double racc = 0.0;
        if (go) {
            const BInst& in = I[k.inst];
            pn::OpArgs<T> a;
            a.x = X[k.inst];
            a.y = Y[k.inst];
            a.bvec = Bv ? Bv[k.inst] : nullptr;
            a.n_q = in.n_q;
            if constexpr (sizeof(T) == 4) {
                a.q = (const T*)in.q_f;
                a.st = (const T*)in.st_f;
                a.ss = (const T*)in.ss_f;
            } else {
                a.q = (const T*)in.q_d;
                a.st = (const T*)in.st_d;
                a.ss = (const T*)in.ss_d;
            }
            a.planes = in.planes;
            a.terms = in.terms;
            a.R = in.R;
            a.nzb = in.nzb;
            a.periodic = in.periodic;
            a.pitch_x = in.pitch_x;
            a.pitch_y = in.pitch_y;
            a.plane_stride = in.plane_stride;
            a.partials = nullptr;
            const int R = in.R;
            const pn::Plane P = in.planes[k.plane];
            const int64_t box = in.pitch_y * in.nzb;
            const int64_t pbase = int64_t(k.plane) * in.plane_stride;
            const int64_t s1 = min(k.s0 + cho, in.plane_stride);
            T rrun = T(0);
            int rcnt = 0;
            for (int64_t s = k.s0 + threadIdx.x; s < s1; s += blockDim.x) {
                const int x = int(s % in.pitch_x);
                const int64_t t = s / in.pitch_x;
                const int y = int(t % (R + 1));
                const int z = int(t / (R + 1));
                const int ext = in.periodic ? 0 : 1;
                const bool active = s < box && x < R + ext * P.px && y < R + ext * P.py && z < R + ext * P.pz;
                T out = T(0);
                if (active) {
                    out = pn::op_point<T, MODE>(a, k.plane, P, x, y, z, s);
                    if (MODE == pn::OP_RESIDUAL) {
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
            racc += double(rrun);
        }
        if (MODE == pn::OP_RESIDUAL && partials != nullptr) {
            const double bs = bsum(racc);
            if (threadIdx.x == 0) partials[c] = bs;
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) kb_op(const BInst* __restrict__ I, const BState* st,
                                             const OpChunk* __restrict__ ch, int nch, int64_t cho,
                                             const T* const* X, T* const* Y, const T* const* Bv, int gate,
                                             double* partials) {
    ph_op<T, MODE>(I, st, ch, nch, cho, X, Y, Bv, gate, partials, blockIdx.x, gridDim.x);
}

// Sums NV1 per-thread FP32 values over the block into out[0..NV1) (nv
// projections in slots 0..nv-1, the self-dot in slot BM_MAX): each warp adds
// its 32 values in FP32, the 8 warp sums are added in FP64.
__device__ __forceinline__ void block_sum_nv(const float (&part)[NV1], int nv, double* out) {
    __shared__ double red[NV1][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV1; ++v) {
        if (v < nv || v == BM_MAX) {
            float t = part[v];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) red[v][warp] = double(t);
        }
    }
    __syncthreads();
    if (threadIdx.x < NV1 && (int(threadIdx.x) < nv || threadIdx.x == BM_MAX)) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[threadIdx.x][q];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// partials[c][v] = chunk c's share of V_v . w (v <= j) and w . w (slot BM_MAX),
// w = V_{j+1}, for live instances (products summed per thread in FP32).
__device__ __forceinline__ void ph_mdot(const BInst* __restrict__ I, const BState* st,
                                        const VecChunk* __restrict__ ch, int nch, int64_t chv, int j,
                                        double* partials, int cta, int ncta) {
    const int nv = j + 1;
    for (int c = cta; c < nch; c += ncta) {
        const VecChunk k = ch[c];
        float part[NV1];
#pragma unroll
        for (int v = 0; v < NV1; ++v) part[v] = 0.0f;
        if (st[k.inst].live) {
            const BInst& in = I[k.inst];
            const int64_t n4 = in.n / 4;
            const float4* V = reinterpret_cast<const float4*>(in.V);
            const float4* w = V + int64_t(nv) * n4;
            const int64_t i0 = k.e0 / 4, i1 = min(i0 + chv / 4, n4);
            for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const float4 wi = w[i];
#pragma unroll
                for (int v = 0; v < BM_MAX; ++v) {
                    if (v < nv) {
                        const float4 q = V[int64_t(v) * n4 + i];
                        part[v] = fmaf(q.w, wi.w, fmaf(q.z, wi.z, fmaf(q.y, wi.y, fmaf(q.x, wi.x, part[v]))));
                    }
                }
                part[BM_MAX] = fmaf(wi.w, wi.w, fmaf(wi.z, wi.z, fmaf(wi.y, wi.y, fmaf(wi.x, wi.x, part[BM_MAX]))));
            }
        }
        block_sum_nv(part, nv, partials + int64_t(c) * NV1);
    }
}

__global__ void __launch_bounds__(256) kb_mdot(const BInst* __restrict__ I, const BState* st,
                                               const VecChunk* __restrict__ ch, int nch, int64_t chv, int j,
                                               double* partials) {
    ph_mdot(I, st, ch, nch, chv, j, partials, blockIdx.x, gridDim.x);
}

// Block-wide sums over one instance's chunk partials (256 threads, fixed
// assignment of chunks to threads and a fixed tree: deterministic): out[v]
// for v < nv, and out[BM_MAX] if `self`, of partials with `stride` values per
// chunk.  Must be called by every thread of the block.
__device__ __forceinline__ void block_chunk_sums(const double* partials, int stride, int first, int count, int nv,
                                                 bool self, double* out) {
    __shared__ double red[NV1][8];
    double acc[NV1];
#pragma unroll
    for (int v = 0; v < NV1; ++v) acc[v] = 0.0;
    for (int c = threadIdx.x; c < count; c += blockDim.x) {
        const double* p = partials + int64_t(first + c) * stride;
#pragma unroll
        for (int v = 0; v < NV1; ++v)
            if (v < nv || (self && v == BM_MAX)) acc[v] += p[v];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV1; ++v) {
        if (v < nv || (self && v == BM_MAX)) {
            double t = acc[v];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) red[v][warp] = t;
        }
    }
    __syncthreads();
    const int v = threadIdx.x;
    if (v < NV1 && (v < nv || (self && v == BM_MAX))) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[v][q];
        out[v] = t;
    }
    __syncthreads();
}

// Arnoldi bookkeeping of step j for every live instance (one block of 256
// threads per instance): projections and |w|^2 from the chunk partials,
// Hessenberg column, previous rotations, rotation j, residual estimate;
// freezes an instance that reached its target or the end of the cycle.
__device__ __forceinline__ void ph_givens(const BInst* __restrict__ I, BState* st, const int* vc_first,
                                          const int* vc_count, const double* partials, int j, int m, int inst) {
    BState& S = st[inst];
    if (!S.live) return;  // uniform over the block
    const BInst& in = I[inst];
    __shared__ double vals[NV1];
    // the column and the earlier rotations in shared memory: thread 0's
    // rotation chain then reads no global memory (on the global arrays, which
    // may alias, each step was a dependent round trip to L2)
    __shared__ double cc[BM_MAX + 2], css[BM_MAX], sns[BM_MAX];
    block_chunk_sums(partials, NV1, vc_first[inst], vc_count[inst], j + 1, true, vals);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        css[i] = in.cs[i];
        sns[i] = in.sn[i];
    }
    __syncthreads();
    const int ldh = m + 1;
    double* col = in.H + int64_t(j) * ldh;
    if (threadIdx.x == 0) {
        const double w2 = vals[BM_MAX];
        double hh = 0.0;
        for (int i = 0; i <= j; ++i) {
            cc[i] = vals[i];
            hh += vals[i] * vals[i];
        }
        // one Gram-Schmidt pass: |w - V h|^2 = |w|^2 - |h|^2 for orthonormal V
        double nrm2 = w2 - hh;
        if (!(nrm2 > 1e-12 * w2)) nrm2 = 0.0;  // breakdown: the Krylov space is invariant
        const double hn = sqrt(fmax(nrm2, 0.0));
        cc[j + 1] = hn;
        S.scale = hn > 0.0 ? 1.0 / hn : 0.0;
        for (int i = 0; i < j; ++i) {
            const double t = css[i] * cc[i] + sns[i] * cc[i + 1];
            cc[i + 1] = -sns[i] * cc[i] + css[i] * cc[i + 1];
            cc[i] = t;
        }
        const double a = cc[j], b = cc[j + 1];
        const double den = hypot(a, b);
        const double c = den > 0.0 ? a / den : 1.0;
        const double s = den > 0.0 ? b / den : 0.0;
        in.cs[j] = c;
        in.sn[j] = s;
        cc[j] = den;
        cc[j + 1] = 0.0;
        const double gj = in.g[j];
        in.g[j + 1] = -s * gj;
        in.g[j] = c * gj;
        S.res = fabs(-s * gj);
        S.kdim = j + 1;
        if (S.res <= S.target || j + 1 >= m || !(hn > 0.0)) S.live = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) {
        col[i] = cc[i];
        if (i <= j) in.proj[i] = vals[i];
    }
}

__global__ void kb_givens(const BInst* __restrict__ I, BState* st, const int* vc_first, const int* vc_count,
                          const double* partials, int j, int m) {
    ph_givens(I, st, vc_first, vc_count, partials, j, m, blockIdx.x);
}

// V_{j+1} = (V_{j+1} - sum_{i <= j} proj_i V_i) / |.| for live instances.
__device__ __forceinline__ void ph_maxpy(const BInst* __restrict__ I, const BState* st,
                                                const VecChunk* __restrict__ ch, int nch, int64_t chv, int j, int cta, int ncta) {
    const int nv = j + 1;
    for (int c = cta; c < nch; c += ncta) {
        const VecChunk k = ch[c];
        const BState& S = st[k.inst];
        if (!S.live) continue;
        const BInst& in = I[k.inst];
        float cj[BM_MAX];
#pragma unroll
        for (int v = 0; v < BM_MAX; ++v) cj[v] = v < nv ? -float(in.proj[v]) : 0.0f;
        const float sc = float(S.scale);
        const int64_t n4 = in.n / 4;
        float4* V = reinterpret_cast<float4*>(in.V);
        float4* w = V + int64_t(nv) * n4;
        const int64_t i0 = k.e0 / 4, i1 = min(i0 + chv / 4, n4);
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            float4 acc = w[i];
#pragma unroll
            for (int v = 0; v < BM_MAX; ++v) {
                if (v < nv) {
                    const float4 q = V[int64_t(v) * n4 + i];
                    acc.x = fmaf(cj[v], q.x, acc.x);
                    acc.y = fmaf(cj[v], q.y, acc.y);
                    acc.z = fmaf(cj[v], q.z, acc.z);
                    acc.w = fmaf(cj[v], q.w, acc.w);
                }
            }
            acc.x *= sc;
            acc.y *= sc;
            acc.z *= sc;
            acc.w *= sc;
            w[i] = acc;
        }
    }
}

__global__ void __launch_bounds__(256) kb_maxpy(const BInst* __restrict__ I, const BState* st,
                                                const VecChunk* __restrict__ ch, int nch, int64_t chv, int j)  {
    ph_maxpy(I, st, ch, nch, chv, j, blockIdx.x, gridDim.x);
}

// Cycle start, one block per running instance: beta = |r0| from the
// residual partials, g = beta e_0, 1 / beta for the first basis vector.
__device__ __forceinline__ void ph_cycle_init(const BInst* __restrict__ I, BState* st, const int* oc_first,
                                              const int* oc_count, const double* partials, int m, int inst) {
    BState& S = st[inst];
    if (!S.run) return;  // uniform over the block
    __shared__ double b2s[NV1];
    block_chunk_sums(partials, 1, oc_first[inst], oc_count[inst], 1, false, b2s);
    if (threadIdx.x != 0) return;
    const BInst& in = I[inst];
    const double beta = sqrt(fmax(b2s[0], 0.0));
    for (int i = 0; i <= m; ++i) in.g[i] = 0.0;
    in.g[0] = beta;
    S.res = beta;
    S.kdim = 0;
    S.scale = beta > 0.0 ? 1.0 / beta : 0.0;
    S.live = (beta > S.target && isfinite(beta)) ? 1 : 0;
}

__global__ void kb_cycle_init(const BInst* __restrict__ I, BState* st, const int* oc_first, const int* oc_count,
                              const double* partials, int m) {
    ph_cycle_init(I, st, oc_first, oc_count, partials, m, blockIdx.x);
}

// v *= scale on V_0 of live instances.
__device__ __forceinline__ void ph_scale0(const BInst* __restrict__ I, const BState* st,
                                                 const VecChunk* __restrict__ ch, int nch, int64_t chv, int cta, int ncta) {
    for (int c = cta; c < nch; c += ncta) {
        const VecChunk k = ch[c];
        const BState& S = st[k.inst];
        if (!S.live) continue;
        const BInst& in = I[k.inst];
        const float sc = float(S.scale);
        float4* v = reinterpret_cast<float4*>(in.V);
        const int64_t i0 = k.e0 / 4, i1 = min(i0 + chv / 4, in.n / 4);
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            float4 a = v[i];
            a.x *= sc;
            a.y *= sc;
            a.z *= sc;
            a.w *= sc;
            v[i] = a;
        }
    }
}

__global__ void __launch_bounds__(256) kb_scale0(const BInst* __restrict__ I, const BState* st,
                                                 const VecChunk* __restrict__ ch, int nch, int64_t chv)  {
    ph_scale0(I, st, ch, nch, chv, blockIdx.x, gridDim.x);
}

// y = H^{-1} g (kdim x kdim, upper triangular), one thread per instance.
__device__ __forceinline__ void ph_backsolve(const BInst* __restrict__ I, const BState* st, int m,
                                             int inst) {
    const BState& S = st[inst];
    if (!S.run) return;
    const BInst& in = I[inst];
    const int k = S.kdim, ldh = m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double t = in.g[i];
        for (int c = i + 1; c < k; ++c) t -= in.H[int64_t(c) * ldh + i] * in.y[c];
        const double d = in.H[int64_t(i) * ldh + i];
        in.y[i] = d != 0.0 ? t / d : 0.0;
    }
}

__global__ void kb_backsolve(const BInst* __restrict__ I, const BState* st, int n_inst, int m) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst < n_inst) ph_backsolve(I, st, m, inst);
}

// d += sum_{i < kdim} y_i V_i for running instances.
__device__ __forceinline__ void ph_update(const BInst* __restrict__ I, const BState* st,
                                                 const VecChunk* __restrict__ ch, int nch, int64_t chv, int cta, int ncta) {
    for (int c = cta; c < nch; c += ncta) {
        const VecChunk k = ch[c];
        const BState& S = st[k.inst];
        if (!S.run || S.kdim == 0) continue;
        const BInst& in = I[k.inst];
        const int nv = S.kdim;
        float yj[BM_MAX];
#pragma unroll
        for (int v = 0; v < BM_MAX; ++v) yj[v] = v < nv ? float(in.y[v]) : 0.0f;
        const int64_t n4 = in.n / 4;
        const float4* V = reinterpret_cast<const float4*>(in.V);
        float4* d = reinterpret_cast<float4*>(in.d32);
        const int64_t i0 = k.e0 / 4, i1 = min(i0 + chv / 4, n4);
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            float4 acc = d[i];
#pragma unroll
            for (int v = 0; v < BM_MAX; ++v) {
                if (v < nv) {
                    const float4 q = V[int64_t(v) * n4 + i];
                    acc.x = fmaf(yj[v], q.x, acc.x);
                    acc.y = fmaf(yj[v], q.y, acc.y);
                    acc.z = fmaf(yj[v], q.z, acc.z);
                    acc.w = fmaf(yj[v], q.w, acc.w);
                }
            }
            d[i] = acc;
        }
    }
}

__global__ void __launch_bounds__(256) kb_update(const BInst* __restrict__ I, const BState* st,
                                                 const VecChunk* __restrict__ ch, int nch, int64_t chv)  {
    ph_update(I, st, ch, nch, chv, blockIdx.x, gridDim.x);
}

// FP64 residual norms: rr = sum of the op partials, for unfinished instances.
__global__ void kb_outer_reduce(BState* st, const int* oc_first, const int* oc_count, const double* partials) {
    const int inst = blockIdx.x;
    BState& S = st[inst];
    if (S.done) return;  // uniform over the block
    __shared__ double t[NV1];
    block_chunk_sums(partials, 1, oc_first[inst], oc_count[inst], 1, false, t);
    if (threadIdx.x == 0) S.rr = t[0];
}

// r32 = r64 / |r|, d32 = 0 for running instances (|r| = sqrt(rr)).
__global__ void __launch_bounds__(256) kb_to_f32(const BInst* __restrict__ I, BState* st,
                                                 const VecChunk* __restrict__ ch, int nch, int64_t chv) {
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const VecChunk k = ch[c];
        const BState& S = st[k.inst];
        if (!S.run) continue;
        const BInst& in = I[k.inst];
        const double rn = sqrt(fmax(S.rr, 0.0));
        const double inv = rn > 0.0 ? 1.0 / rn : 0.0;
        const int64_t e1 = min(k.e0 + chv, in.n);
        for (int64_t i = k.e0 + threadIdx.x; i < e1; i += blockDim.x) {
            in.r32[i] = float(in.r64[i] * inv);
            in.d32[i] = 0.0f;
        }
    }
}

// x += |r| d for running instances.
__global__ void __launch_bounds__(256) kb_x_update(const BInst* __restrict__ I, const BState* st,
                                                   const VecChunk* __restrict__ ch, int nch, int64_t chv,
                                                   double* const* X) {
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const VecChunk k = ch[c];
        const BState& S = st[k.inst];
        if (!S.run) continue;
        const BInst& in = I[k.inst];
        const double rn = sqrt(fmax(S.rr, 0.0));
        double* x = X[k.inst];
        const int64_t e1 = min(k.e0 + chv, in.n);
        for (int64_t i = k.e0 + threadIdx.x; i < e1; i += blockDim.x) x[i] += rn * double(in.d32[i]);
    }
}

// ---- persistent mode: one cooperative launch per restart cycle ------------

// Grid barrier for a cooperative launch (every CTA resident).  Thread 0 of
// each CTA reads the generation, arrives, and the last arrival resets the
// count and advances the generation; the others wait for the generation to
// change.  The wait is bounded: after `limit` polls (each followed by a
// ~100 ns sleep) a CTA sets the error flag and returns false, and every CTA
// that sees the flag returns false too, so a kernel that cannot complete a
// barrier ends instead of hanging and the host reads PN_ERR_TIMEOUT.
struct GridBar {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

__device__ bool grid_sync(GridBar* bar, unsigned int expected, long long limit) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* vgen = &bar->gen;
        volatile int* verr = &bar->err;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            long long polls = 0;
            while (*vgen == g) {
                if (*verr || ++polls > limit) {
                    atomicExch(&bar->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        if (*verr) ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

struct CycleArgs {
    const BInst* I;
    BState* st;
    const OpChunk* opc;
    int nopc;
    int64_t cho;
    const VecChunk* vc;
    int nvc;
    int64_t chv;
    const int* oc_first;
    const int* oc_count;
    const int* vc_first;
    const int* vc_count;
    double* part_op;
    double* part_vec;
    void* const* ptrs;   // V_j of every instance at (j n), then r32, d32
    size_t p_r32, p_d32;
    int n, m;
    GridBar* bar;
    long long limit;
};

// One restart cycle of every running instance (the same phases as the
// captured graph, separated by grid barriers instead of kernel boundaries).
__global__ void __launch_bounds__(256, 2) kb_cycle_persistent(CycleArgs a) {
    const int cta = blockIdx.x, ncta = gridDim.x;
    const unsigned int nb = gridDim.x;
    const float* const* V = (const float* const*)a.ptrs;
    ph_op<float, pn::OP_RESIDUAL>(a.I, a.st, a.opc, a.nopc, a.cho, (const float* const*)(a.ptrs + a.p_d32),
                                  (float* const*)a.ptrs, (const float* const*)(a.ptrs + a.p_r32), G_RUN, a.part_op,
                                  cta, ncta);
    if (!grid_sync(a.bar, nb, a.limit)) return;
    for (int inst = cta; inst < a.n; inst += ncta)
        ph_cycle_init(a.I, a.st, a.oc_first, a.oc_count, a.part_op, a.m, inst);
    if (!grid_sync(a.bar, nb, a.limit)) return;
    ph_scale0(a.I, a.st, a.vc, a.nvc, a.chv, cta, ncta);
    if (!grid_sync(a.bar, nb, a.limit)) return;
    for (int j = 0; j < a.m; ++j) {
        ph_op<float, pn::OP_APPLY>(a.I, a.st, a.opc, a.nopc, a.cho, V + size_t(j) * a.n,
                                   (float* const*)(a.ptrs + size_t(j + 1) * a.n), nullptr, G_LIVE, nullptr, cta,
                                   ncta);
        if (!grid_sync(a.bar, nb, a.limit)) return;
        ph_mdot(a.I, a.st, a.vc, a.nvc, a.chv, j, a.part_vec, cta, ncta);
        if (!grid_sync(a.bar, nb, a.limit)) return;
        for (int inst = cta; inst < a.n; inst += ncta)
            ph_givens(a.I, a.st, a.vc_first, a.vc_count, a.part_vec, j, a.m, inst);
        if (!grid_sync(a.bar, nb, a.limit)) return;
        ph_maxpy(a.I, a.st, a.vc, a.nvc, a.chv, j, cta, ncta);
        if (!grid_sync(a.bar, nb, a.limit)) return;
    }
    for (int inst = cta * blockDim.x + threadIdx.x; inst < a.n; inst += ncta * blockDim.x)
        ph_backsolve(a.I, a.st, a.m, inst);
    if (!grid_sync(a.bar, nb, a.limit)) return;
    ph_update(a.I, a.st, a.vc, a.nvc, a.chv, cta, ncta);
}

// One barrier expecting `expected` arrivals (tests of the timeout path use
// expected > gridDim.x: the wait then runs out).
__global__ void kb_barrier_test(GridBar* bar, unsigned int expected, long long limit) {
    grid_sync(bar, expected, limit);
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace

struct pn_batch {
    int n = 0, m = 0;
    std::vector<pn_handle*> hs;
    std::vector<BInst> inst;
    BInst* d_inst = nullptr;
    BState* d_state = nullptr;
    BState* h_state = nullptr;  // pinned mirror
    // work lists
    int64_t cho = 16384, chv = 65536;
    int op_mult = 4, vec_mult = 4;  // CTAs per SM of the persistent grids
    std::vector<OpChunk> opc;
    std::vector<VecChunk> vc;
    std::vector<int> oc_first, oc_count, vc_first, vc_count;
    OpChunk* d_opc = nullptr;
    VecChunk* d_vc = nullptr;
    int* d_counts = nullptr;        // oc_first, oc_count, vc_first, vc_count (4 n ints)
    double* d_part_op = nullptr;    // opc.size()
    double* d_part_vec = nullptr;   // vc.size() * NV1
    size_t cap_opc = 0, cap_vc = 0;
    // pointer arrays: V_j of every instance ((m + 1) n), r32, d32, r64, x, and apply scratch
    void** d_ptrs = nullptr;
    size_t ptr_count = 0;
    // storage
    void* d_vecs = nullptr;
    double* d_scal = nullptr;
    cudaStream_t s = nullptr;
    cudaGraphExec_t cycle = nullptr;
    int mode = 0;                   // PN_BATCH_GRAPH or PN_BATCH_PERSISTENT
    // instances with at least this many unknowns fill the GPU alone: pn_batch_solve
    // solves them with pn_solve, a few at a time on their own streams (<= 0: none)
    int64_t solo_min = int64_t(1) << 18;
    int64_t graph_solo = -1;        // solo_min the captured cycle was built for (its tiled launches skip solo instances)
    bool lists_all = true;          // the work lists hold every instance (else the members of lists_solo)
    int64_t lists_solo = 0;
    int use_tiled = 1;              // Arnoldi-step operator: per-instance tiled launches on graph branches
    int n_tiled = 0, n_generic = 0;
    static constexpr int NSIDE = 8;
    cudaStream_t side[NSIDE] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[NSIDE] = {};
    int* d_zero = nullptr;          // a device 0: a gated launch that does nothing
    GridBar* d_bar = nullptr;
    long long spin_limit = 1LL << 24;  // barrier polls (~100 ns each) before PN_ERR_TIMEOUT
    std::string err;
};

namespace {

int bfail(pn_batch* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

int bcuda(pn_batch* b, cudaError_t e, const char* where) {
    return bfail(b, PN_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// pointer-array layout in d_ptrs (each block n entries)
enum { P_V0 = 0 };  // V_j at (P_V0 + j) n, j <= m
inline size_t p_r32(const pn_batch* b) { return size_t(b->m + 1) * b->n; }
inline size_t p_d32(const pn_batch* b) { return p_r32(b) + b->n; }
inline size_t p_r64(const pn_batch* b) { return p_d32(b) + b->n; }
inline size_t p_x(const pn_batch* b) { return p_r64(b) + b->n; }
inline size_t p_ax(const pn_batch* b) { return p_x(b) + b->n; }   // apply: inputs
inline size_t p_ay(const pn_batch* b) { return p_ax(b) + b->n; }   // apply: outputs
inline size_t p_total(const pn_batch* b) { return p_ay(b) + b->n; }

// The operator and vector work lists (chunks of every instance, or of the
// instances `members` selects: the others get empty ranges and no chunks).
int build_lists(pn_batch* b, const std::vector<char>* members = nullptr) {
    b->opc.clear();
    b->vc.clear();
    b->oc_first.assign(b->n, 0);
    b->oc_count.assign(b->n, 0);
    b->vc_first.assign(b->n, 0);
    b->vc_count.assign(b->n, 0);
    b->lists_all = members == nullptr;
    b->lists_solo = members ? b->solo_min : 0;
    for (int i = 0; i < b->n; ++i) {
        const BInst& in = b->inst[i];
        if (members && !(*members)[i]) {
            b->oc_first[i] = int(b->opc.size());
            b->vc_first[i] = int(b->vc.size());
            continue;
        }
        b->oc_first[i] = int(b->opc.size());
        for (int p = 0; p < in.K; ++p)
            for (int64_t s0 = 0; s0 < in.plane_stride; s0 += b->cho) b->opc.push_back(OpChunk{i, p, s0});
        b->oc_count[i] = int(b->opc.size()) - b->oc_first[i];
        b->vc_first[i] = int(b->vc.size());
        for (int64_t e0 = 0; e0 < in.n; e0 += b->chv) b->vc.push_back(VecChunk{i, 0, e0});
        b->vc_count[i] = int(b->vc.size()) - b->vc_first[i];
    }
    if (b->opc.size() > size_t(INT32_MAX / 2) || b->vc.size() > size_t(INT32_MAX / 2))
        return bfail(b, PN_ERR_TOO_LARGE, "pn_batch: work lists too long");
    cudaError_t e = cudaSuccess;
    if (b->opc.size() > b->cap_opc) {
        cudaFree(b->d_opc);
        cudaFree(b->d_part_op);
        b->d_opc = nullptr;
        b->d_part_op = nullptr;
        b->cap_opc = 0;
        if ((e = cudaMalloc(&b->d_opc, b->opc.size() * sizeof(OpChunk))) != cudaSuccess ||
            (e = cudaMalloc(&b->d_part_op, b->opc.size() * sizeof(double))) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, PN_ERR_ALLOC, "pn_batch: work list allocation");
        }
        b->cap_opc = b->opc.size();
    }
    if (b->vc.size() > b->cap_vc) {
        cudaFree(b->d_vc);
        cudaFree(b->d_part_vec);
        b->d_vc = nullptr;
        b->d_part_vec = nullptr;
        b->cap_vc = 0;
        if ((e = cudaMalloc(&b->d_vc, b->vc.size() * sizeof(VecChunk))) != cudaSuccess ||
            (e = cudaMalloc(&b->d_part_vec, b->vc.size() * NV1 * sizeof(double))) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, PN_ERR_ALLOC, "pn_batch: work list allocation");
        }
        b->cap_vc = b->vc.size();
    }
    std::vector<int> counts;
    counts.insert(counts.end(), b->oc_first.begin(), b->oc_first.end());
    counts.insert(counts.end(), b->oc_count.begin(), b->oc_count.end());
    counts.insert(counts.end(), b->vc_first.begin(), b->vc_first.end());
    counts.insert(counts.end(), b->vc_count.begin(), b->vc_count.end());
    if (!b->opc.empty())
        e = cudaMemcpy(b->d_opc, b->opc.data(), b->opc.size() * sizeof(OpChunk), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !b->vc.empty())
        e = cudaMemcpy(b->d_vc, b->vc.data(), b->vc.size() * sizeof(VecChunk), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_counts, counts.data(), counts.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch: uploading work lists");
    if (b->cycle) {
        cudaGraphExecDestroy(b->cycle);
        b->cycle = nullptr;
    }
    return PN_OK;
}

int grid_of(const pn_batch* b, size_t items, int mult) {
    const int64_t g = std::min<int64_t>(int64_t(items), int64_t(mult) * pn_sm_count());
    return int(std::max<int64_t>(g, 1));
}

// Kernel sequences (all on b->s).
void launch_op32(pn_batch* b, size_t px, size_t py, size_t pb, int gate, bool residual) {
    const int grid = grid_of(b, b->opc.size(), b->op_mult);
    const float* const* X = (const float* const*)(b->d_ptrs + px);
    float* const* Y = (float* const*)(b->d_ptrs + py);
    if (residual)
        kb_op<float, pn::OP_RESIDUAL><<<grid, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_opc, int(b->opc.size()),
                                                              b->cho, X, Y, (const float* const*)(b->d_ptrs + pb),
                                                              gate, b->d_part_op);
    else
        kb_op<float, pn::OP_APPLY><<<grid, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_opc, int(b->opc.size()),
                                                           b->cho, X, Y, nullptr, gate, nullptr);
}

// y_i = A_i V_j(i) -> V_{j+1}(i) for live instances: the tiled operator of
// every tiled-capable instance as its own launch on one of the side streams
// (independent graph branches that run concurrently), gated by the
// instance's live flag, and one generic launch for the others.
void launch_step_apply(pn_batch* b, int j, const int* const* live, const std::vector<char>* running = nullptr) {
    if (!b->use_tiled || b->n_tiled == 0) {
        launch_op32(b, size_t(P_V0 + j) * b->n, size_t(P_V0 + j + 1) * b->n, 0, G_LIVE, false);
        return;
    }
    cudaEventRecord(b->ev_fork, b->s);
    for (int k = 0; k < pn_batch::NSIDE; ++k) cudaStreamWaitEvent(b->side[k], b->ev_fork, 0);
    int q = 0;
    for (int i = 0; i < b->n; ++i) {
        const BInst& in = b->inst[i];
        if (in.generic || (running && !(*running)[i])) continue;
        pn::launch_tiled_gated(b->hs[i], pn::OP_APPLY, in.V + size_t(j) * in.n, in.V + size_t(j + 1) * in.n, nullptr,
                               nullptr, live[i], b->side[q++ % pn_batch::NSIDE]);
    }
    if (b->n_generic > 0)
        launch_op32(b, size_t(P_V0 + j) * b->n, size_t(P_V0 + j + 1) * b->n, 0, G_LIVE_GENERIC, false);
    for (int k = 0; k < pn_batch::NSIDE; ++k) {
        cudaEventRecord(b->ev_join[k], b->side[k]);
        cudaStreamWaitEvent(b->s, b->ev_join[k], 0);
    }
}

std::vector<const int*> live_flags(const pn_batch* b) {
    std::vector<const int*> f(b->n);
    for (int i = 0; i < b->n; ++i) f[i] = &b->d_state[i].live;
    return f;
}

void launch_cycle(pn_batch* b, const std::vector<char>* running = nullptr) {
    const int gv = grid_of(b, b->vc.size(), b->vec_mult);
    const int nch = int(b->vc.size());
    const int* oc_first = b->d_counts;
    const int* oc_count = b->d_counts + b->n;
    const int* vc_first = b->d_counts + 2 * b->n;
    const int* vc_count = b->d_counts + 3 * b->n;
    // V_0 = r32 - A d32, beta, V_0 /= beta
    launch_op32(b, p_d32(b), P_V0, p_r32(b), G_RUN, true);
    kb_cycle_init<<<b->n, 256, 0, b->s>>>(b->d_inst, b->d_state, oc_first, oc_count, b->d_part_op, b->m);
    kb_scale0<<<gv, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_vc, nch, b->chv);
    const std::vector<const int*> live = live_flags(b);
    for (int j = 0; j < b->m; ++j) {
        launch_step_apply(b, j, live.data(), running);
        kb_mdot<<<gv, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_vc, nch, b->chv, j, b->d_part_vec);
        kb_givens<<<b->n, 256, 0, b->s>>>(b->d_inst, b->d_state, vc_first, vc_count, b->d_part_vec, j, b->m);
        kb_maxpy<<<gv, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_vc, nch, b->chv, j);
    }
    kb_backsolve<<<(b->n + 63) / 64, 64, 0, b->s>>>(b->d_inst, b->d_state, b->n, b->m);
    kb_update<<<gv, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_vc, nch, b->chv);
}

// The captured restart cycle.  `members` (or null: every instance) selects the
// instances that get a tiled operator launch in it; the others (the ones
// pn_batch_solve hands to pn_solve) are left out instead of being launched
// gated in every Arnoldi step.
int ensure_graph(pn_batch* b, const std::vector<char>* members = nullptr) {
    if (b->cycle) return PN_OK;
    if (b->use_tiled && b->n_tiled > 0) {
        // one gated launch per tiled instance outside the capture (a device 0
        // flag: nothing runs) sets the kernels' shared-memory attributes
        for (int i = 0; i < b->n; ++i)
            if (!b->inst[i].generic)
                pn::launch_tiled_gated(b->hs[i], pn::OP_APPLY, b->inst[i].V, b->inst[i].V + b->inst[i].n, nullptr,
                                       nullptr, b->d_zero, b->s);
        const cudaError_t e0 = cudaStreamSynchronize(b->s);
        if (e0 != cudaSuccess) return bcuda(b, e0, "pn_batch: preparing the tiled operator");
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch: begin capture");
    launch_cycle(b, members);
    const cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(b->s, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bcuda(b, le, "pn_batch: capturing the cycle");
    }
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch: end capture");
    e = cudaGraphInstantiate(&b->cycle, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->cycle = nullptr;
        return bcuda(b, e, "pn_batch: instantiating the cycle graph");
    }
    return PN_OK;
}

// One cycle as a cooperative launch; PN_ERR_TIMEOUT when a barrier wait ran out.
int launch_persistent(pn_batch* b) {
    // resident CTAs per SM, cached per device ordinal
    static std::atomic<int> occ_cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, PN_ERR_CUDA, "pn_batch: cudaGetDevice failed");
    }
    int occ = (dev >= 0 && dev < 64) ? occ_cache[dev].load(std::memory_order_relaxed) : 0;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_cycle_persistent, 256, 0) != cudaSuccess ||
            occ < 1) {
            cudaGetLastError();
            return bfail(b, PN_ERR_CUDA, "pn_batch: the persistent kernel cannot be resident");
        }
        if (dev >= 0 && dev < 64) occ_cache[dev].store(occ, std::memory_order_relaxed);
    }
    const int grid = std::max(1, std::min(occ * pn_sm_count(), int(std::max(b->opc.size(), b->vc.size()))));
    CycleArgs a;
    a.I = b->d_inst;
    a.st = b->d_state;
    a.opc = b->d_opc;
    a.nopc = int(b->opc.size());
    a.cho = b->cho;
    a.vc = b->d_vc;
    a.nvc = int(b->vc.size());
    a.chv = b->chv;
    a.oc_first = b->d_counts;
    a.oc_count = b->d_counts + b->n;
    a.vc_first = b->d_counts + 2 * b->n;
    a.vc_count = b->d_counts + 3 * b->n;
    a.part_op = b->d_part_op;
    a.part_vec = b->d_part_vec;
    a.ptrs = b->d_ptrs;
    a.p_r32 = p_r32(b);
    a.p_d32 = p_d32(b);
    a.n = b->n;
    a.m = b->m;
    a.bar = b->d_bar;
    a.limit = b->spin_limit;
    cudaError_t e = cudaMemsetAsync(b->d_bar, 0, sizeof(GridBar), b->s);
    void* args[] = {&a};
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void*)kb_cycle_persistent, dim3(grid), dim3(256), args, 0, b->s);
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch: persistent cycle launch");
    GridBar hb{};
    e = cudaMemcpyAsync(&hb, b->d_bar, sizeof(GridBar), cudaMemcpyDeviceToHost, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch: persistent cycle");
    if (hb.err) return bfail(b, PN_ERR_TIMEOUT, "pn_batch: a grid barrier wait ran out in the persistent cycle");
    return PN_OK;
}

void free_batch(pn_batch* b) {
    if (b->cycle) cudaGraphExecDestroy(b->cycle);
    void* ptrs[] = {b->d_inst, b->d_state, b->d_opc, b->d_vc, b->d_counts, b->d_part_op, b->d_part_vec,
                    b->d_ptrs, b->d_vecs, b->d_scal, b->d_bar};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->h_state) cudaFreeHost(b->h_state);
    for (int k = 0; k < pn_batch::NSIDE; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->d_zero) cudaFree(b->d_zero);
    if (b->s) cudaStreamDestroy(b->s);
}

int read_state(pn_batch* b) {
    cudaError_t e = cudaMemcpyAsync(b->h_state, b->d_state, size_t(b->n) * sizeof(BState), cudaMemcpyDeviceToHost, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch: reading the instance state");
    return PN_OK;
}

int write_state(pn_batch* b) {
    const cudaError_t e =
        cudaMemcpyAsync(b->d_state, b->h_state, size_t(b->n) * sizeof(BState), cudaMemcpyHostToDevice, b->s);
    return e == cudaSuccess ? PN_OK : bcuda(b, e, "pn_batch: writing the instance state");
}

}  // namespace

extern "C" {

int pn_batch_create(pn_batch** out, pn_handle* const* handles, int count, int restart, void* stream) {
    if (!out) return PN_ERR_ARG;
    *out = nullptr;
    if (!handles || count < 1 || restart < 1 || restart > BM_MAX) return PN_ERR_ARG;
    for (int i = 0; i < count; ++i)
        if (!handles[i]) return PN_ERR_ARG;
    pn_batch* b = new (std::nothrow) pn_batch();
    if (!b) return PN_ERR_ALLOC;
    b->n = count;
    b->m = restart;
    b->hs.assign(handles, handles + count);
    cudaStreamSynchronize((cudaStream_t)stream);
    int rc = PN_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete b;
        return PN_ERR_CUDA;
    }
    // storage: per instance (m + 1 + 2) FP32 and one FP64 vector, FP64 scalars
    const int m = restart, ldh = m + 1;
    const size_t scal_per = size_t(ldh) * m + 5 * size_t(m + 1);
    size_t bytes = 0;
    std::vector<size_t> off(count);
    for (int i = 0; i < count; ++i) {
        off[i] = bytes;
        bytes += size_t(handles[i]->n_elems) * (4 * (m + 3) + 8);
        bytes = size_t(round_up(int64_t(bytes), 256));
    }
    if ((e = cudaMalloc(&b->d_vecs, bytes)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_scal, scal_per * count * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_inst, count * sizeof(BInst))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_state, count * sizeof(BState))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_counts, 4 * size_t(count) * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_bar, sizeof(GridBar))) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_state, count * sizeof(BState))) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        delete b;
        return PN_ERR_ALLOC;
    }
    cudaMemsetAsync(b->d_vecs, 0, bytes, b->s);
    cudaMemsetAsync(b->d_scal, 0, scal_per * count * sizeof(double), b->s);
    b->ptr_count = p_total(b);
    if ((e = cudaMalloc(&b->d_ptrs, b->ptr_count * sizeof(void*))) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        delete b;
        return PN_ERR_ALLOC;
    }
    for (int k = 0; k < pn_batch::NSIDE && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_zero, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_zero, 0, sizeof(int), b->s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        delete b;
        return PN_ERR_CUDA;
    }
    b->inst.resize(count);
    std::vector<void*> ptrs(b->ptr_count, nullptr);
    for (int i = 0; i < count; ++i) {
        const pn_handle* h = handles[i];
        BInst& in = b->inst[i];
        in.R = h->R;
        in.K = h->K;
        in.n_q = h->n_q_planes;
        in.generic = pn::tiled_serves(h) ? 0 : 1;
        in.periodic = h->periodic;
        if (in.generic) ++b->n_generic;
        else ++b->n_tiled;
        in.nzb = int(h->nz_box);
        in.pitch_x = h->pitch_x;
        in.pitch_y = h->pitch_y;
        in.plane_stride = h->plane_stride;
        in.n = h->n_elems;
        in.planes = h->d_planes;
        in.terms = h->d_terms;
        in.st_f = h->d_st_f;
        in.ss_f = h->d_ss_f;
        in.st_d = h->d_st_d;
        in.ss_d = h->d_ss_d;
        in.q_f = h->d_q_f;
        in.q_d = h->d_q_d;
        char* base = (char*)b->d_vecs + off[i];
        in.V = (float*)base;
        in.r32 = in.V + size_t(m + 1) * in.n;
        in.d32 = in.r32 + in.n;
        in.r64 = (double*)(in.d32 + in.n);
        double* sc = b->d_scal + scal_per * i;
        in.H = sc;
        in.cs = in.H + size_t(ldh) * m;
        in.sn = in.cs + (m + 1);
        in.g = in.sn + (m + 1);
        in.y = in.g + (m + 1);
        in.proj = in.y + (m + 1);
        for (int j = 0; j <= m; ++j) ptrs[size_t(P_V0 + j) * count + i] = in.V + size_t(j) * in.n;
        ptrs[p_r32(b) + i] = in.r32;
        ptrs[p_d32(b) + i] = in.d32;
        ptrs[p_r64(b) + i] = in.r64;
    }
    e = cudaMemcpy(b->d_inst, b->inst.data(), count * sizeof(BInst), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ptrs, ptrs.data(), ptrs.size() * sizeof(void*), cudaMemcpyHostToDevice);
    std::memset(b->h_state, 0, count * sizeof(BState));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_state, b->h_state, count * sizeof(BState), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_batch(b);
        delete b;
        return PN_ERR_CUDA;
    }
    rc = build_lists(b);
    if (rc == PN_OK) {
        e = cudaStreamSynchronize(b->s);
        if (e != cudaSuccess) rc = PN_ERR_CUDA;
    }
    if (rc != PN_OK) {
        free_batch(b);
        delete b;
        return rc;
    }
    *out = b;
    return PN_OK;
}

int pn_batch_destroy(pn_batch* b) {
    if (!b) return PN_OK;
    free_batch(b);
    delete b;
    return PN_OK;
}

const char* pn_batch_last_error(const pn_batch* b) { return b ? b->err.c_str() : ""; }

int pn_batch_set_tiling(pn_batch* b, int64_t op_chunk, int64_t vec_chunk, int op_ctas_per_sm, int vec_ctas_per_sm) {
    if (!b) return PN_ERR_ARG;
    if (op_chunk < 256 || op_chunk % 256 || vec_chunk < 1024 || vec_chunk % 1024 || op_ctas_per_sm < 1 ||
        op_ctas_per_sm > 64 || vec_ctas_per_sm < 1 || vec_ctas_per_sm > 64)
        return bfail(b, PN_ERR_ARG, "pn_batch_set_tiling: chunks must be multiples of 256 (op) / 1024 (vector), "
                                    "CTAs per SM in [1, 64]");
    b->cho = op_chunk;
    b->chv = vec_chunk;
    b->op_mult = op_ctas_per_sm;
    b->vec_mult = vec_ctas_per_sm;
    return build_lists(b);
}

int pn_batch_set_solo(pn_batch* b, long long min_unknowns) {
    if (!b) return PN_ERR_ARG;
    b->solo_min = int64_t(min_unknowns);
    return PN_OK;
}

int pn_batch_set_mode(pn_batch* b, int mode, long long spin_limit) {
    if (!b) return PN_ERR_ARG;
    if ((mode != PN_BATCH_GRAPH && mode != PN_BATCH_PERSISTENT) || spin_limit < 1)
        return bfail(b, PN_ERR_ARG, "pn_batch_set_mode: bad mode or spin limit");
    b->mode = mode;
    b->spin_limit = spin_limit;
    return PN_OK;
}

int pn_batch_set_op_path(pn_batch* b, int tiled) {
    if (!b) return PN_ERR_ARG;
    b->use_tiled = tiled ? 1 : 0;
    if (b->cycle) {
        cudaGraphExecDestroy(b->cycle);
        b->cycle = nullptr;
    }
    return PN_OK;
}

int pn_batch_get_op_path(const pn_batch* b, int* tiled) {
    if (!b || !tiled) return PN_ERR_ARG;
    *tiled = (b->use_tiled && b->n_tiled > 0) ? 1 : 0;
    return PN_OK;
}

int pn_batch_barrier_test(int blocks, int expected, long long spin_limit, int* timed_out, void* stream) {
    if (blocks < 1 || expected < blocks || spin_limit < 1 || !timed_out) return PN_ERR_ARG;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_barrier_test, 256, 0) != cudaSuccess ||
        blocks > occ * pn_sm_count()) {
        cudaGetLastError();
        return PN_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    GridBar* bar = nullptr;
    if (cudaMalloc(&bar, sizeof(GridBar)) != cudaSuccess) {
        cudaGetLastError();
        return PN_ERR_ALLOC;
    }
    unsigned int ex = unsigned(expected);
    long long lim = spin_limit;
    void* args[] = {&bar, &ex, &lim};
    GridBar hb{};
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void*)kb_barrier_test, dim3(blocks), dim3(256), args, 0, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(bar);
    if (e != cudaSuccess) return PN_ERR_CUDA;
    *timed_out = hb.err ? 1 : 0;
    return hb.err ? PN_ERR_TIMEOUT : PN_OK;
}

int pn_batch_get_tiling(const pn_batch* b, int64_t* op_chunk, int64_t* vec_chunk, int* op_ctas_per_sm,
                        int* vec_ctas_per_sm) {
    if (!b) return PN_ERR_ARG;
    if (op_chunk) *op_chunk = b->cho;
    if (vec_chunk) *vec_chunk = b->chv;
    if (op_ctas_per_sm) *op_ctas_per_sm = b->op_mult;
    if (vec_ctas_per_sm) *vec_ctas_per_sm = b->vec_mult;
    return PN_OK;
}

int pn_batch_tune(pn_batch* b, void* stream) {
    if (!b) return PN_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch_tune");
    // the instances of the batched launches under the current solo threshold
    // (pn_batch_solve hands the others to pn_solve): the tiling is chosen for
    // the work lists those launches sweep
    std::vector<char> members(b->n, 1);
    int n_members = b->n;
    for (int i = 0; i < b->n; ++i)
        if (b->solo_min > 0 && b->hs[i]->n_active >= b->solo_min) {
            members[i] = 0;
            --n_members;
        }
    const std::vector<char>* mem = (n_members > 0 && n_members < b->n) ? &members : nullptr;
    // every member live for the timing; the basis holds whatever it holds
    for (int i = 0; i < b->n; ++i) {
        std::memset(&b->h_state[i], 0, sizeof(BState));
        b->h_state[i].run = b->h_state[i].live = (mem == nullptr || members[i]) ? 1 : 0;
    }
    int rc = write_state(b);
    if (rc != PN_OK) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, PN_ERR_CUDA, "pn_batch_tune: events");
    }
    const int jmid = b->m / 2;
    const std::vector<const int*> live = live_flags(b);
    auto time_it = [&](int what) -> float {  // 0: vector kernels, 1: generic operator, 2: tiled branches
        const int gv = grid_of(b, b->vc.size(), b->vec_mult);
        const int nch = int(b->vc.size());
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            // the Givens kernel freezes instances (the basis is arbitrary
            // here): every repetition starts with every instance live
            if (what == 0 && write_state(b) != PN_OK) return -1.0f;
            cudaEventRecord(e0, b->s);
            if (what == 1) {
                launch_op32(b, size_t(P_V0) * b->n, size_t(P_V0 + 1) * b->n, 0, G_LIVE, false);
            } else if (what == 2) {
                const int keep = b->use_tiled;
                b->use_tiled = 1;
                launch_step_apply(b, 0, live.data(), mem);
                b->use_tiled = keep;
            } else {
                kb_mdot<<<gv, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_vc, nch, b->chv, jmid, b->d_part_vec);
                kb_givens<<<b->n, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_counts + 2 * b->n,
                                                  b->d_counts + 3 * b->n, b->d_part_vec, jmid, b->m);
            }
            cudaEventRecord(e1, b->s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (what == 0) {
                // the multi-axpy as a second segment, every instance live again
                if (write_state(b) != PN_OK) return -1.0f;
                cudaEventRecord(e0, b->s);
                kb_maxpy<<<gv, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_vc, nch, b->chv, jmid);
                cudaEventRecord(e1, b->s);
                if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
                float ms2 = 0.0f;
                cudaEventElapsedTime(&ms2, e0, e1);
                ms += ms2;
            }
            if (rep > 0) best = std::min(best, ms);  // the first run warms up
        }
        return best;
    };
    const int64_t op_chunks[] = {4096, 16384, 65536};
    const int64_t vec_chunks[] = {16384, 65536, 262144};
    const int mults[] = {2, 4, 8};
    int64_t bo = b->cho, bv = b->chv;
    int bmo = b->op_mult, bmv = b->vec_mult;
    float best_op = 1e30f, best_vec = 1e30f;
    for (int64_t oc : op_chunks)
        for (int mu : mults) {
            b->cho = oc;
            b->op_mult = mu;
            if ((rc = build_lists(b, mem)) != PN_OK) break;
            const float t = time_it(1);
            if (t < 0.0f) {
                rc = bcuda(b, cudaGetLastError(), "pn_batch_tune");
                break;
            }
            if (t < best_op) {
                best_op = t;
                bo = oc;
                bmo = mu;
            }
        }
    b->cho = bo;
    b->op_mult = bmo;
    if (rc == PN_OK && (rc = build_lists(b, mem)) == PN_OK && b->n_tiled > 0) {
        // the Arnoldi-step operator: per-instance tiled launches vs the generic launch
        const float tt = time_it(2);
        if (tt < 0.0f) rc = bcuda(b, cudaGetLastError(), "pn_batch_tune");
        else b->use_tiled = tt < best_op ? 1 : 0;
    }
    for (int64_t vcn : vec_chunks) {
        if (rc != PN_OK) break;
        for (int mu : mults) {
            b->chv = vcn;
            b->vec_mult = mu;
            if ((rc = build_lists(b, mem)) != PN_OK) break;
            const float t = time_it(0);
            if (t < 0.0f) {
                rc = bcuda(b, cudaGetLastError(), "pn_batch_tune");
                break;
            }
            if (t < best_vec) {
                best_vec = t;
                bv = vcn;
                bmv = mu;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chv = bv;
    b->vec_mult = bmv;
    const int rc2 = build_lists(b, mem);
    std::memset(b->h_state, 0, size_t(b->n) * sizeof(BState));
    const int rc3 = write_state(b);
    e = cudaStreamSynchronize(b->s);
    if (rc != PN_OK) return rc;
    if (rc2 != PN_OK) return rc2;
    if (rc3 != PN_OK) return rc3;
    return e == cudaSuccess ? PN_OK : bcuda(b, e, "pn_batch_tune");
}

int pn_batch_apply(pn_batch* b, const void* const* x, void* const* y, int dtype, void* stream) {
    if (!b) return PN_ERR_ARG;
    if (!x || !y || (dtype != PN_F32 && dtype != PN_F64)) return bfail(b, PN_ERR_ARG, "pn_batch_apply: bad argument");
    for (int i = 0; i < b->n; ++i) {
        if (!x[i] || !y[i] || x[i] == y[i]) return bfail(b, PN_ERR_ARG, "pn_batch_apply: NULL or aliased vector");
        if ((reinterpret_cast<uintptr_t>(x[i]) | reinterpret_cast<uintptr_t>(y[i])) & 15u)
            return bfail(b, PN_ERR_ARG, "pn_batch_apply: vectors must be 16-byte aligned");
    }
    cudaStream_t us = (cudaStream_t)stream;
    if (!b->lists_all) {
        // the last solve left the solo instances out of the work lists
        const cudaError_t es = cudaStreamSynchronize(b->s);
        if (es != cudaSuccess) return bcuda(b, es, "pn_batch_apply");
        const int rl = build_lists(b);
        if (rl != PN_OK) return rl;
    }
    // the pointer arrays are batch-owned: order after earlier work on b->s
    std::vector<const void*> p(2 * size_t(b->n));
    for (int i = 0; i < b->n; ++i) {
        p[i] = x[i];
        p[b->n + i] = y[i];
    }
    cudaError_t e = cudaStreamSynchronize(b->s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_ptrs + p_ax(b), p.data(), p.size() * sizeof(void*), cudaMemcpyHostToDevice, us);
    if (e == cudaSuccess) e = cudaStreamSynchronize(us);  // the host array p dies with this call
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch_apply");
    const int grid = grid_of(b, b->opc.size(), b->op_mult);
    if (dtype == PN_F32)
        kb_op<float, pn::OP_APPLY><<<grid, 256, 0, us>>>(b->d_inst, b->d_state, b->d_opc, int(b->opc.size()), b->cho,
                                                         (const float* const*)(b->d_ptrs + p_ax(b)),
                                                         (float* const*)(b->d_ptrs + p_ay(b)), nullptr, G_ALL,
                                                         nullptr);
    else
        kb_op<double, pn::OP_APPLY><<<grid, 256, 0, us>>>(b->d_inst, b->d_state, b->d_opc, int(b->opc.size()),
                                                          b->cho, (const double* const*)(b->d_ptrs + p_ax(b)),
                                                          (double* const*)(b->d_ptrs + p_ay(b)), nullptr, G_ALL,
                                                          nullptr);
    e = cudaGetLastError();
    return e == cudaSuccess ? PN_OK : bcuda(b, e, "pn_batch_apply");
}

int pn_batch_solve(pn_batch* b, double* const* u, const pn_solve_opts* opts, pn_solve_stats* stats, void* stream) {
    if (!b) return PN_ERR_ARG;
    if (!u || !opts || !stats) return bfail(b, PN_ERR_ARG, "pn_batch_solve: NULL argument");
    const pn_solve_opts o = *opts;
    if (o.solver != PN_SOLVER_IR_GMRES) return bfail(b, PN_ERR_UNSUPPORTED, "pn_batch_solve: only PN_SOLVER_IR_GMRES is batched");
    if (o.restart != b->m) return bfail(b, PN_ERR_ARG, "pn_batch_solve: opts->restart must equal the batch's restart");
    if (o.basis != PN_BASIS_F32) return bfail(b, PN_ERR_UNSUPPORTED, "pn_batch_solve: the batch keeps an FP32 basis");
    if (!(o.tol > 0.0) || o.max_iter < 1 || o.max_outer < 1 || !(o.inner_tol > 0.0))
        return bfail(b, PN_ERR_ARG, "pn_batch_solve: bad tolerances or caps");
    for (int i = 0; i < b->n; ++i)
        if (!u[i] || (reinterpret_cast<uintptr_t>(u[i]) & 15u))
            return bfail(b, PN_ERR_ARG, "pn_batch_solve: NULL or misaligned u");
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);  // u is ready
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch_solve");
    e = cudaMemcpyAsync(b->d_ptrs + p_x(b), u, size_t(b->n) * sizeof(void*), cudaMemcpyHostToDevice, b->s);
    if (e != cudaSuccess) return bcuda(b, e, "pn_batch_solve");
    const int n = b->n;
    // the instances pn_solve takes (b->solo_min unknowns or more; see below)
    std::vector<char> solo(n, 0), members(n, 1);
    int n_members = n;  // instances of the batched launches
    for (int i = 0; i < n; ++i)
        if (b->solo_min > 0 && b->hs[i]->n_active >= b->solo_min) {
            solo[i] = 1;
            members[i] = 0;
            --n_members;
        }
    if (b->cycle && b->graph_solo != b->solo_min) {
        cudaGraphExecDestroy(b->cycle);
        b->cycle = nullptr;
    }
    // work lists of the batched instances only: the kernels that sweep them
    // (every Arnoldi step) then never visit a solo instance's chunks
    int rc = PN_OK;
    if (n_members < n && (b->lists_all || b->lists_solo != b->solo_min))
        rc = build_lists(b, &members);
    else if (n_members == n && !b->lists_all)
        rc = build_lists(b);
    if (rc != PN_OK) return rc;
    rc = b->mode == PN_BATCH_GRAPH ? ensure_graph(b, &members) : PN_OK;
    if (rc != PN_OK) return rc;
    b->graph_solo = b->solo_min;
    std::vector<int> inner(n, 0), outer(n, 0), status(n, PN_OK);
    std::vector<double> rel(n, 0.0);
    int64_t launches = 0;
    // Instances large enough to fill the GPU alone (b->solo_min unknowns) gain
    // nothing from sharing launches: they are solved first by pn_solve with
    // the same refinement and inner GMRES (FP32 basis, one
    // Gram-Schmidt pass, the batch's restart), and left out of the batched
    // launches (marked done).
    // kSoloWorkers host threads take them, largest first, each on its own
    // stream (side streams, idle until the batched cycles): every pn_solve
    // synchronises with the host between its restart cycles, and the other
    // solve's kernels fill those gaps.  Each solve runs on its own handle and
    // stream, so its result does not depend on the other.
    std::vector<pn_solve_stats> solo_st(n);
    std::vector<int> order;
    for (int i = 0; i < n; ++i)
        if (solo[i]) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int c) { return b->hs[a]->n_active > b->hs[c]->n_active; });
    std::atomic<int> next{0};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return bcuda(b, e, "pn_batch_solve");
    auto worker = [&](cudaStream_t ws) {
        cudaSetDevice(dev);  // the current device is per host thread
        for (int q = next.fetch_add(1); q < int(order.size()); q = next.fetch_add(1)) {
            const int i = order[q];
            pn_solve_opts os = o;
            os.solver = PN_SOLVER_IR_GMRES;
            os.basis = PN_BASIS_F32;
            os.ortho = PN_ORTHO_CGS1;
            os.augment = 0;
            os.profile = 0;
            os.precond = nullptr;
            std::memset(&solo_st[i], 0, sizeof(pn_solve_stats));
            const int r = pn_solve(b->hs[i], u[i], &os, &solo_st[i], ws);
            solo_st[i].status = r;
        }
    };
    constexpr int kSoloWorkers = 3;
    static_assert(kSoloWorkers <= pn_batch::NSIDE, "one side stream per worker");
    std::vector<std::thread> helpers;
    for (int t = 1; t < kSoloWorkers && t < int(order.size()); ++t) {
        try {
            helpers.emplace_back(worker, b->side[t]);
        } catch (...) {
            break;  // fewer threads: the running ones take what is left
        }
    }
    worker(b->side[0]);
    for (auto& t : helpers) t.join();
    for (int i = 0; i < n; ++i)
        if (solo[i]) launches += solo_st[i].launches;
    for (int i = 0; i < n; ++i) {
        BState& S = b->h_state[i];
        std::memset(&S, 0, sizeof(BState));
        S.done = solo[i];
    }
    rc = write_state(b);
    if (rc != PN_OK) return rc;
    const int gv = grid_of(b, b->vc.size(), b->vec_mult);
    const int nch = int(b->vc.size());
    const int* oc_first = b->d_counts;
    const int* oc_count = b->d_counts + n;
    for (int step = 0;; ++step) {
        // FP64 residual of every unfinished instance
        const int grid = grid_of(b, b->opc.size(), b->op_mult);
        kb_op<double, pn::OP_RESIDUAL><<<grid, 256, 0, b->s>>>(
            b->d_inst, b->d_state, b->d_opc, int(b->opc.size()), b->cho, (const double* const*)(b->d_ptrs + p_x(b)),
            (double* const*)(b->d_ptrs + p_r64(b)), nullptr, G_NOT_DONE, b->d_part_op);
        kb_outer_reduce<<<n, 256, 0, b->s>>>(b->d_state, oc_first, oc_count, b->d_part_op);
        launches += 2;
        if ((e = cudaGetLastError()) != cudaSuccess) return bcuda(b, e, "pn_batch_solve: residual");
        if ((rc = read_state(b)) != PN_OK) return rc;
        int left = 0;
        for (int i = 0; i < n; ++i) {
            BState& S = b->h_state[i];
            S.run = 0;
            if (S.done) continue;
            const double q2 = b->hs[i]->q_norm2;
            rel[i] = q2 > 0.0 ? std::sqrt(S.rr / q2) : std::sqrt(S.rr);
            if (!std::isfinite(rel[i])) {
                status[i] = PN_ERR_NONFINITE;
                S.done = 1;
            } else if (rel[i] <= o.tol) {
                S.done = 1;
            } else if (outer[i] >= o.max_outer || inner[i] >= o.max_iter) {
                status[i] = PN_ERR_NOT_CONVERGED;
                S.done = 1;
            } else {
                double itol = o.inner_tol;
                if (rel[i] > 0.0 && o.tol / rel[i] > itol) itol = std::min(0.5, o.tol / rel[i]);
                S.target = itol;
                S.run = 1;
                ++left;
            }
        }
        if ((rc = write_state(b)) != PN_OK) return rc;
        if (left == 0) break;
        kb_to_f32<<<gv, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_vc, nch, b->chv);
        ++launches;
        // inner GMRES cycles (graph replays) until every running instance met its target
        for (;;) {
            int n_run = 0;
            for (int i = 0; i < n; ++i) n_run += b->h_state[i].run ? 1 : 0;
            if (b->mode == PN_BATCH_GRAPH && 4 * n_run <= n_members && b->use_tiled && b->n_tiled > 0) {
                // few of the batched instances left: launch this cycle
                // directly, with tiled operator launches for the running
                // instances only (the captured graph would launch every
                // member's, gated).  The solo instances do not count: the
                // graph has no launches of theirs.
                std::vector<char> running(n);
                for (int i = 0; i < n; ++i) running[i] = b->h_state[i].run ? 1 : 0;
                launch_cycle(b, &running);
                if ((e = cudaGetLastError()) != cudaSuccess) return bcuda(b, e, "pn_batch_solve: cycle");
                launches += 4 * int64_t(b->m) + 5;
            } else if (b->mode == PN_BATCH_GRAPH) {
                if ((e = cudaGraphLaunch(b->cycle, b->s)) != cudaSuccess) return bcuda(b, e, "pn_batch_solve: cycle");
                launches += 4 * int64_t(b->m) + 5;
            } else {
                if ((rc = launch_persistent(b)) != PN_OK) return rc;
                launches += 1;
            }
            if ((rc = read_state(b)) != PN_OK) return rc;
            int running = 0;
            bool changed = false;
            for (int i = 0; i < n; ++i) {
                BState& S = b->h_state[i];
                if (!S.run) continue;
                inner[i] += S.kdim;
                if (!std::isfinite(S.res)) {
                    status[i] = PN_ERR_NONFINITE;
                    S.run = 0;
                    changed = true;
                } else if (S.res <= S.target || S.kdim == 0 || inner[i] >= o.max_iter) {
                    S.run = 0;
                    changed = true;
                } else {
                    ++running;
                }
            }
            if (running == 0) {
                // every unfinished instance took part in this step: all get x += |r| d
                for (int i = 0; i < n; ++i) b->h_state[i].run = b->h_state[i].done ? 0 : 1;
                if ((rc = write_state(b)) != PN_OK) return rc;
                break;
            }
            if (changed && (rc = write_state(b)) != PN_OK) return rc;
        }
        kb_x_update<<<gv, 256, 0, b->s>>>(b->d_inst, b->d_state, b->d_vc, nch, b->chv,
                                          (double* const*)(b->d_ptrs + p_x(b)));
        ++launches;
        for (int i = 0; i < n; ++i)
            if (!b->h_state[i].done) ++outer[i];
    }
    if ((e = cudaStreamSynchronize(b->s)) != cudaSuccess) return bcuda(b, e, "pn_batch_solve");
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int worst = PN_OK;
    for (int i = 0; i < n; ++i) {
        pn_solve_stats& st = stats[i];
        std::memset(&st, 0, sizeof(st));
        if (solo[i]) {
            st = solo_st[i];
            status[i] = st.status;
        } else {
            st.status = status[i];
            st.iterations = inner[i];
            st.outer_iterations = outer[i];
            st.rel_residual = rel[i];
        }
        st.seconds = secs;
        st.launches = launches;
        if (status[i] != PN_OK && worst == PN_OK) worst = status[i];
    }
    if (worst != PN_OK) bfail(b, worst, "pn_batch_solve: not every instance converged (see the per-instance status)");
    return worst;
}

}  // extern "C"
