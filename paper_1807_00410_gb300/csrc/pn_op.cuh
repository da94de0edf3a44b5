// The staggered P_N operator at one output slot, shared by the single-system
// and batched kernels (appendix "Final equation"; half-cell central
// differences between the staggered grids, section "Precomputation";
// Dirichlet dropping, section "Runtime").
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pn_internal.h"

namespace pn {

template <typename T>
struct OpArgs {
    const T* x;
    T* y;
    const T* q;        // source planes (n_q) or null
    int n_q;
    const T* bvec;     // residual against this full vector instead of Q (or null)
    const T* st;       // clamped sigma_t at voxel centres, R^3
    const T* ss;       // sigma_s at voxel centres, R^3
    const Plane* planes;
    const Term* terms;
    int R;
    int nzb;           // z-slices of a plane box (R + 1; 1 for the 2D reduction)
    int periodic;      // 1: every axis wraps, R slots per axis for every class (test mode)
    int64_t pitch_x, pitch_y, plane_stride;
    double* partials;  // residual: per-block sums of r^2
};

template <typename T> __device__ __forceinline__ T term_coef(const Term& t);
template <> __device__ __forceinline__ float term_coef<float>(const Term& t) { return t.cf; }
template <> __device__ __forceinline__ double term_coef<double>(const Term& t) { return t.cd; }
template <typename T> __device__ __forceinline__ T plane_fl(const Plane& p);
template <> __device__ __forceinline__ float plane_fl<float>(const Plane& p) { return p.fl_f; }
template <> __device__ __forceinline__ double plane_fl<double>(const Plane& p) { return p.fl_d; }

// Rounding of each step pinned (no contraction left to the compiler), so that
// every kernel that forms an output from the same inputs -- this per-point
// form, the FP64 class-mean kernel -- gets the same bits.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Mean of a centre field over the in-domain voxel centres adjacent to slot
// (x, y, z) of a grid with parity bits (px, py, pz).  Along an odd axis the
// candidates are slots i-1 and i; clamping both into [0, R) repeats the single
// in-domain centre at a boundary face, which leaves the mean unchanged.
template <typename T>
__device__ __forceinline__ T centre_mean(const T* F, int R, int x, int y, int z, int px, int py, int pz) {
    const int x0 = px ? max(x - 1, 0) : x, x1 = px ? min(x, R - 1) : x;
    const int y0 = py ? max(y - 1, 0) : y, y1 = py ? min(y, R - 1) : y;
    const int z0 = pz ? max(z - 1, 0) : z, z1 = pz ? min(z, R - 1) : z;
    const int64_t R2 = int64_t(R) * R;
    T s = F[z0 * R2 + y0 * R + x0] + F[z0 * R2 + y0 * R + x1] + F[z0 * R2 + y1 * R + x0] +
          F[z0 * R2 + y1 * R + x1] + F[z1 * R2 + y0 * R + x0] + F[z1 * R2 + y0 * R + x1] +
          F[z1 * R2 + y1 * R + x0] + F[z1 * R2 + y1 * R + x1];
    return s * T(0.125);
}

// The same with every axis wrapping (periodic test mode): face i lies
// between centres i - 1 (mod R) and i.
template <typename T>
__device__ __forceinline__ T centre_mean_periodic(const T* F, int R, int x, int y, int z, int px, int py, int pz) {
    const int x0 = px ? (x + R - 1) % R : x, y0 = py ? (y + R - 1) % R : y, z0 = pz ? (z + R - 1) % R : z;
    const int64_t R2 = int64_t(R) * R;
    T s = F[z0 * R2 + y0 * R + x0] + F[z0 * R2 + y0 * R + x] + F[z0 * R2 + y * R + x0] + F[z0 * R2 + y * R + x] +
          F[z * R2 + y0 * R + x0] + F[z * R2 + y0 * R + x] + F[z * R2 + y * R + x0] + F[z * R2 + y * R + x];
    return s * T(0.125);
}

// One output of the operator at slot (x, y, z) of plane p (active slot).  The
// 2D reduction has no z terms, every plane has pz = 0 and z = 0, and its
// centre fields are R^2: the same code serves it.
template <typename T, int MODE>
__device__ __forceinline__ T op_point(const OpArgs<T>& a, int p, const Plane& P, int x, int y, int z, int64_t s) {
    const int R = a.R;
    const int64_t pbase = int64_t(p) * a.plane_stride;
    const T diag = a.periodic ? fma_rn(-plane_fl<T>(P), centre_mean_periodic(a.ss, R, x, y, z, P.px, P.py, P.pz),
                                       centre_mean_periodic(a.st, R, x, y, z, P.px, P.py, P.pz))
                              : fma_rn(-plane_fl<T>(P), centre_mean(a.ss, R, x, y, z, P.px, P.py, P.pz),
                                       centre_mean(a.st, R, x, y, z, P.px, P.py, P.pz));
    T acc = mul_rn(diag, a.x[pbase + s]);
    T tr = T(0);
    for (int ti = P.t0; ti < P.t1; ++ti) {
        const Term tm = a.terms[ti];
        int i, b;
        int64_t stride;
        if (tm.axis == 0) { i = x; b = P.px; stride = 1; }
        else if (tm.axis == 1) { i = y; b = P.py; stride = a.pitch_x; }
        else { i = z; b = P.pz; stride = a.pitch_y; }
        const int64_t qb = int64_t(tm.q) * a.plane_stride + s;
        // plus neighbour at slot i + 1 - b (exists iff < R + 1 - b),
        // minus neighbour at slot i - b (exists iff >= 0); periodic: both wrap mod R
        T vp, vm;
        if (a.periodic) {
            const int ip = (i + 1 - b) % R, im = (i - b + R) % R;
            vp = a.x[qb + (ip - i) * stride];
            vm = a.x[qb + (im - i) * stride];
        } else {
            vp = (i + 1 - b < R + 1 - b) ? a.x[qb + (1 - b) * stride] : T(0);
            vm = (i - b >= 0) ? a.x[qb - b * stride] : T(0);
        }
        tr = fma_rn(term_coef<T>(tm), sub_rn(vp, vm), tr);
    }
    acc = (MODE == OP_APPLY_T) ? sub_rn(acc, tr) : add_rn(acc, tr);
    if (MODE == OP_RESIDUAL) {
        const T bq = a.bvec ? a.bvec[pbase + s] : ((p < a.n_q) ? a.q[pbase + s] : T(0));
        return sub_rn(bq, acc);
    }
    return acc;
}

}  // namespace pn
