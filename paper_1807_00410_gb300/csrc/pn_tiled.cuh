// Tables and arguments shared by the two tiled FP32 operator kernels
// (register-staged, pn_apply_tiled.cu; TMA-staged, pn_apply_tma.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pn_couplings.h"
#include "pn_internal.h"

namespace pn {
namespace tiled {

constexpr int TX = 32;
constexpr int NG = 4;          // thread groups: (bx, by) in {0,1}^2
constexpr int MAXT = 10;       // max transport terms per row per axis
constexpr int MAXC = 10;       // max coefficients per class (N <= 7)

struct ClassRow {
    int k, l;
    int nt[3];
    int j[3][MAXT];     // index of the input within the neighbour class along that axis
    float c[3][MAXT];   // A_d (dimensionless; 1/h applied per output)
};
struct ClassTab {
    int n;
    int plane0;
    ClassRow row[MAXC];
};
struct Tab {
    int K;
    int maxc;
    ClassTab cls[8];
};

constexpr Tab make_tab(int N) {
    Tab t{};
    t.K = (N + 1) * (N + 1);
    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int cls_of_k[64] = {};
    int j_of_k[64] = {};
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m) {
            const int k = l * l + l + m;
            const int c = cpl::parity_class(l, m);
            cls_of_k[k] = c;
            j_of_k[k] = cnt[c]++;
        }
    int base = 0;
    for (int c = 0; c < 8; ++c) {
        t.cls[c].n = cnt[c];
        t.cls[c].plane0 = base;
        base += cnt[c];
        if (cnt[c] > t.maxc) t.maxc = cnt[c];
    }
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m) {
            const int k = l * l + l + m;
            ClassRow& r = t.cls[cls_of_k[k]].row[j_of_k[k]];
            r.k = k;
            r.l = l;
            const cpl::RowTerms rt = cpl::row_terms(N, l, m);
            for (int i = 0; i < rt.n; ++i) {
                const int a = rt.t[i].axis;
                const int kp = rt.t[i].lp * rt.t[i].lp + rt.t[i].lp + rt.t[i].mp;
                r.j[a][r.nt[a]] = j_of_k[kp];
                r.c[a][r.nt[a]] = float(rt.t[i].coef);
                r.nt[a]++;
            }
        }
    return t;
}

template <int N>
struct TabN {
    static constexpr Tab value = make_tab(N);
};

struct Args {
    const float* x;
    float* y;
    const float* q;      // source planes (n_q of them) or null
    const float* bvec;   // full right-hand side vector or null
    int n_q;
    const float* st;     // clamped sigma_t, R^3 voxel centres
    const float* ss;     // sigma_s, R^3
    int R;
    int pitch_x;
    uint32_t pitch_y, plane_stride;  // element strides (the launcher checks they fit)
    int zc;              // slices per CTA (z chunk)
    float inv_h;         // R
    float tsign;         // +1: A, -1: A^T
    float fl[8];         // g^l
    unsigned char pcls[64];  // parity class of plane p
    double* partials;    // residual: per-CTA FP64 sums of r^2
    const int* live;     // null, or a device flag: the launch does nothing while it is 0
    unsigned int* err;   // TMA kernel: set to 1 where a bounded wait ran out (else untouched)
    int late_wait;       // TMA kernel under programmatic dependent launch after the face-column
                         // kernel: wait for it at the end instead of the start (see launch_n)
};

// Right-hand side of one class at slot s of this thread's column (residual
// mode): the full vector bvec, or Q (planes beyond n_q are 0); read only at
// active slots.  Issued at the start of a z-step so that the step's staging,
// barrier and arithmetic hide the load latency.
template <int N, int C>
__device__ __forceinline__ void load_rhs(const Args& a, bool act, uint32_t col, int s, float (&r)[MAXC]) {
    constexpr ClassTab CT = TabN<N>::value.cls[C];
    const uint32_t ps = a.plane_stride;
    const float* base = a.bvec ? a.bvec : a.q;
    const int nq = a.bvec ? 64 : a.n_q;
    const size_t off = size_t(CT.plane0) * ps + size_t(uint32_t(s) * a.pitch_y) + col;
#pragma unroll
    for (int i = 0; i < MAXC; ++i)
        if (i < CT.n) r[i] = (act && CT.plane0 + i < nq) ? __ldg(base + off + uint32_t(i) * ps) : 0.0f;
}

// xy-mean of a staged sigma slice (rows of gx centres) at this thread's
// location for bits (bx, by): the mean over the in-domain centres adjacent to
// it (indices clamped at the domain boundary when the slice was staged).
__device__ __forceinline__ float xy_mean_g(const float* g, int gx, int tx, int ty, int bx, int by) {
    const int gx1 = tx + 1, gy1 = ty + 1;
    const int gx0 = bx ? tx : gx1, gy0 = by ? ty : gy1;
    return 0.25f * (g[gy0 * gx + gx0] + g[gy0 * gx + gx1] + g[gy1 * gx + gx0] + g[gy1 * gx + gx1]);
}

}  // namespace tiled

// The TMA-staged main kernel (pn_apply_tma.cu) over the grid `grid` of the
// plan with z chunks of a.zc slices; the face-column kernel is launched by
// the caller.  Returns cudaErrorNotSupported where the TMA kernel does not
// serve the handle (tma_serves).
cudaError_t launch_tma_main(const pn_handle* h, int mode, const tiled::Args& a, dim3 grid, cudaStream_t s);

}  // namespace pn
