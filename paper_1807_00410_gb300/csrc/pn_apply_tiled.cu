// Tiled FP32 operator of the staggered P_N system for GB300.
//
// The operator (appendix "Final equation"; half-cell central differences
// between the staggered grids, section "Precomputation"; Dirichlet dropping,
// section "Runtime") couples each coefficient only to coefficients of the
// three parity classes that differ from its own in exactly one axis, half a
// cell away along that axis.  The kernel exploits that structure:
//
//  * A CTA owns a TX x TY block of (x, y) slots and marches along z through a
//    chunk of slices.  Thread group g = (bx, by) owns the two classes
//    (bx, by, 0) and (bx, by, 1), which differ only in z, so every z-coupling
//    is between values the thread already holds in registers (the even class
//    at slots s-1 and s, the odd class at s and s+1).
//  * Each step writes slice s of every plane (plus a one-sided halo: the left
//    or right column, the lower or upper row, depending on the plane's class)
//    into a double-buffered shared-memory slice; x- and y-couplings read it.
//    One barrier per step.
//  * Each input value is read from HBM once; halos are re-read from L2.
//  * Couplings are compile-time constants (constexpr closed forms); the 1/h
//    factor is applied once per output.  sigma_t and sigma_s are staged per
//    slice at voxel centres and averaged in registers.
//  * Global loads for slice s+1 (own values, halo, sigma) are issued before
//    slice s is computed, so memory latency overlaps the arithmetic.
//
// Inactive slots read as zero, which realises the Dirichlet rule without
// branches in the stencil.  Output slots outside the tiles (x >= tiles' end,
// plane tails) are written by the generic slab kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "pn_pdl.cuh"
#include "pn_tiled.cuh"

namespace pn {
namespace tiled {

// Load n values of one class at slot z of this thread's column; inactive
// slots read 0.  `base` points at the class's first plane, z = 0, this column;
// planes are ps elements apart, slices py elements apart (both < 2^32 / 4 /
// MAXC bytes, checked by the launcher).
template <int NV>
__device__ __forceinline__ void load_class(const float* base, uint32_t ps, uint32_t py, bool colact, int z, int zext,
                                           float (&v)[MAXC]) {
    const bool act = colact && z >= 0 && z < zext;
    const float* q = base + size_t(uint32_t(z) * py);
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = act ? __ldg(q + uint32_t(i) * ps) : 0.0f;
}

template <int TY>
struct Geo {
    static constexpr int SX = TX + 2;           // shared slice row (one halo column each side)
    static constexpr int SY = TY + 2;
    static constexpr int SLICE = SX * SY;
    static constexpr int GX = TX + 1;           // sigma tile: centres x0-1 .. x0+TX-1
    static constexpr int GY = TY + 1;
    static constexpr int GSL = GX * GY;
    static constexpr int NT = TX * TY * NG;     // threads per CTA
    static constexpr int HALO = TX + TY;        // halo cells per plane per slice
};

// Compute and store the outputs of one class (C: bits (bx, by, bz)) at slot s.
//   own[i]   : this class's values at slot s
//   zp[j], zm[j]: the z-neighbour class's values at the plus / minus slot
//   st, ss   : sigma_t, sigma_s interpolated to this class's location
template <int N, int TY, int C, int MODE>
__device__ __forceinline__ void compute_class(const Args& a, const float* buf, int tx, int ty, bool store_ok,
                                              bool active, size_t outoff, const float (&own)[MAXC],
                                              const float (&zp)[MAXC], const float (&zm)[MAXC], float st, float ss,
                                              const float (&rhs)[MAXC], float& rrun) {
    constexpr Tab T = TabN<N>::value;
    constexpr ClassTab CT = T.cls[C];
    constexpr int bx = C & 1, by = (C >> 1) & 1;
    constexpr int CXn = C ^ 1, CYn = C ^ 2, CZn = C ^ 4;
    constexpr int nX = T.cls[CXn].n, nY = T.cls[CYn].n, nZ = T.cls[CZn].n;
    constexpr int pX = T.cls[CXn].plane0, pY = T.cls[CYn].plane0;
    using G = Geo<TY>;
    if (CT.n == 0) return;
    const uint32_t ps = a.plane_stride;
    float* yb = a.y + size_t(CT.plane0) * ps + outoff;
    const float tscale = a.tsign * a.inv_h;
    // differences of the neighbour classes across this location
    float dx[MAXC], dy[MAXC], dz[MAXC];
    const int cy = ty + 1, cx = tx + 1;
#pragma unroll
    for (int j = 0; j < MAXC; ++j) {
        if (j < nX) {
            const float* b = buf + (pX + j) * G::SLICE + cy * G::SX;
            dx[j] = b[cx + 1 - bx] - b[cx - bx];
        }
        if (j < nY) {
            const float* b = buf + (pY + j) * G::SLICE + cx;
            dy[j] = b[(cy + 1 - by) * G::SX] - b[(cy - by) * G::SX];
        }
        if (j < nZ) dz[j] = zp[j] - zm[j];
    }
#pragma unroll
    for (int i = 0; i < MAXC; ++i) {
        if (i < CT.n) {
            float tr = 0.0f;
#pragma unroll
            for (int t = 0; t < MAXT; ++t)
                if (t < CT.row[i].nt[0]) tr = fmaf(CT.row[i].c[0][t], dx[CT.row[i].j[0][t]], tr);
#pragma unroll
            for (int t = 0; t < MAXT; ++t)
                if (t < CT.row[i].nt[1]) tr = fmaf(CT.row[i].c[1][t], dy[CT.row[i].j[1][t]], tr);
#pragma unroll
            for (int t = 0; t < MAXT; ++t)
                if (t < CT.row[i].nt[2]) tr = fmaf(CT.row[i].c[2][t], dz[CT.row[i].j[2][t]], tr);
            const float d = fmaf(-a.fl[CT.row[i].l], ss, st);
            float out = fmaf(d, own[i], tscale * tr);
            if (MODE == OP_RESIDUAL) {
                if (N <= 6) {
                    out = rhs[i] - out;  // loaded at the start of the step
                } else {
                    // P7 has no registers to spare for the early loads: read here
                    float b = 0.0f;
                    if (active) {
                        if (a.bvec) b = __ldg(a.bvec + size_t(CT.plane0) * ps + outoff + uint32_t(i) * ps);
                        else if (CT.plane0 + i < a.n_q)
                            b = __ldg(a.q + size_t(CT.plane0) * ps + outoff + uint32_t(i) * ps);
                    }
                    out = b - out;
                }
            }
            out = active ? out : 0.0f;
            if (MODE == OP_RESIDUAL) rrun = fmaf(out, out, rrun);
            if (store_ok) yb[uint32_t(i) * ps] = out;
        }
    }
}

// xy-mean of a staged sigma slice at this thread's location for bits (bx, by).
template <int TY>
__device__ __forceinline__ float xy_mean(const float* g, int tx, int ty, int bx, int by) {
    using G = Geo<TY>;
    const int gx1 = tx + 1, gy1 = ty + 1;
    const int gx0 = bx ? tx : gx1, gy0 = by ? ty : gy1;
    return 0.25f * (g[gy0 * G::GX + gx0] + g[gy0 * G::GX + gx1] + g[gy1 * G::GX + gx0] + g[gy1 * G::GX + gx1]);
}

template <int N, int TY, int GRP, int MODE>
__device__ __forceinline__ void run_group(const Args& a, float* smem, int tx, int ty, int x, int y, int za, int zb,
                                          double& racc) {
    using G = Geo<TY>;
    constexpr Tab T = TabN<N>::value;
    constexpr int K = T.K;
    constexpr int C0 = GRP, C1 = GRP + 4;
    constexpr int bx = GRP & 1, by = GRP >> 1;
    constexpr int n0 = T.cls[C0].n, n1 = T.cls[C1].n;
    constexpr int p0 = T.cls[C0].plane0, p1 = T.cls[C1].plane0;
    const int R = a.R;
    float* buf = smem;                       // [2][K][SLICE]
    float* sg = smem + 2 * K * G::SLICE;     // [2][2][GSL]  (sigma_t, sigma_s)
    const int tid = tx + TX * (ty + TY * GRP);
    const int x0 = x - tx, y0 = y - ty;
    const bool colact0 = x < R + bx && y < R + by;
    const bool colact1 = colact0;  // same x/y bits
    const uint32_t col = uint32_t(y) * uint32_t(a.pitch_x) + uint32_t(x);
    const bool store_ok = x < a.pitch_x && y <= R;
    const uint32_t ps = a.plane_stride, py = a.pitch_y;
    const float* xb0 = a.x + size_t(p0) * ps + col;  // class C0, z = 0, this column
    const float* xb1 = a.x + size_t(p1) * ps + col;

    // halo cells owned by this thread: plane p, shared index, global column offset
    constexpr int NH = (K * G::HALO + G::NT - 1) / G::NT;
    int h_sidx[NH];
    const float* h_ptr[NH];
    int h_zext[NH];  // 0: cell inactive in x/y; else the plane's z extent
#pragma unroll
    for (int u = 0; u < NH; ++u) {
        const int h = tid + u * G::NT;
        h_sidx[u] = -1;
        h_ptr[u] = a.x;
        h_zext[u] = 0;
        if (h < K * G::HALO) {
            const int p = h / G::HALO, r = h % G::HALO;
            const int pc = a.pcls[p];
            const int pbx = pc & 1, pby = (pc >> 1) & 1, pbz = pc >> 2;
            int hx, hy, sx, sy;
            if (r < TX) {
                hx = x0 + r;
                hy = pby ? y0 + TY : y0 - 1;
                sx = r + 1;
                sy = pby ? TY + 1 : 0;
            } else {
                hy = y0 + (r - TX);
                hx = pbx ? x0 + TX : x0 - 1;
                sy = r - TX + 1;
                sx = pbx ? TX + 1 : 0;
            }
            h_sidx[u] = p * G::SLICE + sy * G::SX + sx;
            const bool act = hx >= 0 && hy >= 0 && hx < R + pbx && hy < R + pby;
            h_zext[u] = act ? R + pbz : 0;
            if (act) h_ptr[u] = a.x + size_t(p) * ps + uint32_t(hy) * uint32_t(a.pitch_x) + uint32_t(hx);
        }
    }
    // sigma tile cell owned by this thread (two fields)
    const bool sg_own = tid < 2 * G::GSL;
    const int sg_field = tid / G::GSL, sg_cell = tid % G::GSL;
    int64_t sg_off = 0;
    {
        const int gx = sg_cell % G::GX, gy = sg_cell / G::GX;
        const int cxr = min(max(x0 - 1 + gx, 0), R - 1), cyr = min(max(y0 - 1 + gy, 0), R - 1);
        sg_off = int64_t(cyr) * R + cxr;
    }
    const float* sgsrc = sg_field == 0 ? a.st : a.ss;
    const int64_t R2 = int64_t(R) * R;
    auto sg_load = [&](int s) -> float {
        const int zc = min(max(s, 0), R - 1);
        return sg_own ? __ldg(sgsrc + zc * R2 + sg_off) : 0.0f;
    };

    // priming: sigma slice za-1 -> xy-means of the previous slice
    if (sg_own) sg[((za + 1) & 1) * 2 * G::GSL + tid] = sg_load(za - 1);
    float v0p[MAXC] = {}, v0c[MAXC] = {}, v0n[MAXC] = {}, v1c[MAXC] = {}, v1n[MAXC] = {};
    load_class<n0>(xb0, ps, py, colact0, za - 1, R, v0p);
    load_class<n0>(xb0, ps, py, colact0, za, R, v0c);
    load_class<n1>(xb1, ps, py, colact1, za, R + 1, v1c);
    load_class<n1>(xb1, ps, py, colact1, za + 1, R + 1, v1n);
    float hreg[NH];
#pragma unroll
    for (int u = 0; u < NH; ++u)
        hreg[u] = (za < h_zext[u]) ? __ldg(h_ptr[u] + size_t(uint32_t(za) * py)) : 0.0f;
    float sreg = sg_load(za);
    __syncthreads();
    float mt_prev, ms_prev;
    {
        const float* g = sg + ((za + 1) & 1) * 2 * G::GSL;
        mt_prev = xy_mean<TY>(g, tx, ty, bx, by);
        ms_prev = xy_mean<TY>(g + G::GSL, tx, ty, bx, by);
    }
    float rrun = 0.0f;
    int rcnt = 0;
    for (int s = za; s < zb; ++s) {
        float* b = buf + (s & 1) * K * G::SLICE;
        float* g = sg + (s & 1) * 2 * G::GSL;
        float rhs0[MAXC], rhs1[MAXC];
        if (MODE == OP_RESIDUAL && N <= 6) {
            load_rhs<N, C0>(a, colact0 && s < R, col, s, rhs0);
            load_rhs<N, C1>(a, colact1, col, s, rhs1);
        }
        // stage slice s: own values, halo, sigma
        const int sidx = (ty + 1) * G::SX + (tx + 1);
#pragma unroll
        for (int i = 0; i < n0; ++i) b[(p0 + i) * G::SLICE + sidx] = v0c[i];
#pragma unroll
        for (int i = 0; i < n1; ++i) b[(p1 + i) * G::SLICE + sidx] = v1c[i];
#pragma unroll
        for (int u = 0; u < NH; ++u)
            if (h_sidx[u] >= 0) b[h_sidx[u]] = hreg[u];
        if (sg_own) g[tid] = sreg;
        // prefetch slice s+1 (and s+2 for the odd class)
        load_class<n0>(xb0, ps, py, colact0, s + 1, R, v0n);
        float v1t[MAXC] = {};
        load_class<n1>(xb1, ps, py, colact1, s + 2, R + 1, v1t);
#pragma unroll
        for (int u = 0; u < NH; ++u)
            hreg[u] = (s + 1 < h_zext[u]) ? __ldg(h_ptr[u] + size_t(uint32_t(s + 1) * py)) : 0.0f;
        sreg = sg_load(s + 1);
        __syncthreads();
        const float mt = xy_mean<TY>(g, tx, ty, bx, by);
        const float ms = xy_mean<TY>(g + G::GSL, tx, ty, bx, by);
        const size_t outoff = size_t(uint32_t(s) * py) + col;
        // even class (bz = 0): z-neighbours are the odd class at s+1 (plus) and s (minus)
        compute_class<N, TY, C0, MODE>(a, b, tx, ty, store_ok, colact0 && s < R, outoff, v0c, v1n, v1c, mt, ms,
                                       rhs0, rrun);
        // odd class (bz = 1): z-neighbours are the even class at s (plus) and s-1 (minus)
        compute_class<N, TY, C1, MODE>(a, b, tx, ty, store_ok, colact1, outoff, v1c, v0c, v0p,
                                       0.5f * (mt + mt_prev), 0.5f * (ms + ms_prev), rhs1, rrun);
        if (MODE == OP_RESIDUAL && ++rcnt == 4) {
            racc += double(rrun);
            rrun = 0.0f;
            rcnt = 0;
        }
        mt_prev = mt;
        ms_prev = ms;
#pragma unroll
        for (int i = 0; i < n0; ++i) {
            v0p[i] = v0c[i];
            v0c[i] = v0n[i];
        }
#pragma unroll
        for (int i = 0; i < n1; ++i) {
            v1c[i] = v1n[i];
            v1n[i] = v1t[i];
        }
    }
    racc += double(rrun);
}

template <int N, int TY, int MODE>
__global__ void __launch_bounds__(TX * TY * NG, 1) k_apply_tiled(Args a) {
    pdl_wait();  // programmatic dependent launch (pn_pdl.cuh)
    if (a.live && !*a.live) return;  // uniform over the grid
    extern __shared__ float smem[];
    // warp w runs group w % 4 (one group's code per scheduler; see pn_apply_tma.cu)
    const int tx = threadIdx.x, grp = threadIdx.y, ty = threadIdx.z;
    const int x = blockIdx.x * TX + tx, y = blockIdx.y * TY + ty;
    const int za = blockIdx.z * a.zc;
    const int zb = min(za + a.zc, a.R + 1);
    double racc = 0.0;
    switch (grp) {
        case 0: run_group<N, TY, 0, MODE>(a, smem, tx, ty, x, y, za, zb, racc); break;
        case 1: run_group<N, TY, 1, MODE>(a, smem, tx, ty, x, y, za, zb, racc); break;
        case 2: run_group<N, TY, 2, MODE>(a, smem, tx, ty, x, y, za, zb, racc); break;
        default: run_group<N, TY, 3, MODE>(a, smem, tx, ty, x, y, za, zb, racc); break;
    }
    pdl_trigger();
    if (MODE == OP_RESIDUAL && a.partials != nullptr) {
        __shared__ double red[TX * TY * NG / 32];
        for (int o = 16; o > 0; o >>= 1) racc += __shfl_down_sync(0xffffffffu, racc, o);
        const int tid = tx + TX * (ty + TY * grp);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = racc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int i = 0; i < TX * TY * NG / 32; ++i) t += red[i];
            a.partials[(int64_t(blockIdx.z) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
        }
    }
}


// Output of plane i of face class C (p_x = 1) at x = R of row (y, z), from
// global memory, with the same compile-time couplings as the tiled kernel:
// only this row's own terms are read (at most two loads per term).
template <int N, int C, int MODE>
__device__ __forceinline__ void face_out(const Args& a, int y, int z, int i, float& rrun) {
    constexpr Tab T = TabN<N>::value;
    constexpr ClassTab CT = T.cls[C];
    constexpr int by = (C >> 1) & 1, bz = C >> 2;
    constexpr int pX = T.cls[C ^ 1].plane0, pY = T.cls[C ^ 2].plane0, pZ = T.cls[C ^ 4].plane0;
    const int R = a.R;
    const uint32_t ps = a.plane_stride, py = a.pitch_y, px = uint32_t(a.pitch_x);
    const bool active = y < R + by && z < R + bz;
    const size_t rowoff = size_t(uint32_t(z) * py) + uint32_t(y) * px;
    auto val = [&](int plane, int xx, int yy, int zz, int ext_y, int ext_z) -> float {
        if (yy < 0 || zz < 0 || yy >= ext_y || zz >= ext_z) return 0.0f;
        return __ldg(a.x + size_t(plane) * ps + size_t(uint32_t(zz) * py) + uint32_t(yy) * px + uint32_t(xx));
    };
    float tr = 0.0f;
    int l = 0;
    if (active) {
#pragma unroll
        for (int ii = 0; ii < MAXC; ++ii) {
            if (ii < CT.n && ii == i) {
                l = CT.row[ii].l;
                // x: the centre class at slot R - 1 (its slot R lies outside the domain)
#pragma unroll
                for (int q = 0; q < MAXT; ++q)
                    if (q < CT.row[ii].nt[0])
                        tr = fmaf(CT.row[ii].c[0][q], -val(pX + CT.row[ii].j[0][q], R - 1, y, z, R + by, R + bz), tr);
                // y and z: the neighbour class with the other bit, slots i + 1 - b and i - b
#pragma unroll
                for (int q = 0; q < MAXT; ++q)
                    if (q < CT.row[ii].nt[1]) {
                        const int jj = pY + CT.row[ii].j[1][q];
                        tr = fmaf(CT.row[ii].c[1][q],
                                  val(jj, R, y + 1 - by, z, R + 1 - by, R + bz) - val(jj, R, y - by, z, R + 1 - by, R + bz),
                                  tr);
                    }
#pragma unroll
                for (int q = 0; q < MAXT; ++q)
                    if (q < CT.row[ii].nt[2]) {
                        const int jj = pZ + CT.row[ii].j[2][q];
                        tr = fmaf(CT.row[ii].c[2][q],
                                  val(jj, R, y, z + 1 - bz, R + by, R + 1 - bz) - val(jj, R, y, z - bz, R + by, R + 1 - bz),
                                  tr);
                    }
            }
        }
    }
    const size_t off = size_t(CT.plane0 + i) * ps + rowoff + uint32_t(R);
    float out = 0.0f;
    if (active) {
        // sigma at the face x = R: centre x = R - 1, mean over the y and z neighbours
        const int64_t R2 = int64_t(R) * R;
        const int y0 = by ? max(y - 1, 0) : y, y1 = by ? min(y, R - 1) : y;
        const int z0 = bz ? max(z - 1, 0) : z, z1 = bz ? min(z, R - 1) : z;
        const int64_t c = R - 1;
        const float st = 0.25f * (__ldg(a.st + z0 * R2 + y0 * R + c) + __ldg(a.st + z0 * R2 + y1 * R + c) +
                                  __ldg(a.st + z1 * R2 + y0 * R + c) + __ldg(a.st + z1 * R2 + y1 * R + c));
        const float ss = 0.25f * (__ldg(a.ss + z0 * R2 + y0 * R + c) + __ldg(a.ss + z0 * R2 + y1 * R + c) +
                                  __ldg(a.ss + z1 * R2 + y0 * R + c) + __ldg(a.ss + z1 * R2 + y1 * R + c));
        out = fmaf(fmaf(-a.fl[l], ss, st), __ldg(a.x + off), a.tsign * a.inv_h * tr);
        if (MODE == OP_RESIDUAL) {
            float b = 0.0f;
            if (a.bvec) b = __ldg(a.bvec + off);
            else if (CT.plane0 + i < a.n_q) b = __ldg(a.q + off);
            out = b - out;
            rrun = fmaf(out, out, rrun);
        }
    }
    // x = R is the first of the row's last four slots (R a multiple of 32, the
    // only case with outputs right of the tiles): the output and three zeros
    if (a.pitch_x - R == 4)
        *reinterpret_cast<float4*>(a.y + off) = make_float4(out, 0.0f, 0.0f, 0.0f);
    else
        a.y[off] = out;
}

template <int N, int C, int MODE>
__device__ __forceinline__ void face_class_items(const Args& a, int64_t t0, int64_t stride, float& rrun) {
    constexpr ClassTab CT = TabN<N>::value.cls[C];
    if (CT.n == 0) return;
    const int R = a.R;
    const int64_t rows = int64_t(R + 1) * (R + 1);
    // consecutive threads take consecutive rows of the same plane (warp-uniform plane)
    for (int64_t u = t0; u < rows * CT.n; u += stride) {
        const int i = int(u / rows);
        const int64_t row = u % rows;
        face_out<N, C, MODE>(a, int(row % (R + 1)), int(row / (R + 1)), i, rrun);
    }
}

// Slots right of the tiles: x in [x_lo, pitch_x) of every (y, z) row, and the
// plane tails.  Only x = R can hold unknowns (face classes, p_x = 1).
// blockIdx.y = 0 writes 0 to every other such slot and to the plane tails,
// one slot per thread; blockIdx.y = 1..4 computes the x = R outputs of face
// class 1, 3, 5, 7, one (row, plane) per thread.
// Block ranges of the face kernel's tasks in one 1D grid: [b[0], b[1]) writes
// the zeros, [b[k], b[k+1]) computes face class 2k - 1 (k = 1..4).
struct FaceRanges {
    int b[6];
};

template <int N, int MODE>
__device__ __forceinline__ void face_body(const Args& a, int x_lo, const FaceRanges& fr) {
    if (a.live && !*a.live) return;  // uniform over the grid
    constexpr Tab T = TabN<N>::value;
    constexpr int K = T.K;
    const int R = a.R;
    const uint32_t ps = a.plane_stride, py = a.pitch_y;
    const uint32_t px = uint32_t(a.pitch_x);
    const int64_t rows = int64_t(R + 1) * (R + 1);
    const int w = a.pitch_x - x_lo;
    const uint32_t box = py * uint32_t(R + 1);
    const uint32_t tail = ps - box;
    int task = 0;
    while (task < 4 && int(blockIdx.x) >= fr.b[task + 1]) ++task;
    const int64_t t0 = int64_t(int(blockIdx.x) - fr.b[task]) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(fr.b[task + 1] - fr.b[task]) * blockDim.x;
    float rrun = 0.0f;
    if (task == 0 && w == 4 && x_lo + 4 == a.pitch_x) {
        // four slots per row, 16-byte aligned: one vector store each; the face
        // planes' rows are written with their x = R output by tasks 1..4
        const int64_t nz = int64_t(K) * rows;
        for (int64_t u = t0; u < nz + int64_t(K) * tail; u += stride) {
            if (u < nz) {
                const int64_t row = u % rows;
                const int p = int(u / rows);
                if ((a.pcls[p] & 1) && x_lo <= R) continue;
                const int y = int(row % (R + 1)), z = int(row / (R + 1));
                *reinterpret_cast<float4*>(a.y + size_t(p) * ps + size_t(uint32_t(z) * py) + uint32_t(y) * px +
                                           uint32_t(x_lo)) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            } else {
                const int64_t v = u - nz;
                a.y[size_t(v / tail) * ps + box + uint32_t(v % tail)] = 0.0f;
            }
        }
    } else if (task == 0) {
        const int64_t nz = w > 0 ? int64_t(K) * rows * w : 0;
        for (int64_t u = t0; u < nz + int64_t(K) * tail; u += stride) {
            if (u < nz) {
                const int xo = int(u % w);
                const int64_t q = u / w;
                const int64_t row = q % rows;
                const int p = int(q / rows);
                const int x = x_lo + xo;
                if (x == R && (a.pcls[p] & 1)) continue;  // a face unknown: computed below
                const int y = int(row % (R + 1)), z = int(row / (R + 1));
                a.y[size_t(p) * ps + size_t(uint32_t(z) * py) + uint32_t(y) * px + uint32_t(x)] = 0.0f;
            } else {
                const int64_t v = u - nz;
                a.y[size_t(v / tail) * ps + box + uint32_t(v % tail)] = 0.0f;
            }
        }
    } else if (x_lo <= R) {
        switch (task) {
            case 1: face_class_items<N, 1, MODE>(a, t0, stride, rrun); break;
            case 2: face_class_items<N, 3, MODE>(a, t0, stride, rrun); break;
            case 3: face_class_items<N, 5, MODE>(a, t0, stride, rrun); break;
            default: face_class_items<N, 7, MODE>(a, t0, stride, rrun); break;
        }
    }
    if (MODE == OP_RESIDUAL && a.partials != nullptr) {
        double v = double(rrun);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __shared__ double red[8];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tsum = 0.0;
            for (int i = 0; i < 8; ++i) tsum += red[i];
            a.partials[blockIdx.x] = tsum;
        }
    }
}

// Ahead of the TMA main kernel under programmatic dependent launch: waits for
// the input's producer, then lets the main kernel start at once (the two
// write disjoint outputs); the main kernel waits for this one at its end.
template <int N, int MODE>
__global__ void __launch_bounds__(256) k_face_x_first(Args a, int x_lo, FaceRanges fr) {
    pdl_wait();
    pdl_trigger();
    face_body<N, MODE>(a, x_lo, fr);
}

template <int N, int MODE>
__global__ void __launch_bounds__(256) k_face_x(Args a, int x_lo, FaceRanges fr) {
    // Launched right after the main kernel (programmatic dependent launch:
    // its CTAs become resident during the main kernel's last wave), it waits
    // for the main kernel before any work, so the two run one after the other
    // (running them side by side slowed the main kernel down).
    pdl_wait();
    face_body<N, MODE>(a, x_lo, fr);
    pdl_trigger();
}

}  // namespace tiled

namespace {

struct TiledPlan {
    dim3 grid, block;
    int zc;
    size_t smem;
    int x_end;  // tiles cover x < x_end
};

template <int TY>
TiledPlan plan_for(const pn_handle* h) {
    using G = tiled::Geo<TY>;
    TiledPlan p;
    const int R = h->R;
    const int nxt = (R + tiled::TX - 1) / tiled::TX;
    const int nyt = (R + 1 + TY - 1) / TY;
    const int sms = pn_sm_count();
    // z chunks: enough CTAs for about tile_ctas_per_sm per SM, chunks of at
    // least 4 slices
    const int target = std::max(1, h->tile_ctas_per_sm) * sms;
    int nzc = std::max(1, (target + nxt * nyt - 1) / (nxt * nyt));
    nzc = std::min(nzc, std::max(1, (R + 1) / 4));
    const int zc = (R + 1 + nzc - 1) / nzc;
    nzc = (R + 1 + zc - 1) / zc;
    p.grid = dim3(nxt, nyt, nzc);
    p.block = dim3(tiled::TX, tiled::NG, TY);
    p.zc = zc;
    p.smem = (size_t(2) * h->K * G::SLICE + 4 * G::GSL) * sizeof(float);
    p.x_end = std::min<int>(int(h->pitch_x), nxt * tiled::TX);
    return p;
}

constexpr int kTY = 4;

// Block ranges of the face kernel: enough blocks for each task (one item per
// thread), capped at 4 per SM for the zeros (grid-stride beyond).
tiled::FaceRanges face_ranges(const pn_handle* h) {
    const int64_t rows = int64_t(h->R + 1) * (h->R + 1);
    const int64_t x_lo = std::min<int64_t>(h->pitch_x, int64_t((h->R + tiled::TX - 1) / tiled::TX) * tiled::TX);
    const int64_t w = h->pitch_x - x_lo;
    const int64_t tail = h->plane_stride - h->pitch_y * (h->R + 1);
    auto blocks = [](int64_t items, int64_t cap) {
        return int(std::max<int64_t>(1, std::min<int64_t>(cap, (items + 255) / 256)));
    };
    int ncls[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = 0; p < h->K; ++p) ++ncls[h->plane_class[p]];
    tiled::FaceRanges fr{};
    fr.b[0] = 0;
    const int64_t zero_items = w == 4 && x_lo + 4 == h->pitch_x ? rows : rows * w;  // vector stores when w = 4
    fr.b[1] = blocks(int64_t(h->K) * (zero_items + tail), 4 * int64_t(pn_sm_count()));
    for (int k = 1; k <= 4; ++k) {
        const int c = 2 * k - 1;
        const int nb = (x_lo <= h->R && ncls[c] > 0) ? blocks(rows * ncls[c], 4 * int64_t(pn_sm_count())) : 0;
        fr.b[k + 1] = fr.b[k] + nb;
    }
    return fr;
}

int face_blocks(const pn_handle* h) { return face_ranges(h).b[5]; }

template <int N, int MODE>
cudaError_t launch_n(const pn_handle* h, const tiled::Args& a, const TiledPlan& p, cudaStream_t s) {
    auto kern = tiled::k_apply_tiled<N, kTY, MODE>;
    static std::atomic<unsigned long long> configured{0};
    {
        cudaError_t e = pn_smem_attr_once(configured, reinterpret_cast<const void*>(kern), 200 * 1024);
        if (e != cudaSuccess) return e;
    }
    // columns right of the tiles and plane tails: disjoint outputs and partial
    // slots, same inputs; on the handle's side stream, concurrently, or after
    // the main kernel on the same stream (h->face_serial, chosen by the tuner)
    // With programmatic dependent launch (h->pdl, inside the Arnoldi loop) both
    // kernels go to s (k_face_x waits for the main kernel).
    const bool pdl = h->pdl != 0;
    cudaStream_t fs = (h->side && !h->face_serial && !pdl) ? h->side : s;
    cudaError_t e = cudaSuccess;
    if (fs != s) {
        e = cudaEventRecord(h->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(fs, h->ev_fork, 0);
        if (e != cudaSuccess) return e;
    }
    const bool tma_main = h->tile_kernel == PN_APPLY_KERNEL_TMA && tma_serves(h);
    if (pdl && tma_main && a.live == nullptr) {
        // face-column kernel first, then the main kernel overlapping it (both
        // on s; k_face_x_first and late_wait above)
        tiled::Args af = a;
        if (af.partials) af.partials += p.grid.x * p.grid.y * p.grid.z;
        const tiled::FaceRanges fr = face_ranges(h);
        e = launch_pdl(true, tiled::k_face_x_first<N, MODE>, dim3(fr.b[5]), dim3(256), 0, s, af, p.x_end, fr);
        if (e != cudaSuccess) return e;
        tiled::Args am = a;
        am.late_wait = 1;
        return launch_tma_main(h, MODE, am, p.grid, s);
    }
    if (tma_main) {
        e = launch_tma_main(h, MODE, a, p.grid, s);
    } else {
        e = launch_pdl(pdl, kern, p.grid, p.block, p.smem, s, a);
    }
    if (e != cudaSuccess) return e;
    tiled::Args af = a;
    if (af.partials) af.partials += p.grid.x * p.grid.y * p.grid.z;
    const tiled::FaceRanges fr = face_ranges(h);
    e = launch_pdl(pdl, tiled::k_face_x<N, MODE>, dim3(fr.b[5]), dim3(256), 0, fs, af, p.x_end, fr);
    if (e != cudaSuccess || fs == s) return e;
    e = cudaEventRecord(h->ev_join, fs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_join, 0);
    return e;
}

template <int MODE>
cudaError_t launch_mode(const pn_handle* h, const tiled::Args& a, const TiledPlan& p, cudaStream_t s) {
    switch (h->N) {
        case 0: return launch_n<0, MODE>(h, a, p, s);
        case 1: return launch_n<1, MODE>(h, a, p, s);
        case 2: return launch_n<2, MODE>(h, a, p, s);
        case 3: return launch_n<3, MODE>(h, a, p, s);
        case 4: return launch_n<4, MODE>(h, a, p, s);
        case 5: return launch_n<5, MODE>(h, a, p, s);
        case 6: return launch_n<6, MODE>(h, a, p, s);
        default: return launch_n<7, MODE>(h, a, p, s);
    }
}

}  // namespace

int tiled_partial_count(const pn_handle* h) {
    const TiledPlan p = plan_for<kTY>(h);
    return int(p.grid.x * p.grid.y * p.grid.z) + face_blocks(h);
}

int tiled_partial_bound(const pn_handle* h) {
    const int nxt = (h->R + tiled::TX - 1) / tiled::TX;
    const int nyt = (h->R + 1 + kTY - 1) / kTY;
    const int nzc_max = std::max(1, (h->R + 1) / 4);
    return nxt * nyt * nzc_max + face_blocks(h);
}

int tiled_x_end(const pn_handle* h) { return plan_for<kTY>(h).x_end; }

cudaError_t launch_tiled(const pn_handle* h, int mode, const float* x, float* y, const float* bvec,
                         double* partials, cudaStream_t s) {
    return launch_tiled_gated(h, mode, x, y, bvec, partials, nullptr, s);
}

cudaError_t launch_tiled_gated(const pn_handle* h, int mode, const float* x, float* y, const float* bvec,
                               double* partials, const int* live, cudaStream_t s) {
    const TiledPlan p = plan_for<kTY>(h);
    tiled::Args a{};
    a.x = x;
    a.y = y;
    a.q = h->d_q_f;
    a.bvec = bvec;
    a.n_q = h->n_q_planes;
    a.st = h->d_st_f;
    a.ss = h->d_ss_f;
    a.R = h->R;
    a.pitch_x = int(h->pitch_x);
    a.pitch_y = uint32_t(h->pitch_y);
    a.plane_stride = uint32_t(h->plane_stride);
    a.zc = p.zc;
    a.inv_h = float(h->R);
    a.tsign = mode == OP_APPLY_T ? -1.0f : 1.0f;
    for (int l = 0; l < 8; ++l) a.fl[l] = l == 0 ? 1.0f : float(std::pow(h->g, l));
    for (int q = 0; q < 64; ++q) a.pcls[q] = q < h->K ? (unsigned char)h->plane_class[q] : 0;
    a.partials = partials;
    a.live = live;
    a.err = reinterpret_cast<unsigned int*>(h->d_scalars + PN_S_FAULT);
    if (mode == OP_RESIDUAL) return launch_mode<OP_RESIDUAL>(h, a, p, s);
    return launch_mode<OP_APPLY>(h, a, p, s);
}

}  // namespace pn
