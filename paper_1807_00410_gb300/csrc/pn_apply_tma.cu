// TMA-staged tiled FP32 operator of the staggered P_N system for GB300.
//
// The operator and its arithmetic are those of the register-staged kernel in
// pn_apply_tiled.cu, operation for operation (the outputs are bitwise equal);
// the data path differs:
//
//  * The input planes of one parity class reach shared memory as one 4D TMA
//    box per z-slice (x: 36 slots, y: 5 rows, z: 1 slice, all n_c planes of
//    the class), from a tensor map whose extents are the class's active
//    extents.  The copy engine fills every slot outside them with 0, which is
//    the Dirichlet rule for inputs (section "Runtime"); whatever the padding
//    slots of x hold is never read.  The box starts at x0 (classes with
//    p_x = 1) or x0 - 4 (p_x = 0), a 16-byte boundary, and holds the one halo
//    column that the x-differences of the neighbouring class need; in y it
//    starts at y0 or y0 - 1 and holds the one halo row.
//  * Each class has a ring of four slice slots.  One thread issues the copies
//    two z-steps ahead (even classes) and three ahead (odd classes, which the
//    even outputs need at s + 1); each slot has one mbarrier per parity that
//    counts the box bytes.  Every wait is bounded (about 2 s of globaltimer),
//    after which the kernel sets the handle's error flag and stops waiting.
//  * Every value a thread reads -- its own, its x and y neighbours, its z
//    neighbours at the adjacent slices -- comes from shared memory, so the
//    four thread groups of a CTA get equal row counts: group g computes the
//    even class g and the odd class {7, 5, 6, 4}[g] (each pair holds K / 4
//    rows for odd N: 16 at P7, 9 at P5, 4 at P3, 1 at P1).  The
//    register-staged kernel pairs each class with its z-neighbour instead and
//    its largest group holds 20 / 12 / 6 / 2 rows.
#include <cuda.h>
#include <cuda_runtime.h>

#include <dlfcn.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "pn_mbar.cuh"
#include "pn_pdl.cuh"
#include "pn_tiled.cuh"

namespace pn {
namespace tma {

using tiled::Args;
using tiled::ClassTab;
using tiled::MAXC;
using tiled::MAXT;
using tiled::NG;
using tiled::Tab;
using tiled::TabN;
using tiled::TX;

constexpr int TY = 4;
constexpr int BX = TX + 4;        // box width (slots)
constexpr int BY = TY + 1;        // box height (rows)
constexpr int TILE = BX * BY;     // floats per plane and slice
constexpr int DEPTH = 4;          // slice slots per class
constexpr int NT = TX * TY * NG;  // threads per CTA
constexpr int GX = TX + 1, GY = TY + 1, GSL = GX * GY;  // sigma tile: centres x0-1.., y0-1..
constexpr int kOdd[4] = {7, 5, 6, 4};                   // odd class computed by group g

struct Lay {
    int off[8];   // float offset of class c's ring
    int slot[8];  // floats per slot of class c (a multiple of 32: slots stay 128-byte aligned)
    int tx[2];    // bytes one batch of copies delivers (even classes, odd classes)
    int floats;   // ring floats
};

constexpr Lay make_lay(int N) {
    Lay L{};
    const Tab T = tiled::make_tab(N);
    int o = 0;
    for (int c = 0; c < 8; ++c) {
        const int n = T.cls[c].n;
        const int sl = ((n * TILE + 31) / 32) * 32;
        L.off[c] = o;
        L.slot[c] = sl;
        o += DEPTH * sl;
        L.tx[c >> 2] += n * TILE * 4;
    }
    L.floats = o;
    return L;
}

template <int N>
struct LayN {
    static constexpr Lay value = make_lay(N);
};

// Orders 6 and 7 (one CTA per SM) write their outputs through shared memory:
// each thread group stages its two classes' outputs of a z-step (n planes x 4
// rows x 32 slots per class) and one thread stores them with TMA tensor
// stores, instead of one global store per output and thread.  Below order 6
// the staging tile would cost the second CTA per SM.
template <int N>
struct StoreTma {
    static constexpr bool value = N >= 6;
};

// output staging tile: K planes x TY rows x TX slots (floats)
constexpr int ost_floats(int N, bool ts) { return ts ? (N + 1) * (N + 1) * TX * TY : 0; }

// ring, output staging tile (orders >= 6), sigma tile (2 slots x 2 fields),
// 2 x DEPTH mbarriers, alignment slack
constexpr size_t smem_bytes(int N) {
    return size_t(make_lay(N).floats) * 4 + size_t(ost_floats(N, N >= 6)) * 4 + size_t(4 * GSL) * 4 +
           2 * DEPTH * 8 + 128;
}

struct Maps {
    CUtensorMap tm[8];  // one per parity class (unused where the class is empty)
};

// ---- PTX wrappers (mbarriers: pn_mbar.cuh) ----------------------------------

using mbar::smem_u32;

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) { mbar::init(bar, count); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    mbar::arrive_expect_tx(bar, bytes);
}
__device__ __forceinline__ void mbar_wait(uint32_t bar, uint32_t parity, unsigned int* err, bool& failed) {
    mbar::wait(bar, parity, err, failed);
}

// TMA tensor store of a 4D box from shared memory (bulk async-group of the
// issuing thread), its group commit and waits, and the proxy fence that makes
// this thread's shared-memory writes visible to the copy engine
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, uint32_t src, int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// barrier of one thread group (4 warps); id 1 + group (0 is __syncthreads)
__device__ __forceinline__ void group_sync(int grp) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(TX * TY) : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Copies of slice t of every class of parity P (0: classes 0..3, 1: 4..7) into
// ring slot k & 3, completing on that slot's mbarrier.
template <int N, int P>
__device__ __forceinline__ void issue(const Maps& m, uint32_t ring_s, uint32_t bar_s, int k, int t, int x0, int y0) {
    constexpr Lay L = LayN<N>::value;
    constexpr Tab T = TabN<N>::value;
    const int slot = k & (DEPTH - 1);
    const uint32_t bar = bar_s + uint32_t(P * DEPTH + slot) * 8u;
    mbar_arrive_expect_tx(bar, uint32_t(L.tx[P]));
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        const int c = 4 * P + cc;
        if (T.cls[c].n == 0) continue;
        const int bx = c & 1, by = (c >> 1) & 1;
        tma_load_4d(ring_s + uint32_t(L.off[c] + slot * L.slot[c]) * 4u, &m.tm[c], x0 - 4 * (1 - bx), y0 - (1 - by), t,
                    0, bar);
    }
}

// Outputs of class C at slot s from the staged slices.  u: ring slot of the
// even slice s - 1 and the odd slice s; u1: of the even slice s and the odd
// slice s + 1.  Same arithmetic, in the same order, as the register-staged
// kernel's compute_class.
template <int N, int C, int MODE>
__device__ __forceinline__ void tma_class(const Args& a, const float* ring, float* ost, int tx, int ty, int u,
                                          int u1, bool store_ok, bool active, size_t outoff, float st, float ss,
                                          const float (&rhs)[MAXC], float& rrun) {
    constexpr bool TS = StoreTma<N>::value;
    constexpr Tab T = TabN<N>::value;
    constexpr ClassTab CT = T.cls[C];
    constexpr Lay L = LayN<N>::value;
    constexpr int bx = C & 1, by = (C >> 1) & 1, bz = C >> 2;
    constexpr int CXn = C ^ 1, CYn = C ^ 2, CZn = C ^ 4;
    constexpr int nX = T.cls[CXn].n, nY = T.cls[CYn].n, nZ = T.cls[CZn].n;
    if (CT.n == 0) return;
    const int so = bz ? u : u1;  // slot of slice s of this parity
    const int po = (ty + 1 - by) * BX + tx + 4 * (1 - bx);
    const float* own = ring + L.off[C] + so * L.slot[C] + po;
    const float* xb = ring + L.off[CXn] + so * L.slot[CXn] + (ty + 1 - by) * BX + tx + 3 * bx;  // x - bx
    const float* yb = ring + L.off[CYn] + so * L.slot[CYn] + ty * BX + tx + 4 * (1 - bx);       // y - by
    const float* zp = ring + L.off[CZn] + u1 * L.slot[CZn] + po;  // z-neighbour at s + 1 - bz
    const float* zm = ring + L.off[CZn] + u * L.slot[CZn] + po;   // at s - bz
    const uint32_t ps = a.plane_stride;
    float* yo = a.y + size_t(CT.plane0) * ps + outoff;
    const float tscale = a.tsign * a.inv_h;
    float dx[MAXC], dy[MAXC], dz[MAXC];
#pragma unroll
    for (int j = 0; j < MAXC; ++j) {
        if (j < nX) dx[j] = xb[j * TILE + 1] - xb[j * TILE];
        if (j < nY) dy[j] = yb[j * TILE + BX] - yb[j * TILE];
        if (j < nZ) dz[j] = zp[j * TILE] - zm[j * TILE];
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
            float out = fmaf(d, own[i * TILE], tscale * tr);
            if (MODE == OP_RESIDUAL) out = rhs[i] - out;
            out = active ? out : 0.0f;
            if (MODE == OP_RESIDUAL) rrun = fmaf(out, out, rrun);
            if (TS) ost[(CT.plane0 + i) * (TX * TY) + ty * TX + tx] = out;  // rows beyond R: clipped by the store
            else if (store_ok) yo[uint32_t(i) * ps] = out;
        }
    }
}

template <int N, int GRP, int MODE>
__device__ __forceinline__ void run_group(const Maps& m, const Maps& ms, const Args& a, float* ring, float* ost,
                                          float* sg, uint32_t bar_s, int tx, int ty, int za, int zb, double& racc) {
    constexpr bool TS = StoreTma<N>::value;
    const bool elected = tx == 0 && ty == 0;  // issues this group's output stores
    constexpr int CE = GRP, CO = kOdd[GRP];
    constexpr int bxe = CE & 1, bye = (CE >> 1) & 1, bxo = CO & 1, byo = (CO >> 1) & 1;
    constexpr bool same_xy = bxe == bxo && bye == byo;
    const int R = a.R;
    const int tid = tx + TX * (ty + TY * GRP);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool store_ok = x < a.pitch_x && y <= R;
    const bool acte = x < R + bxe && y < R + bye;
    const bool acto = x < R + bxo && y < R + byo;
    const uint32_t col = uint32_t(y) * uint32_t(a.pitch_x) + uint32_t(x);
    const uint32_t ring_s = smem_u32(ring);
    unsigned int* err = a.err;
    bool failed = false;

    // sigma tile cell owned by this thread (two fields), one slice ahead
    const bool sg_own = tid < 2 * GSL;
    const int sg_field = tid / GSL, sg_cell = tid % GSL;
    int64_t sg_off = 0;
    {
        const int gx = sg_cell % GX, gy = sg_cell / GX;
        const int cxr = min(max(x0 - 1 + gx, 0), R - 1), cyr = min(max(y0 - 1 + gy, 0), R - 1);
        sg_off = int64_t(cyr) * R + cxr;
    }
    const float* sgsrc = sg_field == 0 ? a.st : a.ss;
    const int64_t R2 = int64_t(R) * R;
    auto sg_load = [&](int s) -> float {
        const int zc = min(max(s, 0), R - 1);
        return sg_own ? __ldg(sgsrc + zc * R2 + sg_off) : 0.0f;
    };

    if (tid == 0) {
        // prologue copies: even slices za-1 .. za+1, odd za .. za+2 (those consumed)
        issue<N, 0>(m, ring_s, bar_s, 0, za - 1, x0, y0);
        issue<N, 0>(m, ring_s, bar_s, 1, za, x0, y0);
        if (za + 1 <= zb - 1) issue<N, 0>(m, ring_s, bar_s, 2, za + 1, x0, y0);
        issue<N, 1>(m, ring_s, bar_s, 0, za, x0, y0);
        issue<N, 1>(m, ring_s, bar_s, 1, za + 1, x0, y0);
        if (za + 2 <= zb) issue<N, 1>(m, ring_s, bar_s, 2, za + 2, x0, y0);
    }
    if (sg_own) sg[((za + 1) & 1) * 2 * GSL + tid] = sg_load(za - 1);
    float sreg = sg_load(za);
    __syncthreads();
    float mot_prev, mos_prev;  // the odd class's xy-means of the previous slice
    {
        const float* g = sg + ((za + 1) & 1) * 2 * GSL;
        mot_prev = tiled::xy_mean_g(g, GX, tx, ty, bxo, byo);
        mos_prev = tiled::xy_mean_g(g + GSL, GX, tx, ty, bxo, byo);
    }
    float rrun = 0.0f;
    int rcnt = 0;
    for (int s = za; s < zb; ++s) {
        float rhse[MAXC], rhso[MAXC];
        if (MODE == OP_RESIDUAL) {
            tiled::load_rhs<N, CE>(a, acte && s < R, col, s, rhse);
            tiled::load_rhs<N, CO>(a, acto, col, s, rhso);
        }
        float* g = sg + (s & 1) * 2 * GSL;
        if (sg_own) g[tid] = sreg;
        sreg = sg_load(s + 1);
        __syncthreads();
        const int k = s - za;  // ring index of the odd slice s (the even slice s - 1)
        if (tid == 0) {
            if (s + 2 <= zb - 1) issue<N, 0>(m, ring_s, bar_s, k + 3, s + 2, x0, y0);
            if (s + 3 <= zb) issue<N, 1>(m, ring_s, bar_s, k + 3, s + 3, x0, y0);
        }
        const int u = k & (DEPTH - 1), u1 = (k + 1) & (DEPTH - 1);
        if (s == za) {
            mbar_wait(bar_s, 0u, err, failed);
            mbar_wait(bar_s + DEPTH * 8u, 0u, err, failed);
        }
        const uint32_t ph = uint32_t((k + 1) >> 2) & 1u;
        mbar_wait(bar_s + uint32_t(u1) * 8u, ph, err, failed);
        mbar_wait(bar_s + uint32_t(DEPTH + u1) * 8u, ph, err, failed);
        const float met = tiled::xy_mean_g(g, GX, tx, ty, bxe, bye);
        const float mes = tiled::xy_mean_g(g + GSL, GX, tx, ty, bxe, bye);
        const float mot = same_xy ? met : tiled::xy_mean_g(g, GX, tx, ty, bxo, byo);
        const float mos = same_xy ? mes : tiled::xy_mean_g(g + GSL, GX, tx, ty, bxo, byo);
        const size_t outoff = size_t(uint32_t(s) * a.pitch_y) + col;
        if (TS) {
            // the group's staging tile is free once its previous stores have read it
            if (elected) bulk_wait_read0();
            group_sync(GRP);
        }
        tma_class<N, CE, MODE>(a, ring, ost, tx, ty, u, u1, store_ok, acte && s < R, outoff, met, mes, rhse, rrun);
        tma_class<N, CO, MODE>(a, ring, ost, tx, ty, u, u1, store_ok, acto, outoff, 0.5f * (mot + mot_prev),
                               0.5f * (mos + mos_prev), rhso, rrun);
        if (TS) {
            constexpr Tab T = TabN<N>::value;
            fence_async_smem();
            group_sync(GRP);
            if (elected) {
                if (T.cls[CE].n)
                    tma_store_4d(&ms.tm[CE], smem_u32(ost + T.cls[CE].plane0 * (TX * TY)), x0, y0, s, 0);
                if (T.cls[CO].n)
                    tma_store_4d(&ms.tm[CO], smem_u32(ost + T.cls[CO].plane0 * (TX * TY)), x0, y0, s, 0);
                bulk_commit();
            }
        }
        if (MODE == OP_RESIDUAL && ++rcnt == 4) {
            racc += double(rrun);
            rrun = 0.0f;
            rcnt = 0;
        }
        mot_prev = mot;
        mos_prev = mos;
    }
    racc += double(rrun);
    if (TS && elected) bulk_wait0();  // the group's last stores are complete
    if (tid == 0) {
        // every copy issued above was waited for; after a wait that ran out,
        // wait (bounded) for the last copy of each slot before returning
        bool f2 = false;
        if (failed) {
            const int kmax[2] = {zb - za, zb - za};  // even: k in [0, zb-za]; odd: k in [0, zb-za]
            for (int p = 0; p < 2; ++p)
                for (int j = 0; j < DEPTH; ++j) {
                    if (j > kmax[p]) continue;
                    const int kl = j + ((kmax[p] - j) / DEPTH) * DEPTH;
                    mbar_wait(bar_s + uint32_t(p * DEPTH + j) * 8u, uint32_t(kl >> 2) & 1u, err, f2);
                }
        }
    }
}

// two CTAs per SM where their shared memory fits and 64 registers suffice
template <int N, int MODE>
__global__ void __launch_bounds__(NT, (N <= 4 || (N == 5 && MODE != OP_RESIDUAL)) ? 2 : 1)
    k_apply_tma(const __grid_constant__ Maps m, const __grid_constant__ Maps ms, Args a) {
    // programmatic dependent launch: the input (and the gate) come from the
    // previous kernel; the next kernel may start once every CTA has finished
    // its z-march (the trigger below).  With a.late_wait the previous kernel
    // is the face-column kernel, which triggered right after its own wait:
    // the input is complete already, and the wait at the end makes this
    // kernel complete only after the face outputs (for the kernel after it).
    if (!a.late_wait) pdl_wait();
    if (a.live && !*a.live) return;  // uniform over the grid (never with late_wait)
    constexpr Lay L = LayN<N>::value;
    extern __shared__ __align__(128) unsigned char dsm[];
    float* ring = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(dsm) + 127) & ~uintptr_t(127));
    float* ost = ring + L.floats;  // output staging tile (orders >= 6), 128-byte aligned
    float* sg = ost + ost_floats(N, StoreTma<N>::value);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sg + 4 * GSL);
    const uint32_t bar_s = smem_u32(bars);
    // warp w runs group w % 4: each of the SM's four schedulers (warps are
    // spread over them by warp index) executes one group's code, so its
    // instruction cache holds one of the four specialised bodies
    const int tx = threadIdx.x, grp = threadIdx.y, ty = threadIdx.z;
    const int tid = tx + TX * (ty + TY * grp);
    const int za = blockIdx.z * a.zc;
    const int zb = min(za + a.zc, a.R + 1);
    if (tid == 0) {
        for (int i = 0; i < 2 * DEPTH; ++i) mbar_init(bar_s + uint32_t(i) * 8u, 1u);
        mbar::fence_init();
    }
    __syncthreads();
    double racc = 0.0;
    switch (grp) {
        case 0: run_group<N, 0, MODE>(m, ms, a, ring, ost, sg, bar_s, tx, ty, za, zb, racc); break;
        case 1: run_group<N, 1, MODE>(m, ms, a, ring, ost, sg, bar_s, tx, ty, za, zb, racc); break;
        case 2: run_group<N, 2, MODE>(m, ms, a, ring, ost, sg, bar_s, tx, ty, za, zb, racc); break;
        default: run_group<N, 3, MODE>(m, ms, a, ring, ost, sg, bar_s, tx, ty, za, zb, racc); break;
    }
    if (a.late_wait) pdl_wait();
    pdl_trigger();
    if (MODE == OP_RESIDUAL && a.partials != nullptr) {
        __shared__ double red[NT / 32];
        for (int o = 16; o > 0; o >>= 1) racc += __shfl_down_sync(0xffffffffu, racc, o);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = racc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int i = 0; i < NT / 32; ++i) t += red[i];
            a.partials[(int64_t(blockIdx.z) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
        }
    }
}

// ---- host side ------------------------------------------------------------------

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder: through the runtime's entry-point query,
// else from the driver library itself (some profiler shims do not forward the
// query); null if neither has it (the register-staged kernel then runs).
EncodeTiled encode_fn() {
    static const EncodeTiled fn = []() -> EncodeTiled {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && p)
            return reinterpret_cast<EncodeTiled>(p);
        cudaGetLastError();
        void* lib = dlopen("libcuda.so.1", RTLD_NOW | RTLD_LOCAL);
        if (!lib) return nullptr;
        p = dlsym(lib, "cuTensorMapEncodeTiled");
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

// Tensor maps of recently used input vectors (the Krylov solvers apply the
// operator to a fixed set of buffers).
struct Cache {
    struct Entry {
        const void* x;
        bool store;  // maps of an output vector (the whole padded box of each class)
        Maps m;
    };
    std::vector<Entry> e;
    size_t next = 0;
};
constexpr size_t kCacheEntries = 48;

// Load maps (store = false): each class's active extents, so that the copy
// engine writes 0 for inactive and out-of-domain slots.  Store maps: the whole
// padded box of each class's planes (the kernel writes 0 into the inactive
// slots of its tile; rows beyond the box are clipped).
bool encode_maps(const pn_handle* h, const void* x, Maps& m, bool store) {
    const EncodeTiled enc = encode_fn();
    if (!enc) return false;
    std::memset(&m, 0, sizeof(m));
    int n[8] = {0, 0, 0, 0, 0, 0, 0, 0}, p0[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = h->K - 1; p >= 0; --p) {
        ++n[h->plane_class[p]];
        p0[h->plane_class[p]] = p;
    }
    for (int c = 0; c < 8; ++c) {
        if (n[c] == 0) continue;
        const int bx = c & 1, by = (c >> 1) & 1, bz = c >> 2;
        const cuuint64_t dim[4] = {store ? cuuint64_t(h->pitch_x) : cuuint64_t(h->R + bx),
                                   cuuint64_t(store ? h->R + 1 : h->R + by), cuuint64_t(store ? h->R + 1 : h->R + bz),
                                   cuuint64_t(n[c])};
        const cuuint64_t str[3] = {cuuint64_t(h->pitch_x) * 4, cuuint64_t(h->pitch_y) * 4,
                                   cuuint64_t(h->plane_stride) * 4};
        const cuuint32_t box[4] = {cuuint32_t(store ? TX : BX), cuuint32_t(store ? TY : BY), 1u, cuuint32_t(n[c])};
        const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
        void* base = const_cast<char*>(static_cast<const char*>(x)) + size_t(p0[c]) * h->plane_stride * 4;
        if (enc(&m.tm[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dim, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

const Maps* maps_for(const pn_handle* h, const void* x, bool store) {
    pn_handle* hm = const_cast<pn_handle*>(h);
    Cache* c = static_cast<Cache*>(hm->tma_cache);
    if (!c) {
        c = new Cache();
        c->e.reserve(kCacheEntries);
        hm->tma_cache = c;
    }
    for (const auto& e : c->e)
        if (e.x == x && e.store == store) return &e.m;
    Cache::Entry ne;
    ne.x = x;
    ne.store = store;
    if (!encode_maps(h, x, ne.m, store)) return nullptr;
    if (c->e.size() < kCacheEntries) {
        c->e.push_back(ne);
        return &c->e.back().m;
    }
    Cache::Entry& slot = c->e[c->next];
    c->next = (c->next + 1) % kCacheEntries;
    slot = ne;
    return &slot.m;
}

template <int N, int MODE>
cudaError_t launch_n(const Maps& m, const Maps& ms, const Args& a, dim3 grid, cudaStream_t s, bool pdl) {
    auto kern = k_apply_tma<N, MODE>;
    static std::atomic<unsigned long long> configured{0};
    const size_t bytes = smem_bytes(N);
    cudaError_t e = pn_smem_attr_once(configured, reinterpret_cast<const void*>(kern), int(bytes));
    if (e != cudaSuccess) return e;
    return launch_pdl(pdl, kern, grid, dim3(TX, NG, TY), bytes, s, m, ms, a);
}

template <int MODE>
cudaError_t launch_mode(const pn_handle* h, const Maps& m, const Maps& ms, const Args& a, dim3 grid,
                        cudaStream_t s) {
    const bool pdl = h->pdl != 0;
    switch (h->N) {
        case 0: return launch_n<0, MODE>(m, ms, a, grid, s, pdl);
        case 1: return launch_n<1, MODE>(m, ms, a, grid, s, pdl);
        case 2: return launch_n<2, MODE>(m, ms, a, grid, s, pdl);
        case 3: return launch_n<3, MODE>(m, ms, a, grid, s, pdl);
        case 4: return launch_n<4, MODE>(m, ms, a, grid, s, pdl);
        case 5: return launch_n<5, MODE>(m, ms, a, grid, s, pdl);
        case 6: return launch_n<6, MODE>(m, ms, a, grid, s, pdl);
        default: return launch_n<7, MODE>(m, ms, a, grid, s, pdl);
    }
}

}  // namespace tma

void* tensor_map_encoder() { return reinterpret_cast<void*>(tma::encode_fn()); }

bool tma_serves(const pn_handle* h) {
    if (!tiled_serves(h) || h->N > 7 || !tma::encode_fn()) return false;
    // the tile geometry is fixed (32 x 4 columns); x must be 16-byte aligned,
    // which every entry point checks
    return tma::smem_bytes(h->N) <= 227 * 1024;
}

cudaError_t launch_tma_main(const pn_handle* h, int mode, const tiled::Args& a, dim3 grid, cudaStream_t s) {
    if (!tma_serves(h)) return cudaErrorNotSupported;
    const tma::Maps* m = tma::maps_for(h, a.x, false);
    if (!m) return cudaErrorInvalidValue;
    const tma::Maps* ms = m;  // unused below order 6
    if (h->N >= 6) {
        // the output's maps (the tile store needs a 16-byte aligned, padded y)
        ms = tma::maps_for(h, a.y, true);
        if (!ms) return cudaErrorInvalidValue;
        m = tma::maps_for(h, a.x, false);  // (the cache may have moved the entry)
        if (!m) return cudaErrorInvalidValue;
    }
    if (mode == OP_RESIDUAL) return tma::launch_mode<OP_RESIDUAL>(h, *m, *ms, a, grid, s);
    return tma::launch_mode<OP_APPLY>(h, *m, *ms, a, grid, s);
}

void tma_cache_free(pn_handle* h) {
    delete static_cast<tma::Cache*>(h->tma_cache);
    h->tma_cache = nullptr;
}

}  // namespace pn
