// 3x3x3 convolution of the learned preconditioner's network on the fifth-
// generation tensor cores (tcgen05), as an implicit GEMM:
//
//     out[v][o] = act(bias[o] + sum_{tap} sum_c in[v + tap][c] w[tap][o][c])
//
// M = 128 voxels of one tile (8 x 16 y 1 z of one sample), N = n <= 64 output
// channels (the host splits wider layers into launches of at most 64), K = 27
// taps x input channels.  BF16 operands, FP32 accumulation in tensor memory
// (TMEM).
//
//  * The tile's input, with its one-voxel halo, reaches shared memory by TMA
//    once per 16-channel block: two boxes (channels c..c+7 and c+8..c+15) of
//    10 x 18 x 3 voxels from a 5D tensor map (channels, x, y, z, sample); the
//    copy engine writes 0 for coordinates outside the grid (the convolution's
//    zero padding).  The weights of all 27 taps for the block come with it:
//    two boxes of 8 channels x n rows x 27 taps ([tap][o][c]).
//  * Both operands are then in the canonical K-major layout without swizzle
//    (core matrices of 8 rows x 16 bytes): for tap (dx, dy, dz) the A operand
//    is the block shifted by (dx, dy, dz) -- rows x = 0..7 of one tile row are
//    8 consecutive 16-byte rows of the block, the next tile row 10 rows (160
//    bytes) on (stride byte offset), the second 8 channels one box on (leading
//    byte offset) -- so one block serves the 27 MMAs of the 16-channel step
//    (tcgen05.mma.cta_group::1.kind::f16, 128 x n x 16).
//  * One thread issues the copies into a ring of slots (one 16-channel block
//    each) and the MMAs; each block's commit frees its slot; after the last
//    one the four warps read the accumulator (tcgen05.ld 32x32b, warp w owns
//    TMEM lanes 32w..32w+31 = voxels of the tile), add the bias, apply the ReLU
//    and store BF16.
//  * Every wait is bounded (about 2 s of %globaltimer); one that runs out sets
//    the network's error word, the kernel waits (bounded) for its copies in
//    flight and for its MMAs, and still frees its TMEM before it returns.
//
// The input gradient of a layer is this kernel on the tap-flipped, transposed
// weights ([tap][c][o]).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "pn_cnn.h"
#include "pn_internal.h"
#include "pn_mbar.cuh"

namespace pn {
namespace cnn {
namespace tc {

constexpr int kThreads = 128;
constexpr int kMaxN = 64;                 // output channels per launch
constexpr int HX = 10, HY = 18, HZ = 3;   // halo'd input block (voxels)
constexpr uint32_t kABytes = 8u * HX * HY * HZ * 2u;  // one 8-channel box: 8640
constexpr uint32_t kASlot = 8704;         // its slot (128-byte multiple)

// bytes of one ring slot for n output channels: two input boxes and two
// weight boxes (27 taps x n rows x 8 channels each), rounded to 1024
__host__ __device__ constexpr uint32_t wbox_bytes(int n) { return 27u * uint32_t(n) * 16u; }
__host__ __device__ constexpr uint32_t slot_bytes(int n) { return (2 * kASlot + 2 * wbox_bytes(n) + 1023u) / 1024u * 1024u; }
__host__ __device__ constexpr int stages_for(int n) { return n <= 32 ? 3 : 2; }
__host__ __device__ constexpr uint32_t smem_bytes(int n) { return uint32_t(stages_for(n)) * slot_bytes(n) + 1024u; }

struct Args {
    int n;               // output channels of this launch (16..64, a multiple of 16)
    int in_co;           // first input channel of the slice read
    int kc;              // input channels / 16
    int o0;              // first output channel (row of the weights, offset of bias and output)
    int ntx, nty;        // tiles per axis (8 x, 16 y; one z slice per tile)
    int X, Y, Z;
    const float* bias;   // or null
    bf16* out;
    int out_cs, out_co;
    int relu;
    uint32_t idesc;      // instruction descriptor (kind::f16, BF16 x BF16 -> F32, M = 128, N = n)
    uint32_t tmem_cols;  // power of two >= max(32, n)
    unsigned int* err;   // set to 1 where a bounded wait ran out
};

// ---- PTX wrappers ---------------------------------------------------------------

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor: start address, leading byte offset (next
// core matrix along K), stride byte offset (next 8 rows), descriptor version
// 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrives on `bar` once every MMA this thread issued before it has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_conv3_tc(const __grid_constant__ CUtensorMap act, const __grid_constant__ CUtensorMap wts, Args a) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    constexpr int kMaxStages = 3;
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], done;
    __shared__ uint32_t tmem_slot;
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
    const uint32_t ring_s = mbar::smem_u32(ring);
    const uint32_t SB = slot_bytes(a.n);
    const int S = stages_for(a.n);
    const uint32_t WB = wbox_bytes(a.n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // tile of this CTA: 8 x 16 y voxels of one z slice of one sample
    int t = blockIdx.x;
    const int tx = t % a.ntx;
    t /= a.ntx;
    const int ty = t % a.nty;
    t /= a.nty;
    const int z0 = t % a.Z;
    const int b = t / a.Z;
    const int x0 = tx * 8, y0 = ty * 16;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar::init(mbar::smem_u32(&full[s]), 1u);
            mbar::init(mbar::smem_u32(&empty[s]), 1u);
        }
        mbar::init(mbar::smem_u32(&done), 1u);
        mbar::fence_init();
    }
    if (warp == 0) {
        // the accumulator: 128 lanes x tmem_cols FP32 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         mbar::smem_u32(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;

    const int steps = a.kc;  // 16-channel blocks
    const uint32_t tx_bytes = 2 * kABytes + 2 * WB;
    bool failed = false;
    if (threadIdx.x == 0) {
        auto issue = [&](int k) {
            const int slot = k % S;
            const uint32_t bar = mbar::smem_u32(&full[slot]);
            const uint32_t sa = ring_s + uint32_t(slot) * SB;
            const uint32_t sb = sa + 2 * kASlot;
            const int c = a.in_co + k * 16;
            mbar::arrive_expect_tx(bar, tx_bytes);
            tma_load_5d(sa, &act, c, x0 - 1, y0 - 1, z0 - 1, b, bar);
            tma_load_5d(sa + kASlot, &act, c + 8, x0 - 1, y0 - 1, z0 - 1, b, bar);
            tma_load_3d(sb, &wts, k * 16, a.o0, 0, bar);
            tma_load_3d(sb + WB, &wts, k * 16 + 8, a.o0, 0, bar);
        };
        const int pro = steps < S ? steps : S;
        int issued = 0;    // blocks whose copies went out
        int consumed = 0;  // blocks whose copies were waited for
        for (int k = 0; k < pro; ++k, ++issued) issue(k);
        for (int k = 0; k < steps && !failed; ++k) {
            const int slot = k % S;
            mbar::wait(mbar::smem_u32(&full[slot]), uint32_t(k / S) & 1u, a.err, failed);
            if (failed) break;
            consumed = k + 1;
            fence_after_sync();
            const uint32_t sa = ring_s + uint32_t(slot) * SB;
            const uint32_t sb = sa + 2 * kASlot;
            for (int tap = 0; tap < 27; ++tap) {
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;  // 0..2: offset + 1
                const uint32_t a0 = sa + uint32_t((dz * HY + dy) * HX + dx) * 16u;
                const uint64_t ad = smem_desc(a0, kASlot, uint32_t(HX) * 16u);
                const uint64_t bd = smem_desc(sb + uint32_t(tap) * uint32_t(a.n) * 16u, WB, 128u);
                mma_bf16(tmem, ad, bd, a.idesc, (k > 0 || tap > 0) ? 1u : 0u);
            }
            mma_commit(mbar::smem_u32(&empty[slot]));
            // refill the previous block's slot with the block S after it
            const int kp = k - 1, kn = kp + S;
            if (kp >= 0 && kn < steps) {
                mbar::wait(mbar::smem_u32(&empty[kp % S]), uint32_t(kp / S) & 1u, a.err, failed);
                if (!failed) {
                    issue(kn);
                    ++issued;
                }
            }
        }
        // every MMA issued has completed once `done` flips
        mma_commit(mbar::smem_u32(&done));
        if (failed) {
            // wait (bounded) for the copies still in flight: blocks [consumed, issued)
            bool f2 = false;
            for (int k = consumed; k < issued; ++k)
                mbar::wait(mbar::smem_u32(&full[k % S]), uint32_t(k / S) & 1u, a.err, f2);
        }
    }
    __syncwarp();
    // the accumulator is complete (or the kernel gave up: the error word is set)
    {
        bool f3 = false;
        mbar::wait(mbar::smem_u32(&done), 0u, a.err, f3);
    }
    fence_after_sync();

    // epilogue: warp w holds voxels 32w..32w+31 of the tile (TMEM lanes)
    const int m = warp * 32 + lane;
    const int vx = x0 + (m & 7), vy = y0 + (m >> 3);
    const bool ok = vx < a.X && vy < a.Y;
    const int64_t v = ((int64_t(b) * a.Z + z0) * a.Y + vy) * a.X + vx;
    bf16* op = a.out + v * a.out_cs + a.out_co + a.o0;
    const float* bias = a.bias ? a.bias + a.o0 : nullptr;
    for (int c0 = 0; c0 < a.n; c0 += 16) {
        float r[16];
        tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), r);
        uint32_t pk[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float lo = r[2 * i], hi = r[2 * i + 1];
            if (bias) {
                lo += bias[c0 + 2 * i];
                hi += bias[c0 + 2 * i + 1];
            }
            if (a.relu) {
                lo = fmaxf(lo, 0.0f);
                hi = fmaxf(hi, 0.0f);
            }
            pk[i] = pack_bf16x2(lo, hi);
        }
        if (ok) {
            uint4* dst = reinterpret_cast<uint4*>(op + c0);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

// ---- weight gradient --------------------------------------------------------------
//
//     dW[tap][o][c] += sum_v gy[v][o] x[v + tap][c]
//
// as D = A B per group of taps: M = 128 rows = (tap of the group, input
// channel) -- 128 / ci taps stacked, the rows beyond them unused -- N = n <= 64
// output channels, K = voxels.  Both operands come straight from the
// channels-last tensors, so both are MN-major (the 8 channels of one 16-byte
// row of a core matrix are the M or N index, its 8 rows 8 consecutive voxels):
// per 128-voxel tile (8 x 16 y 1 z of one sample) the x slice of each stacked
// tap arrives as 8-channel boxes (x, y, z shifted by the tap; coordinates
// outside the grid read as 0), the gradient of the output as 8-channel boxes
// of the unshifted tile.  In a box the voxel rows are 16 bytes apart: the next
// 8 voxels (K) are 128 bytes on (leading byte offset), the next 8 channels (M
// or N) one box (2048 bytes) on (stride byte offset).  Each CTA walks a range
// of tiles, accumulating in TMEM, and adds its sums to dW with FP32 atomics.
constexpr uint32_t kWBox = 2048;  // 8 channels x 128 voxels

struct WArgs {
    int ci, n;           // input channels of the layer; output channels of this launch (16..64)
    int x_co, gy_co;     // channel offsets of the slices read
    int o0;              // first output channel of this launch
    int taps_per;        // taps stacked in M (128 / ci, at most 27); group g holds taps g * taps_per ...
    int nchunks;         // CTAs per group: CTA b takes group b / nchunks, tile chunk b % nchunks
    int ntx, nty, Z;     // tiles per axis and slices (one z slice per tile)
    int64_t tiles;       // tiles in total
    int64_t per;         // tiles per chunk
    float* dw;           // [27][co][ci]
    int co;              // output channels of the layer (row stride of dw)
    uint32_t idesc;
    uint32_t tmem_cols;
    unsigned int* err;
};

__host__ __device__ constexpr uint32_t wslot_bytes(int n) { return 16u * kWBox + uint32_t(n / 8) * kWBox; }
constexpr int kWStages = 3;
__host__ __device__ constexpr uint32_t wsmem_bytes(int n) { return kWStages * wslot_bytes(n) + 1024u; }

__global__ void __launch_bounds__(kThreads, 1)
    k_conv3_wgrad_tc(const __grid_constant__ CUtensorMap xm, const __grid_constant__ CUtensorMap gm, WArgs a) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ __align__(8) uint64_t full[kWStages], empty[kWStages], done;
    __shared__ uint32_t tmem_slot;
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
    const uint32_t ring_s = mbar::smem_u32(ring);
    const uint32_t SB = wslot_bytes(a.n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int group = int(blockIdx.x) / a.nchunks, chunk = int(blockIdx.x) % a.nchunks;
    const int t0 = group * a.taps_per;
    const int ntap = 27 - t0 < a.taps_per ? 27 - t0 : a.taps_per;
    const int64_t tb = int64_t(chunk) * a.per;
    const int64_t te = tb + a.per < a.tiles ? tb + a.per : a.tiles;
    const int steps = te > tb ? int(te - tb) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kWStages; ++s) {
            mbar::init(mbar::smem_u32(&full[s]), 1u);
            mbar::init(mbar::smem_u32(&empty[s]), 1u);
        }
        mbar::init(mbar::smem_u32(&done), 1u);
        mbar::fence_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         mbar::smem_u32(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int cg = a.ci / 8;  // 8-channel groups per tap
    const uint32_t tx_bytes = uint32_t(ntap * cg + a.n / 8) * kWBox;
    bool failed = false;
    if (threadIdx.x == 0 && steps > 0) {
        auto issue = [&](int k) {
            int64_t t = tb + k;
            const int tx = int(t % a.ntx);
            t /= a.ntx;
            const int ty = int(t % a.nty);
            t /= a.nty;
            const int z0 = int(t % a.Z);
            const int b = int(t / a.Z);
            const int x0 = tx * 8, y0 = ty * 16;
            const int slot = k % kWStages;
            const uint32_t bar = mbar::smem_u32(&full[slot]);
            const uint32_t sa = ring_s + uint32_t(slot) * SB;
            mbar::arrive_expect_tx(bar, tx_bytes);
            for (int j = 0; j < ntap; ++j) {
                const int tap = t0 + j;
                const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                for (int g = 0; g < cg; ++g)
                    tma_load_5d(sa + uint32_t(j * cg + g) * kWBox, &xm, a.x_co + 8 * g, x0 + dx, y0 + dy, z0 + dz, b,
                                bar);
            }
            const uint32_t sb = sa + 16u * kWBox;
            for (int g = 0; g < a.n / 8; ++g)
                tma_load_5d(sb + uint32_t(g) * kWBox, &gm, a.gy_co + a.o0 + 8 * g, x0, y0, z0, b, bar);
        };
        const int pro = steps < kWStages ? steps : kWStages;
        int issued = 0, consumed = 0;
        for (int k = 0; k < pro; ++k, ++issued) issue(k);
        for (int k = 0; k < steps && !failed; ++k) {
            const int slot = k % kWStages;
            mbar::wait(mbar::smem_u32(&full[slot]), uint32_t(k / kWStages) & 1u, a.err, failed);
            if (failed) break;
            consumed = k + 1;
            fence_after_sync();
            const uint32_t sa = ring_s + uint32_t(slot) * SB;
            const uint32_t sb = sa + 16u * kWBox;
            for (int kk = 0; kk < 8; ++kk) {  // 16 voxels per MMA
                const uint64_t ad = smem_desc(sa + uint32_t(kk) * 256u, 128u, kWBox);
                const uint64_t bd = smem_desc(sb + uint32_t(kk) * 256u, 128u, kWBox);
                mma_bf16(tmem, ad, bd, a.idesc, (k > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(mbar::smem_u32(&empty[slot]));
            const int kp = k - 1, kn = kp + kWStages;
            if (kp >= 0 && kn < steps) {
                mbar::wait(mbar::smem_u32(&empty[kp % kWStages]), uint32_t(kp / kWStages) & 1u, a.err, failed);
                if (!failed) {
                    issue(kn);
                    ++issued;
                }
            }
        }
        mma_commit(mbar::smem_u32(&done));
        if (failed) {
            bool f2 = false;
            for (int k = consumed; k < issued; ++k)
                mbar::wait(mbar::smem_u32(&full[k % kWStages]), uint32_t(k / kWStages) & 1u, a.err, f2);
        }
    }
    __syncwarp();
    if (steps > 0) {
        bool f3 = false;
        mbar::wait(mbar::smem_u32(&done), 0u, a.err, f3);
        fence_after_sync();
        // row m of D = (tap j of the group, channel c); its n columns = output channels
        const int m = warp * 32 + lane;
        const int j = m / a.ci, c = m % a.ci;
        const bool ok = j < ntap;
        float* dst = a.dw + (int64_t(t0 + j) * a.co + a.o0) * a.ci + c;
        for (int c0 = 0; c0 < a.n; c0 += 16) {
            float r[16];
            tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), r);
            if (ok) {
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(dst + int64_t(c0 + i) * a.ci, r[i]);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

// ---- host ------------------------------------------------------------------------

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace tc

bool conv3_tc_serves(const ConvArgs& a) {
    return tensor_map_encoder() != nullptr && a.ci % 16 == 0 && a.co % 16 == 0 && a.co >= 16 && a.co <= 256 &&
           a.co_total == a.co && a.in_cs % 8 == 0 && a.in_co % 8 == 0 && a.out_cs % 8 == 0 && a.out_co % 8 == 0 &&
           (reinterpret_cast<uintptr_t>(a.in) & 15u) == 0 && (reinterpret_cast<uintptr_t>(a.w) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(a.out) & 15u) == 0 && a.g.nvox > 0;
}

cudaError_t conv3_tc(const ConvArgs& a, unsigned int* err, cudaStream_t s) {
    const tc::EncodeTiled enc = reinterpret_cast<tc::EncodeTiled>(tensor_map_encoder());
    if (!enc || !conv3_tc_serves(a)) return cudaErrorNotSupported;
    CUtensorMap act;
    std::memset(&act, 0, sizeof(act));
    {
        const cuuint64_t dim[5] = {cuuint64_t(a.in_cs), cuuint64_t(a.g.X), cuuint64_t(a.g.Y), cuuint64_t(a.g.Z),
                                   cuuint64_t(a.g.B)};
        const cuuint64_t row = cuuint64_t(a.in_cs) * 2;
        const cuuint64_t str[4] = {row, row * a.g.X, row * a.g.X * a.g.Y, row * a.g.X * a.g.Y * a.g.Z};
        const cuuint32_t box[5] = {8u, cuuint32_t(tc::HX), cuuint32_t(tc::HY), cuuint32_t(tc::HZ), 1u};
        const cuuint32_t es[5] = {1u, 1u, 1u, 1u, 1u};
        if (enc(&act, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(a.in), dim, str, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    static std::atomic<unsigned long long> configured{0};
    uint32_t smem_max = 0;
    for (int n = 16; n <= tc::kMaxN; n += 16) smem_max = std::max(smem_max, tc::smem_bytes(n));
    cudaError_t e = pn_smem_attr_once(configured, reinterpret_cast<const void*>(tc::k_conv3_tc), int(smem_max));
    if (e != cudaSuccess) return e;
    const int ntx = (a.g.X + 7) / 8, nty = (a.g.Y + 15) / 16;
    const int64_t tiles = int64_t(ntx) * nty * a.g.Z * a.g.B;
    if (tiles > 0x7FFFFFFF) return cudaErrorInvalidValue;
    // output channels in launches of at most 64 (the accumulator's width)
    for (int o0 = 0; o0 < a.co; o0 += tc::kMaxN) {
        const int n = std::min(tc::kMaxN, a.co - o0);
        CUtensorMap wts;
        std::memset(&wts, 0, sizeof(wts));
        const cuuint64_t dim[3] = {cuuint64_t(a.ci), cuuint64_t(a.co), 27};
        const cuuint64_t str[2] = {cuuint64_t(a.ci) * 2, cuuint64_t(a.ci) * 2 * a.co};
        const cuuint32_t box[3] = {8u, cuuint32_t(n), 27u};
        const cuuint32_t es[3] = {1u, 1u, 1u};
        if (enc(&wts, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(a.w), dim, str, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        tc::Args p{};
        p.n = n;
        p.in_co = a.in_co;
        p.kc = a.ci / 16;
        p.o0 = o0;
        p.ntx = ntx;
        p.nty = nty;
        p.X = a.g.X;
        p.Y = a.g.Y;
        p.Z = a.g.Z;
        p.bias = a.bias;
        p.out = a.out;
        p.out_cs = a.out_cs;
        p.out_co = a.out_co;
        p.relu = a.relu;
        // kind::f16 instruction descriptor: D F32 (bits 4-5 = 1), A and B BF16
        // (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit
        // 17, M >> 4 at bit 24
        p.idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
        uint32_t cols = 32;
        while (cols < uint32_t(n)) cols <<= 1;
        p.tmem_cols = cols;
        p.err = err;
        tc::k_conv3_tc<<<unsigned(tiles), tc::kThreads, tc::smem_bytes(n), s>>>(act, wts, p);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cnn
}  // namespace pn

namespace pn {
namespace cnn {

bool conv3_wgrad_tc_serves(const WgradArgs& a) {
    return tensor_map_encoder() != nullptr && a.ci % 16 == 0 && a.ci <= 128 && a.co % 16 == 0 && a.co >= 16 &&
           a.x_cs % 8 == 0 && a.x_co % 8 == 0 && a.gy_cs % 8 == 0 && a.gy_co % 8 == 0 &&
           (reinterpret_cast<uintptr_t>(a.x) & 15u) == 0 && (reinterpret_cast<uintptr_t>(a.gy) & 15u) == 0 &&
           a.g.nvox > 0;
}

// dW[tap][o][c] += sum_v gy[v][o] x[v + tap][c] on the tcgen05 tensor cores;
// the bias gradient is left to the caller.
cudaError_t conv3_wgrad_tc(const WgradArgs& a, unsigned int* err, cudaStream_t s) {
    const tc::EncodeTiled enc = reinterpret_cast<tc::EncodeTiled>(tensor_map_encoder());
    if (!enc || !conv3_wgrad_tc_serves(a)) return cudaErrorNotSupported;
    // 5D maps (channels, x, y, z, sample) with 8-channel x 8 x 16 x 1 boxes
    auto map5 = [&](CUtensorMap& m, const bf16* base, int cs) -> bool {
        std::memset(&m, 0, sizeof(m));
        const cuuint64_t dim[5] = {cuuint64_t(cs), cuuint64_t(a.g.X), cuuint64_t(a.g.Y), cuuint64_t(a.g.Z),
                                   cuuint64_t(a.g.B)};
        const cuuint64_t row = cuuint64_t(cs) * 2;
        const cuuint64_t str[4] = {row, row * a.g.X, row * a.g.X * a.g.Y, row * a.g.X * a.g.Y * a.g.Z};
        const cuuint32_t box[5] = {8u, 8u, 16u, 1u, 1u};
        const cuuint32_t es[5] = {1u, 1u, 1u, 1u, 1u};
        return enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(base), dim, str, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap xm, gm;
    if (!map5(xm, a.x, a.x_cs) || !map5(gm, a.gy, a.gy_cs)) return cudaErrorInvalidValue;
    static std::atomic<unsigned long long> configured{0};
    cudaError_t e = pn_smem_attr_once(configured, reinterpret_cast<const void*>(tc::k_conv3_wgrad_tc),
                                      int(tc::wsmem_bytes(tc::kMaxN)));
    if (e != cudaSuccess) return e;
    const int ntx = (a.g.X + 7) / 8, nty = (a.g.Y + 15) / 16;
    const int64_t tiles = int64_t(ntx) * nty * a.g.Z * a.g.B;
    const int taps_per = std::min(27, 128 / a.ci);
    const int groups = (27 + taps_per - 1) / taps_per;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    for (int o0 = 0; o0 < a.co; o0 += tc::kMaxN) {
        const int n = std::min(tc::kMaxN, a.co - o0);
        // one launch: every tap group x chunks of tiles, about four CTAs per SM
        const int64_t want = std::max<int64_t>(1, (4 * int64_t(sms) + groups - 1) / groups);
        const int64_t chunks = std::min<int64_t>(tiles, want);
        const int64_t per = (tiles + chunks - 1) / chunks;
        const int64_t nchunks = (tiles + per - 1) / per;
        tc::WArgs p{};
        p.ci = a.ci;
        p.n = n;
        p.x_co = a.x_co;
        p.gy_co = a.gy_co;
        p.o0 = o0;
        p.taps_per = taps_per;
        p.nchunks = int(nchunks);
        p.ntx = ntx;
        p.nty = nty;
        p.Z = a.g.Z;
        p.tiles = tiles;
        p.per = per;
        p.dw = a.dw;
        p.co = a.co;
        // kind::f16: D F32, A and B BF16, both MN-major (bits 15, 16 = 1), N >> 3 at bit 17, M >> 4 at bit 24
        p.idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | (uint32_t(n >> 3) << 17) |
                  (uint32_t(128 >> 4) << 24);
        uint32_t cols = 32;
        while (cols < uint32_t(n)) cols <<= 1;
        p.tmem_cols = cols;
        p.err = err;
        tc::k_conv3_wgrad_tc<<<unsigned(nchunks * groups), tc::kThreads, tc::wsmem_bytes(n), s>>>(xm, gm, p);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cnn
}  // namespace pn
