// tc_conv.cu - fused teacher inference on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// The whole network of Sec. 2.2 (dense computation with stride-1 max-filtering) runs in one
// persistent kernel; intermediates never leave the SM:
//   layer 1   conv5x5 1->32 + bias + ReLU    FP32 on CUDA cores (weights are kernel constants)
//   maxfilter 2x2 stride 1                    fused into the layer-1 producer
//   layer 2   conv5x5 32->32                  tcgen05.mma, BF16 or E4M3 operands, FP32 in TMEM
//   + bias + ReLU + maxfilter                 fused into the layer-2 epilogue (TMEM -> regs)
//   layer 3   conv5x5 32->32                  tcgen05.mma
//   + bias + ReLU + head 1x1 + sigmoid        fused into the layer-3 epilogue, stored to HBM
//
// Work item: one slice, a strip of 118 output columns, a run of output rows: either chunks of a
// tuned length taken round-robin, or the parts of one equal contiguous range of strip-rows per CTA
// (a compile-time choice, tuned per workload for BF16; always the ranges for FP8). Each CTA walks
// its items row by row. The layer-2/3 implicit GEMM per input row r:
//   M = 128 pixels of the row, K = 32 channels (x 5 column taps dx), N = 5 row taps x 32 outputs.
// The five row taps dy are stacked along N, so one input row is multiplied once and its five
// 32-column result blocks accumulate into the TMEM accumulators of output rows r-4 .. r (a ring
// of 8 row accumulators per layer); the column tap dx is a 16-byte shift of the A descriptor's
// start address in the no-swizzle K-major layout [channel chunk][pixel][16 B].
//
// Warp roles (512 threads): warp 0 owns TMEM and one thread of it issues layer-2 MMAs; one
// thread of warp 2 issues layer-3 MMAs; warp 1 loads uint8 input rows (reflect-101 mirror
// padding, /255); warps 4-7 drain layer-2 accumulators; warps 8-11 drain layer-3 accumulators;
// warps 12-15 compute layer 1. Hand-offs are mbarriers; every
// wait is bounded by a 4 s global-timer limit after which the CTA records MB_ERR_TIMEOUT, stops
// issuing work and leaves cleanly (TMEM is always freed).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace mb {

constexpr int kThreads = 512;
constexpr int kPitch = 136;          // pixels per ring row (128 used + dx overrun)
constexpr int kStrip = 118;          // valid output columns per 128-pixel strip
constexpr int kInCols = 132;         // input columns read per row
constexpr int kInRing = 8;           // input row ring
constexpr int kRingDefault = 6;      // mf1 / mf2 ring slots (the A operands of layers 2 and 3) until tuned
constexpr int kMaxBlocks = 64;       // blocks per launch (kernel-parameter table)
constexpr int kWpackConstOff = 2 * 10 * 5120;  // constants follow the largest packed B (BF16)
constexpr uint64_t kWaitNs = 4000000000ull;

struct TcBlockDesc {
    const uint8_t* in;
    void* out;
    int64_t in_pitch, in_slice, out_pitch, out_slice;
    int h, w;               // source slice size (mirror padding range)
    int ry0, rx0, rh, rw;   // output region
    int z, n_strips, n_chunks, item_start;
    int64_t row_start;      // FP8 split: first strip-row of the block in (block, slice, strip, row) order
};

// Per-channel constants, staged into shared memory at kernel start (floats):
//   w1[25 taps][32 ch] | b1 | ep2 scale | ep2 bias | ep3 scale | ep3 bias | q1 | q2 | head w
// (FP8 folds q1 into w1 and b1 on the host; the slot is kept so that the layout is one for both)
constexpr int kCW1 = 0, kCB1 = 800, kCE2S = 832, kCE2B = 864, kCE3S = 896, kCE3B = 928, kCQ1 = 960,
              kCQ2 = 992, kCHW = 1024, kConsts = 1056;

struct TcParams {
    float hb;
    const uint8_t* wpack;   // global: packed B operands of layers 2 and 3, then the constants
    int* err;               // error word (MB_ERR_TIMEOUT on a timed-out wait)
    int n_blocks, n_items, rows_per_item, lag, out_u8;  // lag: unused (one issuer per layer)
    int64_t total_rows;     // FP8 split: strip-rows of the launch
    int fault_stall;        // test injection: the input loader withholds its arrivals
    uint64_t wait_ns;       // limit of every device-side wait
    TcBlockDesc blk[kMaxBlocks];
};

// RING: depth of the two A-operand rings (staged rows of the layer-2 and layer-3 inputs), a tuning
// parameter chosen at run time among compiled depths (BF16 4, 5, 6; FP8 4, 6, 8).
template <bool FP8, int RING = kRingDefault>
struct Cfg {
    static constexpr int kRing = RING;
    static constexpr int kChunks = FP8 ? 2 : 4;                 // 16-byte channel chunks per pixel
    static constexpr int kSlotBytes = kChunks * kPitch * 16;
    static constexpr int kGroups = FP8 ? 5 : 10;                // MMAs per (layer, input row, run)
    // TMEM row accumulators per layer. BF16: a ring of 8 (windows of 5 rows that wrap are split
    // into two MMAs). FP8: a ring of exactly 5 with the B blocks stored twice in order
    // [0 1 2 3 4 0 1 2 3], so every full window is one N=160 MMA into slots 0..4 whose B rows
    // start at the block that lands in slot 0.
    static constexpr int kAcc = FP8 ? 5 : 8;
    static constexpr int kBBlocks = FP8 ? 9 : 5;                 // 32-row blocks stored per group
    static constexpr int kLboB = kBBlocks * 32 * 16;             // B chunk stride (bytes)
    static constexpr int kGroupB = 2 * kLboB;                    // bytes per B group
    static constexpr int kLayerB = kGroups * kGroupB;
    // shared memory map
    static constexpr int oB = 0;
    static constexpr int oR1 = oB + 2 * kLayerB;
    static constexpr int oR2 = oR1 + kRing * kSlotBytes;
    static constexpr int oIn = oR2 + kRing * kSlotBytes;
    static constexpr int oSt1 = oIn + kInRing * kPitch * 4;
    static constexpr int oSt2 = oSt1 + 2 * 4 * 32 * 4;
    static constexpr int oConst = oSt2 + 2 * 4 * 32 * 4;
    static constexpr int oBar = oConst + kConsts * 4;
    static constexpr int kBars = 2 * kInRing + 4 * kRing + 4 * 8 + 2;
    static constexpr int oMisc = oBar + kBars * 8;
    static constexpr int kSmem = oMisc + 16;
    static_assert(kSmem <= 227 * 1024, "shared memory");
};

struct Bars {
    uint64_t* in_full;
    uint64_t* in_empty;
    uint64_t* m1_full;
    uint64_t* m1_empty;
    uint64_t* m2_full;
    uint64_t* m2_empty;
    uint64_t* a2_full;
    uint64_t* a2_free;
    uint64_t* a3_full;
    uint64_t* a3_free;
    uint64_t* fin;
};

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait. Returns false (and raises the CTA-wide abort flag) when the phase did not
// complete within kWaitNs, or immediately once the CTA is aborting.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                           int* err, uint64_t limit_ns = kWaitNs) {
    if (ptx::mbar_test(bar, parity)) return true;  // a completed phase costs one poll
    if (*abort_flag) return false;
    const uint64_t t0 = gtime();
    uint32_t n = 0;
    while (!ptx::mbar_test(bar, parity)) {
        if ((++n & 255u) == 0) {
            if (*abort_flag) return false;
            if (gtime() - t0 > limit_ns) {
                *abort_flag = 1;
                *(volatile int*)err = MB_ERR_TIMEOUT;
                return false;
            }
        }
    }
    return true;
}

__device__ __forceinline__ int refl_clamp(int t, int n) {
    t = t < 0 ? -t : t;
    t = t >= n ? 2 * (n - 1) - t : t;
    return t < 0 ? 0 : (t >= n ? n - 1 : t);
}

struct ItemInfo {
    int b, zi, x0, y0, rows;
};

__device__ __forceinline__ ItemInfo decode_item(const TcParams& p, int k) {
    int b = 0;
    while (b + 1 < p.n_blocks && p.blk[b + 1].item_start <= k) ++b;
    const TcBlockDesc& d = p.blk[b];
    int r = k - d.item_start;
    const int chunk = r % d.n_chunks;
    r /= d.n_chunks;
    const int strip = r % d.n_strips;
    const int zi = r / d.n_strips;
    ItemInfo it;
    it.b = b;
    it.zi = zi;
    it.x0 = strip * kStrip;
    it.y0 = chunk * p.rows_per_item;
    it.rows = min(p.rows_per_item, d.rh - it.y0);
    return it;
}

// Even-range work split (always for FP8; for BF16 when tuned to rows per item 0): the launch's
// strip-rows, in (block, slice, strip, row) order, are cut into one equal contiguous range per CTA,
// so every CTA computes the same number of rows and no tail wave remains; a CTA's items are the
// parts of its range in one (block, slice, strip) column. The other split walks round-robin items
// of a tuned number of rows. Chosen at compile time (a run-time choice in one kernel cost BF16
// 1.9 %). Every role of a CTA walks the same sequence.
struct RangeIter {
    int64_t r, hi;  // next strip-row, end of this CTA's range
};

__device__ __forceinline__ RangeIter range_begin(const TcParams& p) {
    RangeIter s;
    s.r = p.total_rows * (int64_t)blockIdx.x / gridDim.x;
    s.hi = p.total_rows * (int64_t)(blockIdx.x + 1) / gridDim.x;
    return s;
}

__device__ __forceinline__ bool range_next(const TcParams& p, RangeIter& s, ItemInfo& it) {
    if (s.r >= s.hi) return false;
    int b = 0;
    while (b + 1 < p.n_blocks && p.blk[b + 1].row_start <= s.r) ++b;
    const TcBlockDesc& d = p.blk[b];
    const int64_t off = s.r - d.row_start;
    const int64_t col = off / d.rh;
    it.b = b;
    it.zi = (int)(col / d.n_strips);
    it.x0 = (int)(col % d.n_strips) * kStrip;
    it.y0 = (int)(off - col * d.rh);
    it.rows = (int)min((int64_t)(d.rh - it.y0), s.hi - s.r);
    s.r += it.rows;
    return true;
}

// Pack 8 consecutive channels (BF16) or 16 (E4M3) of one pixel into a 16-byte ring row.
template <bool FP8>
__device__ __forceinline__ void store_pixel(uint8_t* slot, int c, const float (&m)[32], const float* q) {
    if (!FP8) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint4 u;
            __nv_bfloat162 h0 = __floats2bfloat162_rn(m[8 * k + 0], m[8 * k + 1]);
            __nv_bfloat162 h1 = __floats2bfloat162_rn(m[8 * k + 2], m[8 * k + 3]);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(m[8 * k + 4], m[8 * k + 5]);
            __nv_bfloat162 h3 = __floats2bfloat162_rn(m[8 * k + 6], m[8 * k + 7]);
            u.x = *reinterpret_cast<uint32_t*>(&h0);
            u.y = *reinterpret_cast<uint32_t*>(&h1);
            u.z = *reinterpret_cast<uint32_t*>(&h2);
            u.w = *reinterpret_cast<uint32_t*>(&h3);
            *reinterpret_cast<uint4*>(slot + (k * kPitch + c) * 16) = u;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ch = 16 * k + 4 * j;
                __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(
                    make_float2(m[ch] * q[ch], m[ch + 1] * q[ch + 1]), __NV_SATFINITE, __NV_E4M3);
                __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
                    make_float2(m[ch + 2] * q[ch + 2], m[ch + 3] * q[ch + 3]), __NV_SATFINITE, __NV_E4M3);
                w[j] = (uint32_t)lo | ((uint32_t)hi << 16);
            }
            *reinterpret_cast<uint4*>(slot + (k * kPitch + c) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Store 16 channels (one half h of the 32) of one pixel: BF16 chunks 2h and 2h+1, or E4M3 chunk h.
template <bool FP8>
__device__ __forceinline__ void store_half(uint8_t* slot, int c, int h, const float (&m)[16], const float* q) {
    if (!FP8) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            uint4 u;
            __nv_bfloat162 h0 = __floats2bfloat162_rn(m[8 * k + 0], m[8 * k + 1]);
            __nv_bfloat162 h1 = __floats2bfloat162_rn(m[8 * k + 2], m[8 * k + 3]);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(m[8 * k + 4], m[8 * k + 5]);
            __nv_bfloat162 h3 = __floats2bfloat162_rn(m[8 * k + 6], m[8 * k + 7]);
            u.x = *reinterpret_cast<uint32_t*>(&h0);
            u.y = *reinterpret_cast<uint32_t*>(&h1);
            u.z = *reinterpret_cast<uint32_t*>(&h2);
            u.w = *reinterpret_cast<uint32_t*>(&h3);
            *reinterpret_cast<uint4*>(slot + ((2 * h + k) * kPitch + c) * 16) = u;
        }
    } else {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ch = 4 * j;
            __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(m[ch] * q[ch], m[ch + 1] * q[ch + 1]),
                                                               __NV_SATFINITE, __NV_E4M3);
            __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
                make_float2(m[ch + 2] * q[ch + 2], m[ch + 3] * q[ch + 3]), __NV_SATFINITE, __NV_E4M3);
            w[j] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        *reinterpret_cast<uint4*>(slot + (h * kPitch + c) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Store channels 8h .. 8h+7 of one pixel: BF16 chunk h (16 B), or the half h & 1 of E4M3 chunk h >> 1.
template <bool FP8>
__device__ __forceinline__ void store_eighth(uint8_t* slot, int c, int h, const float (&m)[8], const float* q) {
    if (!FP8) {
        uint4 u;
        __nv_bfloat162 h0 = __floats2bfloat162_rn(m[0], m[1]);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(m[2], m[3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(m[4], m[5]);
        __nv_bfloat162 h3 = __floats2bfloat162_rn(m[6], m[7]);
        u.x = *reinterpret_cast<uint32_t*>(&h0);
        u.y = *reinterpret_cast<uint32_t*>(&h1);
        u.z = *reinterpret_cast<uint32_t*>(&h2);
        u.w = *reinterpret_cast<uint32_t*>(&h3);
        *reinterpret_cast<uint4*>(slot + (h * kPitch + c) * 16) = u;
    } else {
        uint32_t w[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int ch = 4 * j;
            // (layer 1 arrives already scaled: the scale is folded into its weights and bias)
            __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(m[ch], m[ch + 1]), __NV_SATFINITE, __NV_E4M3);
            __nv_fp8x2_storage_t hi =
                __nv_cvt_float2_to_fp8x2(make_float2(m[ch + 2], m[ch + 3]), __NV_SATFINITE, __NV_E4M3);
            w[j] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        *reinterpret_cast<uint2*>(slot + ((h >> 1) * kPitch + c) * 16 + (h & 1) * 8) = make_uint2(w[0], w[1]);
    }
}

// Issue the MMAs of groups [g_lo, g_hi) of one input row r for one layer: output rows j = r-4+i of
// the layer for the valid blocks i (0 <= j < n_out). Every MMA accumulates; the epilogue zeroes an accumulator after
// draining it, so a row's first contribution adds to zero. Blocks go to ring slots
// (base + r - 4 + i) mod kAcc; runs of contiguous slots are one MMA each.
template <bool FP8>
__device__ __forceinline__ void issue_row(uint32_t tcol0, uint32_t acc_base_seq, int r, int n_out, uint64_t adesc0,
                                          uint64_t bdesc0, int g_lo, int g_hi) {
    using C = Cfg<FP8>;
    constexpr int G = C::kGroups;
    constexpr int K = C::kAcc;
    constexpr uint32_t fmt = FP8 ? ptx::kFmtE4M3 : ptx::kFmtBF16;
    const int ilo = max(0, 4 - r);
    const int ihi = min(4, n_out + 3 - r);
    if (ilo > ihi) return;
    const int s_lo = (int)((acc_base_seq + (uint32_t)(r - 4 + ilo)) % K);
    uint32_t d[2], boff[2], idesc[2];
    int nrun;
    if (K == 5 && ilo == 0 && ihi == 4) {
        // full window: slots 0..4, B rows rotated so slot 0 receives block (5 - s_lo) mod 5
        const int i0 = (5 - s_lo) % 5;
        d[0] = tcol0;
        boff[0] = (uint32_t)(i0 * 32 * 16) >> 4;
        idesc[0] = ptx::idesc_f32acc(fmt, 128, 160);
        nrun = 1;
    } else {
        const int iw = ilo + (K - s_lo);  // first block whose slot wrapped to 0
        const int hi0 = iw <= ihi ? iw - 1 : ihi;
        d[0] = tcol0 + 32u * (uint32_t)s_lo;
        boff[0] = (uint32_t)(ilo * 32 * 16) >> 4;
        idesc[0] = ptx::idesc_f32acc(fmt, 128, (uint32_t)(32 * (hi0 - ilo + 1)));
        nrun = 1;
        if (iw <= ihi) {
            d[1] = tcol0;
            boff[1] = (uint32_t)(iw * 32 * 16) >> 4;
            idesc[1] = ptx::idesc_f32acc(fmt, 128, (uint32_t)(32 * (ihi - iw + 1)));
            nrun = 2;
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g < g_lo || g >= g_hi) continue;
        const int dx = FP8 ? g : (g >> 1);
        const int hk = FP8 ? 0 : (g & 1);
        const uint64_t ad = adesc0 + (uint64_t)((hk * 2 * kPitch * 16 + dx * 16) >> 4);
        const uint64_t bg = bdesc0 + (uint64_t)((g * C::kGroupB) >> 4);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k < nrun) {
                if (FP8)
                    ptx::mma_e4m3(d[k], ad, bg + boff[k], idesc[k], 1u);
                else
                    ptx::mma_bf16(d[k], ad, bg + boff[k], idesc[k], 1u);
            }
        }
    }
}

template <bool FP8, int RING, bool RNG>
__global__ void __launch_bounds__(kThreads, 1) tc_fused_teacher(const __grid_constant__ TcParams p) {
    using C = Cfg<FP8, RING>;
    constexpr int kRing = C::kRing;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* barmem = reinterpret_cast<uint64_t*>(smem + C::oBar);
    Bars B;
    B.in_full = barmem;
    B.in_empty = B.in_full + kInRing;
    B.m1_full = B.in_empty + kInRing;
    B.m1_empty = B.m1_full + kRing;
    B.m2_full = B.m1_empty + kRing;
    B.m2_empty = B.m2_full + kRing;
    B.a2_full = B.m2_empty + kRing;
    B.a2_free = B.a2_full + 8;
    B.a3_full = B.a2_free + 8;
    B.a3_free = B.a3_full + 8;
    B.fin = B.a3_free + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::oMisc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::oMisc + 4);
    float* in_ring = reinterpret_cast<float*>(smem + C::oIn);
    const float* cst = reinterpret_cast<const float*>(smem + C::oConst);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    // ---- set-up: barriers, B operands, ring padding, TMEM ------------------------------------
    if (tid == 0) {
        for (int i = 0; i < kInRing; ++i) {
            ptx::mbar_init(&B.in_full[i], 32);
            ptx::mbar_init(&B.in_empty[i], 128);
        }
        for (int i = 0; i < kRing; ++i) {
            ptx::mbar_init(&B.m1_full[i], 128);
            ptx::mbar_init(&B.m1_empty[i], 1);
            ptx::mbar_init(&B.m2_full[i], 128);
            ptx::mbar_init(&B.m2_empty[i], 1);
        }
        for (int i = 0; i < C::kAcc; ++i) {
            ptx::mbar_init(&B.a2_full[i], 1);
            ptx::mbar_init(&B.a2_free[i], 128);
            ptx::mbar_init(&B.a3_full[i], 1);
            ptx::mbar_init(&B.a3_free[i], 128);
        }
        ptx::mbar_init(B.fin, 1);
        ptx::mbar_init(B.fin + 1, 1);
        *abort_flag = 0;
        ptx::mbar_fence_init();
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(p.wpack);
        uint4* dst = reinterpret_cast<uint4*>(smem + C::oB);
        for (int i = tid; i < 2 * C::kLayerB / 16; i += kThreads) dst[i] = __ldg(src + i);
        const uint4* csrc = reinterpret_cast<const uint4*>(p.wpack + kWpackConstOff);
        uint4* cdst = reinterpret_cast<uint4*>(smem + C::oConst);
        for (int i = tid; i < kConsts / 4; i += kThreads) cdst[i] = __ldg(csrc + i);
        // zero the whole A rings once (the dx overrun pixels 128..135 are read but never written)
        uint4* r = reinterpret_cast<uint4*>(smem + C::oR1);
        for (int i = tid; i < 2 * kRing * C::kSlotBytes / 16; i += kThreads) r[i] = make_uint4(0, 0, 0, 0);
    }
    if (warp == 0) {
        ptx::tmem_alloc(tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    const uint32_t smem_base = ptx::smem_u32(smem);
    // Register budget per warpgroup (launched with 128 per thread = the whole register file):
    // MMA issuers + loader 64, layer-2 epilogue 136, layer-3 epilogue 112 (both keep their
    // per-channel constants in registers), layer-1 producers 200. Sum 512 = the launch's 4 x 128
    // per thread-slot: the increases take exactly what the decreases release, so they are always
    // satisfiable. (At 128 the layer-2 epilogue spilled in the even-range instantiations.)
    static_assert(64 + 136 + 112 + 200 <= 4 * 128, "register budget exceeds the launch allocation");
    if (warp >= 4 && warp < 12) {
        // every accumulator starts at zero (the MMAs only accumulate)
        const uint32_t col0 = warp < 8 ? 0u : 256u;
        const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
        for (int sl = 0; sl < C::kAcc; ++sl) ptx::tmem_st32_zero(tbase + lanes + col0 + 32u * sl);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();

    if (warp < 4) {
        ptx::setmaxnreg_dec<64>();
        if (warp == 0 || warp == 2) {
        // ================= MMA issuers: warp 0 lane 0 for layer 2, warp 2 lane 0 for layer 3 ======
        // Each issuer commits (and finally drains) only its own MMAs.
        if (lane == 0) {
            const bool l2 = warp == 0;
            uint32_t in_seq = 0, acc_seq = 0;  // A-ring rows consumed, accumulator rows completed
            bool ok = true;
            // ring slot i of the layer's A operand: base descriptor + i slots (start-address field)
            const uint64_t ad = ptx::smem_desc(smem_base + (l2 ? C::oR1 : C::oR2), kPitch * 16, 128);
            const uint64_t bd = ptx::smem_desc(smem_base + C::oB + (l2 ? 0 : C::kLayerB), C::kLboB, 128);
            const uint32_t tcol = tbase + (l2 ? 0u : 256u);
            uint64_t* full = l2 ? B.m1_full : B.m2_full;
            uint64_t* empty = l2 ? B.m1_empty : B.m2_empty;
            uint64_t* afree = l2 ? B.a2_free : B.a3_free;
            uint64_t* afull = l2 ? B.a2_full : B.a3_full;
            // The waits for input row r+1 are taken between the two halves of row r's MMAs, while the
            // first half still queues in the tensor pipe (a poll competes with the operand reads for
            // the shared-memory pipe). The accumulator of output row r+1 shares its slot with output
            // row r+1-kAcc, completed by input row r+5-kAcc: mid-row for the ring of 8 (BF16), but
            // only at the end of row r itself for the ring of 5 (FP8), where that wait stays after
            // the row's commits.
            constexpr int G = C::kGroups;
            constexpr bool kEarlyAcc = C::kAcc >= 6;
            auto wait_in = [&](uint32_t q) {
                ok = ok && wait_phase(&full[q % kRing], (q / kRing) & 1, abort_flag, p.err, p.wait_ns);
            };
            auto wait_acc = [&](uint32_t qa) {
                ok = ok && wait_phase(&afree[qa % C::kAcc], ((qa / C::kAcc) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
            };
            RangeIter range = range_begin(p);
            ItemInfo it;
            for (int k = blockIdx.x; RNG ? range_next(p, range, it) : k < p.n_items; k += gridDim.x) {
                if constexpr (!RNG) it = decode_item(p, k);
                const int NR = it.rows;
                const int n_in = l2 ? NR + 9 : NR + 4;   // input rows of this layer
                const int n_out = l2 ? NR + 5 : NR;      // output rows of this layer
                wait_in(in_seq);
                if (n_out > 0) wait_acc(acc_seq);
                ptx::tc_fence_after();
                for (int r = 0; r < n_in; ++r) {
                    const uint32_t q = in_seq + r, s = q % kRing;
                    const uint64_t arow = ad + (uint64_t)(s * (C::kSlotBytes >> 4));
                    if (ok) issue_row<FP8>(tcol, acc_seq, r, n_out, arow, bd, 0, G / 2);
                    if (r + 1 < n_in) {
                        wait_in(q + 1);
                        if (kEarlyAcc && r + 1 < n_out) wait_acc(acc_seq + r + 1);
                        ptx::tc_fence_after();
                    }
                    if (ok) issue_row<FP8>(tcol, acc_seq, r, n_out, arow, bd, G / 2, G);
                    ptx::mma_commit(&empty[s]);
                    if (r >= 4 && r - 4 < n_out) ptx::mma_commit(&afull[(acc_seq + r - 4) % C::kAcc]);
                    if (!kEarlyAcc && r + 1 < n_in && r + 1 < n_out) {
                        wait_acc(acc_seq + r + 1);
                        ptx::tc_fence_after();
                    }
                }
                in_seq += n_in;
                acc_seq += n_out;
            }
            // drain: all of this issuer's MMAs complete before TMEM is released
            uint64_t* fin = B.fin + (l2 ? 0 : 1);
            ptx::mma_commit(fin);
            const uint64_t t0 = gtime();
            while (!ptx::mbar_test(fin, 0)) {
                if (gtime() - t0 > p.wait_ns) {
                    *(volatile int*)p.err = MB_ERR_TIMEOUT;
                    break;
                }
            }
        }
        __syncwarp();
        } else if (warp == 1) {
        // ================= input loader ======================================================
        // Each lane owns columns lane + 32 i of the 132 read per row. The bytes of row u+1 are
        // requested before waiting for row u's ring slot, so one row's global latency overlaps the
        // wait and the conversion of the row before it.
        uint32_t in_seq = 0;
        RangeIter range = range_begin(p);
        ItemInfo it;
        for (int k = blockIdx.x; RNG ? range_next(p, range, it) : k < p.n_items; k += gridDim.x) {
            if constexpr (!RNG) it = decode_item(p, k);
            const TcBlockDesc& d = p.blk[it.b];
            const uint8_t* src = d.in + (int64_t)it.zi * d.in_slice;
            const int nrows = it.rows + 14;
            int sx[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) sx[i] = refl_clamp(d.rx0 + it.x0 - 7 + lane + 32 * i, d.w);
            auto load_row = [&](int u, uint32_t (&v)[5]) {
                const int sy = refl_clamp(d.ry0 + it.y0 - 7 + u, d.h);
                const uint8_t* row = src + (int64_t)sy * d.in_pitch;
#pragma unroll
                for (int i = 0; i < 5; ++i) v[i] = (lane + 32 * i < kInCols) ? (uint32_t)__ldg(row + sx[i]) : 0u;
            };
            uint32_t v[5];
            load_row(0, v);
            for (int u = 0; u < nrows; ++u) {
                uint32_t nv[5];
                load_row(u + 1 < nrows ? u + 1 : u, nv);
                const uint32_t q = in_seq + u, s = q % kInRing;
                wait_phase(&B.in_empty[s], ((q / kInRing) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
                float* dst = in_ring + s * kPitch;
#pragma unroll
                for (int i = 0; i < 5; ++i)
                    if (lane + 32 * i < kInCols) dst[lane + 32 * i] = (float)v[i] / 255.0f;
                if (!p.fault_stall) ptx::mbar_arrive(&B.in_full[s]);
#pragma unroll
                for (int i = 0; i < 5; ++i) v[i] = nv[i];
            }
            in_seq += nrows;
        }
        }
        // warp 3 has no role
    } else if (warp < 8) {
        ptx::setmaxnreg_inc<136>();
        // ================= layer-2 epilogue: bias, ReLU, max-filter -> A ring of layer 3 =======
        const int c = tid - 128;
        const int pw = warp - 4;
        float* stage = reinterpret_cast<float*>(smem + C::oSt2);
        uint32_t a2_seq = 0, m2_seq = 0;
        float prev[32];
        // per-channel constants in registers (the waits are compiler barriers, so reads from shared
        // memory would repeat every row, beside the MMA operand traffic)
        // (FP8 reads its scales from shared memory: registers would not hold them as well)
        float b2[32];
#pragma unroll
        for (int ch = 0; ch < 32; ++ch) b2[ch] = cst[kCE2B + ch];
        RangeIter range = range_begin(p);
        ItemInfo it;
        for (int k = blockIdx.x; RNG ? range_next(p, range, it) : k < p.n_items; k += gridDim.x) {
            if constexpr (!RNG) it = decode_item(p, k);
            const int N2 = it.rows + 5;
            for (int j = 0; j < N2; ++j) {
                const uint32_t q = a2_seq + j, s = q % C::kAcc;
                wait_phase(&B.a2_full[s], (q / C::kAcc) & 1, abort_flag, p.err, p.wait_ns);
                ptx::tc_fence_after();
                float v[32];
                const uint32_t ta = tbase + ((uint32_t)(32 * pw) << 16) + 32u * s;
                ptx::tmem_ld32(ta, v);
                ptx::tmem_st32_zero(ta);
                ptx::tc_fence_before();
                ptx::mbar_arrive(&B.a2_free[s]);
#pragma unroll
                for (int ch = 0; ch < 32; ++ch)  // BF16: the scales are 1
                    v[ch] = fmaxf(FP8 ? fmaf(v[ch], cst[kCE2S + ch], b2[ch]) : v[ch] + b2[ch], 0.f);
                if (j > 0) {
                    float (&m)[32] = prev;  // vertical max in place; prev is reloaded from v below
#pragma unroll
                    for (int ch = 0; ch < 32; ++ch) m[ch] = fmaxf(prev[ch], v[ch]);
                    float* st = stage + (j & 1) * 128;
                    if (lane == 0)
#pragma unroll
                        for (int ch = 0; ch < 32; ++ch) st[pw * 32 + ch] = m[ch];
                    asm volatile("bar.sync 2, 128;" ::: "memory");
#pragma unroll
                    for (int ch = 0; ch < 32; ++ch) {
                        float nb = __shfl_down_sync(0xffffffffu, m[ch], 1);
                        if (lane == 31) nb = pw < 3 ? st[(pw + 1) * 32 + ch] : m[ch];
                        m[ch] = fmaxf(m[ch], nb);
                    }
                    const uint32_t q2 = m2_seq + j - 1, s2 = q2 % kRing;
                    wait_phase(&B.m2_empty[s2], ((q2 / kRing) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
                    store_pixel<FP8>(smem + C::oR2 + s2 * C::kSlotBytes, c, m, cst + kCQ2);
                    ptx::fence_proxy_async_smem();
                    ptx::mbar_arrive(&B.m2_full[s2]);
                }
#pragma unroll
                for (int ch = 0; ch < 32; ++ch) prev[ch] = v[ch];
            }
            a2_seq += N2;
            m2_seq += N2 - 1;
        }
    } else if (warp < 12) {
        ptx::setmaxnreg_dec<112>();
        // ================= layer-3 epilogue: bias, ReLU, head, sigmoid, store ==================
        const int c = tid - 256;
        const int pw = warp - 8;
        uint32_t a3_seq = 0;
        float b3[32], hw[32];  // per-channel constants in registers (FP8 scales stay in shared memory)
#pragma unroll
        for (int ch = 0; ch < 32; ++ch) {
            b3[ch] = cst[kCE3B + ch];
            hw[ch] = cst[kCHW + ch];
        }
        RangeIter range = range_begin(p);
        ItemInfo it;
        for (int k = blockIdx.x; RNG ? range_next(p, range, it) : k < p.n_items; k += gridDim.x) {
            if constexpr (!RNG) it = decode_item(p, k);
            const TcBlockDesc& d = p.blk[it.b];
            const int NR = it.rows;
            const bool col_ok = c < kStrip && it.x0 + c < d.rw;
            for (int y = 0; y < NR; ++y) {
                const uint32_t q = a3_seq + y, s = q % C::kAcc;
                wait_phase(&B.a3_full[s], (q / C::kAcc) & 1, abort_flag, p.err, p.wait_ns);
                ptx::tc_fence_after();
                float v[32];
                const uint32_t ta = tbase + 256u + ((uint32_t)(32 * pw) << 16) + 32u * s;
                ptx::tmem_ld32(ta, v);
                ptx::tmem_st32_zero(ta);
                ptx::tc_fence_before();
                ptx::mbar_arrive(&B.a3_free[s]);
                float z = p.hb;
#pragma unroll
                for (int ch = 0; ch < 32; ++ch)
                    z = fmaf(hw[ch], fmaxf(FP8 ? fmaf(v[ch], cst[kCE3S + ch], b3[ch]) : v[ch] + b3[ch], 0.f), z);
                const float prob = 1.0f / (1.0f + expf(-z));
                if (col_ok && !*abort_flag) {
                    const int64_t idx = (int64_t)it.zi * d.out_slice + (int64_t)(it.y0 + y) * d.out_pitch + it.x0 + c;
                    if (p.out_u8)
                        static_cast<uint8_t*>(d.out)[idx] = (uint8_t)fminf(floorf(255.0f * prob + 0.5f), 255.0f);
                    else
                        static_cast<float*>(d.out)[idx] = prob;
                }
            }
            a3_seq += NR;
        }
    } else {
        ptx::setmaxnreg_inc<200>();
        // ================= layer 1 + max-filter producer ======================================
        // Thread = (channel group h = warp - 12, column quad): columns c0 = 4 lane .. c0 + 3,
        // channels 8h .. 8h+7. Every weight load is a warp-wide broadcast feeding four columns, and
        // a warp holds all 128 columns, so the max-filter's right neighbour is in the next lane.
        const int h = warp - 12;
        const int c0 = 4 * lane;
        uint32_t in_seq = 0, m1_seq = 0;
        float prev[4][8], cur[4][8];
        RangeIter range = range_begin(p);
        ItemInfo it;
        for (int k = blockIdx.x; RNG ? range_next(p, range, it) : k < p.n_items; k += gridDim.x) {
            if constexpr (!RNG) it = decode_item(p, k);
            const int NR = it.rows;
            const int M1 = NR + 9;
            for (int t = -1; t < M1; ++t) {
                if (t < 0) {
                    for (int u = 0; u < 5; ++u) {
                        const uint32_t q = in_seq + u;
                        wait_phase(&B.in_full[q % kInRing], (q / kInRing) & 1, abort_flag, p.err, p.wait_ns);
                    }
                } else {
                    const uint32_t qi = in_seq + t + 5;
                    wait_phase(&B.in_full[qi % kInRing], (qi / kInRing) & 1, abort_flag, p.err, p.wait_ns);
                }
                // layer 1 at input-frame row t+1: FP32 packed two-channel FMAs, weights broadcast
                float2 acc[4][4];
                {
                    const float4 b0 = *reinterpret_cast<const float4*>(cst + kCB1 + 8 * h);
                    const float4 b1 = *reinterpret_cast<const float4*>(cst + kCB1 + 8 * h + 4);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        acc[c][0] = make_float2(b0.x, b0.y);
                        acc[c][1] = make_float2(b0.z, b0.w);
                        acc[c][2] = make_float2(b1.x, b1.y);
                        acc[c][3] = make_float2(b1.z, b1.w);
                    }
                }
#pragma unroll 1
                for (int ky = 0; ky < 5; ++ky) {
                    // all loads of this row tap first (10 broadcast weight vectors, 8 inputs), then
                    // 80 packed FMAs
                    const float* ir = in_ring + ((in_seq + t + 1 + ky) % kInRing) * kPitch + c0;
                    const float4 xl = *reinterpret_cast<const float4*>(ir);
                    const float4 xh = *reinterpret_cast<const float4*>(ir + 4);
                    const float x[8] = {xl.x, xl.y, xl.z, xl.w, xh.x, xh.y, xh.z, xh.w};
                    const float4* wrow = reinterpret_cast<const float4*>(cst + kCW1 + ky * 5 * 32 + 8 * h);
                    float4 w[5][2];
#pragma unroll
                    for (int kx = 0; kx < 5; ++kx) {
                        w[kx][0] = wrow[kx * 8];
                        w[kx][1] = wrow[kx * 8 + 1];
                    }
#pragma unroll
                    for (int kx = 0; kx < 5; ++kx) {
                        const float2 w01 = make_float2(w[kx][0].x, w[kx][0].y), w23 = make_float2(w[kx][0].z, w[kx][0].w);
                        const float2 w45 = make_float2(w[kx][1].x, w[kx][1].y), w67 = make_float2(w[kx][1].z, w[kx][1].w);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float2 xv = make_float2(x[c + kx], x[c + kx]);
                            acc[c][0] = __ffma2_rn(w01, xv, acc[c][0]);
                            acc[c][1] = __ffma2_rn(w23, xv, acc[c][1]);
                            acc[c][2] = __ffma2_rn(w45, xv, acc[c][2]);
                            acc[c][3] = __ffma2_rn(w67, xv, acc[c][3]);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        cur[c][2 * j] = fmaxf(acc[c][j].x, 0.f);
                        cur[c][2 * j + 1] = fmaxf(acc[c][j].y, 0.f);
                    }
                ptx::mbar_arrive(&B.in_empty[(in_seq + t + 1) % kInRing]);
                if (t >= 0) {
                    // vertical max in place (prev is reloaded from cur below)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
#pragma unroll
                        for (int ch = 0; ch < 8; ++ch) prev[c][ch] = fmaxf(prev[c][ch], cur[c][ch]);
                    // horizontal: column c0 + 3 pairs with the next lane's column c0 + 4; lane 31's
                    // column 127 only feeds discarded output columns and pairs with itself
                    const uint32_t q = m1_seq + t, s = q % kRing;
                    wait_phase(&B.m1_empty[s], ((q / kRing) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
                    uint8_t* slot = smem + C::oR1 + s * C::kSlotBytes;
                    float o[8];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
#pragma unroll
                        for (int ch = 0; ch < 8; ++ch) {
                            float nb;
                            if (c < 3) {
                                nb = prev[c + 1][ch];
                            } else {
                                nb = __shfl_down_sync(0xffffffffu, prev[0][ch], 1);
                                if (lane == 31) nb = prev[3][ch];
                            }
                            o[ch] = fmaxf(prev[c][ch], nb);
                        }
                        store_eighth<FP8>(slot, c0 + c, h, o, cst + kCQ1 + 8 * h);
                    }
                    ptx::fence_proxy_async_smem();
                    ptx::mbar_arrive(&B.m1_full[s]);
                }
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int ch = 0; ch < 8; ++ch) prev[c][ch] = cur[c][ch];
            }
            for (int u = M1 + 1; u < NR + 14; ++u) ptx::mbar_arrive(&B.in_empty[(in_seq + u) % kInRing]);
            in_seq += NR + 14;
            m1_seq += M1;
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------------------------------------
// host side

static uint16_t bf16_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Pack one 5x5 32->32 layer's weights W[co][ci][dy][dx] (already scaled) as the B operand groups:
// group g = (dx, K-half) for BF16 or dx for FP8; in a group, row n = 32 b + co of stored block b
// holds row tap dy = 4 - (b mod 5); K-major [chunk][n][16 B].
template <bool FP8>
static void pack_layer(const float* W, const float* wscale_inv, uint8_t* out) {
    using C = Cfg<FP8>;
    for (int dx = 0; dx < 5; ++dx)
        for (int b = 0; b < C::kBBlocks; ++b) {
            const int dy = 4 - (b % 5);
            for (int co = 0; co < 32; ++co) {
                const int n = b * 32 + co;
                for (int ci = 0; ci < 32; ++ci) {
                    const float w = W[((co * 32 + ci) * 5 + dy) * 5 + dx];
                    if (!FP8) {
                        const int g = dx * 2 + ci / 16, kc = (ci % 16) / 8;
                        uint16_t v = bf16_bits(w);
                        memcpy(out + g * C::kGroupB + kc * C::kLboB + n * 16 + (ci % 8) * 2, &v, 2);
                    } else {
                        const int g = dx, kc = ci / 16;
                        __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(w * wscale_inv[co], __NV_SATFINITE, __NV_E4M3);
                        out[g * C::kGroupB + kc * C::kLboB + n * 16 + (ci % 16)] = q;
                    }
                }
            }
        }
}

struct TcState {
    TcParams base;             // weights and epilogue constants (blocks filled per launch)
    uint8_t* d_wpack = nullptr;
    int* h_err = nullptr;      // mapped pinned host word the kernel writes on a timed-out wait
    int* d_err = nullptr;      // its device alias
};

struct GraphCacheEntry {
    std::vector<mb_block> blocks;
    mb_out_type ot;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static TcState* state_of(mb_net* net) { return reinterpret_cast<TcState*>(net->tc_state); }

mb_status tc_prepare(mb_net* net) {
    const bool fp8 = net->prec == MB_PREC_FP8;
    if (fp8 && !net->calibrated) {
        // calibration provides the activation scales; until then only the FP32 pieces exist
    }
    TcState* S = state_of(net);
    if (!S) {
        S = new (std::nothrow) TcState();
        if (!S) {
            set_error("host allocation failed");
            return MB_ERR_OOM;
        }
        memset(&S->base, 0, sizeof(S->base));
        net->tc_state = S;
    }
    const float* P = net->host_params.data();
    const float* W1 = P;
    const float* B1 = W1 + 800;
    const float* W2 = B1 + 32;
    const float* B2 = W2 + 25600;
    const float* W3 = B2 + 32;
    const float* B3 = W3 + 25600;
    const float* HW = B3 + 32;
    TcParams& q = S->base;
    std::vector<float> cs(kConsts, 0.f);
    for (int co = 0; co < 32; ++co) {
        for (int k = 0; k < 25; ++k) cs[kCW1 + k * 32 + co] = W1[co * 25 + k];
        cs[kCB1 + co] = B1[co];
        cs[kCHW + co] = HW[co];
    }
    q.hb = HW[32];
    const size_t layer_bytes = (size_t)(fp8 ? Cfg<true>::kLayerB : Cfg<false>::kLayerB);
    std::vector<uint8_t> pack(2 * layer_bytes, 0);
    if (!fp8) {
        for (int c = 0; c < 32; ++c) {
            cs[kCE2S + c] = 1.f;
            cs[kCE2B + c] = B2[c];
            cs[kCE3S + c] = 1.f;
            cs[kCE3B + c] = B3[c];
            cs[kCQ1 + c] = 1.f;
            cs[kCQ2 + c] = 1.f;
        }
        pack_layer<false>(W2, nullptr, pack.data());
        pack_layer<false>(W3, nullptr, pack.data() + layer_bytes);
    } else {
        // activation scale s_a = amax / 448 per input channel, folded into the next layer's
        // weights; then a per-output-channel weight scale s_w = amax|W'| / 448.
        const float* Ws[2] = {W2, W3};
        const float* Bs[2] = {B2, B3};
        for (int l = 0; l < 2; ++l) {
            float sa[32];
            for (int ci = 0; ci < 32; ++ci) {
                const float a = net->fp8_amax[l][ci];
                sa[ci] = a > 0.f ? a / 448.f : 1.f;
                cs[(l == 0 ? kCQ1 : kCQ2) + ci] = 1.f / sa[ci];
                if (l == 0) {
                    // layer 1's quantisation scale (> 0) commutes with ReLU and the max-filter: it
                    // is folded into layer 1's weights and bias, so the producers store as they go
                    for (int k = 0; k < 25; ++k) cs[kCW1 + k * 32 + ci] /= sa[ci];
                    cs[kCB1 + ci] /= sa[ci];
                }
            }
            std::vector<float> Wp(25600);
            float inv[32];
            for (int co = 0; co < 32; ++co) {
                float amax = 0.f;
                for (int ci = 0; ci < 32; ++ci)
                    for (int t = 0; t < 25; ++t) {
                        const float v = Ws[l][(co * 32 + ci) * 25 + t] * sa[ci];
                        Wp[(co * 32 + ci) * 25 + t] = v;
                        amax = std::max(amax, std::fabs(v));
                    }
                const float sw = amax > 0.f ? amax / 448.f : 1.f;
                inv[co] = 1.f / sw;
                cs[(l == 0 ? kCE2S : kCE3S) + co] = sw;
                cs[(l == 0 ? kCE2B : kCE3B) + co] = Bs[l][co];
            }
            pack_layer<true>(Wp.data(), inv, pack.data() + l * layer_bytes);
        }
    }
    if (!S->d_wpack) MB_TRY(dev_alloc((void**)&S->d_wpack, kWpackConstOff + kConsts * 4));
    if (!S->h_err) {
        if (fault_oom()) {
            set_error("pinned allocation failed (MB_FAULT_OOM injected)");
            return MB_ERR_OOM;
        }
        MB_CUDA(cudaHostAlloc((void**)&S->h_err, sizeof(int), cudaHostAllocMapped));
        *S->h_err = 0;
        MB_CUDA(cudaHostGetDevicePointer((void**)&S->d_err, S->h_err, 0));
    }
    MB_CUDA(cudaMemcpy(S->d_wpack, pack.data(), pack.size(), cudaMemcpyHostToDevice));
    MB_CUDA(cudaMemcpy(S->d_wpack + kWpackConstOff, cs.data(), kConsts * 4, cudaMemcpyHostToDevice));
    q.wpack = S->d_wpack;
    q.err = S->d_err;
    return MB_OK;
}

static void drop_graphs(mb_net* net) {
    for (GraphCacheEntry* g : net->graphs) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
    }
    net->graphs.clear();
}

void tc_release(mb_net* net) {
    drop_graphs(net);
    TcState* S = state_of(net);
    if (S) {
        dev_free(S->d_wpack);
        if (S->h_err) cudaFreeHost(S->h_err);
        delete S;
        net->tc_state = nullptr;
    }
}

static int g_num_sms = 0;

// A-ring depths compiled per precision; the tuned depth picks the instantiation.
constexpr int kBf16Rings[] = {4, 5, 6};
constexpr int kFp8Rings[] = {4, 6, 8};

static bool ring_supported(bool fp8, int ring) {
    for (int r : fp8 ? kFp8Rings : kBf16Rings)
        if (r == ring) return true;
    return false;
}

template <bool FP8, int RING, bool RNG>
static mb_status launch_ring(TcParams& prm, int grid, cudaStream_t st) {
    using C = Cfg<FP8, RING>;
    static bool attr = false;  // per instantiation
    if (!attr) {
        MB_CUDA(cudaFuncSetAttribute(tc_fused_teacher<FP8, RING, RNG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     C::kSmem));
        attr = true;
    }
    tc_fused_teacher<FP8, RING, RNG><<<grid, kThreads, C::kSmem, st>>>(prm);
    return MB_OK;
}

static mb_status launch_tc(mb_net* net, TcParams& prm, cudaStream_t st) {
    const bool fp8 = net->prec == MB_PREC_FP8;
    if (g_num_sms == 0) {
        int dev = 0;
        MB_CUDA(cudaGetDevice(&dev));
        MB_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    // even split of the rows: one CTA per SM, or fewer when a CTA would get under 64 rows
    const bool rng = fp8 || net->rows_per_item == 0;
    const int grid = rng ? (int)std::max<int64_t>(1, std::min<int64_t>(g_num_sms, (prm.total_rows + 63) / 64))
                         : std::max(1, std::min(prm.n_items, g_num_sms));
    const int ring = ring_supported(fp8, net->stages) ? net->stages : kRingDefault;
    mb_status s = MB_OK;
    if (fp8) {
        switch (ring) {
            case 4: s = launch_ring<true, 4, true>(prm, grid, st); break;
            case 8: s = launch_ring<true, 8, true>(prm, grid, st); break;
            default: s = launch_ring<true, 6, true>(prm, grid, st); break;
        }
    } else if (rng) {
        switch (ring) {
            case 4: s = launch_ring<false, 4, true>(prm, grid, st); break;
            case 5: s = launch_ring<false, 5, true>(prm, grid, st); break;
            default: s = launch_ring<false, 6, true>(prm, grid, st); break;
        }
    } else {
        switch (ring) {
            case 4: s = launch_ring<false, 4, false>(prm, grid, st); break;
            case 5: s = launch_ring<false, 5, false>(prm, grid, st); break;
            default: s = launch_ring<false, 6, false>(prm, grid, st); break;
        }
    }
    MB_TRY(s);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

// Fill the block table for up to kMaxBlocks blocks starting at `first`; returns blocks used.
static int fill_blocks(mb_net* net, TcParams& prm, const mb_block* blocks, int n_blocks, int first,
                       const int64_t* y0, const int64_t* x0, const int64_t* rows, const int64_t* cols,
                       mb_out_type ot) {
    int nb = 0, items = 0;
    int64_t total = 0;
    // Rows per work item: the tuned value, unless the launch would not fill one wave of CTAs (a
    // streamed slab, a few small blocks). Then the candidates R, R/2, .. 64 are compared by the
    // predicted time, waves x (rows + 9) (each item restarts the layer-2 row pipeline, 9 extra
    // rows), ties to the larger R. The choice never changes a result. (The even-range split, rows
    // per item 0, takes its items from the ranges; R then only sizes the unused item table.)
    const bool even_split = net->prec == MB_PREC_FP8 || net->rows_per_item == 0;
    int R = even_split ? 1024 : std::max(8, net->rows_per_item);
    if (!even_split) {
        if (g_num_sms == 0) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                g_num_sms = 0;
            }
        }
        const int64_t sms = std::max(g_num_sms, 1);
        auto n_items = [&](int r) {
            int64_t n = 0;
            int seen = 0;
            for (int i = first; i < n_blocks && seen < kMaxBlocks; ++i) {
                if (blocks[i].z == 0 || rows[i] == 0 || cols[i] == 0) continue;
                n += blocks[i].z * ((cols[i] + kStrip - 1) / kStrip) * ((rows[i] + r - 1) / r);
                ++seen;
            }
            return n;
        };
        if (n_items(R) < sms) {
            int64_t best = INT64_MAX;
            int best_r = R;
            for (int r = R; r >= 64; r /= 2) {
                const int64_t cost = (n_items(r) + sms - 1) / sms * (r + 9);
                if (cost < best) {
                    best = cost;
                    best_r = r;
                }
            }
            R = best_r;
        }
    }
    for (int i = first; i < n_blocks && nb < kMaxBlocks; ++i) {
        const mb_block& b = blocks[i];
        if (b.z == 0 || rows[i] == 0 || cols[i] == 0) continue;
        TcBlockDesc& d = prm.blk[nb];
        d.in = b.in;
        d.out = b.out;
        d.in_pitch = b.in_pitch;
        d.in_slice = b.in_slice_pitch;
        d.out_pitch = b.out_pitch;
        d.out_slice = b.out_slice_pitch;
        d.h = (int)b.h;
        d.w = (int)b.w;
        d.ry0 = (int)y0[i];
        d.rx0 = (int)x0[i];
        d.rh = (int)rows[i];
        d.rw = (int)cols[i];
        d.z = (int)b.z;
        d.n_strips = (d.rw + kStrip - 1) / kStrip;
        d.n_chunks = (d.rh + R - 1) / R;
        d.item_start = items;
        items += d.z * d.n_strips * d.n_chunks;
        d.row_start = total;
        total += (int64_t)d.z * d.n_strips * d.rh;
        ++nb;
    }
    prm.n_blocks = nb;
    prm.n_items = items;
    prm.total_rows = total;
    prm.rows_per_item = R;
    prm.lag = 0;
    prm.out_u8 = ot == MB_OUT_U8;
    // host-side fault injection for tests: MB_FAULT_STALL=1 makes every launch's first wait run
    // out (the loader never signals its rows) after a short limit
    const char* stall = getenv("MB_FAULT_STALL");
    prm.fault_stall = (stall && stall[0] == '1') ? 1 : 0;
    prm.wait_ns = prm.fault_stall ? 200000000ull : kWaitNs;
    int used = first;
    int counted = 0;
    while (used < n_blocks && counted < kMaxBlocks) {
        const mb_block& b = blocks[used];
        if (!(b.z == 0 || rows[used] == 0 || cols[used] == 0)) ++counted;
        ++used;
    }
    return used;
}

// A timed-out device wait is reported by the next call that looks (the word lives in mapped host
// memory, so no synchronisation is needed to read it).
static mb_status check_err(mb_net* net) {
    TcState* S = state_of(net);
    if (S && S->h_err && *(volatile int*)S->h_err) {
        *(volatile int*)S->h_err = 0;
        set_error("a tensor-core launch on this net gave up waiting (device-side wait limit)");
        return MB_ERR_TIMEOUT;
    }
    return MB_OK;
}

mb_status tc_poll_error(mb_net* net) { return check_err(net); }

mb_status tc_infer_blocks(mb_net* net, const mb_block* blocks, int n_blocks, const int64_t* y0, const int64_t* x0,
                          const int64_t* rows, const int64_t* cols, mb_out_type ot, cudaStream_t st,
                          bool use_graph) {
    TcState* S = state_of(net);
    if (!S || !S->d_wpack) {
        set_error("tensor-core weights not prepared");
        return MB_ERR_NOT_READY;
    }
    MB_TRY(check_err(net));
    for (int i = 0; i < n_blocks; ++i)
        if (blocks[i].h > (1 << 30) / 2 || blocks[i].w > (1 << 30) / 2) {
            set_error("block %d too large", i);
            return MB_ERR_SHAPE;
        }
    if (use_graph) {
        for (GraphCacheEntry* g : net->graphs) {
            if (g->ot != ot || (int)g->blocks.size() != n_blocks) continue;
            if (memcmp(g->blocks.data(), blocks, sizeof(mb_block) * n_blocks) != 0) continue;
            MB_CUDA(cudaGraphLaunch(g->exec, st));
            count_launch((int)((n_blocks + kMaxBlocks - 1) / kMaxBlocks));
            return check_err(net);
        }
        if (net->graphs.size() >= 8) drop_graphs(net);
        GraphCacheEntry* g = new (std::nothrow) GraphCacheEntry();
        if (!g) {
            set_error("host allocation failed");
            return MB_ERR_OOM;
        }
        g->blocks.assign(blocks, blocks + n_blocks);
        g->ot = ot;
        cudaStream_t cs = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete g;
            return cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
        }
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        mb_status s = e == cudaSuccess ? MB_OK : cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
        int first = 0;
        const int64_t before = mb_launch_count();
        while (s == MB_OK && first < n_blocks) {
            TcParams prm = S->base;
            int next = fill_blocks(net, prm, blocks, n_blocks, first, y0, x0, rows, cols, ot);
            if (prm.n_items > 0) s = launch_tc(net, prm, cs);
            first = next;
        }
        const int64_t launched = mb_launch_count() - before;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (s == MB_OK && e != cudaSuccess) s = cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        if (s == MB_OK) {
            e = cudaGraphInstantiate(&g->exec, graph, 0);
            if (e != cudaSuccess) s = cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        }
        cudaStreamDestroy(cs);
        g->graph = graph;
        if (s != MB_OK) {
            if (g->exec) cudaGraphExecDestroy(g->exec);
            if (g->graph) cudaGraphDestroy(g->graph);
            delete g;
            return s;
        }
        net->graphs.push_back(g);
        (void)launched;
        MB_CUDA(cudaGraphLaunch(g->exec, st));
        return check_err(net);
    }
    int first = 0;
    while (first < n_blocks) {
        TcParams prm = S->base;
        int next = fill_blocks(net, prm, blocks, n_blocks, first, y0, x0, rows, cols, ot);
        if (prm.n_items > 0) MB_TRY(launch_tc(net, prm, st));
        first = next;
    }
    return check_err(net);
}

}  // namespace mb

namespace mb {

__global__ void fill_bytes(uint8_t* p, int64_t n, uint32_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 2654435761u ^ seed;
        x ^= x >> 15;
        x *= 2246822519u;
        x ^= x >> 13;
        p[i] = (uint8_t)(x >> 24);
    }
}

static std::string tune_key(int dev, mb_precision prec, int64_t z, int64_t h, int64_t w) {
    cudaDeviceProp pr;
    char buf[512];
    const char* name = cudaGetDeviceProperties(&pr, dev) == cudaSuccess ? pr.name : "unknown";
    snprintf(buf, sizeof(buf), "%s|%s|%lldx%lldx%lld", name, prec == MB_PREC_FP8 ? "fp8" : "bf16", (long long)z,
             (long long)h, (long long)w);
    for (char* c = buf; *c; ++c)
        if (*c == '"' || *c == '\\') *c = '_';
    return buf;
}

// Cache file: one JSON object per line, {"key": "...", "rows_per_item": R, "stages": S, "ms": T}.
static bool cache_lookup(const char* path, const std::string& key, int* rows, int* stages) {
    FILE* f = path ? fopen(path, "r") : nullptr;
    if (!f) return false;
    char line[1024];
    bool found = false;
    const std::string pat = "\"key\": \"" + key + "\"";
    while (fgets(line, sizeof(line), f)) {
        if (!strstr(line, pat.c_str())) continue;
        const char* r = strstr(line, "\"rows_per_item\": ");
        const char* s = strstr(line, "\"stages\": ");
        if (r && s) {
            *rows = atoi(r + 17);
            *stages = atoi(s + 10);
            found = *rows >= 0 && *stages > 0;
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const char* path, const std::string& key, int rows, int stages, float ms) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"rows_per_item\": %d, \"stages\": %d, \"ms\": %.4f}\n", key.c_str(), rows, stages,
            ms);
    fclose(f);
}

// Times every candidate on one workload (`run` launches it once on `st`; median of 4 launches
// after one), keeps the fastest in the net and records it under `key` in the cache. A cached entry
// is applied without timing. Candidates whose rows per item exceed twice the workload's tallest
// block are skipped (they equal the largest useful one), except the smallest and the even split.
template <class Run>
static mb_status tune_candidates(mb_net* net, const std::string& key, const char* cache_path, int32_t* choice,
                                 cudaStream_t st, int64_t max_rows, Run run) {
    const bool fp8 = net->prec == MB_PREC_FP8;
    int rows = 0, stages = 0;
    if (cache_lookup(cache_path, key, &rows, &stages) && ring_supported(fp8, stages) && (fp8 || rows >= 0)) {
        if (!fp8) net->rows_per_item = rows;
        net->stages = stages;
        net->tuned = true;
        drop_graphs(net);
        if (choice) {
            choice[0] = fp8 ? 0 : rows;
            choice[1] = stages;
            choice[2] = 1;
        }
        return MB_OK;
    }
    mb_status rc = MB_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    {
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaEventCreate", __FILE__, __LINE__);
    }
    const int saved_rows = net->rows_per_item, saved_stages = net->stages;
    int best_r = saved_rows, best_s = saved_stages;
    float best = 1e30f;
    if (rc == MB_OK) {
        const int cand_rows_bf16[] = {64, 128, 256, 512, 1024, 0};  // 0: the even-range split
        const int cand_rows_fp8[] = {0};
        const int* cand_rows = fp8 ? cand_rows_fp8 : cand_rows_bf16;
        const int n_rows = fp8 ? 1 : 6;
        const int* cand_rings = fp8 ? kFp8Rings : kBf16Rings;
        for (int ir = 0; ir < n_rows && rc == MB_OK; ++ir) {
            const int R = cand_rows[ir];
            if (!fp8 && R > 2 * max_rows && R != cand_rows[0] && R != 0) continue;
            for (int is = 0; is < 3 && rc == MB_OK; ++is) {
                const int S = cand_rings[is];
                net->rows_per_item = fp8 ? saved_rows : R;
                net->stages = S;
                float ms_rep[5] = {};
                for (int rep = 0; rep < 5 && rc == MB_OK; ++rep) {
                    cudaError_t e = cudaEventRecord(e0, st);
                    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaEventRecord", __FILE__, __LINE__); break; }
                    rc = run();
                    if (rc != MB_OK) break;
                    e = cudaEventRecord(e1, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e != cudaSuccess) { rc = cuda_fail(e, "autotune timing", __FILE__, __LINE__); break; }
                    ms_rep[rep] = ms;
                }
                if (rc != MB_OK) break;
                // median of the 4 timed repetitions (the first one warms up)
                std::sort(ms_rep + 1, ms_rep + 5);
                const float med = 0.5f * (ms_rep[2] + ms_rep[3]);
                if (med < best) {
                    best = med;
                    best_r = fp8 ? saved_rows : R;
                    best_s = S;
                }
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc == MB_OK) rc = check_err(net);
    if (rc != MB_OK) {
        net->rows_per_item = saved_rows;
        net->stages = saved_stages;
        return rc;
    }
    net->rows_per_item = best_r;
    net->stages = best_s;
    net->tuned = true;
    drop_graphs(net);
    cache_store(cache_path, key, fp8 ? 0 : best_r, best_s, best);
    if (choice) {
        choice[0] = fp8 ? 0 : best_r;
        choice[1] = best_s;
        choice[2] = 0;
    }
    return MB_OK;
}

mb_status tc_autotune(mb_net* net, int64_t z, int64_t h, int64_t w, const char* cache_path, int32_t* choice,
                      cudaStream_t st) {
    int dev = 0;
    MB_CUDA(cudaGetDevice(&dev));
    const std::string key = tune_key(dev, net->prec, z, h, w);
    uint8_t* in = nullptr;
    float* out = nullptr;
    MB_TRY(dev_alloc((void**)&in, (size_t)(z * h * w)));
    mb_status rc = dev_alloc((void**)&out, (size_t)(z * h * w) * 4);
    if (rc == MB_OK) {
        fill_bytes<<<1024, 256, 0, st>>>(in, z * h * w, 12345u);
        count_launch();
        mb_block b;
        b.in = in;
        b.z = z;
        b.h = h;
        b.w = w;
        b.in_pitch = w;
        b.in_slice_pitch = h * w;
        b.out = out;
        b.out_pitch = w;
        b.out_slice_pitch = h * w;
        const int64_t y0 = 0, x0 = 0;
        rc = tune_candidates(net, key, cache_path, choice, st, h,
                             [&] { return tc_infer_blocks(net, &b, 1, &y0, &x0, &h, &w, MB_OUT_F32, st, false); });
    }
    dev_free(in);
    dev_free(out);
    return rc;
}

mb_status tc_autotune_batch(mb_net* net, const mb_block* blocks, int n_blocks, mb_out_type ot, const char* cache_path,
                            int32_t* choice, cudaStream_t st) {
    int dev = 0;
    MB_CUDA(cudaGetDevice(&dev));
    // key: GPU, precision, output type and the blocks' shapes (FNV-1a over z, h, w of each block)
    uint64_t hsh = 1469598103934665603ull;
    int64_t max_h = 8, vox = 0;
    std::vector<int64_t> y0(n_blocks, 0), x0(n_blocks, 0), rows(n_blocks), cols(n_blocks);
    for (int i = 0; i < n_blocks; ++i) {
        const int64_t v3[3] = {blocks[i].z, blocks[i].h, blocks[i].w};
        for (int64_t v : v3)
            for (int byte = 0; byte < 8; ++byte) {
                hsh ^= (uint64_t)((v >> (8 * byte)) & 0xff);
                hsh *= 1099511628211ull;
            }
        rows[i] = blocks[i].h;
        cols[i] = blocks[i].w;
        max_h = std::max<int64_t>(max_h, blocks[i].h);
        vox += blocks[i].z * blocks[i].h * blocks[i].w;
    }
    cudaDeviceProp pr;
    const char* name = cudaGetDeviceProperties(&pr, dev) == cudaSuccess ? pr.name : "unknown";
    char buf[512];
    snprintf(buf, sizeof(buf), "%s|%s|batch|%s|%d blocks|%lld vox|%016llx", name,
             net->prec == MB_PREC_FP8 ? "fp8" : "bf16", ot == MB_OUT_U8 ? "u8" : "f32", n_blocks, (long long)vox,
             (unsigned long long)hsh);
    std::string key = buf;
    for (char& c : key)
        if (c == '"' || c == '\\') c = '_';
    return tune_candidates(net, key, cache_path, choice, st, max_h, [&] {
        return tc_infer_blocks(net, blocks, n_blocks, y0.data(), x0.data(), rows.data(), cols.data(), ot, st, false);
    });
}

}  // namespace mb

extern "C" mb_status mb_set_tuning(mb_net* net, int32_t rows_per_item, int32_t stages) {
    mb::clear_error();
    if (!net) {
        mb::set_error("mb_set_tuning: net is NULL");
        return MB_ERR_INVALID_ARG;
    }
    if (net->family != mb::FAMILY_TEACHER || net->prec == MB_PREC_FP32) {
        mb::set_error("mb_set_tuning: only the tensor-core teacher (BF16/FP8) has tunables");
        return MB_ERR_UNSUPPORTED;
    }
    const bool fp8 = net->prec == MB_PREC_FP8;
    const bool rows_ok = fp8 ? rows_per_item == 0
                             : (rows_per_item == 0 || rows_per_item == 64 || rows_per_item == 128 ||
                                rows_per_item == 256 || rows_per_item == 512 || rows_per_item == 1024);
    if (!rows_ok || !mb::ring_supported(fp8, stages)) {
        mb::set_error("mb_set_tuning: (%d rows per item, %d stages) is not a candidate for %s", (int)rows_per_item,
                      (int)stages, fp8 ? "FP8 (rows 0; stages 4, 6, 8)" : "BF16 (rows 0 or 64..1024; stages 4, 5, 6)");
        return MB_ERR_INVALID_ARG;
    }
    if (!fp8) net->rows_per_item = rows_per_item;
    net->stages = stages;
    net->tuned = true;
    mb::drop_graphs(net);
    return MB_OK;
}

extern "C" mb_status mb_autotune(mb_net* net, int64_t z, int64_t h, int64_t w, const char* cache_path,
                                 int32_t* choice_out, void* stream) {
    mb::clear_error();
    if (!net) {
        mb::set_error("mb_autotune: net is NULL");
        return MB_ERR_INVALID_ARG;
    }
    if (!net->loaded || (net->prec == MB_PREC_FP8 && !net->calibrated)) {
        mb::set_error("mb_autotune: net not ready (weights / FP8 calibration)");
        return MB_ERR_NOT_READY;
    }
    if (net->family != mb::FAMILY_TEACHER || net->prec == MB_PREC_FP32) {
        mb::set_error("mb_autotune: only the tensor-core teacher (BF16/FP8) has tunables");
        return MB_ERR_UNSUPPORTED;
    }
    if (z <= 0 || h < 8 || w < 8 || z * h * w > ((int64_t)1 << 32)) {
        mb::set_error("mb_autotune: workload %lldx%lldx%lld out of range", (long long)z, (long long)h, (long long)w);
        return MB_ERR_SHAPE;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != net->device) cudaSetDevice(net->device);
    mb_status s = mb::tc_autotune(net, z, h, w, cache_path, choice_out, (cudaStream_t)stream);
    if (prev != net->device) cudaSetDevice(prev);
    return s;
}
