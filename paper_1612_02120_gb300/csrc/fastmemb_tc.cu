// fastmemb_tc.cu - FastMemb's dense form (Sec. 2.2) on the 5th-generation tensor cores: the two
// 32->64 dilated convolutions (+ bias, max-out over channel pairs) and the 32->2 head (+ the
// 2-class softmax), each over the 2x2 max-filter of the previous stage.
//
// Implicit GEMM per output image row y and 128-pixel column strip x0, conv dilation d:
//   D[128 px][N] = sum over 16 taps (ky, kx) and 2 K-halves of
//                  A_{ky,kx}[128 px][16 ch] x B_{ky,kx}[N][16 ch]^T
// A_{ky,kx} is input row y + d ky, pixels x0 + d kx .. x0 + d kx + 127, taken from one staged row
// in the no-swizzle K-major layout [channel chunk][pixel][16 B]: the column tap is a (d kx x 16)-
// byte shift of the descriptor's start address, so 4 staged rows feed all 32 MMAs of a row.
// Output rows are walked in steps of d (one residue class y mod d at a time, the max-pooling
// fragments of Sec. 2.2), so each staged row serves 4 consecutive output rows and is loaded once.
//
// Two operand types, one template: BF16 and FP16 (both kind::f16 MMAs, A and B of the same type).
// BF16 weights are split W = W_hi + W_lo, both BF16 (W_lo = BF16(W - W_hi)), and stacked along N,
// so each MMA applies both and the result carries BF16 activation rounding only; FP16's 11-bit
// significand makes the split unnecessary for the layers (64 columns per row tap):
//   BF16 layers: N = 128 per output row, columns n (hi) and 64 + n (lo) of conv channel n
//   FP16 layers: 64 columns per row tap ky (column n = conv channel n), the 4 row taps stacked
//           along N (N = 256) like the head's, into a ring of 8 row accumulators of 64 columns
//   head:   16 columns per row tap ky: 0, 1 (hi of classes 0, 1) and 2, 3 (lo); the rest zero
//           (both types keep the split here: the head's MMAs cost the same with it).
//           Stacked row taps (head, FP16 layers) instead of MMAs per output row: staged row u is
//           multiplied once per (kx, K-half) into the accumulators of output rows u .. u-3, a
//           ring of 8 row accumulators (N = 16 or 64 x the taps that fall inside the item, split where
//           the window wraps the ring); every stacked MMA accumulates, and the epilogue zeroes
//           the used columns of a row's accumulator after draining it.
//
// Warp roles (512 threads, 1 CTA per SM, persistent over work items):
//   warp 0      TMEM owner; lane 0 issues the MMAs (16-bit operands -> FP32 in TMEM)
//   warps 4-7   epilogue: TMEM -> registers; layers: (hi + lo) + bias, max-out, 16-bit store;
//               head: z_c = hi + lo + bias, p = 1 / (1 + exp(z0 - z1)), FP32 or uint8 store
//   warps 8-15  producers, two groups of 4 warps taking alternate staged rows: max-filter 4 16-bit
//               pixels of the previous stage into the A rows; one thread of each group
//               bulk-prefetches the source rows of its staged row 4 ahead into L2
// Every mbarrier wait is bounded (a global-timer limit), after which the CTA records
// MB_ERR_TIMEOUT in a mapped host word, stops issuing work and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <climits>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace mb {

namespace {

constexpr int kFThreads = 512;
constexpr int kFP = 178;                 // pixels per staged row (>= 128 + 3*16); 178 mod 8 = 2 spreads
                                         // the 4 chunk planes of one pixel pair over distinct banks
constexpr int kFSlot = 4 * kFP * 16;     // bytes per staged row (4 chunks of 8 16-bit channels)
constexpr int kFRing = 8;                // staged rows in flight
constexpr int kFAcc = 4;                 // TMEM accumulators of the 32->64 layers
constexpr int kHAcc = 8;                 // head: ring of row accumulators (16 columns each)
constexpr int kFTasks = 6;               // producer tasks per thread and row: ceil(4 * 176 / 128)
constexpr int kFPrefetch = 4;            // staged rows between a row's L2 prefetch and its loads
constexpr uint64_t kFWaitNs = 4000000000ull;

template <bool HEAD, bool F16>
struct FCfg {
    // BF16 layers: N = 128 (hi + lo) per output row, one B block per (tap, K-half):
    // [2 chunks][128 rows][16 B]. kStack (the head, and the FP16 layers): the 4 row taps stacked
    // along N, N rows each (16 for the head, 4 used; 64 for the FP16 layers), one B block per
    // (column tap, K-half): [2 chunks][4 N rows][16 B]; one MMA per staged row and (column tap,
    // K-half) covers up to 4 output rows of a ring of row accumulators.
    static constexpr bool kStack = HEAD || F16;
    static constexpr int N = HEAD ? 16 : (F16 ? 64 : 128);  // accumulator width per output row (= per row tap when stacked)
    static constexpr int kBRows = kStack ? 4 * N : N;       // B rows per block
    static constexpr int kBlock = 2 * kBRows * 16;
    static constexpr int kBBytes = (kStack ? 8 : 32) * kBlock;
    static constexpr int kAcc = kStack ? kHAcc : kFAcc;
    static constexpr int kTmemCols = kAcc * N;
    static constexpr int oB = 0;
    static constexpr int oRing = oB + kBBytes;
    static constexpr int oBias = oRing + kFRing * kFSlot;
    static constexpr int oBar = oBias + 64 * 4;
    static constexpr int kBars = 2 * kFRing + 2 * kAcc + 1;
    static constexpr int oMisc = oBar + kBars * 8;
    static constexpr int kSmem = oMisc + 16;
    static_assert(kSmem <= 227 * 1024, "shared memory");
    static_assert(kTmemCols == 128 || kTmemCols == 256 || kTmemCols == 512, "TMEM allocation");
};

struct FmTcParams {
    const uint16_t* in;        // previous stage, [slice][y][x][32] BF16 or FP16, before its max-filter
    void* out;                 // layers: [slice][y][x][32] of the same type; head: FP32 or uint8 [slice][y][x]
    const uint8_t* wpack;      // B operands then 64 FP32 biases
    int* err;
    int64_t in_slice, in_pitch, out_slice, out_pitch;  // elements / pixels
    int in_rows, in_cols;      // domain of the (max-filtered, strided) input
    int stride;                // input (r, c) is the max-filter at source (stride r, stride c)
    int64_t src_cols;          // source pixels per row that may be read (prefetch bound)
    int out_h, out_w;
    int d, dm;                 // conv dilation, max-filter dilation
    int nz, n_strips;
    int64_t total_rows;        // strip-rows of the launch: nz x n_strips x out_h
    int out_u8;                // head: uint8 output round(255 p)
    int fault_stall;           // test injection: producers withhold their arrivals
    uint64_t wait_ns;
};

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                         uint64_t limit_ns) {
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

struct FmItem {
    int z, ry, x0, m0, rows;  // output rows y = ry + d (m0 + j), j < rows; rows may be 0
};

// Work split: the launch's strip-rows, in (slice z, residue class ry, strip, row) order, are cut
// into one equal contiguous range per CTA (no tail wave); a CTA's items are the parts of its range
// in one (z, ry, strip) column. Residue class ry has hr = ceil((out_h - ry) / d) rows per strip:
// base + 1 for ry < rem and base after (out_h = d base + rem), so n_strips (ry base + min(ry, rem))
// strip-rows of a slice precede it. Every role of a CTA walks the same sequence.
struct FmCursor {
    int64_t g, hi;  // next strip-row, end of this CTA's range
};

__device__ __forceinline__ FmCursor fm_begin(const FmTcParams& p) {
    FmCursor c;
    c.g = p.total_rows * (int64_t)blockIdx.x / gridDim.x;
    c.hi = p.total_rows * (int64_t)(blockIdx.x + 1) / gridDim.x;
    return c;
}

__device__ __forceinline__ bool fm_next(const FmTcParams& p, FmCursor& c, FmItem& it) {
    if (c.g >= c.hi) return false;
    const int64_t per_slice = (int64_t)p.n_strips * p.out_h;
    it.z = (int)(c.g / per_slice);
    const int r = (int)(c.g - (int64_t)it.z * per_slice);  // strip-row within the slice
    const int base = p.out_h / p.d, rem = p.out_h % p.d;
    auto before = [&](int ry) { return p.n_strips * (ry * base + min(ry, rem)); };
    int ry = 0;
    while (ry + 1 < p.d && before(ry + 1) <= r) ++ry;
    const int hr = base + (ry < rem ? 1 : 0);  // > 0: before(ry) <= r < before(ry + 1)
    const int off = r - before(ry);
    const int strip = off / hr;
    it.ry = ry;
    it.x0 = strip * 128;
    it.m0 = off - strip * hr;
    it.rows = (int)min((int64_t)(hr - it.m0), c.hi - c.g);
    c.g += it.rows;
    return true;
}

// element-wise max of 8 packed 16-bit values
template <bool F16>
__device__ __forceinline__ uint4 bmax(uint4 a, uint4 b) {
    using T2 = typename std::conditional<F16, __half2, __nv_bfloat162>::type;
    uint4 r;
    const T2* x = reinterpret_cast<const T2*>(&a);
    const T2* y = reinterpret_cast<const T2*>(&b);
    T2* o = reinterpret_cast<T2*>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = __hmax2(x[i], y[i]);
    return r;
}

template <bool HEAD, bool F16>
__global__ void __launch_bounds__(kFThreads, 1) fm_tc_conv(const __grid_constant__ FmTcParams p) {
    using C = FCfg<HEAD, F16>;
    constexpr uint32_t kFmt = F16 ? ptx::kFmtF16 : ptx::kFmtBF16;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* row_full = reinterpret_cast<uint64_t*>(smem + C::oBar);
    uint64_t* row_empty = row_full + kFRing;
    uint64_t* acc_full = row_empty + kFRing;
    uint64_t* acc_free = acc_full + C::kAcc;
    uint64_t* fin = acc_free + C::kAcc;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::oMisc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::oMisc + 4);
    const float* bias = reinterpret_cast<const float*>(smem + C::oBias);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < kFRing; ++i) {
            ptx::mbar_init(&row_full[i], 128);
            ptx::mbar_init(&row_empty[i], 1);
        }
        for (int i = 0; i < C::kAcc; ++i) {
            ptx::mbar_init(&acc_full[i], 1);
            ptx::mbar_init(&acc_free[i], 128);
        }
        ptx::mbar_init(fin, 1);
        *abort_flag = 0;
        ptx::mbar_fence_init();
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(p.wpack);
        uint4* dst = reinterpret_cast<uint4*>(smem + C::oB);
        for (int i = tid; i < C::kBBytes / 16; i += kFThreads) dst[i] = __ldg(src + i);
        const uint4* bsrc = reinterpret_cast<const uint4*>(p.wpack + C::kBBytes);
        uint4* bdst = reinterpret_cast<uint4*>(smem + C::oBias);
        for (int i = tid; i < 64 * 4 / 16; i += kFThreads) bdst[i] = __ldg(bsrc + i);
    }
    if (warp == 0) {
        ptx::tmem_alloc(tmem_slot, C::kTmemCols);
        ptx::tmem_relinquish();
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    const uint32_t sbase = ptx::smem_u32(smem);
    const int d = p.d;
    if constexpr (C::kStack) {
        // stacked MMAs only accumulate (a staged row adds to up to 4 rows at once): the used
        // accumulator columns start at zero, and the epilogue re-zeroes them after each drain
        if (warp >= 4 && warp < 8) {
            const uint32_t lanes = (uint32_t)(32 * (warp - 4)) << 16;
            for (int sl = 0; sl < C::kAcc; ++sl) {
                if constexpr (HEAD) {
                    ptx::tmem_st4_zero(tbase + lanes + (uint32_t)C::N * sl);
                } else {
                    ptx::tmem_st32_zero(tbase + lanes + (uint32_t)C::N * sl);
                    ptx::tmem_st32_zero(tbase + lanes + (uint32_t)C::N * sl + 32u);
                }
            }
        }
        ptx::tc_fence_before();
        __syncthreads();
        ptx::tc_fence_after();
    }

    if (warp == 0) {
        // ================= MMA issuer ================================================================
        if (lane == 0) {
            const uint64_t adesc0 = ptx::smem_desc(sbase + C::oRing, kFP * 16, 128);
            const uint64_t bdesc0 = ptx::smem_desc(sbase + C::oB, C::kBRows * 16, 128);
            constexpr uint32_t idesc = ptx::idesc_f32acc(kFmt, 128, C::N);
            uint32_t row_seq = 0, acc_seq = 0;
            bool ok = true;
            // The waits for output row j+1 (its one new staged row and its accumulator) are taken
            // between the two halves of row j's MMAs, while the first half still queues in the tensor
            // pipe: at N = 128 the operand reads take the whole shared-memory bandwidth and a poll
            // costs hundreds of cycles.
            auto wait_row = [&](uint32_t q) {
                ok = ok && wait_bar(&row_full[q % kFRing], (q / kFRing) & 1, abort_flag, p.err, p.wait_ns);
            };
            auto wait_acc = [&](uint32_t qa) {
                ok = ok && wait_bar(&acc_free[qa % kFAcc], ((qa / kFAcc) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
            };
            auto issue_half = [&](uint32_t j, uint32_t s, int ky0) {
                const uint32_t dcol = tbase + (uint32_t)C::N * s;
#pragma unroll
                for (int dky = 0; dky < 2; ++dky) {
                    const int ky = ky0 + dky;
                    const uint32_t slot = (row_seq + j + ky) % kFRing;
                    const uint64_t arow = adesc0 + (uint64_t)((slot * kFSlot) >> 4);
#pragma unroll
                    for (int kx = 0; kx < 4; ++kx)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint64_t ad = arow + (uint64_t)((h * 2 * kFP * 16 + d * kx * 16) >> 4);
                            const uint64_t bd = bdesc0 + (uint64_t)((((ky * 4 + kx) * 2 + h) * C::kBlock) >> 4);
                            ptx::mma_bf16(dcol, ad, bd, idesc, (ky | kx | h) ? 1u : 0u);
                        }
                }
            };
            if constexpr (C::kStack) {
                // Staged row u of an item feeds output rows u - ky for ky = 0..3 (the row taps stacked
                // along N): one MMA per (column tap, K-half) with D = the accumulators of rows u, u-1,
                // u-2, u-3. Output row sequence q lives in ring slot K-1 - q mod K, so these rows sit in
                // increasing slots; a window that wraps the ring is split in two MMAs. Only the rows of
                // the item are written (N = 16 x the valid taps).
                constexpr int K = C::kAcc;
                auto slot_of = [](uint32_t q) { return (uint32_t)(K - 1) - q % (uint32_t)K; };
                const uint64_t adesc = ptx::smem_desc(sbase + C::oRing, kFP * 16, 128);
                const uint64_t bdesc = ptx::smem_desc(sbase + C::oB, C::kBRows * 16, 128);
                const uint32_t idn[4] = {ptx::idesc_f32acc(kFmt, 128, C::N), ptx::idesc_f32acc(kFmt, 128, 2 * C::N),
                                         ptx::idesc_f32acc(kFmt, 128, 3 * C::N), ptx::idesc_f32acc(kFmt, 128, 4 * C::N)};
                FmCursor cur = fm_begin(p);
                FmItem it;
                while (fm_next(p, cur, it)) {
                    const int nst = it.rows + 3;
                    for (int u = 0; u < nst; ++u) {
                        const int blo = max(0, u - it.rows + 1), bhi = min(3, u);
                        wait_row(row_seq + u);
                        if (blo == 0) {  // output row u starts here: its slot must have been drained
                            const uint32_t q = acc_seq + u;
                            ok = ok && wait_bar(&acc_free[slot_of(q)], ((q / K) & 1) ^ 1, abort_flag, p.err,
                                                p.wait_ns);
                        }
                        ptx::tc_fence_after();
                        if (ok) {
                            const uint32_t s0 = slot_of(acc_seq + u - blo);
                            const int nb = bhi - blo + 1;
                            const int n1 = min(nb, K - (int)s0);  // taps before the ring wraps
                            const uint64_t arow =
                                adesc + (uint64_t)((((row_seq + u) % kFRing) * kFSlot) >> 4);
#pragma unroll
                            for (int kx = 0; kx < 4; ++kx)
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
                                    const uint64_t ad = arow + (uint64_t)((h * 2 * kFP * 16 + d * kx * 16) >> 4);
                                    const uint64_t bg = bdesc + (uint64_t)(((kx * 2 + h) * C::kBlock) >> 4);
                                    ptx::mma_bf16(tbase + (uint32_t)C::N * s0, ad,
                                                  bg + (uint64_t)((blo * C::N * 16) >> 4), idn[n1 - 1], 1u);
                                    if (n1 < nb)
                                        ptx::mma_bf16(tbase, ad, bg + (uint64_t)(((blo + n1) * C::N * 16) >> 4),
                                                      idn[nb - n1 - 1], 1u);
                                }
                        }
                        ptx::mma_commit(&row_empty[(row_seq + u) % kFRing]);
                        if (u >= 3) ptx::mma_commit(&acc_full[slot_of(acc_seq + u - 3)]);
                    }
                    row_seq += nst;
                    acc_seq += it.rows;
                }
            } else {
            FmCursor cur = fm_begin(p);
            FmItem it;
            while (fm_next(p, cur, it)) {
                for (int u = 0; u < 4; ++u) wait_row(row_seq + u);
                wait_acc(acc_seq);
                ptx::tc_fence_after();
                for (int j = 0; j < it.rows; ++j) {
                    const uint32_t s = (acc_seq + j) % kFAcc;
                    if (ok) issue_half(j, s, 0);
                    if (j + 1 < it.rows) {
                        wait_row(row_seq + j + 4);
                        wait_acc(acc_seq + j + 1);
                        ptx::tc_fence_after();
                    }
                    if (ok) issue_half(j, s, 2);
                    ptx::mma_commit(&acc_full[s]);
                    ptx::mma_commit(&row_empty[(row_seq + j) % kFRing]);
                }
                // the last three staged rows of the item are free once its MMAs are done
                for (int u = it.rows; u < it.rows + 3; ++u) ptx::mma_commit(&row_empty[(row_seq + u) % kFRing]);
                row_seq += it.rows + 3;
                acc_seq += it.rows;
            }
            }
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
    } else if (warp >= 4 && warp < 8) {
        // ================= epilogue ===================================================================
        const int px = tid - 128;  // TMEM lane = pixel of the strip
        const uint32_t lanes = (uint32_t)(32 * (warp - 4)) << 16;
        uint32_t acc_seq = 0;
        FmCursor cur = fm_begin(p);
        FmItem it;
        while (fm_next(p, cur, it)) {
            const int x = it.x0 + px;
            for (int j = 0; j < it.rows; ++j) {
                const uint32_t qa = acc_seq + j;
                const uint32_t s = C::kStack ? (uint32_t)(C::kAcc - 1) - qa % (uint32_t)C::kAcc : qa % (uint32_t)C::kAcc;
                wait_bar(&acc_full[s], (qa / C::kAcc) & 1, abort_flag, p.err, p.wait_ns);
                ptx::tc_fence_after();
                const uint32_t ta = tbase + lanes + (uint32_t)C::N * s;
                const int y = it.ry + d * (it.m0 + j);
                const bool store = x < p.out_w && y < p.out_h && !*abort_flag;
                if constexpr (HEAD) {
                    float c[4];
                    ptx::tmem_ld4(ta, c);
                    ptx::tmem_st4_zero(ta);
                    ptx::tc_fence_before();
                    ptx::mbar_arrive(&acc_free[s]);
                    const float z0 = (c[0] + c[2]) + bias[0], z1 = (c[1] + c[3]) + bias[1];
                    const float prob = 1.0f / (1.0f + expf(z0 - z1));
                    if (store) {
                        const int64_t idx = (int64_t)it.z * p.out_slice + (int64_t)y * p.out_pitch + x;
                        if (p.out_u8)
                            static_cast<uint8_t*>(p.out)[idx] = (uint8_t)fminf(floorf(255.0f * prob + 0.5f), 255.0f);
                        else
                            static_cast<float*>(p.out)[idx] = prob;
                    }
                } else {
                    uint32_t w[16];
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        // conv channels 32 half .. 32 half + 31: column n (BF16: hi; lo in 64 + n)
                        float hi[32];
                        ptx::tmem_ld32(ta + 32u * half, hi);
                        if constexpr (C::kStack) ptx::tmem_st32_zero(ta + 32u * half);  // accumulated into
                        if constexpr (F16) {
#pragma unroll
                            for (int c = 0; c < 16; c += 2) {
                                const int n = 32 * half + 2 * c;
                                const float a0 = fmaxf(hi[2 * c] + bias[n], hi[2 * c + 1] + bias[n + 1]);
                                const float a1 = fmaxf(hi[2 * c + 2] + bias[n + 2], hi[2 * c + 3] + bias[n + 3]);
                                __half2 v = __floats2half2_rn(a0, a1);
                                w[8 * half + c / 2] = *reinterpret_cast<uint32_t*>(&v);
                            }
                        } else {
                            float lo[32];
                            ptx::tmem_ld32(ta + 64u + 32u * half, lo);
#pragma unroll
                            for (int c = 0; c < 16; c += 2) {
                                const int n = 32 * half + 2 * c;
                                const float a0 = fmaxf((hi[2 * c] + lo[2 * c]) + bias[n],
                                                       (hi[2 * c + 1] + lo[2 * c + 1]) + bias[n + 1]);
                                const float a1 = fmaxf((hi[2 * c + 2] + lo[2 * c + 2]) + bias[n + 2],
                                                       (hi[2 * c + 3] + lo[2 * c + 3]) + bias[n + 3]);
                                __nv_bfloat162 v = __floats2bfloat162_rn(a0, a1);
                                w[8 * half + c / 2] = *reinterpret_cast<uint32_t*>(&v);
                            }
                        }
                    }
                    ptx::tc_fence_before();
                    ptx::mbar_arrive(&acc_free[s]);
                    if (store) {
                        uint4* o = reinterpret_cast<uint4*>(static_cast<uint16_t*>(p.out) +
                                                            (int64_t)it.z * p.out_slice +
                                                            ((int64_t)y * p.out_pitch + x) * 32);
                        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
                        o[1] = make_uint4(w[4], w[5], w[6], w[7]);
                        o[2] = make_uint4(w[8], w[9], w[10], w[11]);
                        o[3] = make_uint4(w[12], w[13], w[14], w[15]);
                    }
                }
            }
            acc_seq += it.rows;
        }
    } else if (warp >= 8) {
        // ================= producers: max-filtered input rows into the A ring =========================
        // Group g = warps 8-11 / 12-15 stages the rows u = g mod 2 of every item. Thread tasks
        // e = pt + 128 i (chunk e & 3 of pixel e >> 2); all loads of a row are issued before the
        // slot wait so their latency overlaps the wait.
        const int grp = (warp - 8) >> 2;
        const int pt = tid - 256 - 128 * grp;
        const int ntask = 4 * (128 + 3 * d);
        const int64_t dxo = (int64_t)p.dm * 32, dyo = (int64_t)p.dm * p.in_pitch * 32;
        uint32_t row_seq = 0;
        FmCursor cur = fm_begin(p);
        FmItem it;
        while (fm_next(p, cur, it)) {
            const uint16_t* src = p.in + (int64_t)it.z * p.in_slice;
            // source pixels one staged row reads: stride (npix - 1) + dm + 1 from stride x0, clipped
            const int sx0 = p.stride * it.x0;
            const int pf_cols = (int)min((int64_t)(p.stride * (127 + 3 * d) + p.dm + 1), p.src_cols - sx0);
            for (int u = grp; u < it.rows + 3; u += 2) {
                const uint32_t q = row_seq + u, slot = q % kFRing;
                const int yin = it.ry + d * (it.m0 + u);
                // bulk-prefetch into L2 the two source rows of staged row u + kFPrefetch
                if (pt == 0 && u + kFPrefetch < it.rows + 3) {
                    const int yp = it.ry + d * (it.m0 + u + kFPrefetch);
                    if (yp < p.in_rows && pf_cols > 0) {
                        const uint16_t* r0 = src + ((int64_t)(p.stride * yp) * p.in_pitch + sx0) * 32;
                        ptx::prefetch_l2_bulk(r0, (uint32_t)pf_cols * 64u);
                        ptx::prefetch_l2_bulk(r0 + dyo, (uint32_t)pf_cols * 64u);
                    }
                }
                uint4 v[kFTasks];
#pragma unroll
                for (int i = 0; i < kFTasks; ++i) {
                    const int e = pt + 128 * i;
                    const int xin = it.x0 + (e >> 2);
                    v[i] = make_uint4(0, 0, 0, 0);
                    if (e < ntask && yin < p.in_rows && xin < p.in_cols) {
                        const uint16_t* a =
                            src + ((int64_t)(p.stride * yin) * p.in_pitch + p.stride * xin) * 32 + (e & 3) * 8;
                        const uint4 r0 = __ldg(reinterpret_cast<const uint4*>(a));
                        const uint4 r1 = __ldg(reinterpret_cast<const uint4*>(a + dxo));
                        const uint4 r2 = __ldg(reinterpret_cast<const uint4*>(a + dyo));
                        const uint4 r3 = __ldg(reinterpret_cast<const uint4*>(a + dyo + dxo));
                        v[i] = bmax<F16>(bmax<F16>(r0, r1), bmax<F16>(r2, r3));
                    }
                }
                wait_bar(&row_empty[slot], ((q / kFRing) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
                uint8_t* dst = smem + C::oRing + slot * kFSlot;
#pragma unroll
                for (int i = 0; i < kFTasks; ++i) {
                    const int e = pt + 128 * i;
                    if (e < ntask) *reinterpret_cast<uint4*>(dst + ((e & 3) * kFP + (e >> 2)) * 16) = v[i];
                }
                ptx::fence_proxy_async_smem();
                if (!p.fault_stall) ptx::mbar_arrive(&row_full[slot]);
            }
            row_seq += it.rows + 3;
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tbase, C::kTmemCols);
}

uint16_t bf16_bits_rn(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

uint16_t f16_bits_rn(float f) {
    const __half h = __float2half_rn(f);
    uint16_t u;
    memcpy(&u, &h, 2);
    return u;
}

float f16_value(uint16_t b) {
    __half h;
    memcpy(&h, &b, 2);
    return __half2float(h);
}

// Pack a conv 4x4 32->C layer W[c][ci][ky][kx], b[c] as B operands: blocks of [chunk kc][row][8
// 16-bit], ci = 16 h + 8 kc + e, per (tap t = 4 ky + kx, K-half h) for the layers and per (column
// tap kx, K-half h) for the head, whose row taps are stacked along the rows. Part 0 of a weight is
// T(W), part 1 T(W - T(W)) for T = BF16 (layers and head) or FP16 (the head only: FP16 layers
// carry part 0 alone). Then 64 FP32 biases.
template <bool HEAD, bool F16>
void fm_pack(const float* W, const float* b, int channels, std::vector<uint8_t>& out) {
    using C = FCfg<HEAD, F16>;
    constexpr bool kLo = HEAD || !F16;
    out.assign(C::kBBytes + 64 * 4, 0);
    for (int c = 0; c < channels; ++c)
        for (int ci = 0; ci < 32; ++ci)
            for (int ky = 0; ky < 4; ++ky)
                for (int kx = 0; kx < 4; ++kx) {
                    const int t = ky * 4 + kx, h = ci / 16, kc = (ci % 16) / 8, e = ci % 8;
                    const float w = W[((c * 32 + ci) * 4 + ky) * 4 + kx];
                    const uint16_t whi = F16 ? f16_bits_rn(w) : bf16_bits_rn(w);
                    const uint16_t wlo =
                        F16 ? f16_bits_rn(w - f16_value(whi)) : bf16_bits_rn(w - bf16_value(whi));
                    // BF16 layers: block (tap, K-half), rows c (hi) and 64 + c (lo); FP16 layers: block
                    // (column tap, K-half), rows 64 ky + c; head: block (column tap, K-half), rows
                    // 16 ky + c (hi) and 16 ky + 2 + c (lo)
                    const int rhi = HEAD ? 16 * ky + c : (F16 ? 64 * ky + c : c);
                    const int rlo = HEAD ? 16 * ky + 2 + c : 64 + c;
                    const int blk_i = C::kStack ? kx * 2 + h : t * 2 + h;
                    uint8_t* blk = out.data() + blk_i * C::kBlock + kc * C::kBRows * 16;
                    memcpy(blk + rhi * 16 + e * 2, &whi, 2);
                    if (kLo) memcpy(blk + rlo * 16 + e * 2, &wlo, 2);
                }
    std::vector<float> bias(64, 0.f);
    for (int c = 0; c < channels; ++c) bias[c] = b[c];
    memcpy(out.data() + C::kBBytes, bias.data(), 64 * 4);
}

template <bool HEAD, bool F16>
mb_status launch_fm_tc(const FmTcParams& p, cudaStream_t st) {
    using C = FCfg<HEAD, F16>;
    static int n_sms = 0;
    if (n_sms == 0) {
        int dev = 0;
        MB_CUDA(cudaGetDevice(&dev));
        MB_CUDA(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    static bool attr = false;
    if (!attr) {
        MB_CUDA(cudaFuncSetAttribute(fm_tc_conv<HEAD, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem));
        attr = true;
    }
    // one range per SM, or fewer when a range would get under 8 rows
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_sms, (p.total_rows + 7) / 8));
    fm_tc_conv<HEAD, F16><<<grid, kFThreads, C::kSmem, st>>>(p);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

}  // namespace

struct FmTcState {
    uint8_t* d_wpack[4] = {nullptr, nullptr, nullptr, nullptr};  // the 32->64 convs, then the head
    int* h_err = nullptr;
    int* d_err = nullptr;
};

mb_status fm_tc_prepare(mb_net* net) {
    FmTcState* S = reinterpret_cast<FmTcState*>(net->fm_state);
    if (!S) {
        S = new (std::nothrow) FmTcState();
        if (!S) {
            set_error("host allocation failed");
            return MB_ERR_OOM;
        }
        net->fm_state = S;
    }
    // API layout: W1 [64][1][4][4], b1 [64], then per 32->64 conv W [64][32][4][4], b [64], then the
    // head W [2][32][4][4], b [2]
    const int nc = fastmemb_convs(net->family);
    const float* P = net->host_params.data() + 64 * 16 + 64;
    std::vector<uint8_t> pk;
    const bool f16 = net->prec == MB_PREC_FP16;
    for (int l = 0; l < nc - 1; ++l) {
        const bool head = l == nc - 2;
        const int co = head ? 2 : 64;
        if (!head)
            f16 ? fm_pack<false, true>(P, P + co * 32 * 16, co, pk) : fm_pack<false, false>(P, P + co * 32 * 16, co, pk);
        else
            f16 ? fm_pack<true, true>(P, P + co * 32 * 16, co, pk) : fm_pack<true, false>(P, P + co * 32 * 16, co, pk);
        P += co * 32 * 16 + co;
        if (!S->d_wpack[l]) MB_TRY(dev_alloc((void**)&S->d_wpack[l], pk.size()));
        MB_CUDA(cudaMemcpy(S->d_wpack[l], pk.data(), pk.size(), cudaMemcpyHostToDevice));
    }
    if (!S->h_err) {
        if (fault_oom()) {
            set_error("pinned allocation failed (MB_FAULT_OOM injected)");
            return MB_ERR_OOM;
        }
        MB_CUDA(cudaHostAlloc((void**)&S->h_err, sizeof(int), cudaHostAllocMapped));
        *S->h_err = 0;
        MB_CUDA(cudaHostGetDevicePointer((void**)&S->d_err, S->h_err, 0));
    }
    return MB_OK;
}

void fm_tc_release(mb_net* net) {
    FmTcState* S = reinterpret_cast<FmTcState*>(net->fm_state);
    if (!S) return;
    for (uint8_t* w : S->d_wpack) dev_free(w);
    if (S->h_err) cudaFreeHost(S->h_err);
    delete S;
    net->fm_state = nullptr;
}

mb_status fm_tc_poll_error(mb_net* net) {
    FmTcState* S = reinterpret_cast<FmTcState*>(net->fm_state);
    if (S && S->h_err && *(volatile int*)S->h_err) {
        *(volatile int*)S->h_err = 0;
        set_error("a FastMemb tensor-core launch gave up waiting (device-side wait limit)");
        return MB_ERR_TIMEOUT;
    }
    return MB_OK;
}

mb_status fm_tc_layer(mb_net* net, int layer, const void* in, int64_t in_slice, int64_t in_pitch, int64_t src_rows,
                      int64_t src_cols, int in_rows, int in_cols, int dm, int stride, void* out, int64_t out_slice,
                      int64_t out_pitch, int out_h, int out_w, int d, int nz, int out_u8, cudaStream_t st) {
    FmTcState* S = reinterpret_cast<FmTcState*>(net->fm_state);
    if (!S || !S->d_wpack[layer]) {
        set_error("FastMemb tensor-core weights not prepared");
        return MB_ERR_NOT_READY;
    }
    FmTcParams p{};
    p.in = static_cast<const uint16_t*>(in);
    p.out = out;
    p.wpack = S->d_wpack[layer];
    p.err = S->d_err;
    p.in_slice = in_slice;
    p.in_pitch = in_pitch;
    p.out_slice = out_slice;
    p.out_pitch = out_pitch;
    p.in_rows = in_rows;
    p.in_cols = in_cols;
    p.stride = stride;
    p.src_cols = src_cols;
    if ((int64_t)stride * (in_rows - 1) + dm >= src_rows || (int64_t)stride * (in_cols - 1) + dm >= src_cols) {
        set_error("FastMemb: input domain exceeds its source");
        return MB_ERR_INVALID_ARG;
    }
    p.out_h = out_h;
    p.out_w = out_w;
    p.d = d;
    p.dm = dm;
    p.nz = nz;
    p.out_u8 = out_u8;
    p.n_strips = (out_w + 127) / 128;
    p.total_rows = (int64_t)nz * p.n_strips * out_h;
    const char* stall = getenv("MB_FAULT_STALL");
    p.fault_stall = (stall && stall[0] == '1') ? 1 : 0;
    p.wait_ns = p.fault_stall ? 200000000ull : kFWaitNs;
    const bool head = layer == fastmemb_convs(net->family) - 2;
    if (net->prec == MB_PREC_FP16) return head ? launch_fm_tc<true, true>(p, st) : launch_fm_tc<false, true>(p, st);
    return head ? launch_fm_tc<true, false>(p, st) : launch_fm_tc<false, false>(p, st);
}

}  // namespace mb
