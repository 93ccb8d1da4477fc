// student_tc.cu - inference of the distilled student (the fast pass of the multi-pass idea, Sec. 1)
// in one fused kernel on the 5th-generation tensor cores, for BF16 student nets:
//   x = u/255 (mirror-padded by 2) -> conv3x3 1->16 + b, ReLU -> conv3x3 16->16 + b, ReLU
//   -> conv1x1 16->1 + b -> sigmoid
// Both convolutions are implicit GEMMs per 128-pixel strip row (M = 128 pixels, operands in the
// no-swizzle K-major layout [8-element chunk][pixel][16 B]):
//   layer 1  D1[px][co] = sum_kx A1[px + kx][ky] x W1[co][ky][kx] with A1[q][ky] = u(r - 1 + ky, q):
//            the three row taps are stacked along K (an input byte is exact in BF16), the column tap
//            kx is a kx x 16-byte shift of the descriptor start; 3 MMAs (N = 16, K = 16) per row.
//            The epilogue scales by 1/255 in FP32, adds the bias, applies ReLU and rounds to BF16
//            into a ring of staged feature rows.
//   layer 2  each staged row r is multiplied once per column tap kx with the three row taps stacked
//            along N (N = 48: blocks for output rows r-2, r-1, r with row taps 2, 1, 0), accumulating
//            into a ring of 12 row accumulators (windows that wrap the ring are split in two MMAs).
//            The epilogue adds the bias, applies ReLU, the head and the sigmoid in FP32 and stores.
// A strip covers 126 output columns (128 layer-1 pixels, the last two only feed the column taps).
//
// Warp roles (384 threads, two CTAs per SM, persistent over work items):
//   warp 0      TMEM owner (256 columns: layer-2 ring 0..191, layer-1 ring 192..255); lane 0
//               issues the layer-1 MMAs
//   warp 3      lane 0 issues the layer-2 MMAs (a thread stalls ~200 cycles on each commit; with
//               two issuing threads the tensor core keeps working meanwhile)
//   warps 1-2   operand builders: keep three input rows per column in registers and write the
//               layer-1 operand row (one 16-byte store per pixel per row)
//   warps 4-7   layer-1 epilogue (TMEM lane = layer-1 pixel)
//   warps 8-11  layer-2 epilogue and head (TMEM lane = output pixel)
// Every mbarrier wait is bounded (a global-timer limit), after which the CTA records
// MB_ERR_TIMEOUT in a mapped host word, stops issuing work and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"
#include "tc_ptx.cuh"

namespace mb {

namespace {

constexpr int kSThreads = 384;
constexpr int kSW = 126;                  // output columns per strip
constexpr int kSPitch = 136;              // pixels per operand row (128 + the column taps' overrun)
constexpr int kSRowB = 2 * kSPitch * 16;  // bytes per operand row: 2 chunks (K = 16 BF16)
constexpr int kNA1 = 4;                   // layer-1 operand rows in flight
constexpr int kNS = 6;                    // staged layer-1 feature rows
constexpr int kKL = 4;                    // layer-1 accumulators, 16 TMEM columns each
constexpr int kKA = 12;                   // layer-2 row accumulators, 16 TMEM columns each
constexpr int kSTmem = 256;
constexpr int kL1Col = 16 * kKA;          // first TMEM column of the layer-1 ring
constexpr int kB1 = 3 * 2 * 16 * 16;      // per column tap: [2 chunks][16 co][16 B]
constexpr int kB2Group = 2 * 48 * 16;     // per column tap: [2 chunks][48 rows][16 B]
constexpr int kB2 = 3 * kB2Group;
constexpr int kSConst = 64;               // b1[16] | b2[16] | head w[16] | head b | 1/255
constexpr int kCB1 = 0, kCB2 = 16, kCWH = 32, kCBH = 48, kCInv = 49;
constexpr int oSB1 = 0;
constexpr int oSB2 = oSB1 + kB1;
constexpr int oSA1 = oSB2 + kB2;
constexpr int oSS = oSA1 + kNA1 * kSRowB;
constexpr int oSConst = oSS + kNS * kSRowB;
constexpr int oSBar = oSConst + kSConst * 4;
constexpr int kSBars = 2 * kNA1 + 2 * kKL + 2 * kNS + 2 * kKA + 2;
constexpr int oSMisc = oSBar + kSBars * 8;
constexpr int kSUsed = oSMisc + 16;
// Requested shared memory: at most two CTAs fit on an SM, so their TMEM (2 x 256 columns) always
// fits and no CTA waits in tcgen05.alloc.
constexpr int kSSmem = 80 * 1024;
constexpr int kWpack = kB1 + kB2 + kSConst * 4;
constexpr uint64_t kSWaitNs = 4000000000ull;
// forward layout of the student's parameters (as packed for the CUDA-core path)
constexpr int kFW1 = 0, kFB1 = 144, kFW2 = 160, kFB2 = 2464, kFWH = 2480, kFBH = 2496;
static_assert(kSUsed <= kSSmem && 3 * kSSmem > 227 * 1024, "shared memory");
static_assert(oSA1 % 16 == 0 && oSS % 16 == 0 && oSBar % 8 == 0, "alignment");
static_assert(2 * kSTmem <= 512 && kL1Col + 16 * kKL <= kSTmem, "TMEM of two CTAs");

struct StTcParams {
    const uint8_t* in;        // slice z at in + z in_slice; row pitch in_pitch
    void* out;                // region output, [z][rows][cols] with out_pitch / out_slice
    const uint8_t* wpack;     // B operands then the FP32 constants
    int* err;
    int64_t in_slice, in_pitch, out_slice, out_pitch;
    int h, w;                 // slice
    int y0, x0, rows, cols;   // region
    int n_strips;
    int64_t total_rows;       // strip-rows of the launch: z x n_strips x rows
    int out_u8;
    int fault_stall;
    uint64_t wait_ns;
};

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A completed phase costs one poll: the abort flag is read only once the phase is found incomplete.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                         uint64_t limit_ns) {
    if (ptx::mbar_test(bar, parity)) return true;
    if (*abort_flag) return false;
    const uint64_t t0 = gtime();
    uint32_t n = 0;
    // mbarrier.try_wait suspends the thread for a while by itself; no extra sleep between polls
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

__device__ __forceinline__ int refl(int t, int n) { return t < 0 ? -t : (t >= n ? 2 * (n - 1) - t : t); }

struct StItem {
    int z, m0, rows, s0, ncol;  // region rows m0 .. m0 + rows - 1, region columns s0 .. s0 + ncol - 1
};

// Work split: the launch's strip-rows, in (slice, strip, row) order, are cut into one equal
// contiguous range per CTA (every CTA gets the same number of rows, no tail wave); a CTA's items
// are the parts of its range in one (slice, strip) column. Every role of a CTA walks the same
// sequence.
struct StCursor {
    int64_t g, hi;  // next strip-row, end of this CTA's range
};

__device__ __forceinline__ StCursor st_begin(const StTcParams& p) {
    StCursor c;
    c.g = p.total_rows * (int64_t)blockIdx.x / gridDim.x;
    c.hi = p.total_rows * (int64_t)(blockIdx.x + 1) / gridDim.x;
    return c;
}

__device__ __forceinline__ bool st_next(const StTcParams& p, StCursor& c, StItem& it) {
    if (c.g >= c.hi) return false;
    const int64_t col = c.g / p.rows;  // (slice, strip) column
    it.z = (int)(col / p.n_strips);
    const int strip = (int)(col - (int64_t)it.z * p.n_strips);
    it.m0 = (int)(c.g - col * p.rows);
    it.rows = (int)min((int64_t)(p.rows - it.m0), c.hi - c.g);
    it.s0 = strip * kSW;
    it.ncol = min(kSW, p.cols - it.s0);
    c.g += it.rows;
    return true;
}

// BF16 bits of a byte value (exact: every integer up to 256 has at most 8 significant bits).
__device__ __forceinline__ uint32_t bf16_of_byte(uint32_t v) { return __float_as_uint((float)v) >> 16; }

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__global__ void __launch_bounds__(kSThreads, 2) st_tc_infer(const __grid_constant__ StTcParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* a1_full = reinterpret_cast<uint64_t*>(smem + oSBar);
    uint64_t* a1_empty = a1_full + kNA1;
    uint64_t* l1_full = a1_empty + kNA1;
    uint64_t* l1_free = l1_full + kKL;
    uint64_t* s_full = l1_free + kKL;
    uint64_t* s_empty = s_full + kNS;
    uint64_t* l2_full = s_empty + kNS;
    uint64_t* l2_free = l2_full + kKA;
    uint64_t* fin = l2_free + kKA;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + oSMisc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + oSMisc + 4);
    const float* cst = reinterpret_cast<const float*>(smem + oSConst);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < kNA1; ++i) {
            ptx::mbar_init(&a1_full[i], 64);
            ptx::mbar_init(&a1_empty[i], 1);
        }
        for (int i = 0; i < kKL; ++i) {
            ptx::mbar_init(&l1_full[i], 1);
            ptx::mbar_init(&l1_free[i], 128);
        }
        for (int i = 0; i < kNS; ++i) {
            ptx::mbar_init(&s_full[i], 128);
            ptx::mbar_init(&s_empty[i], 1);
        }
        for (int i = 0; i < kKA; ++i) {
            ptx::mbar_init(&l2_full[i], 1);
            ptx::mbar_init(&l2_free[i], 128);
        }
        ptx::mbar_init(fin, 1);
        ptx::mbar_init(fin + 1, 1);
        *abort_flag = 0;
        ptx::mbar_fence_init();
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(p.wpack);
        uint4* dst = reinterpret_cast<uint4*>(smem + oSB1);
        for (int i = tid; i < (kB1 + kB2) / 16; i += kSThreads) dst[i] = __ldg(src + i);
        const float* csrc = reinterpret_cast<const float*>(p.wpack + kB1 + kB2);
        float* cdst = reinterpret_cast<float*>(smem + oSConst);
        for (int i = tid; i < kSConst; i += kSThreads) cdst[i] = __ldg(csrc + i);
        // both operand rings start zero: the second K chunk of the layer-1 operand and the pixels
        // past 127 of every row (read by the column taps, never written) stay zero
        uint4* r = reinterpret_cast<uint4*>(smem + oSA1);
        for (int i = tid; i < (kNA1 + kNS) * kSRowB / 16; i += kSThreads) r[i] = make_uint4(0, 0, 0, 0);
    }
    if (warp == 0) {
        ptx::tmem_alloc(tmem_slot, kSTmem);
        ptx::tmem_relinquish();
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    const uint32_t sbase = ptx::smem_u32(smem);
    if (warp >= 8) {
        // every layer-2 accumulator starts at zero (its MMAs only accumulate)
        const uint32_t lanes = (uint32_t)(32 * (warp - 8)) << 16;
        for (int sl = 0; sl < kKA; ++sl) ptx::tmem_st16_zero(tbase + lanes + 16u * sl);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();

    if (warp == 0 || warp == 3) {
        // ================= MMA issuers: warp 0 lane 0 layer 1, warp 3 lane 0 layer 2 ================
        // Each issues, commits and finally drains only its own MMAs; they meet only through the
        // layer-1 epilogue (layer 1 runs ahead as far as its 4 accumulators allow). A single thread's
        // per-row instruction chain is what bounds the issue rate of MMAs this small, so ring
        // positions are running slot/phase counters (no division per row), and a full layer-2 window
        // is issued from one of three branches with compile-time instruction descriptors: it starts
        // at most two slots before the ring's end (one N = 48 MMA per column tap) or in one of the last
        // two slots (split where it wraps).
        if (lane == 0) {
            constexpr uint32_t id16 = ptx::idesc_f32acc(ptx::kFmtBF16, 128, 16);
            constexpr uint32_t id32 = ptx::idesc_f32acc(ptx::kFmtBF16, 128, 32);
            constexpr uint32_t id48 = ptx::idesc_f32acc(ptx::kFmtBF16, 128, 48);
            bool ok = true;
            if (warp == 0) {
                static_assert(kNA1 == kKL, "one counter serves both layer-1 rings");
                const uint64_t a1d = ptx::smem_desc(sbase + oSA1, kSPitch * 16, 128);
                const uint64_t b1d = ptx::smem_desc(sbase + oSB1, 16 * 16, 128);
                uint32_t s1 = 0, ph1 = 0;  // operand slot = layer-1 accumulator slot, and its phase
                StCursor cur = st_begin(p);
                StItem it;
                while (st_next(p, cur, it)) {
                    const int n_rows = it.rows + 2;
                    for (int u = 0; u < n_rows; ++u) {
                        ok = ok && wait_bar(&a1_full[s1], ph1, abort_flag, p.err, p.wait_ns);
                        ok = ok && wait_bar(&l1_free[s1], ph1 ^ 1, abort_flag, p.err, p.wait_ns);
                        ptx::tc_fence_after();
                        if (ok) {
                            const uint64_t arow = a1d + (uint64_t)((s1 * kSRowB) >> 4);
#pragma unroll
                            for (int kx = 0; kx < 3; ++kx)
                                ptx::mma_bf16(tbase + kL1Col + 16u * s1, arow + (uint64_t)kx,
                                              b1d + (uint64_t)((kx * 512) >> 4), id16, kx ? 1u : 0u);
                        }
                        ptx::mma_commit(&a1_empty[s1]);
                        ptx::mma_commit(&l1_full[s1]);
                        if (++s1 == kKL) {
                            s1 = 0;
                            ph1 ^= 1;
                        }
                    }
                }
            } else {
                // staged row u of an item feeds output rows u-2+i, i = 0..2, with row tap 2-i; output
                // row o of the item accumulates in slot (aq + o) mod kKA, aq = output rows before it
                const uint64_t sd = ptx::smem_desc(sbase + oSS, kSPitch * 16, 128);
                const uint64_t b2d = ptx::smem_desc(sbase + oSB2, 48 * 16, 128);
                uint32_t ss = 0, sph = 0;  // staged slot and phase
                uint32_t as = 0, aph = 0;  // slot and phase of the next output row to start
                uint32_t ws = kKA - 2;     // slot of output row u - 2 (may be a row of no item)
                StCursor cur = st_begin(p);
                StItem it;
                while (st_next(p, cur, it)) {
                    const int R = it.rows, n_rows = R + 2;
                    for (int u = 0; u < n_rows; ++u) {
                        ok = ok && wait_bar(&s_full[ss], sph, abort_flag, p.err, p.wait_ns);
                        if (u < R)  // output row u starts here: its accumulator must have been drained
                            ok = ok && wait_bar(&l2_free[as], aph ^ 1, abort_flag, p.err, p.wait_ns);
                        ptx::tc_fence_after();
                        const uint64_t arow = sd + (uint64_t)((ss * kSRowB) >> 4);
                        if (ok && u >= 2 && u < R) {
                            if (ws < kKA - 2) {
#pragma unroll
                                for (int kx = 0; kx < 3; ++kx)
                                    ptx::mma_bf16(tbase + 16u * ws, arow + (uint64_t)kx,
                                                  b2d + (uint64_t)((kx * kB2Group) >> 4), id48, 1u);
                            } else if (ws == kKA - 2) {  // blocks 0-1 in the last two slots, block 2 in slot 0
#pragma unroll
                                for (int kx = 0; kx < 3; ++kx) {
                                    const uint64_t bg = b2d + (uint64_t)((kx * kB2Group) >> 4);
                                    ptx::mma_bf16(tbase + 16u * (kKA - 2), arow + (uint64_t)kx, bg, id32, 1u);
                                    ptx::mma_bf16(tbase, arow + (uint64_t)kx, bg + 32u, id16, 1u);
                                }
                            } else {  // block 0 in the last slot, blocks 1-2 in slots 0-1
#pragma unroll
                                for (int kx = 0; kx < 3; ++kx) {
                                    const uint64_t bg = b2d + (uint64_t)((kx * kB2Group) >> 4);
                                    ptx::mma_bf16(tbase + 16u * (kKA - 1), arow + (uint64_t)kx, bg, id16, 1u);
                                    ptx::mma_bf16(tbase, arow + (uint64_t)kx, bg + 16u, id32, 1u);
                                }
                            }
                        } else if (ok) {  // the first and last two staged rows: part of the window
                            const int ilo = max(0, 2 - u), ihi = min(2, R + 1 - u);
                            if (ilo <= ihi) {
                                const int s_lo = (int)((ws + (uint32_t)ilo) % kKA);
                                const int iw = ilo + (kKA - s_lo);  // first block whose slot wraps to 0
                                const int hi0 = iw <= ihi ? iw - 1 : ihi;
#pragma unroll
                                for (int kx = 0; kx < 3; ++kx) {
                                    const uint64_t bg = b2d + (uint64_t)((kx * kB2Group) >> 4);
                                    ptx::mma_bf16(tbase + 16u * s_lo, arow + (uint64_t)kx, bg + (uint64_t)(16 * ilo),
                                                  ptx::idesc_f32acc(ptx::kFmtBF16, 128, (uint32_t)(16 * (hi0 - ilo + 1))), 1u);
                                    if (iw <= ihi)
                                        ptx::mma_bf16(tbase, arow + (uint64_t)kx, bg + (uint64_t)(16 * iw),
                                                      ptx::idesc_f32acc(ptx::kFmtBF16, 128, (uint32_t)(16 * (ihi - iw + 1))), 1u);
                                }
                            }
                        }
                        ptx::mma_commit(&s_empty[ss]);
                        if (u >= 2) ptx::mma_commit(&l2_full[ws]);  // output row u - 2 is complete
                        if (++ss == kNS) {
                            ss = 0;
                            sph ^= 1;
                        }
                        if (u < R && ++as == kKA) {
                            as = 0;
                            aph ^= 1;
                        }
                        if (++ws == kKA) ws = 0;
                    }
                    // the next item's first window starts two rows before its output row 0
                    ws = (ws + kKA - 2) % kKA;
                }
            }
            uint64_t* f = fin + (warp == 0 ? 0 : 1);
            ptx::mma_commit(f);
            const uint64_t t0 = gtime();
            while (!ptx::mbar_test(f, 0)) {
                if (gtime() - t0 > p.wait_ns) {
                    *(volatile int*)p.err = MB_ERR_TIMEOUT;
                    break;
                }
            }
        }
        __syncwarp();
    } else if (warp == 1 || warp == 2) {
        // ================= layer-1 operand builder ====================================================
        // Operand row u of an item belongs to layer-1 row r = y0 + m0 - 1 + u: pixel q holds the input
        // bytes of rows r - 1 .. r + 1 (elements 0..2 of K chunk 0) at column x0 + s0 - 2 + q, both
        // mirror-padded at the slice borders. Builder thread b (warps 1-2) owns pixels b + 64 k; it
        // keeps its three rows in registers and has the loads of the kLd rows after them in flight
        // (one thread also bulk-prefetches rows into L2). A loaded byte is converted only when its
        // row enters the window: converting it at the load would stall the thread on the load.
        const int bt = tid - 32;
        uint32_t slot = 0, sph = 0;  // operand slot and its phase
        StCursor cur = st_begin(p);
        StItem it;
        while (st_next(p, cur, it)) {
            const int R = it.rows, n_rows = R + 2, last = R + 3;  // input rows 0 .. R + 3 of the item
            const uint8_t* src = p.in + (int64_t)it.z * p.in_slice;
            const int c0 = p.x0 + it.s0 - 2;
            const int nin = min(130, it.ncol + 4);  // input columns the strip's outputs depend on
            const int rbase = p.y0 + it.m0 - 2;
            int col[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) col[i] = bt + 64 * i < nin ? refl(c0 + bt + 64 * i, p.w) : -1;
            auto load_row = [&](int i, uint32_t (&v)[3]) {  // raw bytes (columns past the strip read column 0)
                const uint8_t* row = src + (int64_t)refl(rbase + min(i, last), p.h) * p.in_pitch;
#pragma unroll
                for (int j = 0; j < 3; ++j) v[j] = (uint32_t)__ldg(row + max(col[j], 0));
            };
            auto bf16_row = [&](uint32_t (&v)[3]) {  // raw bytes -> BF16 bits, zero past the strip
#pragma unroll
                for (int j = 0; j < 3; ++j) v[j] = col[j] >= 0 ? bf16_of_byte(v[j]) : 0u;
            };
            constexpr int kPf = 8;
            auto prefetch_row = [&](int i) {
                if (bt != 0 || i > last) return;
                const uint8_t* base = src + (int64_t)refl(rbase + i, p.h) * p.in_pitch;
                const uintptr_t lo = (uintptr_t)(base + max(0, c0)) & ~(uintptr_t)15;
                const uintptr_t hi = (uintptr_t)(base + min(p.w, c0 + nin)) & ~(uintptr_t)15;
                if (hi > lo) ptx::prefetch_l2_bulk((const void*)lo, (uint32_t)(hi - lo));
            };
            for (int i = 3; i < 3 + kPf; ++i) prefetch_row(i);
            constexpr int kLd = 3;  // input rows whose loads are in flight
            uint32_t w0[3], w1[3], w2[3], pend[kLd][3];
            load_row(0, w0);
            load_row(1, w1);
            load_row(2, w2);
            bf16_row(w0);
            bf16_row(w1);
            bf16_row(w2);
#pragma unroll
            for (int t = 0; t < kLd; ++t) load_row(3 + t, pend[t]);  // rows past the last are clamped to it
            for (int u0 = 0; u0 < n_rows; u0 += kLd) {
#pragma unroll
                for (int t = 0; t < kLd; ++t) {
                    const int u = u0 + t;
                    if (u >= n_rows) break;
                    prefetch_row(u + 3 + kPf);
                    wait_bar(&a1_empty[slot], sph ^ 1, abort_flag, p.err, p.wait_ns);
                    uint8_t* dst = smem + oSA1 + slot * kSRowB;
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int px = bt + 64 * j;
                        if (px < 130)
                            *reinterpret_cast<uint4*>(dst + px * 16) = make_uint4(w0[j] | (w1[j] << 16), w2[j], 0u, 0u);
                    }
                    ptx::fence_proxy_async_smem();
                    if (!p.fault_stall) ptx::mbar_arrive(&a1_full[slot]);
                    if (++slot == kNA1) {
                        slot = 0;
                        sph ^= 1;
                    }
                    // rows u+1 .. u+3 become the window; the loads of row u + 3 + kLd take row u+3's place
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        w0[j] = w1[j];
                        w1[j] = w2[j];
                        w2[j] = col[j] >= 0 ? bf16_of_byte(pend[t][j]) : 0u;
                    }
                    load_row(u + 3 + kLd, pend[t]);
                }
            }
        }
    } else if (warp >= 4 && warp < 8) {
        // ================= layer-1 epilogue: x 1/255, bias, ReLU, BF16 -> staged feature ring =======
        const int px = tid - 128;
        const uint32_t lanes = (uint32_t)(32 * (warp - 4)) << 16;
        const float inv = cst[kCInv];
        uint32_t sl = 0, lph = 0, ss = 0, sph = 0;  // accumulator and staged slots, their phases
        StCursor cur = st_begin(p);
        StItem it;
        while (st_next(p, cur, it)) {
            const int n_rows = it.rows + 2;
            for (int u = 0; u < n_rows; ++u) {
                wait_bar(&l1_full[sl], lph, abort_flag, p.err, p.wait_ns);
                ptx::tc_fence_after();
                float d[16];
                ptx::tmem_ld16(tbase + lanes + kL1Col + 16u * sl, d);
                ptx::tc_fence_before();
                ptx::mbar_arrive(&l1_free[sl]);
                if (++sl == kKL) {
                    sl = 0;
                    lph ^= 1;
                }
                uint32_t wd[8];
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    wd[c] = pack_bf16x2(fmaxf(fmaf(d[2 * c], inv, cst[kCB1 + 2 * c]), 0.f),
                                        fmaxf(fmaf(d[2 * c + 1], inv, cst[kCB1 + 2 * c + 1]), 0.f));
                wait_bar(&s_empty[ss], sph ^ 1, abort_flag, p.err, p.wait_ns);
                uint8_t* dst = smem + oSS + ss * kSRowB;
                *reinterpret_cast<uint4*>(dst + px * 16) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                *reinterpret_cast<uint4*>(dst + (kSPitch + px) * 16) = make_uint4(wd[4], wd[5], wd[6], wd[7]);
                ptx::fence_proxy_async_smem();
                ptx::mbar_arrive(&s_full[ss]);
                if (++ss == kNS) {
                    ss = 0;
                    sph ^= 1;
                }
            }
        }
    } else if (warp >= 8) {
        // ================= layer-2 epilogue: bias, ReLU, head, sigmoid, store ========================
        const int px = tid - 256;  // TMEM lane = output pixel of the strip
        const uint32_t lanes = (uint32_t)(32 * (warp - 8)) << 16;
        uint32_t sl = 0, aph = 0;  // accumulator slot and its phase
        // the head's constants in registers (shared-memory reads would repeat every row: the waits
        // are compiler barriers)
        float b2r[16], whr[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            b2r[c] = cst[kCB2 + c];
            whr[c] = cst[kCWH + c];
        }
        const float bhr = cst[kCBH];
        StCursor cur = st_begin(p);
        StItem it;
        while (st_next(p, cur, it)) {
            const bool col = px < it.ncol;
            int64_t idx = (int64_t)it.z * p.out_slice + (int64_t)it.m0 * p.out_pitch + it.s0 + px;
            for (int j = 0; j < it.rows; ++j, idx += p.out_pitch) {
                wait_bar(&l2_full[sl], aph, abort_flag, p.err, p.wait_ns);
                const bool live = !*abort_flag;  // read early: its latency overlaps the drain
                ptx::tc_fence_after();
                float d[16];
                const uint32_t ta = tbase + lanes + 16u * sl;
                ptx::tmem_ld16(ta, d);
                ptx::tmem_st16_zero(ta);
                ptx::tc_fence_before();
                ptx::mbar_arrive(&l2_free[sl]);
                if (++sl == kKA) {
                    sl = 0;
                    aph ^= 1;
                }
                float z = bhr;
#pragma unroll
                for (int c = 0; c < 16; ++c) z = fmaf(whr[c], fmaxf(d[c] + b2r[c], 0.f), z);
                // the correctly rounded reciprocal is the correctly rounded quotient 1 / x
                const float prob = __frcp_rn(1.0f + expf(-z));
                if (col && live) {
                    if (p.out_u8)
                        static_cast<uint8_t*>(p.out)[idx] = (uint8_t)fminf(floorf(255.0f * prob + 0.5f), 255.0f);
                    else
                        static_cast<float*>(p.out)[idx] = prob;
                }
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tbase, kSTmem);
}

// Operands and constants from the forward-layout parameters (W1t[tap][co], b1, W2t[ci][tap][co], b2,
// wh, bh; tap = 3 ky + kx):
//   B1, per column tap kx: [chunk][co][8] BF16 with element k = ky < 3 holding W1[co][ky][kx]
//   B2, per column tap kx: [chunk][n][8] BF16, n = 16 i + co, element ci holding W2[co][ci][2 - i][kx]
//   constants: b1, b2, head weights, head bias, 1/255
__global__ void st_tc_pack(const float* fwd, uint8_t* wpack) {
    __nv_bfloat16* b1 = reinterpret_cast<__nv_bfloat16*>(wpack);
    for (int i = threadIdx.x; i < kB1 / 2; i += blockDim.x) {
        const int kx = i / 256, rem = i % 256, kk = (rem / 128) * 8 + rem % 8, co = (rem / 8) % 16;
        b1[i] = __float2bfloat16_rn(kk < 3 ? fwd[kFW1 + (kk * 3 + kx) * 16 + co] : 0.f);
    }
    __nv_bfloat16* b2 = reinterpret_cast<__nv_bfloat16*>(wpack + kB1);
    for (int i = threadIdx.x; i < kB2 / 2; i += blockDim.x) {
        const int kx = i / 768, rem = i % 768, ci = (rem / 384) * 8 + rem % 8, n = (rem / 8) % 48;
        const int ky = 2 - n / 16, co = n % 16;
        b2[i] = __float2bfloat16_rn(fwd[kFW2 + (ci * 9 + ky * 3 + kx) * 16 + co]);
    }
    float* c = reinterpret_cast<float*>(wpack + kB1 + kB2);
    for (int i = threadIdx.x; i < kSConst; i += blockDim.x) {
        float v = 0.f;
        if (i < 16) v = fwd[kFB1 + i];
        else if (i < 32) v = fwd[kFB2 + (i - 16)];
        else if (i < 48) v = fwd[kFWH + (i - 32)];
        else if (i == kCBH) v = fwd[kFBH];
        else if (i == kCInv) v = 1.0f / 255.0f;
        c[i] = v;
    }
}

struct StTcState {
    uint8_t* d_wpack = nullptr;
    int* h_err = nullptr;
    int* d_err = nullptr;
    int n_sms = 0;
};

}  // namespace

void st_tc_release(mb_net* net) {
    StTcState* S = reinterpret_cast<StTcState*>(net->st_state);
    if (!S) return;
    dev_free(S->d_wpack);
    if (S->h_err) cudaFreeHost(S->h_err);
    delete S;
    net->st_state = nullptr;
}

mb_status st_tc_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                       int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                       int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st) {
    if (z == 0 || rows == 0 || cols == 0) return MB_OK;
    StTcState* S = reinterpret_cast<StTcState*>(net->st_state);
    if (!S) {
        S = new (std::nothrow) StTcState();
        if (!S) {
            set_error("host allocation failed");
            return MB_ERR_OOM;
        }
        net->st_state = S;
    }
    if (!S->d_wpack) MB_TRY(dev_alloc((void**)&S->d_wpack, kWpack));
    if (!S->h_err) {
        if (fault_oom()) {
            set_error("pinned allocation failed (MB_FAULT_OOM injected)");
            return MB_ERR_OOM;
        }
        MB_CUDA(cudaHostAlloc((void**)&S->h_err, sizeof(int), cudaHostAllocMapped));
        *S->h_err = 0;
        MB_CUDA(cudaHostGetDevicePointer((void**)&S->d_err, S->h_err, 0));
    }
    if (*(volatile int*)S->h_err) {
        *(volatile int*)S->h_err = 0;
        set_error("a student tensor-core launch gave up waiting (device-side wait limit)");
        return MB_ERR_TIMEOUT;
    }
    if (!S->n_sms) {
        int dev = 0;
        MB_CUDA(cudaGetDevice(&dev));
        MB_CUDA(cudaDeviceGetAttribute(&S->n_sms, cudaDevAttrMultiProcessorCount, dev));
        MB_CUDA(cudaFuncSetAttribute(st_tc_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kSSmem));
    }
    // the forward copy changes while the student trains: pack it on every call
    st_tc_pack<<<1, 256, 0, st>>>(net->d_simt, S->d_wpack);
    count_launch();
    MB_CUDA(cudaGetLastError());
    StTcParams p{};
    p.in = in;
    p.out = out;
    p.wpack = S->d_wpack;
    p.err = S->d_err;
    p.in_slice = in_slice;
    p.in_pitch = in_pitch;
    p.out_slice = out_slice;
    p.out_pitch = out_pitch;
    p.h = (int)h;
    p.w = (int)w;
    p.y0 = (int)y0;
    p.x0 = (int)x0;
    p.rows = (int)rows;
    p.cols = (int)cols;
    p.out_u8 = ot == MB_OUT_U8 ? 1 : 0;
    p.n_strips = (int)((cols + kSW - 1) / kSW);
    const int64_t slots = (int64_t)S->n_sms * 2;
    p.total_rows = z * p.n_strips * rows;
    const char* stall = getenv("MB_FAULT_STALL");
    p.fault_stall = (stall && stall[0] == '1') ? 1 : 0;
    p.wait_ns = p.fault_stall ? 200000000ull : kSWaitNs;
    // one range per CTA slot, or fewer when a range would get under 8 rows
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(slots, (p.total_rows + 7) / 8));
    st_tc_infer<<<grid, kSThreads, kSSmem, st>>>(p);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

}  // namespace mb
