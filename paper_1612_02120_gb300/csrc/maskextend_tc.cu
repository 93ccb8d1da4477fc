// maskextend_tc.cu - MaskExtend's five max-out convolutions (Sec. 3.2) on the 5th-generation tensor
// cores, FP16 operands and FP32 accumulation; the last one ends with the 1x1 64->3 head and the
// 3-class softmax in its epilogue.
//
// Implicit GEMM per output row y and 128-pixel column strip x0 of a conv with dilation D:
//   D[128 px][N] = sum over taps (ky, kx) and K chunks kc of  A[128 px][16 ch] x B[N][16 ch]^T
// N = 2 x features (the max-out pairs, channels 2c and 2c+1 -> feature c), K = input channels
// padded to a multiple of 16 (12 -> 16, 40 -> 48, 56 -> 64). A for tap (ky, kx) is staged input row
// y + D ky at pixels x0 + D kx .. + 127: one staged row in the no-swizzle K-major layout
// [8-channel chunk][pixel][16 B], the column tap a (D kx x 16)-byte shift of the descriptor.
//
// The weights of the deeper layers (up to 16 taps x 64 x 128 FP16 = 256 KB) do not fit in shared
// memory beside the staged rows, so B is streamed in units of 4 taps (2 for the widest layer) and
// reused over a group of R output rows of one residue class y mod D (R TMEM accumulators: 8 at
// N = 64, else 4). A group's taps run ky-major: step ky reads staged rows m + ky .. m + ky + R - 1,
// so the window of staged rows slides by one row per step. In step 0 the rows are issued one after
// the other (all four taps of ky = 0 resident), so an accumulator is only waited for when its row
// starts while the epilogue drains the previous group's rows in the same order. The issuing thread
// polls one mbarrier per weight unit and per staged row and commits once per unit, per staged row
// and per group: with the tensor pipe reading shared memory at its full rate, each poll or commit
// costs tens of cycles of MMA issue.
//
// Warp roles (512 threads, 1 CTA per SM, persistent over work items):
//   warp 0       TMEM owner; lane 0 issues the MMAs
//   warp 1       lane 0 streams the weight units into their ring with bulk asynchronous copies
//                (completion counted on the unit's mbarrier)
//   warps 4-7    epilogue: TMEM -> registers, + bias, max-out, FP16 store (head: the 1x1 conv to 3
//                classes and the softmax, FP32 probabilities)
//   warps 8-15   A producers, groups taking staged rows in turn (4 groups of 2 warps for the first
//                layer, 2 of 4 after): the 2x2 max-filter (dilation dm) of the previous layer's
//                output, or the assembled input stack, into the staged-row ring (as deep as shared
//                memory allows, up to 12 rows)
// Every mbarrier wait is bounded (a global-timer limit), after which the CTA records
// MB_ERR_TIMEOUT in a mapped host word, stops issuing work, waits (bounded) for its bulk copies in
// flight and frees its TMEM.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace mb {

namespace {

constexpr int kMThreads = 512;
constexpr int kMBRing = 3;   // weight units in flight (a unit is 4 or 2 tap tiles)
constexpr uint64_t kMWaitNs = 4000000000ull;

// Staged pixels per row: >= 128 + 3 D, and chosen so that the 8 threads of a quarter-warp, which
// store consecutive (chunk, pixel) tasks, hit distinct 16-byte bank groups (pixel pitch of a chunk
// plane = MP x 16 bytes).
__host__ __device__ constexpr int me_mp(int chunks, int D) {
    return chunks == 2 ? 132 : chunks == 4 ? 138 : D <= 4 ? 141 : D <= 8 ? 153 : 177;
}

template <int KC, int N, int D, bool HEAD>
struct MCfg {
    static constexpr int kChunks = 2 * KC;              // 8-channel chunks per staged pixel
    static constexpr int kMP = me_mp(kChunks, D);
    static constexpr int kNpix = 128 + 3 * D;            // staged pixels a row needs
    static constexpr int kARow = kChunks * kMP * 16;     // bytes per staged row
    static constexpr int kBTap = kChunks * N * 16;       // bytes per tap tile [chunk][N][16 B]
    static constexpr int kConsts = N + (HEAD ? 3 * 64 + 3 : 0);  // biases (+ head W[3][64], b[3])
    // output rows per group = TMEM accumulators (512 columns, 64 or 128 apart)
    static constexpr int kR = N <= 64 ? 8 : 4;
    static constexpr int kAccStride = 512 / kR;
    // taps per weight unit (one mbarrier, one release): a whole step's 4 taps, or 2 for the widest
    static constexpr int kBU = KC == 4 ? 2 : 4;
    static constexpr int kBUnit = kBU * kBTap;
    // staged rows: kR in use by a step, the rest filled ahead (as many as fit, up to 12)
    static constexpr int kFixed = kMBRing * kBUnit + kConsts * 4 + 16 + (2 * kMBRing + kR + 2) * 8 + 16;
    static constexpr int kARing = (227 * 1024 - kFixed) / (kARow + 16) < 12 ? (227 * 1024 - kFixed) / (kARow + 16) : 12;
    // producer groups taking staged rows in turn (more for the short rows of the first layer)
    static constexpr int kGroups = KC == 1 ? 4 : 2;
    static constexpr int kGThreads = 256 / kGroups;
    static constexpr int oA = 0;
    static constexpr int oB = oA + kARing * kARow;
    static constexpr int oConst = oB + kMBRing * kBUnit;
    static constexpr int oBar = oConst + ((kConsts * 4 + 15) & ~15);
    static constexpr int kBars = 2 * kARing + 2 * kMBRing + 1 + kR + 1;
    static constexpr int oMisc = oBar + kBars * 8;
    static constexpr int kSmem = oMisc + 16;
    static constexpr int kATasks = (kNpix * kChunks + kGThreads - 1) / kGThreads;
    static_assert(kNpix <= kMP, "staged row too short");
    static_assert(kARing >= kR + 1, "staged-row ring");
    static_assert(N % 16 == 0 && N <= 128, "MMA N");
    static_assert(kSmem <= 227 * 1024, "shared memory");
};

struct MeTcParams {
    const __half* in;       // source [src rows][in_pitch][cs] FP16
    __half* out;            // layers: [out_h][out_pitch][N/2] FP16
    float* probs;           // head: [3][out_h][out_pitch] FP32, planes probs_plane apart
    const uint8_t* wpack;   // 16 tap tiles, then the FP32 constants
    int* err;
    int64_t in_pitch, out_pitch, probs_plane;  // pixels
    int cs;                 // source channels (a multiple of 8, <= 16 KC)
    int in_rows, in_cols;   // conv input domain: input (r, c) = 2x2 max (dilation dm) at source (r, c)
    int out_h, out_w, dm;
    int n_strips;
    int total_rows;         // strip-rows of the launch: n_strips x out_h (< 2^31, checked)
    int fault_stall;        // test injection: producers withhold their arrivals
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

struct MeItem {
    int ry, x0, m0, rows;  // output rows y = ry + D (m0 + j), j < rows; rows may be 0
};

// Work split: the launch's strip-rows, in (residue class ry, strip, row) order, are cut into one
// equal contiguous range per CTA (every CTA gets the same number of rows, no tail wave); a CTA's
// items are the parts of its range in one (ry, strip) column. Residue class ry has
// hr = ceil((out_h - ry) / D) rows per strip, i.e. base + 1 for ry < rem and base after
// (out_h = D base + rem), so n_strips (ry base + min(ry, rem)) strip-rows precede it. Every role of
// a CTA walks the same sequence.
struct MeCursor {
    int g, hi;  // next strip-row, end of this CTA's range
};

__device__ __forceinline__ MeCursor me_begin(const MeTcParams& p) {
    MeCursor c;
    c.g = (int)((int64_t)p.total_rows * blockIdx.x / gridDim.x);
    c.hi = (int)((int64_t)p.total_rows * (blockIdx.x + 1) / gridDim.x);
    return c;
}

template <int D>
__device__ __forceinline__ bool me_next(const MeTcParams& p, MeCursor& c, MeItem& it) {
    if (c.g >= c.hi) return false;
    const int base = p.out_h / D, rem = p.out_h % D;
    auto before = [&](int ry) { return p.n_strips * (ry * base + min(ry, rem)); };
    int ry = 0;
    while (ry + 1 < D && before(ry + 1) <= c.g) ++ry;
    const int hr = base + (ry < rem ? 1 : 0);  // > 0: before(ry) <= g < before(ry + 1)
    const int off = c.g - before(ry);
    const int strip = off / hr;
    it.ry = ry;
    it.x0 = strip * 128;
    it.m0 = off - strip * hr;
    it.rows = min(hr - it.m0, c.hi - c.g);
    c.g += it.rows;
    return true;
}

__device__ __forceinline__ uint4 hmax4(uint4 a, uint4 b) {
    uint4 r;
    const __half2* x = reinterpret_cast<const __half2*>(&a);
    const __half2* y = reinterpret_cast<const __half2*>(&b);
    __half2* o = reinterpret_cast<__half2*>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = __hmax2(x[i], y[i]);
    return r;
}

template <int KC, int N, int D, bool HEAD>
__global__ void __launch_bounds__(kMThreads, 1) me_tc_conv(const __grid_constant__ MeTcParams p) {
    using C = MCfg<KC, N, D, HEAD>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* a_full = reinterpret_cast<uint64_t*>(smem + C::oBar);
    uint64_t* a_empty = a_full + C::kARing;
    uint64_t* b_full = a_empty + C::kARing;
    uint64_t* b_empty = b_full + kMBRing;
    uint64_t* acc_full = b_empty + kMBRing;  // one per CTA: a group's accumulators are complete
    uint64_t* acc_free = acc_full + 1;       // per accumulator: drained by the epilogue
    uint64_t* fin = acc_free + C::kR;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::oMisc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::oMisc + 4);
    const float* cst = reinterpret_cast<const float*>(smem + C::oConst);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < C::kARing; ++i) {
            ptx::mbar_init(&a_full[i], C::kGThreads);
            ptx::mbar_init(&a_empty[i], 1);
        }
        for (int i = 0; i < kMBRing; ++i) {
            ptx::mbar_init(&b_full[i], 1);
            ptx::mbar_init(&b_empty[i], 1);
        }
        ptx::mbar_init(acc_full, 1);
        for (int i = 0; i < C::kR; ++i) ptx::mbar_init(&acc_free[i], 128);
        ptx::mbar_init(fin, 1);
        *abort_flag = 0;
        ptx::mbar_fence_init();
    }
    {
        const float* src = reinterpret_cast<const float*>(p.wpack + 16 * C::kBTap);
        float* dst = reinterpret_cast<float*>(smem + C::oConst);
        for (int i = tid; i < C::kConsts; i += kMThreads) dst[i] = __ldg(src + i);
    }
    if (warp == 0) {
        ptx::tmem_alloc(tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    const uint32_t sbase = ptx::smem_u32(smem);

    if (warp == 0) {
        // ================= MMA issuer ================================================================
        if (lane == 0) {
            const uint64_t adesc0 = ptx::smem_desc(sbase + C::oA, C::kMP * 16, 128);
            const uint64_t bdesc0 = ptx::smem_desc(sbase + C::oB, N * 16, 128);
            constexpr uint32_t idesc = ptx::idesc_f32acc(ptx::kFmtF16, 128, N);
            constexpr int kR = C::kR, kBU = C::kBU;
            uint32_t a_seq = 0, u_seq = 0;
            uint32_t free_par = 0;  // bit j: parity of the next use of accumulator j
            bool ok = true;
            // Row j of every group accumulates in TMEM columns kAccStride j (a group always starts
            // at accumulator 0, so a group cannot complete before the epilogue has taken the one
            // before it). Rows are runtime loops and only taps and K chunks are unrolled (the tap
            // shift D kx and the chunk kc are compile-time offsets): a short issue loop stays in
            // the instruction cache beside the other roles' code.
            auto mma_taps = [&](uint64_t ad, uint32_t dcol, uint64_t bd, auto kx0, auto ntaps, bool zero_first) {
#pragma unroll
                for (int t = 0; t < decltype(ntaps)::value; ++t)
#pragma unroll
                    for (int kc = 0; kc < KC; ++kc) {
                        const int kx = decltype(kx0)::value + t;
                        ptx::mma_bf16(dcol, ad + (uint64_t)((D * kx * 16 + kc * 2 * C::kMP * 16) >> 4),
                                      bd + (uint64_t)(((kx % kBU) * C::kBTap + kc * 2 * N * 16) >> 4), idesc,
                                      (zero_first && t == 0 && kc == 0) ? 0u : 1u);
                    }
            };
            auto unit_desc = [&](uint32_t q) { return bdesc0 + (uint64_t)(((q % kMBRing) * C::kBUnit) >> 4); };
            auto wait_unit = [&](uint32_t q) {
                ok = ok && wait_bar(&b_full[q % kMBRing], (q / kMBRing) & 1, abort_flag, p.err, p.wait_ns);
            };
            MeCursor cur = me_begin(p);
            MeItem it;
            while (me_next<D>(p, cur, it)) {
                const int groups = (it.rows + kR - 1) / kR;
                int a_known = 0;  // staged rows [0, a_known) of the item are known full
                int a_rel = 0;    // staged rows [0, a_rel) are released
                auto release_upto = [&](int last) {
                    for (; a_rel <= last; ++a_rel) ptx::mma_commit(&a_empty[(a_seq + a_rel) % C::kARing]);
                };
                for (int g = 0; g < groups; ++g) {
                    const int rg = min(kR, it.rows - kR * g);
                    for (int ky = 0; ky < 4; ++ky) {
                        const int s = kR * g + ky;  // staged rows s .. s + rg - 1
                        for (; a_known < s + rg; ++a_known) {
                            const uint32_t q = a_seq + a_known;
                            ok = ok && wait_bar(&a_full[q % C::kARing], (q / C::kARing) & 1, abort_flag, p.err, p.wait_ns);
                        }
                        const uint32_t aslot0 = (a_seq + s) % C::kARing;
                        auto arow = [&](int j) {
                            const uint32_t sl = aslot0 + j < (uint32_t)C::kARing ? aslot0 + j : aslot0 + j - C::kARing;
                            return adesc0 + (uint64_t)((sl * C::kARow) >> 4);
                        };
                        if (ky == 0) {
                            // the step's weight units, then rows one after the other, each waiting
                            // only for its own accumulator
                            for (int u = 0; u < 4 / kBU; ++u) wait_unit(u_seq + u);
                            const uint64_t bd0 = unit_desc(u_seq), bd1 = unit_desc(u_seq + (4 / kBU) - 1);
                            for (int j = 0; j < rg; ++j) {
                                ok = ok && wait_bar(&acc_free[j], ((free_par >> j) & 1) ^ 1, abort_flag, p.err,
                                                    p.wait_ns);
                                free_par ^= 1u << j;
                                ptx::tc_fence_after();
                                const uint64_t ad = arow(j);
                                const uint32_t dcol = tbase + (uint32_t)(C::kAccStride * j);
                                if (ok) {
                                    if constexpr (kBU == 4) {
                                        mma_taps(ad, dcol, bd0, std::integral_constant<int, 0>{},
                                                 std::integral_constant<int, 4>{}, true);
                                    } else {
                                        mma_taps(ad, dcol, bd0, std::integral_constant<int, 0>{},
                                                 std::integral_constant<int, 2>{}, true);
                                        mma_taps(ad, dcol, bd1, std::integral_constant<int, 2>{},
                                                 std::integral_constant<int, 2>{}, false);
                                    }
                                }
                            }
                            for (int u = 0; u < 4 / kBU; ++u) ptx::mma_commit(&b_empty[(u_seq + u) % kMBRing]);
                            u_seq += 4 / kBU;
                        } else {
                            for (int u = 0; u < 4 / kBU; ++u) {
                                wait_unit(u_seq);
                                ptx::tc_fence_after();
                                const uint64_t bd = unit_desc(u_seq);
                                if (ok) {
                                    for (int j = 0; j < rg; ++j) {
                                        const uint64_t ad = arow(j);
                                        const uint32_t dcol = tbase + (uint32_t)(C::kAccStride * j);
                                        if constexpr (kBU == 4) {
                                            mma_taps(ad, dcol, bd, std::integral_constant<int, 0>{},
                                                     std::integral_constant<int, 4>{}, false);
                                        } else if (u == 0) {
                                            mma_taps(ad, dcol, bd, std::integral_constant<int, 0>{},
                                                     std::integral_constant<int, 2>{}, false);
                                        } else {
                                            mma_taps(ad, dcol, bd, std::integral_constant<int, 2>{},
                                                     std::integral_constant<int, 2>{}, false);
                                        }
                                    }
                                }
                                ptx::mma_commit(&b_empty[u_seq % kMBRing]);
                                ++u_seq;
                            }
                        }
                        // staged row s is not read by any later step
                        release_upto(s);
                    }
                    ptx::mma_commit(acc_full);
                    // rows before the next group's first are done; after the last group, all rows
                    release_upto(g + 1 < groups ? kR * (g + 1) - 1 : it.rows + 2);
                }
                a_seq += it.rows + 3;
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
        uint32_t n_groups = 0;
        MeCursor cur = me_begin(p);
        MeItem it;
        while (me_next<D>(p, cur, it)) {
            const int x = it.x0 + px;
            for (int j = 0; j < it.rows; ++j) {
                if (j % C::kR == 0) {  // a new group: all its accumulators are complete together
                    wait_bar(acc_full, n_groups & 1, abort_flag, p.err, p.wait_ns);
                    ++n_groups;
                    ptx::tc_fence_after();
                }
                const uint32_t s = j % C::kR;  // accumulator of this row
                const uint32_t ta = tbase + lanes + (uint32_t)C::kAccStride * s;
                const int y = it.ry + D * (it.m0 + j);
                const bool store = x < p.out_w && y < p.out_h && !*abort_flag;
                if constexpr (HEAD) {
                    // features c = 0..63 -> logits z_k = b_k + sum_c W[k][c] f_c, in order of c
                    const float* hw = cst + N;
                    float z0 = hw[192], z1 = hw[193], z2 = hw[194];
#pragma unroll
                    for (int q = 0; q < N / 32; ++q) {
                        float v[32];
                        ptx::tmem_ld32(ta + 32u * q, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int c = 16 * q + i;
                            const float f = fmaxf(v[2 * i] + cst[2 * c], v[2 * i + 1] + cst[2 * c + 1]);
                            z0 = fmaf(hw[c], f, z0);
                            z1 = fmaf(hw[64 + c], f, z1);
                            z2 = fmaf(hw[128 + c], f, z2);
                        }
                    }
                    ptx::tc_fence_before();
                    ptx::mbar_arrive(&acc_free[s]);
                    const float m = fmaxf(z0, fmaxf(z1, z2));
                    const float e0 = expf(z0 - m), e1 = expf(z1 - m), e2 = expf(z2 - m);
                    const float den = e0 + e1 + e2;
                    if (store) {
                        float* o = p.probs + (int64_t)y * p.out_pitch + x;
                        o[0] = e0 / den;
                        o[p.probs_plane] = e1 / den;
                        o[2 * p.probs_plane] = e2 / den;
                    }
                } else {
                    // conv channels 2c, 2c+1 -> feature c; N/2 FP16 features = N/16 16-byte words
                    uint32_t w[N / 4];
#pragma unroll
                    for (int q = 0; q < N / 32; ++q) {
                        float v[32];
                        ptx::tmem_ld32(ta + 32u * q, v);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int n = 32 * q + 4 * i;
                            const float f0 = fmaxf(v[4 * i] + cst[n], v[4 * i + 1] + cst[n + 1]);
                            const float f1 = fmaxf(v[4 * i + 2] + cst[n + 2], v[4 * i + 3] + cst[n + 3]);
                            __half2 h2 = __floats2half2_rn(f0, f1);
                            w[8 * q + i] = *reinterpret_cast<uint32_t*>(&h2);
                        }
                    }
                    if constexpr (N % 32 != 0) {
                        constexpr int q = N / 32;
                        float v[16];
                        ptx::tmem_ld16(ta + 32u * q, v);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int n = 32 * q + 4 * i;
                            const float f0 = fmaxf(v[4 * i] + cst[n], v[4 * i + 1] + cst[n + 1]);
                            const float f1 = fmaxf(v[4 * i + 2] + cst[n + 2], v[4 * i + 3] + cst[n + 3]);
                            __half2 h2 = __floats2half2_rn(f0, f1);
                            w[8 * q + i] = *reinterpret_cast<uint32_t*>(&h2);
                        }
                    }
                    ptx::tc_fence_before();
                    ptx::mbar_arrive(&acc_free[s]);
                    if (store) {
                        uint4* o = reinterpret_cast<uint4*>(p.out + ((int64_t)y * p.out_pitch + x) * (N / 2));
#pragma unroll
                        for (int i = 0; i < N / 16; ++i) o[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ================= B producer: weight units, in the issuer's order ==========================
        if (lane == 0) {
            uint32_t issued = 0;
            bool go = true;
            MeCursor cur = me_begin(p);
            MeItem it;
            while (go && me_next<D>(p, cur, it)) {
                const int groups = (it.rows + C::kR - 1) / C::kR;
                for (int g = 0; go && g < groups; ++g)
                    for (int t0 = 0; go && t0 < 16; t0 += C::kBU) {
                        const uint32_t slot = issued % kMBRing;
                        go = wait_bar(&b_empty[slot], ((issued / kMBRing) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
                        if (go && !p.fault_stall) {
                            ptx::mbar_arrive_expect_tx(&b_full[slot], C::kBUnit);
                            for (int t = 0; t < C::kBU; ++t)
                                ptx::bulk_copy_g2s(smem + C::oB + slot * C::kBUnit + t * C::kBTap,
                                                   p.wpack + (size_t)(t0 + t) * C::kBTap, C::kBTap, &b_full[slot]);
                            ++issued;
                        }
                    }
            }
            // the copies still in flight land before the CTA exits (bounded, abort or not)
            for (uint32_t q = issued > (uint32_t)kMBRing ? issued - kMBRing : 0; q < issued; ++q) {
                const uint64_t t0 = gtime();
                while (!ptx::mbar_test(&b_full[q % kMBRing], (q / kMBRing) & 1))
                    if (gtime() - t0 > p.wait_ns) {
                        *(volatile int*)p.err = MB_ERR_TIMEOUT;
                        break;
                    }
            }
        }
        __syncwarp();
    } else if (warp >= 8) {
        // ================= A producers: staged input rows ===========================================
        // Group grp (kGroups groups of 8 / kGroups warps) stages the rows u = grp mod kGroups. Task
        // e = pt + kGThreads i: chunk e % kChunks of staged pixel e / kChunks (consecutive threads read
        // consecutive 16-byte chunks of one source pixel). All loads of a row are issued before the
        // slot wait so their latency overlaps it.
        const int grp = (tid - 256) / C::kGThreads;
        const int pt = tid - 256 - C::kGThreads * grp;
        const int64_t dxo = (int64_t)p.dm * p.cs, dyo = (int64_t)p.dm * p.in_pitch * p.cs;
        const int src_chunks = p.cs / 8;
        uint32_t a_seq = 0;
        MeCursor cur = me_begin(p);
        MeItem it;
        while (me_next<D>(p, cur, it)) {
            for (int u = grp; u < it.rows + 3; u += C::kGroups) {
                const uint32_t q = a_seq + u, slot = q % C::kARing;
                const int yin = it.ry + D * (it.m0 + u);
                uint4 v[C::kATasks];
#pragma unroll
                for (int i = 0; i < C::kATasks; ++i) {
                    const int e = pt + C::kGThreads * i;
                    const int c = e % C::kChunks, xin = it.x0 + e / C::kChunks;
                    v[i] = make_uint4(0, 0, 0, 0);
                    if (e < C::kNpix * C::kChunks && c < src_chunks && yin < p.in_rows && xin < p.in_cols) {
                        const __half* a = p.in + ((int64_t)yin * p.in_pitch + xin) * p.cs + c * 8;
                        const uint4 r0 = __ldg(reinterpret_cast<const uint4*>(a));
                        if (p.dm > 0) {
                            const uint4 r1 = __ldg(reinterpret_cast<const uint4*>(a + dxo));
                            const uint4 r2 = __ldg(reinterpret_cast<const uint4*>(a + dyo));
                            const uint4 r3 = __ldg(reinterpret_cast<const uint4*>(a + dyo + dxo));
                            v[i] = hmax4(hmax4(r0, r1), hmax4(r2, r3));
                        } else {
                            v[i] = r0;
                        }
                    }
                }
                wait_bar(&a_empty[slot], ((q / C::kARing) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
                uint8_t* dst = smem + C::oA + slot * C::kARow;
#pragma unroll
                for (int i = 0; i < C::kATasks; ++i) {
                    const int e = pt + C::kGThreads * i;
                    if (e < C::kNpix * C::kChunks)
                        *reinterpret_cast<uint4*>(dst + ((e % C::kChunks) * C::kMP + e / C::kChunks) * 16) = v[i];
                }
                ptx::fence_proxy_async_smem();
                if (!p.fault_stall) ptx::mbar_arrive(&a_full[slot]);
            }
            a_seq += it.rows + 3;
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tbase, 512);
}

uint16_t f16_bits(float f) {
    const __half h = __float2half_rn(f);
    uint16_t b;
    memcpy(&b, &h, 2);
    return b;
}

// Pack conv layer W[n][cin][4][4], b[n] (n < N conv channels) as 16 tap tiles: tile t = 4 ky + kx is
// [chunk kc][row n][8 FP16], input channel 8 kc + e (zero beyond cin); then the N FP32 biases and,
// for the last layer, the head W[3][64] and b[3].
void me_tc_pack(const float* W, const float* b, int cin, int n, int kc, const float* head, std::vector<uint8_t>& out) {
    const int chunks = 2 * kc, tap = chunks * n * 16;
    const size_t consts = (size_t)n + (head ? 3 * 64 + 3 : 0);
    out.assign((size_t)16 * tap + consts * 4, 0);
    for (int o = 0; o < n; ++o)
        for (int ci = 0; ci < cin; ++ci)
            for (int t = 0; t < 16; ++t) {
                const uint16_t h = f16_bits(W[((size_t)o * cin + ci) * 16 + t]);
                memcpy(out.data() + (size_t)t * tap + ((size_t)(ci / 8) * n + o) * 16 + (ci % 8) * 2, &h, 2);
            }
    float* c = reinterpret_cast<float*>(out.data() + (size_t)16 * tap);
    for (int o = 0; o < n; ++o) c[o] = b[o];
    if (head)
        for (int i = 0; i < 3 * 64 + 3; ++i) c[n + i] = head[i];
}

template <int KC, int N, int D, bool HEAD>
mb_status launch_me_tc(const MeTcParams& p, cudaStream_t st) {
    using C = MCfg<KC, N, D, HEAD>;
    static int n_sms = 0;
    if (n_sms == 0) {
        int dev = 0;
        MB_CUDA(cudaGetDevice(&dev));
        MB_CUDA(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    static bool attr = false;
    if (!attr) {
        MB_CUDA(cudaFuncSetAttribute(me_tc_conv<KC, N, D, HEAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     C::kSmem));
        attr = true;
    }
    // one range per SM, or fewer when a range would get under 8 rows
    const int grid = std::max(1, std::min(n_sms, (p.total_rows + 7) / 8));
    me_tc_conv<KC, N, D, HEAD><<<grid, kMThreads, C::kSmem, st>>>(p);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

// Layer table: input channels, K chunks of 16, N (= 2 x features), dilation.
constexpr int kMeCin[5] = {12, 32, 40, 48, 56};
constexpr int kMeKc[5] = {1, 2, 3, 3, 4};
constexpr int kMeN[5] = {64, 80, 96, 112, 128};

struct MeTcState {
    uint8_t* d_wpack[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int* h_err = nullptr;
    int* d_err = nullptr;
    int n_sms = 0;
};

}  // namespace

mb_status me_tc_prepare(mb_net* net) {
    MeTcState* S = reinterpret_cast<MeTcState*>(net->me_state);
    if (!S) {
        S = new (std::nothrow) MeTcState();
        if (!S) {
            set_error("host allocation failed");
            return MB_ERR_OOM;
        }
        net->me_state = S;
    }
    // API layout: per conv W [N][cin][4][4], b [N]; then the head W [3][64], b [3]
    const float* P = net->host_params.data();
    const float* head = P;
    for (int l = 0; l < 5; ++l) head += (size_t)kMeN[l] * kMeCin[l] * 16 + kMeN[l];
    std::vector<uint8_t> pk;
    for (int l = 0; l < 5; ++l) {
        const size_t nw = (size_t)kMeN[l] * kMeCin[l] * 16;
        me_tc_pack(P, P + nw, kMeCin[l], kMeN[l], kMeKc[l], l == 4 ? head : nullptr, pk);
        P += nw + kMeN[l];
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
    if (!S->n_sms) {
        int dev = 0;
        MB_CUDA(cudaGetDevice(&dev));
        MB_CUDA(cudaDeviceGetAttribute(&S->n_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return MB_OK;
}

void me_tc_release(mb_net* net) {
    MeTcState* S = reinterpret_cast<MeTcState*>(net->me_state);
    if (!S) return;
    for (uint8_t* w : S->d_wpack) dev_free(w);
    if (S->h_err) cudaFreeHost(S->h_err);
    delete S;
    net->me_state = nullptr;
}

mb_status me_tc_poll_error(mb_net* net) {
    MeTcState* S = reinterpret_cast<MeTcState*>(net->me_state);
    if (S && S->h_err && *(volatile int*)S->h_err) {
        *(volatile int*)S->h_err = 0;
        set_error("a MaskExtend tensor-core launch gave up waiting (device-side wait limit)");
        return MB_ERR_TIMEOUT;
    }
    return MB_OK;
}

// Rows per work item: the cost of a launch is taken as waves x (rows + 5) staged-row steps (3 rows
// of context and ~2 of pipeline fill per item); the smallest cost wins, ties to more rows.

mb_status me_tc_layer(mb_net* net, int layer, const void* in, int64_t in_pitch, int cs, int in_rows, int in_cols,
                      int dm, void* out, int64_t out_pitch, int out_h, int out_w, float* probs, int64_t probs_plane,
                      cudaStream_t st) {
    MeTcState* S = reinterpret_cast<MeTcState*>(net->me_state);
    if (!S || !S->d_wpack[layer]) {
        set_error("MaskExtend tensor-core weights not prepared");
        return MB_ERR_NOT_READY;
    }
    static const int kD[5] = {1, 2, 4, 8, 16};
    const int d = kD[layer];
    if (cs % 8 != 0 || cs > 16 * kMeKc[layer] || in_rows < out_h + 3 * d || in_cols < out_w + 3 * d) {
        set_error("MaskExtend: inconsistent layer geometry");
        return MB_ERR_INVALID_ARG;
    }
    MeTcParams p{};
    p.in = static_cast<const __half*>(in);
    p.out = static_cast<__half*>(out);
    p.probs = probs;
    p.wpack = S->d_wpack[layer];
    p.err = S->d_err;
    p.in_pitch = in_pitch;
    p.out_pitch = out_pitch;
    p.probs_plane = probs_plane;
    p.cs = cs;
    p.in_rows = in_rows;
    p.in_cols = in_cols;
    p.out_h = out_h;
    p.out_w = out_w;
    p.dm = dm;
    p.n_strips = (out_w + 127) / 128;
    if ((int64_t)p.n_strips * out_h > 0x7fffffffLL) {
        set_error("MaskExtend: too many strip-rows for one launch");
        return MB_ERR_SHAPE;
    }
    p.total_rows = p.n_strips * out_h;
    const char* stall = getenv("MB_FAULT_STALL");
    p.fault_stall = (stall && stall[0] == '1') ? 1 : 0;
    p.wait_ns = p.fault_stall ? 200000000ull : kMWaitNs;
    switch (layer) {
        case 0: return launch_me_tc<1, 64, 1, false>(p, st);
        case 1: return launch_me_tc<2, 80, 2, false>(p, st);
        case 2: return launch_me_tc<3, 96, 4, false>(p, st);
        case 3: return launch_me_tc<3, 112, 8, false>(p, st);
        default: return launch_me_tc<4, 128, 16, true>(p, st);
    }
}

}  // namespace mb
