// student_tc.cu - inference of the distilled student (the fast pass of the multi-pass idea, Sec. 1)
// in one fused kernel on the 5th-generation tensor cores, for BF16 student nets:
//   x = u/255 (mirror-padded by 2) -> conv3x3 1->16 + b, ReLU -> conv3x3 16->16 + b, ReLU
//   -> conv1x1 16->1 + b -> sigmoid
// Layer 1 runs on CUDA cores in FP32 (packed FP32x2 FMAs) and is rounded to BF16 into a ring of
// staged rows; layer 2 is an implicit GEMM per output row and 128-pixel strip:
//   D[128 px][16 co] = sum over taps (ky, kx) of A_{ky,kx}[128 px][16 ci] x B_{ky,kx}[16 co][16 ci]^T
// where A_{ky,kx} is staged row y - 1 + ky at pixels kx .. kx + 127 (a kx x 16-byte shift of the
// descriptor start in the no-swizzle K-major layout [8-channel chunk][pixel][16 B]). The epilogue
// adds the bias, applies ReLU, the head and the sigmoid in FP32 and stores the probability.
//
// Warp roles (256 threads, several CTAs per SM, persistent over work items):
//   warp 0      TMEM owner (128 columns: 8 accumulators of 16); lane 0 issues the MMAs
//   warps 1-3   layer-1 producers: 130 pixels x 2 channel halves per staged row, from input rows
//               staged once each in shared memory
//   warps 4-7   epilogue: TMEM lane = pixel of the strip
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

constexpr int kSThreads = 256;
constexpr int kSP = 132;                  // staged pixels per row (>= 130; 132 mod 8 = 4 spreads the
                                          // two chunk planes of 4 consecutive pixels over distinct banks)
constexpr int kSRow = 2 * kSP * 16;       // bytes per staged row
constexpr int kSRing = 8;                 // staged rows
constexpr int kSAcc = 8;                  // accumulators, 16 TMEM columns each
constexpr int kSTmem = 128;
constexpr int kSB = 9 * 2 * 16 * 16;      // B: 9 taps x [2 chunks][16 co][16 B]
constexpr int kSConst = 193;              // W1t[9][16], b1[16], b2[16], wh[16], bh
constexpr int oSB = 0;
constexpr int oSRing = oSB + kSB;
constexpr int oSConst = oSRing + kSRing * kSRow;
constexpr int oSIn = oSConst + ((kSConst * 4 + 15) & ~15);  // 4 input rows x 136 floats
constexpr int oSBar = oSIn + 4 * 136 * 4;
constexpr int kSBars = 2 * kSRing + 2 * kSAcc + 1;
constexpr int oSMisc = oSBar + kSBars * 8;
constexpr int kSSmem = oSMisc + 16;
constexpr int kSProdThreads = 96;
constexpr int kSTasks = (130 * 2 + kSProdThreads - 1) / kSProdThreads;
constexpr uint64_t kSWaitNs = 4000000000ull;
// forward layout of the student's parameters (as packed for the CUDA-core path)
constexpr int kFW1 = 0, kFB1 = 144, kFW2 = 160, kFB2 = 2464, kFWH = 2480, kFBH = 2496;
static_assert(kSSmem <= 100 * 1024, "shared memory");

struct StTcParams {
    const uint8_t* in;        // slice z at in + z in_slice; row pitch in_pitch
    void* out;                // region output, [z][rows][cols] with out_pitch / out_slice
    const uint8_t* wpack;     // B tiles then the FP32 constants
    int* err;
    int64_t in_slice, in_pitch, out_slice, out_pitch;
    int h, w;                 // slice
    int y0, x0, rows, cols;   // region
    int n_strips, n_chunks, rows_per_item, n_items;
    int out_u8;
    int fault_stall;
    uint64_t wait_ns;
};

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                         uint64_t limit_ns) {
    if (*abort_flag) return false;
    if (ptx::mbar_test(bar, parity)) return true;
    const uint64_t t0 = gtime();
    uint32_t n = 0;
    while (!ptx::mbar_test(bar, parity)) {
        __nanosleep(32);
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

__device__ __forceinline__ StItem st_item(const StTcParams& p, int k) {
    StItem it;
    const int chunk = k % p.n_chunks;
    k /= p.n_chunks;
    const int strip = k % p.n_strips;
    it.z = k / p.n_strips;
    it.m0 = chunk * p.rows_per_item;
    it.rows = max(0, min(p.rows_per_item, p.rows - it.m0));
    it.s0 = strip * 128;
    it.ncol = min(128, p.cols - it.s0);
    return it;
}

__global__ void __launch_bounds__(kSThreads, 2) st_tc_infer(const __grid_constant__ StTcParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* a_full = reinterpret_cast<uint64_t*>(smem + oSBar);
    uint64_t* a_empty = a_full + kSRing;
    uint64_t* acc_full = a_empty + kSRing;
    uint64_t* acc_free = acc_full + kSAcc;
    uint64_t* fin = acc_free + kSAcc;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + oSMisc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + oSMisc + 4);
    const float* cst = reinterpret_cast<const float*>(smem + oSConst);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < kSRing; ++i) {
            ptx::mbar_init(&a_full[i], kSProdThreads);
            ptx::mbar_init(&a_empty[i], 1);
        }
        for (int i = 0; i < kSAcc; ++i) {
            ptx::mbar_init(&acc_full[i], 1);
            ptx::mbar_init(&acc_free[i], 128);
        }
        ptx::mbar_init(fin, 1);
        *abort_flag = 0;
        ptx::mbar_fence_init();
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(p.wpack);
        uint4* dst = reinterpret_cast<uint4*>(smem + oSB);
        for (int i = tid; i < kSB / 16; i += kSThreads) dst[i] = __ldg(src + i);
        const float* csrc = reinterpret_cast<const float*>(p.wpack + kSB);
        float* cdst = reinterpret_cast<float*>(smem + oSConst);
        for (int i = tid; i < kSConst; i += kSThreads) cdst[i] = __ldg(csrc + i);
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

    if (warp == 0) {
        // ================= MMA issuer ================================================================
        if (lane == 0) {
            const uint64_t adesc0 = ptx::smem_desc(sbase + oSRing, kSP * 16, 128);
            const uint64_t bdesc0 = ptx::smem_desc(sbase + oSB, 16 * 16, 128);
            constexpr uint32_t idesc = ptx::idesc_f32acc(ptx::kFmtBF16, 128, 16);
            uint32_t a_seq = 0, acc_seq = 0;
            bool ok = true;
            auto wait_row = [&](uint32_t q) {
                ok = ok && wait_bar(&a_full[q % kSRing], (q / kSRing) & 1, abort_flag, p.err, p.wait_ns);
            };
            for (int k = blockIdx.x; k < p.n_items; k += gridDim.x) {
                const StItem it = st_item(p, k);
                if (it.rows == 0) continue;
                wait_row(a_seq);
                wait_row(a_seq + 1);
                for (int j = 0; j < it.rows; ++j) {
                    wait_row(a_seq + j + 2);
                    const uint32_t qa = acc_seq + j, s = qa % kSAcc;
                    ok = ok && wait_bar(&acc_free[s], ((qa / kSAcc) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
                    ptx::tc_fence_after();
                    if (ok) {
                        const uint32_t dcol = tbase + 16u * s;
#pragma unroll
                        for (int ky = 0; ky < 3; ++ky) {
                            const uint64_t arow =
                                adesc0 + (uint64_t)((((a_seq + j + ky) % kSRing) * kSRow) >> 4);
#pragma unroll
                            for (int kx = 0; kx < 3; ++kx)
                                ptx::mma_bf16(dcol, arow + (uint64_t)kx, bdesc0 + (uint64_t)(((ky * 3 + kx) * 512) >> 4),
                                              idesc, (ky | kx) ? 1u : 0u);
                        }
                    }
                    ptx::mma_commit(&acc_full[s]);
                    ptx::mma_commit(&a_empty[(a_seq + j) % kSRing]);  // staged row j is done
                }
                ptx::mma_commit(&a_empty[(a_seq + it.rows) % kSRing]);
                ptx::mma_commit(&a_empty[(a_seq + it.rows + 1) % kSRing]);
                a_seq += it.rows + 2;
                acc_seq += it.rows;
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
    } else if (warp < 4) {
        // ================= layer-1 producers ========================================================
        // Staged row u of an item is layer-1 row r = y0 + m0 - 1 + u of the slice, at columns
        // c = x0 + s0 - 1 + px (px < 130), computed from input rows r - 1 .. r + 1 (reflect-101).
        // Input rows go through a ring of 4 rows of x = u/255 in shared memory (columns c - 1 .. c + 1
        // of every staged pixel: 132 values from x0 + s0 - 2); each is loaded once, one row ahead
        // (its loads are in flight while the current row is computed). The three producer warps
        // synchronise on named barrier 1. Task e = pt + 96 i: staged pixel e >> 1, channels 8 (e & 1)..+7.
        const int pt = tid - 32;
        float* xr = reinterpret_cast<float*>(smem + oSIn);
        // a thread's tasks all have channel half pt & 1 (96 is even): its 72 weights and 8 biases
        // stay in registers
        const int hf = pt & 1;
        float2 wr[9][4], br[4];  // channel pairs, for packed FP32x2 FMAs
#pragma unroll
        for (int t = 0; t < 9; ++t)
#pragma unroll
            for (int o = 0; o < 4; ++o) wr[t][o] = make_float2(cst[t * 16 + 8 * hf + 2 * o], cst[t * 16 + 8 * hf + 2 * o + 1]);
#pragma unroll
        for (int o = 0; o < 4; ++o) br[o] = make_float2(cst[kFB1 + 8 * hf + 2 * o], cst[kFB1 + 8 * hf + 2 * o + 1]);
        uint32_t a_seq = 0;
        auto bar_prod = [] { asm volatile("bar.sync 1, 96;" ::: "memory"); };
        for (int k = blockIdx.x; k < p.n_items; k += gridDim.x) {
            const StItem it = st_item(p, k);
            if (it.rows == 0) continue;
            const uint8_t* src = p.in + (int64_t)it.z * p.in_slice;
            const int c0 = p.x0 + it.s0 - 2;           // input column of ring entry 0
            const int nin = min(132, it.ncol + 4);     // input columns this strip needs
            const int rfirst = p.y0 + it.m0 - 2;       // input row feeding staged row 0's ky = 0
            // input row i (slice row rfirst + i) -> registers, as raw bytes (converted to x = u/255 when
            // put into the ring, so the loads stay in flight meanwhile): columns pt, pt + 96 of the ring
            // row; the item reads input rows 0 .. rows + 3
            auto load_in = [&](int i, uint32_t (&v)[2]) {
                const bool need = i <= it.rows + 3;
                const int row = refl(rfirst + min(i, it.rows + 3), p.h);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int j = pt + 96 * q;
                    v[q] = need && j < nin ? (uint32_t)src[(int64_t)row * p.in_pitch + refl(c0 + j, p.w)] : 0u;
                }
            };
            auto put_in = [&](int i, const uint32_t (&v)[2]) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int j = pt + 96 * q;
                    if (j < 132) xr[(i & 3) * 136 + j] = (float)v[q] / 255.0f;
                }
            };
            // input rows come from DRAM on first touch: one thread bulk-prefetches the strip of the
            // row kPf staged rows ahead into L2, so the loads issued one staged row ahead hit L2
            constexpr int kPf = 8;
            auto prefetch_in = [&](int i) {
                if (pt != 0 || i > it.rows + 3) return;
                const int row = refl(rfirst + i, p.h);
                const uint8_t* base = src + (int64_t)row * p.in_pitch;
                const uintptr_t lo = (uintptr_t)(base + max(0, c0)) & ~(uintptr_t)15;
                const uintptr_t hi = (uintptr_t)(base + min(p.w, c0 + nin)) & ~(uintptr_t)15;
                if (hi > lo) ptx::prefetch_l2_bulk((const void*)lo, (uint32_t)(hi - lo));
            };
            {
                for (int i = 3; i < 3 + kPf; ++i) prefetch_in(i);
                uint32_t v0[2], v1[2], v2[2];
                load_in(0, v0);
                load_in(1, v1);
                load_in(2, v2);
                bar_prod();  // the previous item's readers are done with the ring
                put_in(0, v0);
                put_in(1, v1);
                put_in(2, v2);
            }
            for (int u = 0; u < it.rows + 2; ++u) {
                const uint32_t q = a_seq + u, slot = q % kSRing;
                uint32_t nxt[2];
                load_in(u + 3, nxt);  // the input row of the next staged row
                prefetch_in(u + 3 + kPf);
                bar_prod();  // input rows u .. u + 2 are in the ring
                const float* x0r = xr + (u & 3) * 136;
                const float* x1r = xr + ((u + 1) & 3) * 136;
                const float* x2r = xr + ((u + 2) & 3) * 136;
                uint4 v[kSTasks];
#pragma unroll
                for (int i = 0; i < kSTasks; ++i) {
                    const int e = pt + kSProdThreads * i;
                    const int px = e >> 1;
                    v[i] = make_uint4(0, 0, 0, 0);
                    if (e < 260 && px < it.ncol + 2) {
                        float x[9];
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx) {
                            x[kx] = x0r[px + kx];
                            x[3 + kx] = x1r[px + kx];
                            x[6 + kx] = x2r[px + kx];
                        }
                        float2 a[4];
#pragma unroll
                        for (int o = 0; o < 4; ++o) a[o] = br[o];
#pragma unroll
                        for (int t = 0; t < 9; ++t) {
                            const float2 xv = make_float2(x[t], x[t]);
#pragma unroll
                            for (int o = 0; o < 4; ++o) a[o] = __ffma2_rn(wr[t][o], xv, a[o]);
                        }
                        uint32_t wd[4];
#pragma unroll
                        for (int o = 0; o < 4; ++o) {
                            __nv_bfloat162 b2 = __floats2bfloat162_rn(fmaxf(a[o].x, 0.f), fmaxf(a[o].y, 0.f));
                            wd[o] = *reinterpret_cast<uint32_t*>(&b2);
                        }
                        v[i] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                    }
                }
                // ring slot of row u + 3 held row u - 1, which every producer finished reading before
                // this row's barrier; row u + 3 becomes visible at the next row's barrier
                put_in(u + 3, nxt);
                wait_bar(&a_empty[slot], ((q / kSRing) & 1) ^ 1, abort_flag, p.err, p.wait_ns);
                uint8_t* dst = smem + oSRing + slot * kSRow;
#pragma unroll
                for (int i = 0; i < kSTasks; ++i) {
                    const int e = pt + kSProdThreads * i;
                    if (e < 260) *reinterpret_cast<uint4*>(dst + ((e & 1) * kSP + (e >> 1)) * 16) = v[i];
                }
                ptx::fence_proxy_async_smem();
                if (!p.fault_stall) ptx::mbar_arrive(&a_full[slot]);
            }
            a_seq += it.rows + 2;
        }
    } else {
        // ================= epilogue ===================================================================
        const int px = tid - 128;  // TMEM lane = pixel of the strip
        const uint32_t lanes = (uint32_t)(32 * (warp - 4)) << 16;
        uint32_t acc_seq = 0;
        for (int k = blockIdx.x; k < p.n_items; k += gridDim.x) {
            const StItem it = st_item(p, k);
            for (int j = 0; j < it.rows; ++j) {
                const uint32_t qa = acc_seq + j, s = qa % kSAcc;
                wait_bar(&acc_full[s], (qa / kSAcc) & 1, abort_flag, p.err, p.wait_ns);
                ptx::tc_fence_after();
                float d[16];
                ptx::tmem_ld16(tbase + lanes + 16u * s, d);
                ptx::tc_fence_before();
                ptx::mbar_arrive(&acc_free[s]);
                float z = cst[kSConst - 1];
#pragma unroll
                for (int c = 0; c < 16; ++c) z = fmaf(cst[176 + c], fmaxf(d[c] + cst[160 + c], 0.f), z);
                const float prob = 1.0f / (1.0f + expf(-z));
                if (px < it.ncol && !*abort_flag) {
                    const int64_t idx = (int64_t)it.z * p.out_slice + (int64_t)(it.m0 + j) * p.out_pitch + it.s0 + px;
                    if (p.out_u8)
                        static_cast<uint8_t*>(p.out)[idx] = (uint8_t)fminf(floorf(255.0f * prob + 0.5f), 255.0f);
                    else
                        static_cast<float*>(p.out)[idx] = prob;
                }
            }
            acc_seq += it.rows;
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tbase, kSTmem);
}

// B tiles (BF16) and FP32 constants from the forward-layout parameters (W1t[tap][co], b1,
// W2t[ci][tap][co], b2, wh, bh): tile tap = [ci / 8][co][ci % 8].
__global__ void st_tc_pack(const float* fwd, uint8_t* wpack) {
    __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(wpack);
    float* c = reinterpret_cast<float*>(wpack + kSB);
    for (int i = threadIdx.x; i < 9 * 16 * 16; i += blockDim.x) {
        const int tap = i / 256, co = (i / 16) % 16, ci = i % 16;
        b[tap * 256 + ((ci / 8) * 16 + co) * 8 + (ci % 8)] = __float2bfloat16_rn(fwd[kFW2 + (ci * 9 + tap) * 16 + co]);
    }
    for (int i = threadIdx.x; i < 160; i += blockDim.x) c[i] = fwd[kFW1 + i];  // W1t and b1
    for (int i = threadIdx.x; i < 33; i += blockDim.x) c[160 + i] = fwd[kFB2 + i];  // b2, wh, bh
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
    if (!S->d_wpack) MB_TRY(dev_alloc((void**)&S->d_wpack, kSB + 208 * 4));
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
    // the forward copy changes while the student trains: pack it on every call (2,497 values)
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
    p.n_strips = (int)((cols + 127) / 128);
    // rows per item: at least two items per CTA slot when the region is large, 64 at most
    const int64_t slots = (int64_t)S->n_sms * 2;
    int rpi = 64;
    while (rpi > 8 && z * p.n_strips * ((rows + rpi - 1) / rpi) < 2 * slots) rpi /= 2;
    p.rows_per_item = rpi;
    p.n_chunks = (int)((rows + rpi - 1) / rpi);
    const int64_t items = z * p.n_strips * p.n_chunks;
    if (items > 0x7fffffffLL) {
        set_error("student: too many work items for one launch");
        return MB_ERR_SHAPE;
    }
    p.n_items = (int)items;
    const char* stall = getenv("MB_FAULT_STALL");
    p.fault_stall = (stall && stall[0] == '1') ? 1 : 0;
    p.wait_ns = p.fault_stall ? 200000000ull : kSWaitNs;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, slots));
    st_tc_infer<<<grid, kSThreads, kSSmem, st>>>(p);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

}  // namespace mb
