// fm_conv.cuh - the FP32 CUDA-core convolution kernel of the max-out networks (FastMemb,
// FastMemb_3nm, MaskExtend; Sec. 2.2 and Sec. 3.2), shared by fastmemb.cu and maskextend.cu.
//
// A conv with dilation d restricted to one residue class (y mod d, x mod d) of its output is a
// plain 4x4 conv on the d-strided sub-grid (a max-pooling fragment), so each CTA computes a
// TH x 32 tile of one fragment: 4 consecutive fragment pixels x CPT conv channels per thread,
// input channels staged CC at a time with the previous stage's dilated 2x2 max-filter (and an
// optional source stride) applied while staging. Epilogues: max-out of adjacent channel pairs
// (FP32, BF16 or FP16 out), or the 2-class softmax.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mb {

namespace {

enum { FM_IN_U8 = 0, FM_IN_F32 = 1 };
enum { FM_OUT_MAXOUT = 0, FM_OUT_SOFTMAX_F32 = 1, FM_OUT_SOFTMAX_U8 = 2, FM_OUT_MAXOUT_BF16 = 3, FM_OUT_MAXOUT_F16 = 4 };

struct FmArgs {
    const void* in;
    int64_t in_slice;      // u8: bytes per slice; f32: floats per slice
    int64_t in_pitch;      // u8: bytes per row; f32: pixels per row
    int in_rows, in_cols;  // extent of this conv's (max-filtered) input domain
    int src_h, src_w;      // u8: slice size for reflect-101
    int off_y, off_x;      // u8: input (r, c) reads slice (refl(r + off_y), refl(c + off_x))
    int d;                 // conv dilation = fragment step
    int dm;                // dilation of the 2x2 max-filter applied to the staged input (0: none)
    int in_stride;         // f32: input (r, c) is the max-filter at source (s r, s c); 0 or 1: s = 1
    int out_h, out_w;
    int fy_tiles, fx_tiles;  // tiles per fragment along y / x
    void* out;
    int64_t out_slice, out_pitch;  // elements
    const float* wt;               // [CIN][4][4][CO]
    const float* bias;             // [CO]
};

__device__ __forceinline__ int refl101(int t, int n) {
    t = t < 0 ? -t : t;
    return t >= n ? 2 * (n - 1) - t : t;
}

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 max4(float4 a, float4 b) {
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}
// TH output rows per CTA: NT = 8 x (CO / CPT) x TH threads (at most 256).
template <int CIN, int CC, int CO, int CPT, int IN, int OUT, int TH = 256 / (8 * (CO / CPT))>
__global__ void __launch_bounds__(256) fm_conv(const FmArgs a) {
    constexpr int K = 4;
    constexpr int NCG = CO / CPT;
    constexpr int NT = 8 * NCG * TH;
    constexpr int TW = 32;
    constexpr int IH = TH + K - 1;
    constexpr int IW = TW + K - 1;
    constexpr int IWP = 36;
    static_assert(CO % CPT == 0 && (CPT == 16 || CPT == 8 || CPT == 2), "channel split");
    static_assert(CIN % CC == 0 && (CC == 1 || CC == 4 || CC == 8), "channel chunking");
    static_assert(NT <= 256 && TH >= 1, "block size");
    __shared__ __align__(16) float s_in[CC * IH * IWP];
    __shared__ __align__(16) float s_w[CC * K * K * CO];

    const int t = threadIdx.x;
    const int tx = t & 7, cg = (t >> 3) % NCG, ty = (t >> 3) / NCG;
    const int d = a.d;
    // blockIdx.x = ((ry * d + rx) * fy_tiles + fy_tile) * fx_tiles + fx_tile
    int b = blockIdx.x;
    const int fxt = b % a.fx_tiles;
    b /= a.fx_tiles;
    const int fyt = b % a.fy_tiles;
    b /= a.fy_tiles;
    const int rx = b % d, ry = b / d;
    const int fx0 = fxt * TW, fy0 = fyt * TH;
    const int zi = blockIdx.y;

    float acc[4][CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const float bv = a.bias[cg * CPT + c];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j][c] = bv;
    }

    for (int c0 = 0; c0 < CIN; c0 += CC) {
        __syncthreads();
        for (int e = t; e < IH * IWP; e += NT) {
            const int r = e / IWP, c = e - (e / IWP) * IWP;
            const int gy = ry + d * (fy0 + r), gx = rx + d * (fx0 + c);
            const bool ok = c < IW && gy < a.in_rows && gx < a.in_cols;
            if constexpr (IN == FM_IN_U8) {
                float v = 0.f;
                if (ok) {
                    const uint8_t* src = static_cast<const uint8_t*>(a.in) + (int64_t)zi * a.in_slice;
                    const int sy = refl101(gy + a.off_y, a.src_h), sx = refl101(gx + a.off_x, a.src_w);
                    v = (float)src[(int64_t)sy * a.in_pitch + sx] / 255.0f;
                }
                s_in[r * IWP + c] = v;
            } else {
                float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
                if (ok) {
                    const int st = a.in_stride > 1 ? a.in_stride : 1;
                    const float* p = static_cast<const float*>(a.in) + (int64_t)zi * a.in_slice +
                                     ((int64_t)(st * gy) * a.in_pitch + st * gx) * CIN + c0;
                    v0 = ld4(p);
                    if constexpr (CC == 8) v1 = ld4(p + 4);
                    if (a.dm > 0) {
                        const float* q = p + (int64_t)a.dm * CIN;
                        const float* s = p + (int64_t)a.dm * a.in_pitch * CIN;
                        const float* u = s + (int64_t)a.dm * CIN;
                        v0 = max4(max4(v0, ld4(q)), max4(ld4(s), ld4(u)));
                        if constexpr (CC == 8) v1 = max4(max4(v1, ld4(q + 4)), max4(ld4(s + 4), ld4(u + 4)));
                    }
                }
                const float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                for (int cc = 0; cc < CC; ++cc) s_in[(cc * IH + r) * IWP + c] = vv[cc];
            }
        }
        {
            const float4* src = reinterpret_cast<const float4*>(a.wt + (int64_t)c0 * K * K * CO);
            float4* dst = reinterpret_cast<float4*>(s_w);
            for (int e = t; e < CC * K * K * CO / 4; e += NT) dst[e] = __ldg(src + e);
        }
        __syncthreads();
#pragma unroll 1
        for (int cc = 0; cc < CC; ++cc) {
#pragma unroll
            for (int ky = 0; ky < K; ++ky) {
                const float* row = s_in + (cc * IH + ty + ky) * IWP + 4 * tx;
                const float4 p0 = *reinterpret_cast<const float4*>(row);
                const float4 p1 = *reinterpret_cast<const float4*>(row + 4);
                const float v[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
                const float* wr = s_w + ((cc * K + ky) * K) * CO + CPT * cg;
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    float wv[CPT];
                    if constexpr (CPT >= 8) {
#pragma unroll
                        for (int q = 0; q < CPT / 4; ++q) {
                            const float4 w4 = *reinterpret_cast<const float4*>(wr + kx * CO + 4 * q);
                            wv[4 * q] = w4.x; wv[4 * q + 1] = w4.y; wv[4 * q + 2] = w4.z; wv[4 * q + 3] = w4.w;
                        }
                    } else {
                        const float2 w0 = *reinterpret_cast<const float2*>(wr + kx * CO);
                        wv[0] = w0.x; wv[1] = w0.y;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int c = 0; c < CPT; ++c) acc[j][c] = fmaf(v[j + kx], wv[c], acc[j][c]);
                }
            }
        }
    }

    const int oy = ry + d * (fy0 + ty);
    if (oy >= a.out_h) return;
    if constexpr (OUT == FM_OUT_MAXOUT_BF16 || OUT == FM_OUT_MAXOUT_F16) {
        // 16-bit activations (BF16 or FP16), the tensor-core layers' input
        static_assert(CPT >= 8, "max-out epilogue writes 4 channels per 8 conv channels");
        uint16_t* o = static_cast<uint16_t*>(a.out) + (int64_t)zi * a.out_slice;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ox = rx + d * (fx0 + 4 * tx + j);
            if (ox < a.out_w) {
#pragma unroll
                for (int q = 0; q < CPT / 8; ++q) {
                    const float* v = acc[j] + 8 * q;
                    const float2 l = make_float2(fmaxf(v[0], v[1]), fmaxf(v[2], v[3]));
                    const float2 h = make_float2(fmaxf(v[4], v[5]), fmaxf(v[6], v[7]));
                    uint2 u;
                    if constexpr (OUT == FM_OUT_MAXOUT_F16) {
                        __half2 lo = __floats2half2_rn(l.x, l.y), hi = __floats2half2_rn(h.x, h.y);
                        u.x = *reinterpret_cast<uint32_t*>(&lo);
                        u.y = *reinterpret_cast<uint32_t*>(&hi);
                    } else {
                        __nv_bfloat162 lo = __floats2bfloat162_rn(l.x, l.y), hi = __floats2bfloat162_rn(h.x, h.y);
                        u.x = *reinterpret_cast<uint32_t*>(&lo);
                        u.y = *reinterpret_cast<uint32_t*>(&hi);
                    }
                    *reinterpret_cast<uint2*>(o + ((int64_t)oy * a.out_pitch + ox) * (CO / 2) + (CPT / 2) * cg + 4 * q) =
                        u;
                }
            }
        }
    } else if constexpr (OUT == FM_OUT_MAXOUT) {
        static_assert(CPT >= 8, "max-out epilogue writes 4 channels per 8 conv channels");
        float* o = static_cast<float*>(a.out) + (int64_t)zi * a.out_slice;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ox = rx + d * (fx0 + 4 * tx + j);
            if (ox < a.out_w) {
#pragma unroll
                for (int q = 0; q < CPT / 8; ++q) {
                    const float* v = acc[j] + 8 * q;
                    const float4 m = make_float4(fmaxf(v[0], v[1]), fmaxf(v[2], v[3]), fmaxf(v[4], v[5]), fmaxf(v[6], v[7]));
                    *reinterpret_cast<float4*>(o + ((int64_t)oy * a.out_pitch + ox) * (CO / 2) + (CPT / 2) * cg + 4 * q) = m;
                }
            }
        }
    } else {
        static_assert(CPT == 2 && CO == 2, "softmax epilogue: two classes per thread");
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ox = rx + d * (fx0 + 4 * tx + j);
            if (ox < a.out_w) {
                const float p = 1.0f / (1.0f + expf(acc[j][0] - acc[j][1]));
                const int64_t idx = (int64_t)zi * a.out_slice + (int64_t)oy * a.out_pitch + ox;
                if constexpr (OUT == FM_OUT_SOFTMAX_F32) {
                    static_cast<float*>(a.out)[idx] = p;
                } else {
                    const float q = floorf(255.0f * p + 0.5f);
                    static_cast<uint8_t*>(a.out)[idx] = (uint8_t)fminf(q, 255.0f);
                }
            }
        }
    }
}

template <int CIN, int CC, int CO, int CPT, int IN, int OUT, int TH = 256 / (8 * (CO / CPT))>
mb_status launch_fm(FmArgs a, int nz, cudaStream_t st) {
    constexpr int NT = 8 * (CO / CPT) * TH;
    const int fh = (a.out_h + a.d - 1) / a.d, fw = (a.out_w + a.d - 1) / a.d;  // largest fragment
    a.fy_tiles = (fh + TH - 1) / TH;
    a.fx_tiles = (fw + 31) / 32;
    const int64_t nblk = (int64_t)a.d * a.d * a.fy_tiles * a.fx_tiles;
    if (nblk > 0x7fffffffLL) {
        set_error("FastMemb: region too large for one launch");
        return MB_ERR_SHAPE;
    }
    dim3 grid((unsigned)nblk, (unsigned)nz);
    fm_conv<CIN, CC, CO, CPT, IN, OUT, TH><<<grid, NT, 0, st>>>(a);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

}  // namespace

}  // namespace mb
