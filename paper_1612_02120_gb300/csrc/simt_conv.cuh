// simt_conv.cuh - the register-tiled direct-convolution kernel of the FP32 CUDA-core path, shared
// by the layered inference path (simt_conv.cu) and the student's training kernels (student.cu).
//
// One CTA of 256 threads computes a TH x 32 output tile with all COUT channels of a valid
// cross-correlation (K x K, CIN -> COUT) plus bias; each thread holds 4 consecutive pixels x 8
// channels in registers and input channels are staged CC at a time in shared memory.
// Input modes:  IN_U8        uint8 slice, mirror-padded (reflect-101) at an offset, scaled by 1/255
//               IN_F32       [slice][y][x][CIN] FP32 activations
//               IN_F32_MAXF  the same, 2x2 stride-1 max-filtered while staging
//               IN_F32_PAD   the same at an offset, zero outside the source extent
// Output modes: OUT_ACT      ReLU, [slice][y][x][COUT]
//               OUT_HEAD_*   ReLU, then the 1x1 head + sigmoid -> FP32 map or uint8 (round(255 p))
//               OUT_GRADMASK no ReLU; multiplied by (mask > 0) elementwise, [slice][y][x][COUT]
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mb {

enum { IN_U8 = 0, IN_F32 = 1, IN_F32_MAXF = 2, IN_F32_PAD = 3 };
enum { OUT_ACT = 0, OUT_HEAD_F32 = 1, OUT_HEAD_U8 = 2, OUT_GRADMASK = 3 };

struct ConvArgs {
    const void* in;
    int64_t in_slice;  // u8: bytes per slice; f32: floats per slice
    int64_t in_pitch;  // u8: bytes per row; f32: pixels per row
    int in_rows, in_cols;  // extent of the (virtual) input domain this layer reads
    int src_h, src_w;      // u8: slice size (reflect-101 range); f32 pad: source extent
    int off_y, off_x;      // input (r, c) reads source (r + off_y, c + off_x) (u8: reflected)
    int out_h, out_w;
    void* out;
    int64_t out_slice, out_pitch;  // elements
    const float* wt;      // [CIN][K][K][COUT]
    const float* bias;    // [COUT]
    const float* head_w;  // [COUT] followed by the head bias
    const int* zmap;      // u8 input: slice index map (NULL: identity)
    const float* mask;    // OUT_GRADMASK: [slice][y][x][COUT], same layout as out
};

__device__ __forceinline__ int refl101(int t, int n) {
    t = t < 0 ? -t : t;
    return t >= n ? 2 * (n - 1) - t : t;
}

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 max4(float4 a, float4 b) {
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}

// One CTA of 256 threads computes a TH x 32 output tile with all COUT channels; each thread holds
// 4 consecutive pixels x 8 channels in registers. Input channels are staged CC at a time.
template <int K, int CIN, int COUT, int CC, int IN, int OUT>
__global__ void __launch_bounds__(256) conv_simt(const ConvArgs a) {
    constexpr int NCG = COUT / 8;
    constexpr int TW = 32;
    constexpr int TH = 256 / (8 * NCG);
    constexpr int IH = TH + K - 1;
    constexpr int IW = TW + K - 1;
    constexpr int IWP = 36;  // reads reach 4*7 + 7 = 35
    static_assert(IW <= IWP, "tile too wide");
    static_assert(CIN % CC == 0, "channel chunking");
    __shared__ __align__(16) float s_in[CC * IH * IWP];
    __shared__ __align__(16) float s_w[CC * K * K * COUT];

    const int t = threadIdx.x;
    const int tx = t & 7, cg = (t >> 3) % NCG, ty = (t >> 3) / NCG;
    const int ox0 = blockIdx.x * TW, oy0 = blockIdx.y * TH;
    const int zi = blockIdx.z;

    float acc[4][8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float b = a.bias[cg * 8 + c];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j][c] = b;
    }

    for (int c0 = 0; c0 < CIN; c0 += CC) {
        __syncthreads();
        for (int e = t; e < IH * IWP; e += 256) {
            const int r = e / IWP, c = e - (e / IWP) * IWP;
            const int gy = oy0 + r, gx = ox0 + c;
            const bool ok = c < IW && gy < a.in_rows && gx < a.in_cols;
            if (IN == IN_U8) {
                float v = 0.f;
                if (ok) {
                    const int zs = a.zmap ? a.zmap[zi] : zi;
                    const uint8_t* src = static_cast<const uint8_t*>(a.in) + (int64_t)zs * a.in_slice;
                    int sy = refl101(gy + a.off_y, a.src_h), sx = refl101(gx + a.off_x, a.src_w);
                    v = (float)src[(int64_t)sy * a.in_pitch + sx] / 255.0f;
                }
                s_in[r * IWP + c] = v;
            } else if (IN == IN_F32_PAD) {
                float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
                const int sy = gy + a.off_y, sx = gx + a.off_x;
                if (ok && sy >= 0 && sy < a.src_h && sx >= 0 && sx < a.src_w) {
                    const float* q = static_cast<const float*>(a.in) + (int64_t)zi * a.in_slice +
                                     ((int64_t)sy * a.in_pitch + sx) * CIN + c0;
                    v0 = ldg4(q);
                    v1 = ldg4(q + 4);
                }
                float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                for (int cc = 0; cc < CC; ++cc) s_in[(cc * IH + r) * IWP + c] = vv[cc];
            } else {
                float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
                if (ok) {
                    const float* p = static_cast<const float*>(a.in) + (int64_t)zi * a.in_slice +
                                     ((int64_t)gy * a.in_pitch + gx) * CIN + c0;
                    v0 = ldg4(p);
                    v1 = ldg4(p + 4);
                    if (IN == IN_F32_MAXF) {
                        const float* q = p + CIN;
                        const float* s = p + a.in_pitch * CIN;
                        const float* u = s + CIN;
                        v0 = max4(max4(v0, ldg4(q)), max4(ldg4(s), ldg4(u)));
                        v1 = max4(max4(v1, ldg4(q + 4)), max4(ldg4(s + 4), ldg4(u + 4)));
                    }
                }
                float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                for (int cc = 0; cc < CC; ++cc) s_in[(cc * IH + r) * IWP + c] = vv[cc];
            }
        }
        {
            const float4* src = reinterpret_cast<const float4*>(a.wt + (int64_t)c0 * K * K * COUT);
            float4* dst = reinterpret_cast<float4*>(s_w);
            for (int e = t; e < CC * K * K * COUT / 4; e += 256) dst[e] = __ldg(src + e);
        }
        __syncthreads();
#pragma unroll 1
        for (int cc = 0; cc < CC; ++cc) {
#pragma unroll
            for (int ky = 0; ky < K; ++ky) {
                const float* row = s_in + (cc * IH + ty + ky) * IWP + 4 * tx;
                float4 p0 = *reinterpret_cast<const float4*>(row);
                float4 p1 = *reinterpret_cast<const float4*>(row + 4);
                float v[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
                const float* wr = s_w + ((cc * K + ky) * K) * COUT + 8 * cg;
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    float4 w0 = *reinterpret_cast<const float4*>(wr + kx * COUT);
                    float4 w1 = *reinterpret_cast<const float4*>(wr + kx * COUT + 4);
                    float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int c = 0; c < 8; ++c) acc[j][c] = fmaf(v[j + kx], wv[c], acc[j][c]);
                }
            }
        }
    }

    const int oy = oy0 + ty;
    if (OUT == OUT_GRADMASK) {
        if (oy < a.out_h) {
            float* o = static_cast<float*>(a.out) + (int64_t)zi * a.out_slice;
            const float* mk = a.mask + (int64_t)zi * a.out_slice;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ox = ox0 + 4 * tx + j;
                if (ox < a.out_w) {
                    const int64_t off = ((int64_t)oy * a.out_pitch + ox) * COUT + 8 * cg;
                    const float4 m0 = *reinterpret_cast<const float4*>(mk + off);
                    const float4 m1 = *reinterpret_cast<const float4*>(mk + off + 4);
                    float* d = o + off;
                    *reinterpret_cast<float4*>(d) = make_float4(m0.x > 0.f ? acc[j][0] : 0.f, m0.y > 0.f ? acc[j][1] : 0.f,
                                                                m0.z > 0.f ? acc[j][2] : 0.f, m0.w > 0.f ? acc[j][3] : 0.f);
                    *reinterpret_cast<float4*>(d + 4) = make_float4(m1.x > 0.f ? acc[j][4] : 0.f, m1.y > 0.f ? acc[j][5] : 0.f,
                                                                    m1.z > 0.f ? acc[j][6] : 0.f, m1.w > 0.f ? acc[j][7] : 0.f);
                }
            }
        }
    } else if (OUT == OUT_ACT) {
        if (oy < a.out_h) {
            float* o = static_cast<float*>(a.out) + (int64_t)zi * a.out_slice;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ox = ox0 + 4 * tx + j;
                if (ox < a.out_w) {
                    float* d = o + ((int64_t)oy * a.out_pitch + ox) * COUT + 8 * cg;
                    *reinterpret_cast<float4*>(d) = make_float4(fmaxf(acc[j][0], 0.f), fmaxf(acc[j][1], 0.f),
                                                                fmaxf(acc[j][2], 0.f), fmaxf(acc[j][3], 0.f));
                    *reinterpret_cast<float4*>(d + 4) = make_float4(fmaxf(acc[j][4], 0.f), fmaxf(acc[j][5], 0.f),
                                                                    fmaxf(acc[j][6], 0.f), fmaxf(acc[j][7], 0.f));
                }
            }
        }
    } else {
        float hw[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) hw[c] = a.head_w[cg * 8 + c];
        const float hb = a.head_w[COUT];
        float s[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) v = fmaf(fmaxf(acc[j][c], 0.f), hw[c], v);
#pragma unroll
            for (int m = 8; m < 8 * NCG; m <<= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
            s[j] = v;
        }
        if (cg == 0 && oy < a.out_h) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ox = ox0 + 4 * tx + j;
                if (ox < a.out_w) {
                    float p = 1.0f / (1.0f + expf(-(s[j] + hb)));
                    int64_t idx = (int64_t)zi * a.out_slice + (int64_t)oy * a.out_pitch + ox;
                    if (OUT == OUT_HEAD_F32) {
                        static_cast<float*>(a.out)[idx] = p;
                    } else {
                        float q = floorf(255.0f * p + 0.5f);
                        static_cast<uint8_t*>(a.out)[idx] = (uint8_t)fminf(q, 255.0f);
                    }
                }
            }
        }
    }
}

template <int K, int CIN, int COUT, int CC, int IN, int OUT>
inline mb_status launch_conv(const ConvArgs& a, int nz, cudaStream_t st) {
    constexpr int TH = 256 / COUT;
    dim3 grid((a.out_w + 31) / 32, (a.out_h + TH - 1) / TH, nz);
    conv_simt<K, CIN, COUT, CC, IN, OUT><<<grid, 256, 0, st>>>(a);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

}  // namespace mb
