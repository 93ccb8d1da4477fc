// fastmemb.cu - FastMemb in dense form on CUDA cores (FP32), one kernel per convolution.
//
// The network (Sec. 2.2, "A lightweight network architecture"): three [conv 4x4 -> max-out over
// 2 -> 2x2 stride-2 max-pool] stages, no transfer function, then conv 4x4 to two classes and a
// softmax. Dense computation (Sec. 2.2, "Accelerating dense computation") turns each stride-2
// pool into a stride-1 max-filter plus 2-factor sub-sampling; here that becomes a max-filter
// with dilation d and a conv with dilation 2d behind it (d = 1, 2, 4; the head has dilation 8).
//
// The paper's max-pooling fragments are also how the kernel tiles the work: a conv with
// dilation d restricted to one residue class (y mod d, x mod d) of the output is a plain 4x4
// conv on the d-strided sub-grid (one fragment), so every CTA works on one fragment tile and
// keeps the register reuse of an undilated conv (each thread's 4 pixels and 7 input columns are
// consecutive in fragment coordinates).
//
// Per CTA of 256 threads: a TH x 32 fragment tile with all CO conv channels; each thread holds 4
// consecutive fragment pixels x CPT channels. The input is staged CC channels at a time; the
// previous stage's dilated 2x2 max-filter is applied while staging. Epilogues: max-out over
// adjacent channel pairs (conv channel 2c+g -> channel c) to FP32 [slice][y][x][32], or the
// 2-class softmax p = 1 / (1 + exp(z0 - z1)).
//
// Domains for an output region rows x cols (radius 26):
//   conv1 out (rows+49)^2 .. conv2 out (rows+42) .. conv3 out (rows+28) .. head out rows
//   (each conv removes 3d, each max-filter d).
// Sub-sampled output (factor 2: the dense map at even rows and columns, the fragment tree of
// Sec. 2.2 pruned at the first pool): conv1 at full resolution on (2H2+48)^2, then a 2x2
// stride-2 max-pool (read while staging, source stride 2) and the remaining stages on the half
// grid with dilations 1, 2, 4: conv2 out H2+21, conv3 out H2+14, head out H2 = ceil(rows/2).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace mb {

namespace {

enum { FM_IN_U8 = 0, FM_IN_F32 = 1 };
enum { FM_OUT_MAXOUT = 0, FM_OUT_SOFTMAX_F32 = 1, FM_OUT_SOFTMAX_U8 = 2, FM_OUT_MAXOUT_BF16 = 3 };

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
template <int CIN, int CC, int CO, int CPT, int IN, int OUT>
__global__ void __launch_bounds__(256) fm_conv(const FmArgs a) {
    constexpr int K = 4;
    constexpr int NCG = CO / CPT;
    constexpr int TW = 32;
    constexpr int TH = 256 / (8 * NCG);
    constexpr int IH = TH + K - 1;
    constexpr int IW = TW + K - 1;
    constexpr int IWP = 36;
    static_assert(CO % CPT == 0 && (CPT == 8 || CPT == 2), "channel split");
    static_assert(CIN % CC == 0 && (CC == 1 || CC == 8), "channel chunking");
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
        for (int e = t; e < IH * IWP; e += 256) {
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
                    v1 = ld4(p + 4);
                    if (a.dm > 0) {
                        const float* q = p + (int64_t)a.dm * CIN;
                        const float* s = p + (int64_t)a.dm * a.in_pitch * CIN;
                        const float* u = s + (int64_t)a.dm * CIN;
                        v0 = max4(max4(v0, ld4(q)), max4(ld4(s), ld4(u)));
                        v1 = max4(max4(v1, ld4(q + 4)), max4(ld4(s + 4), ld4(u + 4)));
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
            for (int e = t; e < CC * K * K * CO / 4; e += 256) dst[e] = __ldg(src + e);
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
                    if constexpr (CPT == 8) {
                        const float4 w0 = *reinterpret_cast<const float4*>(wr + kx * CO);
                        const float4 w1 = *reinterpret_cast<const float4*>(wr + kx * CO + 4);
                        wv[0] = w0.x; wv[1] = w0.y; wv[2] = w0.z; wv[3] = w0.w;
                        wv[4] = w1.x; wv[5] = w1.y; wv[6] = w1.z; wv[7] = w1.w;
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
    if constexpr (OUT == FM_OUT_MAXOUT_BF16) {
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(a.out) + (int64_t)zi * a.out_slice;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ox = rx + d * (fx0 + 4 * tx + j);
            if (ox < a.out_w) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(fmaxf(acc[j][0], acc[j][1]), fmaxf(acc[j][2], acc[j][3]));
                __nv_bfloat162 hi = __floats2bfloat162_rn(fmaxf(acc[j][4], acc[j][5]), fmaxf(acc[j][6], acc[j][7]));
                uint2 u;
                u.x = *reinterpret_cast<uint32_t*>(&lo);
                u.y = *reinterpret_cast<uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(o + ((int64_t)oy * a.out_pitch + ox) * (CO / 2) + 4 * cg) = u;
            }
        }
    } else if constexpr (OUT == FM_OUT_MAXOUT) {
        static_assert(CPT == 8, "max-out epilogue writes 4 channels per thread");
        float* o = static_cast<float*>(a.out) + (int64_t)zi * a.out_slice;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ox = rx + d * (fx0 + 4 * tx + j);
            if (ox < a.out_w) {
                const float4 m = make_float4(fmaxf(acc[j][0], acc[j][1]), fmaxf(acc[j][2], acc[j][3]),
                                             fmaxf(acc[j][4], acc[j][5]), fmaxf(acc[j][6], acc[j][7]));
                *reinterpret_cast<float4*>(o + ((int64_t)oy * a.out_pitch + ox) * (CO / 2) + 4 * cg) = m;
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

template <int CIN, int CC, int CO, int CPT, int IN, int OUT>
mb_status launch_fm(FmArgs a, int nz, cudaStream_t st) {
    constexpr int TH = 256 / (8 * (CO / CPT));
    const int fh = (a.out_h + a.d - 1) / a.d, fw = (a.out_w + a.d - 1) / a.d;  // largest fragment
    a.fy_tiles = (fh + TH - 1) / TH;
    a.fx_tiles = (fw + 31) / 32;
    const int64_t nblk = (int64_t)a.d * a.d * a.fy_tiles * a.fx_tiles;
    if (nblk > 0x7fffffffLL) {
        set_error("FastMemb: region too large for one launch");
        return MB_ERR_SHAPE;
    }
    dim3 grid((unsigned)nblk, (unsigned)nz);
    fm_conv<CIN, CC, CO, CPT, IN, OUT><<<grid, 256, 0, st>>>(a);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

}  // namespace

// Per-stage geometry of one FastMemb pass with NC convolutions (4 for FastMemb, 5 for
// FastMemb_3nm): extents of the conv outputs (conv1 at full resolution; the rest at full resolution
// for the dense map, on the half grid when sub-sampled), the dilation of each conv, and how each
// conv reads its input (max-filter dilation dm, stride st). Walking back from the map, conv k's
// input needs 3 d_k + dm_k more rows than its output.
constexpr int kFmMaxConvs = 5;
struct FmGeom {
    int nc;
    int64_t r[kFmMaxConvs], c[kFmMaxConvs];
    int d[kFmMaxConvs], dm[kFmMaxConvs], st[kFmMaxConvs];
};

static FmGeom fm_geom(int nc, int64_t rows, int64_t cols, int sub) {
    FmGeom g{};
    g.nc = nc;
    for (int k = 0; k < nc; ++k) {
        g.st[k] = 1;
        if (sub == 2) {
            g.d[k] = k == 0 ? 1 : 1 << (k - 1);
            g.dm[k] = k == 0 ? 0 : (k == 1 ? 1 : g.d[k - 1]);
            if (k == 1) g.st[k] = 2;
        } else {
            g.d[k] = 1 << k;
            g.dm[k] = k == 0 ? 0 : g.d[k - 1];
        }
    }
    g.r[nc - 1] = sub == 2 ? (rows + 1) / 2 : rows;
    g.c[nc - 1] = sub == 2 ? (cols + 1) / 2 : cols;
    for (int k = nc - 1; k >= 1; --k) {
        const int64_t in_r = g.r[k] + 3 * g.d[k], in_c = g.c[k] + 3 * g.d[k];  // conv k's input domain
        g.r[k - 1] = (in_r - 1) * g.st[k] + g.dm[k] + 1;
        g.c[k - 1] = (in_c - 1) * g.st[k] + g.dm[k] + 1;
    }
    if (sub == 2) {  // conv1 covers whole 2x2 pooling windows
        g.r[0] += g.r[0] & 1;
        g.c[0] += g.c[0] & 1;
    }
    return g;
}

// Input domain of conv i >= 1: the (max-filtered, strided) view of conv i-1's output: positions r
// with st r + dm inside the source.
static inline int64_t fm_in_extent(const FmGeom& g, int i, bool rows) {
    const int64_t src = rows ? g.r[i - 1] : g.c[i - 1];
    return (src - 1 - g.dm[i]) / g.st[i] + 1;
}

// Offsets of the SIMT-layout weights of conv k (Wt[ci][ky][kx][co] then b[co]; co = 64 except the
// head's 2; ci = 1 for conv1 and 32 after).
static const float* fm_simt_w(const mb_net* net, int k, int nc, const float** bias) {
    size_t off = 0;
    for (int i = 0; i < k; ++i) off += i == 0 ? 16 * 64 + 64 : 32 * 16 * 64 + 64;
    const float* w = net->d_simt + off;
    const int co = k == nc - 1 ? 2 : 64, ci = k == 0 ? 1 : 32;
    *bias = w + (size_t)ci * 16 * co;
    return w;
}

mb_status simt_fastmemb_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                               int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                               int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st, int sub) {
    if (z == 0 || rows == 0 || cols == 0) return MB_OK;
    const int nc = fastmemb_convs(net->family);
    const int R = nc == 5 ? kFastMemb3nmRadius : kFastMembRadius;
    const FmGeom g = fm_geom(nc, rows, cols, sub);
    size_t per = 0;
    for (int k = 0; k < nc - 1; ++k) per += (size_t)(g.r[k] * g.c[k]) * 32 * sizeof(float);
    const size_t budget = (size_t)3 << 30;
    const int64_t zc = std::min<int64_t>(std::min<int64_t>(std::max<size_t>(1, budget / per), 65535), z);
    MB_TRY(net->ws.ensure(per * (size_t)zc));
    float* act[kFmMaxConvs - 1];
    act[0] = static_cast<float*>(net->ws.ptr);
    for (int k = 1; k < nc - 1; ++k) act[k] = act[k - 1] + (size_t)zc * g.r[k - 1] * g.c[k - 1] * 32;
    for (int64_t z0 = 0; z0 < z; z0 += zc) {
        const int nz = (int)std::min<int64_t>(zc, z - z0);
        FmArgs a{};
        a.in = in + z0 * in_slice;
        a.in_slice = in_slice;
        a.in_pitch = in_pitch;
        a.in_rows = (int)(g.r[0] + 3);
        a.in_cols = (int)(g.c[0] + 3);
        a.src_h = (int)h;
        a.src_w = (int)w;
        a.off_y = (int)(y0 - R);
        a.off_x = (int)(x0 - R);
        a.d = 1;
        a.out_h = (int)g.r[0];
        a.out_w = (int)g.c[0];
        a.out = act[0];
        a.out_slice = g.r[0] * g.c[0] * 32;
        a.out_pitch = g.c[0];
        a.wt = fm_simt_w(net, 0, nc, &a.bias);
        MB_TRY((launch_fm<1, 1, 64, 8, FM_IN_U8, FM_OUT_MAXOUT>(a, nz, st)));
        for (int k = 1; k < nc; ++k) {
            FmArgs b{};
            b.in = act[k - 1];
            b.in_slice = g.r[k - 1] * g.c[k - 1] * 32;
            b.in_pitch = g.c[k - 1];
            b.in_rows = (int)fm_in_extent(g, k, true);
            b.in_cols = (int)fm_in_extent(g, k, false);
            b.d = g.d[k];
            b.dm = g.dm[k];
            b.in_stride = g.st[k];
            b.out_h = (int)g.r[k];
            b.out_w = (int)g.c[k];
            b.wt = fm_simt_w(net, k, nc, &b.bias);
            if (k < nc - 1) {
                b.out = act[k];
                b.out_slice = g.r[k] * g.c[k] * 32;
                b.out_pitch = g.c[k];
                MB_TRY((launch_fm<32, 8, 64, 8, FM_IN_F32, FM_OUT_MAXOUT>(b, nz, st)));
            } else {
                b.out_slice = out_slice;
                b.out_pitch = out_pitch;
                if (ot == MB_OUT_F32) {
                    b.out = static_cast<float*>(out) + z0 * out_slice;
                    MB_TRY((launch_fm<32, 8, 2, 2, FM_IN_F32, FM_OUT_SOFTMAX_F32>(b, nz, st)));
                } else {
                    b.out = static_cast<uint8_t*>(out) + z0 * out_slice;
                    MB_TRY((launch_fm<32, 8, 2, 2, FM_IN_F32, FM_OUT_SOFTMAX_U8>(b, nz, st)));
                }
            }
        }
    }
    return MB_OK;
}

// BF16 path: layer 1 on CUDA cores (FP32 arithmetic, BF16 out); the two 32->64 dilated convs and
// the head on the tensor cores (fastmemb_tc.cu); activations between layers are BF16 [slice][y][x][32].
mb_status bf16_fastmemb_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                               int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                               int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st, int sub) {
    if (z == 0 || rows == 0 || cols == 0) return MB_OK;
    MB_TRY(fm_tc_poll_error(net));
    const int nc = fastmemb_convs(net->family);
    const int R = nc == 5 ? kFastMemb3nmRadius : kFastMembRadius;
    const FmGeom g = fm_geom(nc, rows, cols, sub);
    auto up = [](int64_t n) { return (n + 127) & ~(int64_t)127; };  // 256-byte aligned sub-buffers
    int64_t n[kFmMaxConvs - 1];
    size_t per = 0;
    for (int k = 0; k < nc - 1; ++k) {
        n[k] = up(g.r[k] * g.c[k] * 32);
        per += (size_t)n[k] * 2;
    }
    const size_t budget = (size_t)3 << 30;
    const int64_t zc = std::min<int64_t>(std::min<int64_t>(std::max<size_t>(1, budget / per), 65535), z);
    MB_TRY(net->ws.ensure(per * (size_t)zc));
    __nv_bfloat16* act[kFmMaxConvs - 1];
    act[0] = static_cast<__nv_bfloat16*>(net->ws.ptr);
    for (int k = 1; k < nc - 1; ++k) act[k] = act[k - 1] + (size_t)zc * n[k - 1];
    const size_t osz = ot == MB_OUT_F32 ? 4 : 1;
    for (int64_t z0 = 0; z0 < z; z0 += zc) {
        const int nz = (int)std::min<int64_t>(zc, z - z0);
        FmArgs a{};
        a.in = in + z0 * in_slice;
        a.in_slice = in_slice;
        a.in_pitch = in_pitch;
        a.in_rows = (int)(g.r[0] + 3);
        a.in_cols = (int)(g.c[0] + 3);
        a.src_h = (int)h;
        a.src_w = (int)w;
        a.off_y = (int)(y0 - R);
        a.off_x = (int)(x0 - R);
        a.d = 1;
        a.out_h = (int)g.r[0];
        a.out_w = (int)g.c[0];
        a.out = act[0];
        a.out_slice = n[0];
        a.out_pitch = g.c[0];
        a.wt = fm_simt_w(net, 0, nc, &a.bias);
        MB_TRY((launch_fm<1, 1, 64, 8, FM_IN_U8, FM_OUT_MAXOUT_BF16>(a, nz, st)));
        for (int k = 1; k < nc; ++k) {
            const bool head = k == nc - 1;
            void* o = head ? static_cast<void*>(static_cast<uint8_t*>(out) + z0 * out_slice * osz) : act[k];
            MB_TRY(fm_tc_layer(net, k - 1, act[k - 1], n[k - 1], g.c[k - 1], g.r[k - 1], g.c[k - 1],
                               (int)fm_in_extent(g, k, true), (int)fm_in_extent(g, k, false), g.dm[k], g.st[k], o,
                               head ? out_slice : n[k], head ? out_pitch : g.c[k], (int)g.r[k], (int)g.c[k], g.d[k],
                               nz, head && ot == MB_OUT_U8, st));
        }
    }
    return fm_tc_poll_error(net);
}

}  // namespace mb
