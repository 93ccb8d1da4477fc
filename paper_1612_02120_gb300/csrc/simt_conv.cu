// simt_conv.cu - FP32 CUDA-core path: one register-tiled direct-convolution kernel per layer,
// activations kept in a device workspace between layers.
//
// Operation (Sec. 2.2): valid cross-correlation + bias + ReLU; the 2x2 stride-1 max-filter that
// replaces max-pooling for dense computation is applied while the next layer stages its input;
// the 1x1 head + sigmoid is fused into the last convolution. The first layer reads the uint8
// slice directly, mirror-padding it (reflect-101) and scaling by 1/255.
//
// Domains for an output region of rows x cols (teacher, radius 7):
//   layer-1 output (rows+10) x (cols+10) x 32, layer-2 output (rows+5) x (cols+5) x 32,
//   layer-3 + head output rows x cols. Activation buffers are [slice][y][x][c] FP32.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace mb {

enum { IN_U8 = 0, IN_F32 = 1, IN_F32_MAXF = 2 };
enum { OUT_ACT = 0, OUT_HEAD_F32 = 1, OUT_HEAD_U8 = 2 };

struct ConvArgs {
    const void* in;
    int64_t in_slice;  // u8: bytes per slice; f32: floats per slice
    int64_t in_pitch;  // u8: bytes per row; f32: pixels per row
    int in_rows, in_cols;  // extent of the (virtual) input domain this layer reads
    int src_h, src_w;      // u8: slice size (reflect-101 range)
    int off_y, off_x;      // u8: input (r, c) reads slice (refl(r + off_y), refl(c + off_x))
    int out_h, out_w;
    void* out;
    int64_t out_slice, out_pitch;  // elements
    const float* wt;      // [CIN][K][K][COUT]
    const float* bias;    // [COUT]
    const float* head_w;  // [COUT] followed by the head bias
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
                    const uint8_t* src = static_cast<const uint8_t*>(a.in) + (int64_t)zi * a.in_slice;
                    int sy = refl101(gy + a.off_y, a.src_h), sx = refl101(gx + a.off_x, a.src_w);
                    v = (float)src[(int64_t)sy * a.in_pitch + sx] / 255.0f;
                }
                s_in[r * IWP + c] = v;
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
    if (OUT == OUT_ACT) {
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
static mb_status launch_conv(const ConvArgs& a, int nz, cudaStream_t st) {
    constexpr int TH = 256 / COUT;
    dim3 grid((a.out_w + 31) / 32, (a.out_h + TH - 1) / TH, nz);
    conv_simt<K, CIN, COUT, CC, IN, OUT><<<grid, 256, 0, st>>>(a);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

// Per-channel max of a 2x2 max-filtered activation map (all values >= 0 after ReLU, so the
// float bit patterns order like unsigned integers and atomicMax is exact and deterministic).
__global__ void amax_mf_kernel(const float* act, int64_t slice, int rows, int cols, int64_t pitch,
                               unsigned int* out_bits) {
    __shared__ unsigned int s_max[32];
    if (threadIdx.x < 32) s_max[threadIdx.x] = 0u;
    __syncthreads();
    const int c = threadIdx.x & 31;
    float m = 0.f;
    const float* base = act + (int64_t)blockIdx.y * slice;
    for (int64_t px = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; px < (int64_t)rows * cols;
         px += (int64_t)gridDim.x * (blockDim.x / 32)) {
        int y = (int)(px / cols), x = (int)(px - (int64_t)(px / cols) * cols);
        const float* p = base + ((int64_t)y * pitch + x) * 32 + c;
        float v = fmaxf(fmaxf(p[0], p[32]), fmaxf(p[pitch * 32], p[pitch * 32 + 32]));
        m = fmaxf(m, v);
    }
    atomicMax(&s_max[c], __float_as_uint(m));
    __syncthreads();
    if (threadIdx.x < 32) atomicMax(&out_bits[threadIdx.x], s_max[threadIdx.x]);
}

void simt_pack(const mb_net* net, const float* params, std::vector<float>& out) {
    out.clear();
    const float* p = params;
    for (const mb_layer_desc& L : net->layers) {
        if (L.kind == MB_CONV) {
            const int k = L.ksize, ci = L.cin, co = L.cout;
            size_t base = out.size();
            out.resize(base + (size_t)ci * k * k * co + co);
            for (int o = 0; o < co; ++o)
                for (int i = 0; i < ci; ++i)
                    for (int y = 0; y < k; ++y)
                        for (int x = 0; x < k; ++x)
                            out[base + (((size_t)i * k + y) * k + x) * co + o] = p[((o * ci + i) * k + y) * k + x];
            for (int o = 0; o < co; ++o) out[base + (size_t)ci * k * k * co + o] = p[(size_t)co * ci * k * k + o];
            p += (size_t)co * ci * k * k + co;
        } else if (L.kind == MB_HEAD_SIGMOID) {
            for (int i = 0; i < L.cin + 1; ++i) out.push_back(p[i]);
            p += L.cin + 1;
        }
    }
}

static size_t teacher_ws_per_slice(int64_t rows, int64_t cols) {
    return (size_t)((rows + 10) * (cols + 10) + (rows + 5) * (cols + 5)) * 32 * sizeof(float);
}

static int64_t chunk_slices(size_t per_slice, int64_t z) {
    const size_t budget = (size_t)3 << 30;
    int64_t zc = (int64_t)std::max<size_t>(1, budget / std::max<size_t>(per_slice, 1));
    zc = std::min<int64_t>(zc, 65535);
    return std::min<int64_t>(zc, z);
}

mb_status simt_teacher_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                              int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                              int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st) {
    const int64_t r1 = rows + 10, c1 = cols + 10, r2 = rows + 5, c2 = cols + 5;
    const int64_t zc = chunk_slices(teacher_ws_per_slice(rows, cols), z);
    MB_TRY(net->ws.ensure(teacher_ws_per_slice(rows, cols) * (size_t)zc));
    float* act1 = static_cast<float*>(net->ws.ptr);
    float* act2 = act1 + (size_t)zc * r1 * c1 * 32;
    const float* w1 = net->d_simt;
    const float* b1 = w1 + 25 * 32;
    const float* w2 = b1 + 32;
    const float* b2 = w2 + 25 * 32 * 32;
    const float* w3 = b2 + 32;
    const float* b3 = w3 + 25 * 32 * 32;
    const float* hw = b3 + 32;
    for (int64_t z0 = 0; z0 < z; z0 += zc) {
        const int nz = (int)std::min<int64_t>(zc, z - z0);
        ConvArgs a{};
        a.in = in + z0 * in_slice;
        a.in_slice = in_slice;
        a.in_pitch = in_pitch;
        a.in_rows = (int)(r1 + 4);
        a.in_cols = (int)(c1 + 4);
        a.src_h = (int)h;
        a.src_w = (int)w;
        a.off_y = (int)(y0 - 7);
        a.off_x = (int)(x0 - 7);
        a.out_h = (int)r1;
        a.out_w = (int)c1;
        a.out = act1;
        a.out_slice = r1 * c1 * 32;
        a.out_pitch = c1;
        a.wt = w1;
        a.bias = b1;
        MB_TRY((launch_conv<5, 1, 32, 1, IN_U8, OUT_ACT>(a, nz, st)));

        ConvArgs b{};
        b.in = act1;
        b.in_slice = r1 * c1 * 32;
        b.in_pitch = c1;
        b.in_rows = (int)(r2 + 4);
        b.in_cols = (int)(c2 + 4);
        b.out_h = (int)r2;
        b.out_w = (int)c2;
        b.out = act2;
        b.out_slice = r2 * c2 * 32;
        b.out_pitch = c2;
        b.wt = w2;
        b.bias = b2;
        MB_TRY((launch_conv<5, 32, 32, 8, IN_F32_MAXF, OUT_ACT>(b, nz, st)));

        ConvArgs c{};
        c.in = act2;
        c.in_slice = r2 * c2 * 32;
        c.in_pitch = c2;
        c.in_rows = (int)(rows + 4);
        c.in_cols = (int)(cols + 4);
        c.out_h = (int)rows;
        c.out_w = (int)cols;
        c.out_slice = out_slice;
        c.out_pitch = out_pitch;
        c.wt = w3;
        c.bias = b3;
        c.head_w = hw;
        if (ot == MB_OUT_F32) {
            c.out = static_cast<float*>(out) + z0 * out_slice;
            MB_TRY((launch_conv<5, 32, 32, 8, IN_F32_MAXF, OUT_HEAD_F32>(c, nz, st)));
        } else {
            c.out = static_cast<uint8_t*>(out) + z0 * out_slice;
            MB_TRY((launch_conv<5, 32, 32, 8, IN_F32_MAXF, OUT_HEAD_U8>(c, nz, st)));
        }
    }
    return MB_OK;
}

mb_status simt_teacher_amax(mb_net* net, const uint8_t* in, int64_t n, int64_t h, int64_t w, float* d_amax,
                            cudaStream_t st) {
    const int64_t r1 = h + 10, c1 = w + 10, r2 = h + 5, c2 = w + 5;
    const int64_t zc = chunk_slices(teacher_ws_per_slice(h, w), n);
    MB_TRY(net->ws.ensure(teacher_ws_per_slice(h, w) * (size_t)zc));
    float* act1 = static_cast<float*>(net->ws.ptr);
    float* act2 = act1 + (size_t)zc * r1 * c1 * 32;
    MB_CUDA(cudaMemsetAsync(d_amax, 0, 64 * sizeof(float), st));
    const float* w1 = net->d_simt;
    const float* b1 = w1 + 25 * 32;
    const float* w2 = b1 + 32;
    const float* b2 = w2 + 25 * 32 * 32;
    for (int64_t z0 = 0; z0 < n; z0 += zc) {
        const int nz = (int)std::min<int64_t>(zc, n - z0);
        ConvArgs a{};
        a.in = in + z0 * h * w;
        a.in_slice = h * w;
        a.in_pitch = w;
        a.in_rows = (int)(r1 + 4);
        a.in_cols = (int)(c1 + 4);
        a.src_h = (int)h;
        a.src_w = (int)w;
        a.off_y = -7;
        a.off_x = -7;
        a.out_h = (int)r1;
        a.out_w = (int)c1;
        a.out = act1;
        a.out_slice = r1 * c1 * 32;
        a.out_pitch = c1;
        a.wt = w1;
        a.bias = b1;
        MB_TRY((launch_conv<5, 1, 32, 1, IN_U8, OUT_ACT>(a, nz, st)));
        ConvArgs b{};
        b.in = act1;
        b.in_slice = r1 * c1 * 32;
        b.in_pitch = c1;
        b.in_rows = (int)(r2 + 4);
        b.in_cols = (int)(c2 + 4);
        b.out_h = (int)r2;
        b.out_w = (int)c2;
        b.out = act2;
        b.out_slice = r2 * c2 * 32;
        b.out_pitch = c2;
        b.wt = w2;
        b.bias = b2;
        MB_TRY((launch_conv<5, 32, 32, 8, IN_F32_MAXF, OUT_ACT>(b, nz, st)));
        dim3 g1(4 * 152, nz);
        amax_mf_kernel<<<g1, 256, 0, st>>>(act1, r1 * c1 * 32, (int)(r1 - 1), (int)(c1 - 1), c1,
                                           reinterpret_cast<unsigned int*>(d_amax));
        amax_mf_kernel<<<g1, 256, 0, st>>>(act2, r2 * c2 * 32, (int)(r2 - 1), (int)(c2 - 1), c2,
                                           reinterpret_cast<unsigned int*>(d_amax) + 32);
        count_launch(2);
        MB_CUDA(cudaGetLastError());
    }
    return MB_OK;
}

mb_status simt_student_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                              int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                              int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st) {
    const int64_t r1 = rows + 2, c1 = cols + 2;
    const size_t per = (size_t)r1 * c1 * 16 * sizeof(float);
    const int64_t zc = chunk_slices(per, z);
    MB_TRY(net->ws.ensure(per * (size_t)zc));
    float* act1 = static_cast<float*>(net->ws.ptr);
    const float* w1 = net->d_simt;
    const float* b1 = w1 + 9 * 16;
    const float* w2 = b1 + 16;
    const float* b2 = w2 + 9 * 16 * 16;
    const float* hw = b2 + 16;
    for (int64_t z0 = 0; z0 < z; z0 += zc) {
        const int nz = (int)std::min<int64_t>(zc, z - z0);
        ConvArgs a{};
        a.in = in + z0 * in_slice;
        a.in_slice = in_slice;
        a.in_pitch = in_pitch;
        a.in_rows = (int)(r1 + 2);
        a.in_cols = (int)(c1 + 2);
        a.src_h = (int)h;
        a.src_w = (int)w;
        a.off_y = (int)(y0 - 2);
        a.off_x = (int)(x0 - 2);
        a.out_h = (int)r1;
        a.out_w = (int)c1;
        a.out = act1;
        a.out_slice = r1 * c1 * 16;
        a.out_pitch = c1;
        a.wt = w1;
        a.bias = b1;
        MB_TRY((launch_conv<3, 1, 16, 1, IN_U8, OUT_ACT>(a, nz, st)));
        ConvArgs c{};
        c.in = act1;
        c.in_slice = r1 * c1 * 16;
        c.in_pitch = c1;
        c.in_rows = (int)r1;
        c.in_cols = (int)c1;
        c.out_h = (int)rows;
        c.out_w = (int)cols;
        c.out_slice = out_slice;
        c.out_pitch = out_pitch;
        c.wt = w2;
        c.bias = b2;
        c.head_w = hw;
        if (ot == MB_OUT_F32) {
            c.out = static_cast<float*>(out) + z0 * out_slice;
            MB_TRY((launch_conv<3, 16, 16, 8, IN_F32, OUT_HEAD_F32>(c, nz, st)));
        } else {
            c.out = static_cast<uint8_t*>(out) + z0 * out_slice;
            MB_TRY((launch_conv<3, 16, 16, 8, IN_F32, OUT_HEAD_U8>(c, nz, st)));
        }
    }
    return MB_OK;
}

}  // namespace mb
