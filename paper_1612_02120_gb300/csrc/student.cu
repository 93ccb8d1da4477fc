// student.cu - the distilled student network: training on the GPU by hand-written forward,
// backward and Adam kernels, and the multi-pass cascade (student everywhere, teacher on tiles
// the student flags as ambiguous).
//
// Student: conv3x3 1->16 ReLU, conv3x3 16->16 ReLU, conv1x1 16->1 sigmoid, mirror padding 2.
// Loss: L = (1/N) sum (p - t)^2 over all N output pixels of a batch.
// Backward (chain rule):  dz = (2/N)(p - t) p (1 - p)
//   head: dWh[c] = sum dz h2[c], dbh = sum dz;  dy2[c] = dz Wh[c] [h2[c] > 0]
//   conv2: dW2[co][ci][ky][kx] = sum dy2[co](y,x) h1[ci](y+ky, x+kx);  db2 = sum dy2
//          dy1 = (conv of dy2, zero-padded by 2, with W2 flipped and transposed) [h1 > 0]
//   conv1: dW1[co][ky][kx] = sum dy1[co](y,x) xpad(y+ky, x+kx);  db1 = sum dy1
// Every reduction runs in a fixed order (per-CTA partials over a fixed grid, then a per-parameter
// sum over CTAs in FP64), so a run is bitwise reproducible and a resumed run equals an
// uninterrupted one.
// Adam (Kingma and Ba, 2014): FP32 master weights, first/second moments, bias correction, with
// layer 1 optimised in centred-input coordinates (see adam_step); the forward copy is rounded to
// BF16 for BF16 students.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <errno.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "simt_conv.cuh"

namespace mb {

// Parameter offsets (API layout): W1[16][1][3][3] b1[16] W2[16][16][3][3] b2[16] Wh[16] bh.
constexpr int kSW1 = 0, kSB1 = 144, kSW2 = 160, kSB2 = 2464, kSWH = 2480, kSBH = 2496, kSN = 2497;
// Forward (SIMT) layout: W1t[1][3][3][16] b1 | W2t[16][3][3][16] b2 | Wh bh  (same block offsets)
// Backward data layout: W2f[co][ky][kx][ci] = W2[co][ci][2-ky][2-kx]  (2304 floats)
constexpr int kGridHead = 1184;   // 8 x 148: fixed grids make the partial sums reproducible
constexpr int kGridG2 = 592;
constexpr int kGridG1 = 296;

__device__ __forceinline__ int srefl(int t, int n) {
    t = t < 0 ? -t : t;
    return t >= n ? 2 * (n - 1) - t : t;
}

// Block-wide fixed-order sum of one float per thread (256 threads); result valid in thread 0.
__device__ __forceinline__ float block_sum256(float v, float* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    float r = sh[0];
    __syncthreads();
    return r;
}

// Head, loss and dz; h2 is overwritten in place by dy2. Partials per CTA: [loss, dWh[16], dbh].
__global__ void __launch_bounds__(256) student_head_loss(float* h2, const float* target, const int* zmap,
                                                         int64_t tslice, int B, int H, int W, const float* fw,
                                                         float inv_n, float* partial) {
    __shared__ float sh[256];
    const float* hw = fw + kSWH;
    const float hb = fw[kSBH];
    float ls = 0.f, gb = 0.f, gw[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) gw[c] = 0.f;
    const int64_t total = (int64_t)B * H * W;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < total; i += (int64_t)gridDim.x * 256) {
        const int zi = (int)(i / ((int64_t)H * W));
        const int64_t pix = i - (int64_t)zi * H * W;
        float* h = h2 + i * 16;
        float hv[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 v = *reinterpret_cast<const float4*>(h + 4 * q);
            hv[4 * q] = v.x; hv[4 * q + 1] = v.y; hv[4 * q + 2] = v.z; hv[4 * q + 3] = v.w;
        }
        float z = hb;
#pragma unroll
        for (int c = 0; c < 16; ++c) z = fmaf(hw[c], hv[c], z);
        const float p = 1.0f / (1.0f + expf(-z));
        const float t = target[(int64_t)(zmap ? zmap[zi] : zi) * tslice + pix];
        const float e = p - t;
        ls = fmaf(e, e, ls);
        const float dz = 2.0f * inv_n * e * p * (1.0f - p);
        gb += dz;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            gw[c] = fmaf(dz, hv[c], gw[c]);
            hv[c] = hv[c] > 0.f ? dz * hw[c] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4*>(h + 4 * q) = make_float4(hv[4 * q], hv[4 * q + 1], hv[4 * q + 2], hv[4 * q + 3]);
    }
    float r = block_sum256(ls, sh);
    if (threadIdx.x == 0) partial[blockIdx.x * 18 + 0] = r;
    for (int c = 0; c < 16; ++c) {
        r = block_sum256(gw[c], sh);
        if (threadIdx.x == 0) partial[blockIdx.x * 18 + 1 + c] = r;
    }
    r = block_sum256(gb, sh);
    if (threadIdx.x == 0) partial[blockIdx.x * 18 + 17] = r;
}

// conv2 weight gradient over 16x16 pixel tiles. Thread t: input channel ci = t & 15, output
// channels co and co + 8 (co = (t >> 4) & 7), tile rows 8 (t >> 7) .. + 7. Along each row it keeps
// the 3x3 window of h1 in registers and loads one new column (3 values) and the two dy2 values per
// pixel for its 18 FMAs; the two row halves are added (first + second) at the end.
// Partials per CTA: [2304 (co,ci,ky,kx)] then db2[16].
__global__ void __launch_bounds__(256) student_grad2(const float* dy2, const float* h1, int B, int H, int W,
                                                     float* partial) {
    __shared__ __align__(16) float s_d[256 * 16];
    __shared__ __align__(16) float s_h[18 * 18 * 16];
    const int t = threadIdx.x, ci = t & 15, co = (t >> 4) & 7, half = t >> 7;
    float acc0[9], acc1[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc0[k] = acc1[k] = 0.f;
    float db0 = 0.f, db1 = 0.f;
    const int tx_n = (W + 15) / 16, ty_n = (H + 15) / 16;
    const int64_t tiles = (int64_t)B * tx_n * ty_n;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int zi = (int)(tile / ((int64_t)tx_n * ty_n));
        const int rem = (int)(tile - (int64_t)zi * tx_n * ty_n);
        const int y0 = (rem / tx_n) * 16, x0 = (rem % tx_n) * 16;
        __syncthreads();
        for (int e = t; e < 256 * 4; e += 256) {
            const int px = e >> 2, q = e & 3;
            const int y = y0 + (px >> 4), x = x0 + (px & 15);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (y < H && x < W) v = *reinterpret_cast<const float4*>(dy2 + (((int64_t)zi * H + y) * W + x) * 16 + 4 * q);
            *reinterpret_cast<float4*>(s_d + px * 16 + 4 * q) = v;
        }
        for (int e = t; e < 18 * 18 * 4; e += 256) {
            const int px = e >> 2, q = e & 3;
            const int y = y0 + px / 18, x = x0 + px % 18;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (y < H + 2 && x < W + 2)
                v = *reinterpret_cast<const float4*>(h1 + (((int64_t)zi * (H + 2) + y) * (W + 2) + x) * 16 + 4 * q);
            *reinterpret_cast<float4*>(s_h + px * 16 + 4 * q) = v;
        }
        __syncthreads();
        for (int py = 8 * half; py < 8 * half + 8; ++py) {
            float w[3][3];  // h1 at rows py + ky, columns px + kx
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 2; ++kx) w[ky][kx + 1] = s_h[((py + ky) * 18 + kx) * 16 + ci];
#pragma unroll
            for (int px = 0; px < 16; ++px) {
#pragma unroll
                for (int ky = 0; ky < 3; ++ky) {
                    w[ky][0] = w[ky][1];
                    w[ky][1] = w[ky][2];
                    w[ky][2] = s_h[((py + ky) * 18 + px + 2) * 16 + ci];
                }
                const float d0 = s_d[(py * 16 + px) * 16 + co], d1 = s_d[(py * 16 + px) * 16 + co + 8];
                db0 += d0;
                db1 += d1;
#pragma unroll
                for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
                        acc0[ky * 3 + kx] = fmaf(d0, w[ky][kx], acc0[ky * 3 + kx]);
                        acc1[ky * 3 + kx] = fmaf(d1, w[ky][kx], acc1[ky * 3 + kx]);
                    }
            }
        }
    }
    // add the second half's sums to the first's
    __syncthreads();
    float* x = s_d + (t & 127) * 20;
    if (half == 1) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            x[k] = acc0[k];
            x[9 + k] = acc1[k];
        }
        x[18] = db0;
        x[19] = db1;
    }
    __syncthreads();
    if (half == 0) {
        float* out = partial + (int64_t)blockIdx.x * 2320;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            out[(co * 16 + ci) * 9 + k] = acc0[k] + x[k];
            out[((co + 8) * 16 + ci) * 9 + k] = acc1[k] + x[9 + k];
        }
        if (ci == 0) {
            out[2304 + co] = db0 + x[18];
            out[2304 + co + 8] = db1 + x[19];
        }
    }
}

// conv1 weight gradient over the (H+2) x (W+2) layer-1 domain; x is the input mirror-padded by 2.
// Thread t: output channel co = t & 15, tile row r = t >> 4; along the row it keeps the 3x3 window
// of x in registers (one new column of 3 per pixel) for its 9 FMAs and the bias sum. At the end the
// 16 rows' sums are added in row order. Partials per CTA: [144 (co,ky,kx)] then db1[16].
__global__ void __launch_bounds__(256) student_grad1(const float* dy1, const uint8_t* in, const int* zmap,
                                                     int64_t in_slice, int B, int H, int W, float* partial) {
    // dy1 tile [row][16 px][16 co], rows 272 floats apart so the two rows of a warp use distinct banks
    __shared__ __align__(16) float s_d[16 * 272];
    __shared__ __align__(16) float s_x[18 * 18];
    const int t = threadIdx.x, co = t & 15, r = t >> 4;
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.f;
    float db = 0.f;
    const int H1 = H + 2, W1 = W + 2;
    const int tx_n = (W1 + 15) / 16, ty_n = (H1 + 15) / 16;
    const int64_t tiles = (int64_t)B * tx_n * ty_n;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int zi = (int)(tile / ((int64_t)tx_n * ty_n));
        const int rem = (int)(tile - (int64_t)zi * tx_n * ty_n);
        const int y0 = (rem / tx_n) * 16, x0 = (rem % tx_n) * 16;
        __syncthreads();
        for (int e = t; e < 256 * 4; e += 256) {
            const int px = e >> 2, q = e & 3;
            const int y = y0 + (px >> 4), x = x0 + (px & 15);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (y < H1 && x < W1) v = *reinterpret_cast<const float4*>(dy1 + (((int64_t)zi * H1 + y) * W1 + x) * 16 + 4 * q);
            *reinterpret_cast<float4*>(s_d + (px >> 4) * 272 + (px & 15) * 16 + 4 * q) = v;
        }
        const uint8_t* src = in + (int64_t)(zmap ? zmap[zi] : zi) * in_slice;
        for (int e = t; e < 18 * 18; e += 256) {
            const int y = y0 + e / 18, x = x0 + e % 18;
            float v = 0.f;
            if (y < H + 4 && x < W + 4) v = (float)src[(int64_t)srefl(y - 2, H) * W + srefl(x - 2, W)] / 255.0f;
            s_x[e] = v;
        }
        __syncthreads();
        float w[3][3];  // x at rows r + ky, columns px + kx
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 2; ++kx) w[ky][kx + 1] = s_x[(r + ky) * 18 + kx];
#pragma unroll
        for (int px = 0; px < 16; ++px) {
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                w[ky][0] = w[ky][1];
                w[ky][1] = w[ky][2];
                w[ky][2] = s_x[(r + ky) * 18 + px + 2];
            }
            const float d = s_d[r * 272 + px * 16 + co];
            db += d;
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) acc[ky * 3 + kx] = fmaf(d, w[ky][kx], acc[ky * 3 + kx]);
        }
    }
    // rows' sums -> [r][co][10] in shared memory, then added in row order
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 9; ++k) s_d[(r * 16 + co) * 10 + k] = acc[k];
    s_d[(r * 16 + co) * 10 + 9] = db;
    __syncthreads();
    if (t < 160) {
        const int c = t < 144 ? t / 9 : t - 144, k = t < 144 ? t % 9 : 9;
        float sum = 0.f;
        for (int rr = 0; rr < 16; ++rr) sum += s_d[(rr * 16 + c) * 10 + k];
        partial[(int64_t)blockIdx.x * 160 + t] = sum;
    }
}

// grad[off + i] = sum over CTAs (FP64, fixed order) of partial[cta][col0 + i], i < count; with
// loss_out, also *loss_out = inv_n x the sum of column loss_col. One warp per output: lane l adds
// CTAs l, l + 32, ... in order, then the lanes are combined by a fixed xor-shuffle tree. Launch
// with 256-thread blocks, ceil((count + (loss_out != nullptr)) / 8) of them.
__global__ void reduce_partials(const float* partial, int ncta, int width, int col0, int count, float* grad, int off,
                                float* loss_out, int loss_col, float inv_n) {
    const int o = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const bool is_loss = loss_out && o == count;
    if (o >= count && !is_loss) return;
    const int col = is_loss ? loss_col : col0 + o;
    double s = 0.0;
    for (int c = lane; c < ncta; c += 32) s += (double)partial[(int64_t)c * width + col];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) {
        if (is_loss)
            *loss_out = (float)(s * (double)inv_n);
        else
            grad[off + o] = (float)s;
    }
}

__device__ __forceinline__ float fwd_round(float v, int bf16) { return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v; }

// Forward and backward-data layouts from the master weights.
__global__ void student_pack(const float* master, float* fwd, float* w2f, int bf16) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kSN) return;
    const float v = fwd_round(master[i], bf16);
    if (i < kSB1) {  // W1[co][0][ky][kx] -> W1t[tap][co]
        const int co = i / 9, tap = i % 9;
        fwd[tap * 16 + co] = v;
    } else if (i < kSW2) {
        fwd[i] = v;
    } else if (i < kSB2) {  // W2[co][ci][ky][kx] -> W2t[ci][ky][kx][co], W2f[co][2-ky][2-kx][ci]
        const int j = i - kSW2, co = j / 144, ci = (j / 9) % 16, tap = j % 9, ky = tap / 3, kx = tap % 3;
        fwd[kSW2 + (ci * 9 + tap) * 16 + co] = v;
        w2f[(co * 9 + (2 - ky) * 3 + (2 - kx)) * 16 + ci] = v;
    } else {
        fwd[i] = v;
    }
}

// Adam (Kingma & Ba 2014) with bias correction, one thread per parameter, except layer 1, which is
// optimised in centred coordinates: Adam updates W1 and c1 = b1 + (1/2) sum_k W1[co][k], the bias
// of the same network written for the zero-centred input x - 1/2 (conv(pad(x) - 1/2) =
// conv(pad(x)) - (1/2) sum W, since the mirror pad of a constant shift is the same shift). In those
// coordinates the gradients are g_W1 - g_b1 / 2 and g_b1, and the update maps back to the stored
// form as W1 -= dW, b1 -= dc - (1/2) sum_k dW: the trajectory of training on a centred input,
// while the stored network keeps the input u/255. Threads 0..15: one layer-1 output channel each
// (its 9 weights and its bias); the rest: parameters kSW2 .. n-1.
__device__ __forceinline__ float adam_delta(float* m, float* v, int i, float gi, float lr, float b1, float b2,
                                            float eps, float c1, float c2) {
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    return lr * mh / (sqrtf(vh) + eps);
}

__global__ void adam_step(float* w, float* m, float* v, const float* g, int n, float lr, float b1, float b2,
                          float eps, float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 16) {
        const float gb = g[kSB1 + t];
        float dsum = 0.f;
        for (int k = 0; k < 9; ++k) {
            const int i = kSW1 + 9 * t + k;
            const float d = adam_delta(m, v, i, g[i] - 0.5f * gb, lr, b1, b2, eps, c1, c2);
            w[i] -= d;
            dsum += d;
        }
        const float dc = adam_delta(m, v, kSB1 + t, gb, lr, b1, b2, eps, c1, c2);
        w[kSB1 + t] -= dc - 0.5f * dsum;
        return;
    }
    const int i = kSW2 + t - 16;
    if (i >= n) return;
    w[i] -= adam_delta(m, v, i, g[i], lr, b1, b2, eps, c1, c2);
}
static_assert(kSW2 == kSB1 + 16, "layer-1 biases are followed by layer 2");
constexpr int kAdamThreads = 16 + kSN - kSW2;

// Device buffers of one training shape.
struct StudentBufs {
    float* h1 = nullptr;      // [B][H+2][W+2][16]; becomes dy1
    float* h2 = nullptr;      // [B][H][W][16]; becomes dy2
    float* part = nullptr;    // partial sums
    float* grad = nullptr;    // [kSN]
    float* w2f = nullptr;     // [2304]
    float* zero = nullptr;    // [16] zero bias of the data-gradient convolution
    float* m = nullptr;
    float* v = nullptr;
    int* zmap = nullptr;
    float* losses = nullptr;
};

static size_t part_floats() {
    return std::max<size_t>({(size_t)kGridHead * 18, (size_t)kGridG2 * 2320, (size_t)kGridG1 * 160});
}

// Carves the training workspace; every sub-buffer starts on a 256-byte boundary (the convolution
// kernels read weights and activations as float4).
static mb_status ensure_bufs(mb_net* s, int64_t B, int64_t H, int64_t W, int64_t steps, StudentBufs& b) {
    auto up = [](size_t n) { return (n + 63) & ~(size_t)63; };  // floats, rounded to 256 bytes
    const size_t nst = (size_t)std::max<int64_t>(steps, 1);
    const size_t f_h1 = up((size_t)B * (H + 2) * (W + 2) * 16), f_h2 = up((size_t)B * H * W * 16);
    const size_t f_part = up(part_floats()), f_grad = up(kSN), f_w2f = up(2304), f_zero = up(16), f_m = up(kSN),
                 f_v = up(kSN), f_loss = up(nst), f_zmap = up(nst * (size_t)B);
    const size_t floats = f_h1 + f_h2 + f_part + f_grad + f_w2f + f_zero + f_m + f_v + f_loss + f_zmap;
    MB_TRY(s->ws2.ensure(floats * 4));
    float* p = static_cast<float*>(s->ws2.ptr);
    b.h1 = p;
    p += f_h1;
    b.h2 = p;
    p += f_h2;
    b.part = p;
    p += f_part;
    b.grad = p;
    p += f_grad;
    b.w2f = p;
    p += f_w2f;
    b.zero = p;
    p += f_zero;
    b.m = p;
    p += f_m;
    b.v = p;
    p += f_v;
    b.losses = p;
    p += f_loss;
    b.zmap = reinterpret_cast<int*>(p);
    return MB_OK;
}

// Loss and gradient of one batch (slices zmap[0..B) of `in`); the gradient lands in b.grad and the
// mean loss in *loss_dev.
static mb_status batch_grad(mb_net* s, const uint8_t* in, const float* tgt, const int* zmap, int64_t B, int64_t H,
                            int64_t W, StudentBufs& b, float* loss_dev, cudaStream_t st) {
    const float* fwd = s->d_simt;
    const float inv_n = (float)(1.0 / ((double)B * H * W));
    // forward layer 1 -> h1, layer 2 -> h2 (post-ReLU)
    ConvArgs a{};
    a.in = in;
    a.in_slice = H * W;
    a.in_pitch = W;
    a.in_rows = (int)(H + 4);
    a.in_cols = (int)(W + 4);
    a.src_h = (int)H;
    a.src_w = (int)W;
    a.off_y = -2;
    a.off_x = -2;
    a.out_h = (int)(H + 2);
    a.out_w = (int)(W + 2);
    a.out = b.h1;
    a.out_slice = (H + 2) * (W + 2) * 16;
    a.out_pitch = W + 2;
    a.wt = fwd + kSW1;
    a.bias = fwd + kSB1;
    a.zmap = zmap;
    MB_TRY((launch_conv<3, 1, 16, 1, IN_U8, OUT_ACT>(a, (int)B, st)));
    ConvArgs c{};
    c.in = b.h1;
    c.in_slice = (H + 2) * (W + 2) * 16;
    c.in_pitch = W + 2;
    c.in_rows = (int)(H + 2);
    c.in_cols = (int)(W + 2);
    c.out_h = (int)H;
    c.out_w = (int)W;
    c.out = b.h2;
    c.out_slice = H * W * 16;
    c.out_pitch = W;
    c.wt = fwd + kSW2;
    c.bias = fwd + kSB2;
    MB_TRY((launch_conv<3, 16, 16, 8, IN_F32, OUT_ACT>(c, (int)B, st)));
    // head + loss; h2 -> dy2
    student_head_loss<<<kGridHead, 256, 0, st>>>(b.h2, tgt, zmap, H * W, (int)B, (int)H, (int)W, fwd, inv_n, b.part);
    reduce_partials<<<(17 + 1 + 7) / 8, 256, 0, st>>>(b.part, kGridHead, 18, 1, 17, b.grad, kSWH, loss_dev, 0, inv_n);
    count_launch(2);
    // conv2 weight gradient (needs h1 intact)
    student_grad2<<<kGridG2, 256, 0, st>>>(b.h2, b.h1, (int)B, (int)H, (int)W, b.part);
    static_assert(kSB2 == kSW2 + 2304, "W2 and b2 are adjacent in the parameter layout");
    reduce_partials<<<(2320 + 7) / 8, 256, 0, st>>>(b.part, kGridG2, 2320, 0, 2320, b.grad, kSW2, nullptr, 0, 0.f);
    count_launch(2);
    // dy1 = conv(dy2 zero-padded by 2, flipped W2) masked by h1 > 0, in place of h1
    ConvArgs d{};
    d.in = b.h2;
    d.in_slice = H * W * 16;
    d.in_pitch = W;
    d.in_rows = (int)(H + 4);
    d.in_cols = (int)(W + 4);
    d.src_h = (int)H;
    d.src_w = (int)W;
    d.off_y = -2;
    d.off_x = -2;
    d.out_h = (int)(H + 2);
    d.out_w = (int)(W + 2);
    d.out = b.h1;
    d.out_slice = (H + 2) * (W + 2) * 16;
    d.out_pitch = W + 2;
    d.wt = b.w2f;
    d.bias = b.zero;
    d.mask = b.h1;
    MB_TRY((launch_conv<3, 16, 16, 8, IN_F32_PAD, OUT_GRADMASK>(d, (int)B, st)));
    // conv1 weight gradient
    student_grad1<<<kGridG1, 256, 0, st>>>(b.h1, in, zmap, H * W, (int)B, (int)H, (int)W, b.part);
    static_assert(kSB1 == kSW1 + 144, "W1 and b1 are adjacent in the parameter layout");
    reduce_partials<<<(160 + 7) / 8, 256, 0, st>>>(b.part, kGridG1, 160, 0, 160, b.grad, kSW1, nullptr, 0, 0.f);
    count_launch(2);
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

static mb_status pack_forward(mb_net* s, StudentBufs& b, cudaStream_t st) {
    MB_CUDA(cudaMemsetAsync(b.zero, 0, 16 * sizeof(float), st));
    student_pack<<<(kSN + 255) / 256, 256, 0, st>>>(s->d_params, s->d_simt, b.w2f, s->prec == MB_PREC_BF16);
    count_launch();
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

mb_status student_loss_grad(mb_net* s, const uint8_t* in, const float* tgt, int64_t n, int64_t h, int64_t w,
                            double* loss, float* grad, cudaStream_t st) {
    StudentBufs b;
    MB_TRY(ensure_bufs(s, n, h, w, 1, b));
    MB_TRY(pack_forward(s, b, st));
    MB_TRY(batch_grad(s, in, tgt, nullptr, n, h, w, b, b.losses, st));
    MB_CUDA(cudaMemcpyAsync(grad, b.grad, kSN * sizeof(float), cudaMemcpyDeviceToDevice, st));
    float lh = 0.f;
    MB_CUDA(cudaMemcpyAsync(&lh, b.losses, sizeof(float), cudaMemcpyDeviceToHost, st));
    MB_CUDA(cudaStreamSynchronize(st));
    *loss = lh;
    return MB_OK;
}

// ---- checkpoint file: header + master weights + m + v ------------------------------------------
struct CkptHeader {
    char magic[8];      // "MBCKPT02": m and v are the moments of the centred layer-1 coordinates
    int64_t step;       // optimiser steps completed
    int64_t n_params;
    uint64_t sampler;   // SplitMix64 state after the last completed step
    uint64_t seed;
};

static uint64_t sm64(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static mb_status write_ckpt(const char* path, const CkptHeader& hd, const float* d_w, const float* d_m,
                            const float* d_v, cudaStream_t st) {
    std::vector<float> buf(3 * (size_t)kSN);
    MB_CUDA(cudaMemcpyAsync(buf.data(), d_w, kSN * 4, cudaMemcpyDeviceToHost, st));
    MB_CUDA(cudaMemcpyAsync(buf.data() + kSN, d_m, kSN * 4, cudaMemcpyDeviceToHost, st));
    MB_CUDA(cudaMemcpyAsync(buf.data() + 2 * kSN, d_v, kSN * 4, cudaMemcpyDeviceToHost, st));
    MB_CUDA(cudaStreamSynchronize(st));
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) {
        set_error("cannot write checkpoint %s", tmp.c_str());
        return MB_ERR_INVALID_ARG;
    }
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(buf.data(), 4, buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        set_error("writing checkpoint %s failed", path);
        return MB_ERR_INVALID_ARG;
    }
    return MB_OK;
}

// Result of looking for a checkpoint to resume from.
enum class CkptRead { kAbsent, kOk, kInvalid };

// A file that does not exist means a fresh start; a file that exists but is not a complete
// checkpoint of this format (another version, another parameter count, truncated) is an error,
// so that a later checkpoint write never overwrites a file the caller meant to resume from.
static CkptRead read_ckpt(const char* path, CkptHeader& hd, std::vector<float>& buf) {
    FILE* f = fopen(path, "rb");
    if (!f) return errno == ENOENT ? CkptRead::kAbsent : CkptRead::kInvalid;
    buf.resize(3 * (size_t)kSN);
    bool ok = fread(&hd, sizeof(hd), 1, f) == 1 && memcmp(hd.magic, "MBCKPT02", 8) == 0 && hd.n_params == kSN &&
              fread(buf.data(), 4, buf.size(), f) == buf.size();
    if (ok) {
        char extra;
        ok = fread(&extra, 1, 1, f) == 0;  // nothing after the moments
    }
    fclose(f);
    return ok ? CkptRead::kOk : CkptRead::kInvalid;
}

mb_status student_train(mb_net* s, const uint8_t* in, const float* tgt, int64_t n, int64_t h, int64_t w,
                        const mb_train_cfg* cfg, const char* ckpt, float* curve, cudaStream_t st) {
    const int64_t B = cfg->batch;
    StudentBufs b;
    MB_TRY(ensure_bufs(s, B, h, w, cfg->steps, b));
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "MBCKPT02", 8);
    hd.n_params = kSN;
    hd.seed = cfg->seed;
    hd.sampler = cfg->seed ^ 0x5A17E5EEDULL;
    int64_t start = 0;
    std::vector<float> buf;
    const CkptRead found = (ckpt && cfg->resume) ? read_ckpt(ckpt, hd, buf) : CkptRead::kAbsent;
    if (found == CkptRead::kInvalid) {
        set_error("checkpoint %s exists but is not a format-2 checkpoint of this student (version, parameter "
                  "count or size); it was left unchanged",
                  ckpt);
        return MB_ERR_INVALID_ARG;
    }
    if (found == CkptRead::kOk) {
        if (hd.seed != cfg->seed || hd.step > cfg->steps) {
            set_error("checkpoint %s does not match this run (seed or step count)", ckpt);
            return MB_ERR_INVALID_ARG;
        }
        start = hd.step;
        MB_CUDA(cudaMemcpyAsync(s->d_params, buf.data(), kSN * 4, cudaMemcpyHostToDevice, st));
        MB_CUDA(cudaMemcpyAsync(b.m, buf.data() + kSN, kSN * 4, cudaMemcpyHostToDevice, st));
        MB_CUDA(cudaMemcpyAsync(b.v, buf.data() + 2 * kSN, kSN * 4, cudaMemcpyHostToDevice, st));
        MB_CUDA(cudaStreamSynchronize(st));
    } else {
        MB_CUDA(cudaMemsetAsync(b.m, 0, kSN * 4, st));
        MB_CUDA(cudaMemsetAsync(b.v, 0, kSN * 4, st));
    }
    // slice indices of every remaining step, drawn with replacement
    const int64_t nsteps = cfg->steps - start;
    std::vector<int> idx((size_t)std::max<int64_t>(nsteps, 1) * B);
    uint64_t sampler = hd.sampler;
    std::vector<uint64_t> sampler_after((size_t)std::max<int64_t>(nsteps, 1));
    for (int64_t k = 0; k < nsteps; ++k) {
        for (int64_t j = 0; j < B; ++j)
            idx[(size_t)(k * B + j)] = (int)((sm64(&sampler) >> 11) % (uint64_t)n);
        sampler_after[(size_t)k] = sampler;
    }
    if (nsteps > 0)
        MB_CUDA(cudaMemcpyAsync(b.zmap, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    for (int64_t k = 0; k < nsteps; ++k) {
        const int64_t step = start + k + 1;
        MB_TRY(pack_forward(s, b, st));
        MB_TRY(batch_grad(s, in, tgt, b.zmap + k * B, B, h, w, b, b.losses + k, st));
        const double c1 = 1.0 - std::pow((double)cfg->beta1, (double)step);
        const double c2 = 1.0 - std::pow((double)cfg->beta2, (double)step);
        adam_step<<<(kAdamThreads + 255) / 256, 256, 0, st>>>(s->d_params, b.m, b.v, b.grad, kSN, cfg->lr, cfg->beta1,
                                                     cfg->beta2, cfg->eps, (float)c1, (float)c2);
        count_launch();
        MB_CUDA(cudaGetLastError());
        if (ckpt && cfg->ckpt_every > 0 && step % cfg->ckpt_every == 0) {
            hd.step = step;
            hd.sampler = sampler_after[(size_t)k];
            MB_TRY(write_ckpt(ckpt, hd, s->d_params, b.m, b.v, st));
        }
    }
    MB_TRY(pack_forward(s, b, st));
    if (curve && nsteps > 0)
        MB_CUDA(cudaMemcpyAsync(curve, b.losses, nsteps * sizeof(float), cudaMemcpyDeviceToHost, st));
    MB_CUDA(cudaStreamSynchronize(st));
    // the host master copy follows the device
    MB_CUDA(cudaMemcpy(s->host_params.data(), s->d_params, kSN * 4, cudaMemcpyDeviceToHost));
    return MB_OK;
}

// ---- cascade -------------------------------------------------------------------------------------
// One CTA per tile: count student outputs in [lo, hi]; flag when count > max_frac * tile pixels.
__global__ void __launch_bounds__(256) tile_flags(const float* p, int64_t z, int H, int W, int tile, float lo,
                                                  float hi, float max_frac, uint8_t* flags, int* nflag) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int tx_n = (W + tile - 1) / tile, ty_n = (H + tile - 1) / tile;
    const int64_t tid = blockIdx.x;
    const int zi = (int)(tid / ((int64_t)tx_n * ty_n));
    const int rem = (int)(tid - (int64_t)zi * tx_n * ty_n);
    const int y0 = (rem / tx_n) * tile, x0 = (rem % tx_n) * tile;
    const int th = min(tile, H - y0), tw = min(tile, W - x0);
    int cnt = 0;
    for (int i = threadIdx.x; i < th * tw; i += 256) {
        const float v = p[((int64_t)zi * H + y0 + i / tw) * W + x0 + i % tw];
        cnt += (v >= lo && v <= hi) ? 1 : 0;
    }
    atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool f = (double)s_cnt > (double)max_frac * (double)(th * tw);
        flags[tid] = f ? 1 : 0;
        if (f) atomicAdd(nflag, 1);
    }
}

mb_status cascade(mb_net* s, mb_net* t, const uint8_t* in, int64_t z, int64_t h, int64_t w, float* out, int tile,
                  float lo, float hi, float max_frac, double* rate, uint8_t* flags_out, cudaStream_t st) {
    if (z == 0) {
        *rate = 0.0;
        return MB_OK;
    }
    MB_TRY(student_region(s, in, z, h, w, w, h * w, 0, 0, h, w, out, w, h * w, MB_OUT_F32, st));
    const int tx_n = (int)((w + tile - 1) / tile), ty_n = (int)((h + tile - 1) / tile);
    const int64_t ntiles = z * tx_n * ty_n;
    uint8_t* d_flags = nullptr;
    int* d_n = nullptr;
    MB_TRY(dev_alloc((void**)&d_flags, (size_t)ntiles + 64));
    d_n = reinterpret_cast<int*>(d_flags + ((ntiles + 15) / 16) * 16);
    mb_status rc = MB_OK;
    std::vector<uint8_t> hf((size_t)ntiles);
    do {
        cudaError_t e = cudaMemsetAsync(d_n, 0, sizeof(int), st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__); break; }
        tile_flags<<<(unsigned)ntiles, 256, 0, st>>>(out, z, (int)h, (int)w, tile, lo, hi, max_frac, d_flags, d_n);
        count_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess && flags_out)
            e = cudaMemcpyAsync(flags_out, d_flags, (size_t)ntiles, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hf.data(), d_flags, (size_t)ntiles, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "tile flags", __FILE__, __LINE__); break; }
        // the teacher recomputes every flagged tile with its true context, writing into out. Runs of
        // flagged tiles along a tile row, and runs of such rows with the same column span, are
        // recomputed as one region (the teacher's output at a pixel does not depend on the region
        // around it, so this only removes strip and launch overheads).
        struct Region {
            int64_t zi, y0, rows, x0, cols;
        };
        std::vector<Region> regions;
        int64_t nflag = 0;
        for (int64_t zi = 0; zi < z; ++zi) {
            std::vector<Region> open;  // regions that may extend into the next tile row
            for (int64_t ty = 0; ty < ty_n; ++ty) {
                const int64_t y0 = ty * tile, th = std::min<int64_t>(tile, h - y0);
                std::vector<Region> spans;
                for (int64_t tx = 0; tx < tx_n; ++tx) {
                    if (!hf[(size_t)((zi * ty_n + ty) * tx_n + tx)]) continue;
                    ++nflag;
                    const int64_t x0 = tx * tile, tw = std::min<int64_t>(tile, w - x0);
                    if (!spans.empty() && spans.back().x0 + spans.back().cols == x0)
                        spans.back().cols += tw;
                    else
                        spans.push_back({zi, y0, th, x0, tw});
                }
                std::vector<Region> next;
                for (const Region& sp : spans) {
                    bool merged = false;
                    for (Region& o : open)
                        if (!merged && o.x0 == sp.x0 && o.cols == sp.cols && o.y0 + o.rows == sp.y0) {
                            o.rows += sp.rows;
                            next.push_back(o);
                            o.cols = 0;  // taken over by next
                            merged = true;
                        }
                    if (!merged) next.push_back(sp);
                }
                for (const Region& o : open)
                    if (o.cols > 0) regions.push_back(o);
                open.swap(next);
            }
            for (const Region& o : open) regions.push_back(o);
        }
        std::vector<mb_block> blocks;
        std::vector<int64_t> ry, rx, rr, rcn;
        for (const Region& g : regions) {
            if (t->prec == MB_PREC_FP32) {
                rc = simt_teacher_region(t, in + g.zi * h * w, 1, h, w, w, h * w, g.y0, g.x0, g.rows, g.cols,
                                         out + g.zi * h * w + g.y0 * w + g.x0, w, h * w, MB_OUT_F32, st);
                if (rc != MB_OK) break;
                continue;
            }
            mb_block b;
            b.in = in + g.zi * h * w;
            b.z = 1;
            b.h = h;
            b.w = w;
            b.in_pitch = w;
            b.in_slice_pitch = h * w;
            b.out = out + g.zi * h * w + g.y0 * w + g.x0;
            b.out_pitch = w;
            b.out_slice_pitch = h * w;
            blocks.push_back(b);
            ry.push_back(g.y0);
            rx.push_back(g.x0);
            rr.push_back(g.rows);
            rcn.push_back(g.cols);
        }
        if (rc != MB_OK) break;
        if (!blocks.empty())
            rc = tc_infer_blocks(t, blocks.data(), (int)blocks.size(), ry.data(), rx.data(), rr.data(), rcn.data(),
                                 MB_OUT_F32, st, false);
        if (rc != MB_OK) break;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cascade teacher pass", __FILE__, __LINE__); break; }
        *rate = (double)nflag / (double)ntiles;
    } while (0);
    dev_free(d_flags);
    if (rc == MB_OK) rc = tc_poll_error(t);
    return rc;
}

}  // namespace mb
