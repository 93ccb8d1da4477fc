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
#include "simt_conv.cuh"

namespace mb {

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
        if (L.kind == MB_CONV || L.kind == MB_HEAD_SOFTMAX2) {
            const int k = L.ksize, ci = L.cin, co = L.cout * (L.maxout_groups > 1 ? L.maxout_groups : 1);
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
