// maskextend.cu - MaskExtend (Sec. 3.2) on CUDA cores (FP32): the transfer
//   Mask_z = J(CNN(masks z-4..z-1, EM z-1..z+1, membrane maps z-2..z+2))
// recursed in +z, or in -z with every offset mirrored (masks z+4..z+1, EM z+1..z-1, membrane
// maps z+2..z-2: the algorithm continues in either direction). CNN is the dense form of the max-out network: five 4x4 convs with max-out 2
// (32, 40, 48, 56, 64 features; the first four followed by 2x2 pools, i.e. dilations 1, 2, 4, 8,
// 16 with dilated max-filters in between), then a 1x1 head to 3 classes (object, other neurons,
// membrane) with a softmax. J is a 3x3 mean of the object probability (reflect-101 borders)
// followed by >= threshold.
//
// Per step: me_assemble builds the mirror-padded (by 54) 12-map input stack as FP32
// [y][x][16] (channels 12-15 zero); five fm_conv launches (fm_conv.cuh) produce the max-out
// activations; me_head computes the 3 class probabilities; me_smooth_threshold writes the mask,
// which the next step reads as its mask z-1.
//
// Domains for a section of h x w (walking back from the head: conv k's input needs 3 d_k + dm_k
// more rows than its output): conv5 out h, conv4 out h+56, conv3 out h+84, conv2 out h+98,
// conv1 out h+105, input h+108.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "fm_conv.cuh"
#include "internal.h"

namespace mb {

namespace {

constexpr int kMeR = 54;
constexpr int kMeCin = 16;  // 12 maps padded to 16 channels

struct MeMasks {
    const uint8_t* m[4];  // masks of sections z + dz k for k = -4 .. -1, [h][w]
};

// Mirror-padded input stack of section z: out[(r, c)][ch] for r < h + 108, c < w + 108, FP32 or
// (for the tensor-core path) FP16. dz = +1 or -1 is the direction of travel: the maps at offset k
// of the transfer equation are read from section z + dz k.
template <typename T>
__global__ void me_assemble(const uint8_t* __restrict__ em, const float* __restrict__ memb, MeMasks mk, int64_t z,
                            int dz, int h, int w, T* __restrict__ out) {
    const int pw = w + 2 * kMeR, ph = h + 2 * kMeR;
    const int64_t n = (int64_t)ph * pw;
    const int64_t hw = (int64_t)h * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / pw), c = (int)(i - (i / pw) * pw);
        const int y = refl101(r - kMeR, h), x = refl101(c - kMeR, w);
        const int64_t o = (int64_t)y * w + x;
        float v[16];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = (float)em[(z + dz * (k - 1)) * hw + o] / 255.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) v[3 + k] = (float)mk.m[k][o];
#pragma unroll
        for (int k = 0; k < 5; ++k) v[7 + k] = memb[(z + dz * (k - 2)) * hw + o];
#pragma unroll
        for (int k = 12; k < 16; ++k) v[k] = 0.f;
        if constexpr (sizeof(T) == 4) {
            float4* d = reinterpret_cast<float4*>(out + i * kMeCin);
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
        } else {
            uint32_t hw[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                __half2 h2 = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
                hw[k] = *reinterpret_cast<uint32_t*>(&h2);
            }
            uint4* d = reinterpret_cast<uint4*>(out + i * kMeCin);
            d[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            d[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
        }
    }
}

// 1x1 head 64 -> 3 and the softmax: probs[cls][y][x] = exp(z_cls - max) / sum exp(z - max).
__global__ void me_head(const float* __restrict__ act, int h, int w, const float* __restrict__ hw_b,
                        float* __restrict__ probs) {
    __shared__ float s_w[3 * 64 + 3];
    for (int i = threadIdx.x; i < 3 * 64 + 3; i += blockDim.x) s_w[i] = hw_b[i];
    __syncthreads();
    const int64_t n = (int64_t)h * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4* a = reinterpret_cast<const float4*>(act + i * 64);
        float z0 = s_w[192], z1 = s_w[193], z2 = s_w[194];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float4 v = __ldg(a + q);
            const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 4 * q + e;
                z0 = fmaf(s_w[c], x[e], z0);
                z1 = fmaf(s_w[64 + c], x[e], z1);
                z2 = fmaf(s_w[128 + c], x[e], z2);
            }
        }
        const float m = fmaxf(z0, fmaxf(z1, z2));
        const float e0 = expf(z0 - m), e1 = expf(z1 - m), e2 = expf(z2 - m);
        const float den = e0 + e1 + e2;
        probs[i] = e0 / den;
        probs[n + i] = e1 / den;
        probs[2 * n + i] = e2 / den;
    }
}

// J: mask = (3x3 mean of p, reflect-101 borders) >= thr, summed in the row-major window order.
__global__ void me_smooth_threshold(const float* __restrict__ p, int h, int w, float thr, uint8_t* __restrict__ mask) {
    const int64_t n = (int64_t)h * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / w), x = (int)(i - (i / w) * w);
        float s = 0.f;
        for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b) s += p[(int64_t)refl101(y + a, h) * w + refl101(x + b, w)];
        mask[i] = s / 9.0f >= thr ? 1 : 0;
    }
}

}  // namespace

// MaskExtend SIMT weight layout (host): conv1 Wt[16][4][4][64] (input channels 12-15 zero) + b[64];
// conv k >= 2 Wt[cin][4][4][2 cout] + b[2 cout]; head W[3][64] then b[3] (API layout).
void me_pack(const mb_net* net, const float* params, std::vector<float>& out) {
    out.clear();
    const float* p = params;
    for (const mb_layer_desc& L : net->layers) {
        if (L.kind == MB_CONV) {
            const int ci = L.cin, co = L.cout * (L.maxout_groups > 1 ? L.maxout_groups : 1);
            const int cip = ci == 12 ? kMeCin : ci;
            const size_t base = out.size();
            out.resize(base + (size_t)cip * 16 * co + co, 0.f);
            for (int o = 0; o < co; ++o)
                for (int i = 0; i < ci; ++i)
                    for (int t = 0; t < 16; ++t) out[base + ((size_t)i * 16 + t) * co + o] = p[((size_t)o * ci + i) * 16 + t];
            for (int o = 0; o < co; ++o) out[base + (size_t)cip * 16 * co + o] = p[(size_t)co * ci * 16 + o];
            p += (size_t)co * ci * 16 + co;
        } else if (L.kind == MB_HEAD_SOFTMAX) {
            for (int i = 0; i < 3 * 64 + 3; ++i) out.push_back(p[i]);
            p += 3 * 64 + 3;
        }
    }
}

// Masks read by step s (the section z0 + dz s): the four sections before it along the direction of
// travel, step s + k - 4 for k = 0 .. 3; steps before the first are the seeds (seed i = step i - 4).
static void me_masks(MeMasks& mk, const uint8_t* seeds, const uint8_t* masks_out, int64_t s, int64_t hw) {
    for (int k = 0; k < 4; ++k) {
        const int64_t t = s + k - 4;
        mk.m[k] = t < 0 ? seeds + (t + 4) * hw : masks_out + t * hw;
    }
}

static int me_grid(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
}

// FP16 tensor-core form of the recursion: the same stack in FP16, the five convs on the tensor cores
// (maskextend_tc.cu; the last one with the head and the softmax), then J.
static mb_status maskextend_run_tc(mb_net* net, const uint8_t* em, const float* memb, int64_t h, int64_t w,
                                   const uint8_t* seeds, int64_t z0, int64_t n_steps, int dz, float thr,
                                   uint8_t* masks_out, float* probs_out, cudaStream_t st) {
    MB_TRY(me_tc_poll_error(net));  // a wait that timed out in an earlier call on this net
    const int64_t r[5] = {h + 105, h + 98, h + 84, h + 56, h}, c[5] = {w + 105, w + 98, w + 84, w + 56, w};
    const int d[5] = {1, 2, 4, 8, 16}, dm[5] = {0, 1, 2, 4, 8};
    const int64_t feat[5] = {32, 40, 48, 56, 64};
    auto up = [](int64_t n) { return (n + 127) & ~(int64_t)127; };  // 256-byte aligned sub-buffers (FP16)
    const int64_t n_in = up((h + 108) * (w + 108) * kMeCin);
    int64_t n_act[4], total = n_in;
    for (int k = 0; k < 4; ++k) {
        n_act[k] = up(r[k] * c[k] * feat[k]);
        total += n_act[k];
    }
    const int64_t n_prob = up(2 * 3 * h * w);  // FP32 probabilities, counted in FP16 units
    total += n_prob;
    MB_TRY(net->ws.ensure((size_t)total * sizeof(__half)));
    __half* xin = static_cast<__half*>(net->ws.ptr);
    __half* act[4];
    act[0] = xin + n_in;
    for (int k = 1; k < 4; ++k) act[k] = act[k - 1] + n_act[k - 1];
    float* prob_tmp = reinterpret_cast<float*>(act[3] + n_act[3]);
    const int64_t hw = h * w;
    for (int64_t s = 0; s < n_steps; ++s) {
        const int64_t z = z0 + dz * s;
        MeMasks mk;
        me_masks(mk, seeds, masks_out, s, hw);
        me_assemble<__half><<<me_grid((h + 108) * (w + 108)), 256, 0, st>>>(em, memb, mk, z, dz, (int)h, (int)w, xin);
        count_launch();
        MB_CUDA(cudaGetLastError());
        float* probs = probs_out ? probs_out + s * 3 * hw : prob_tmp;
        for (int k = 0; k < 5; ++k) {
            const void* in = k == 0 ? (const void*)xin : (const void*)act[k - 1];
            const int64_t in_pitch = k == 0 ? w + 108 : c[k - 1];
            const int cs = k == 0 ? kMeCin : (int)feat[k - 1];
            MB_TRY(me_tc_layer(net, k, in, in_pitch, cs, (int)(r[k] + 3 * d[k]), (int)(c[k] + 3 * d[k]), dm[k],
                               k < 4 ? (void*)act[k] : nullptr, k < 4 ? c[k] : w, (int)r[k], (int)c[k],
                               k == 4 ? probs : nullptr, hw, st));
        }
        me_smooth_threshold<<<me_grid(hw), 256, 0, st>>>(probs, (int)h, (int)w, thr, masks_out + s * hw);
        count_launch();
        MB_CUDA(cudaGetLastError());
    }
    return me_tc_poll_error(net);
}

mb_status maskextend_run(mb_net* net, const uint8_t* em, const float* memb, int64_t zt, int64_t h, int64_t w,
                         const uint8_t* seeds, int64_t z0, int64_t n_steps, int dz, float thr, uint8_t* masks_out,
                         float* probs_out, cudaStream_t st) {
    (void)zt;
    if (n_steps == 0) return MB_OK;
    if (net->prec == MB_PREC_FP16)
        return maskextend_run_tc(net, em, memb, h, w, seeds, z0, n_steps, dz, thr, masks_out, probs_out, st);
    // geometry (dense): conv outputs and their input domains
    const int64_t r[5] = {h + 105, h + 98, h + 84, h + 56, h}, c[5] = {w + 105, w + 98, w + 84, w + 56, w};
    const int d[5] = {1, 2, 4, 8, 16}, dm[5] = {0, 1, 2, 4, 8};
    const int64_t cout[5] = {32, 40, 48, 56, 64};
    auto up = [](int64_t n) { return (n + 63) & ~(int64_t)63; };  // 256-byte aligned sub-buffers
    const int64_t n_in = up((h + 108) * (w + 108) * kMeCin);
    int64_t n_act[5];
    int64_t total = n_in;
    for (int k = 0; k < 5; ++k) {
        n_act[k] = up(r[k] * c[k] * cout[k]);
        total += n_act[k];
    }
    const int64_t n_prob = up(3 * h * w);
    total += n_prob;
    MB_TRY(net->ws.ensure((size_t)total * sizeof(float)));
    float* xin = static_cast<float*>(net->ws.ptr);
    float* act[5];
    act[0] = xin + n_in;
    for (int k = 1; k < 5; ++k) act[k] = act[k - 1] + n_act[k - 1];
    float* prob_tmp = act[4] + n_act[4];
    // SIMT weights
    const float* wts[5];
    const float* bs[5];
    {
        const float* q = net->d_simt;
        const int cin[5] = {kMeCin, 32, 40, 48, 56};
        for (int k = 0; k < 5; ++k) {
            wts[k] = q;
            bs[k] = q + (size_t)cin[k] * 16 * 2 * cout[k];
            q = bs[k] + 2 * cout[k];
        }
    }
    const float* head = bs[4] + 2 * cout[4];
    const int64_t hw = h * w;
    for (int64_t s = 0; s < n_steps; ++s) {
        const int64_t z = z0 + dz * s;
        MeMasks mk;
        me_masks(mk, seeds, masks_out, s, hw);
        me_assemble<float><<<me_grid((h + 108) * (w + 108)), 256, 0, st>>>(em, memb, mk, z, dz, (int)h, (int)w, xin);
        count_launch();
        MB_CUDA(cudaGetLastError());
        for (int k = 0; k < 5; ++k) {
            FmArgs a{};
            a.in = k == 0 ? xin : act[k - 1];
            a.in_slice = 0;
            a.in_pitch = k == 0 ? w + 108 : c[k - 1];
            a.in_rows = (int)(r[k] + 3 * d[k]);
            a.in_cols = (int)(c[k] + 3 * d[k]);
            a.d = d[k];
            a.dm = dm[k];
            a.in_stride = 1;
            a.out_h = (int)r[k];
            a.out_w = (int)c[k];
            a.out = act[k];
            a.out_slice = 0;
            a.out_pitch = c[k];
            a.wt = wts[k];
            a.bias = bs[k];
            switch (k) {
                case 0: MB_TRY((launch_fm<16, 8, 64, 8, FM_IN_F32, FM_OUT_MAXOUT, 4>(a, 1, st))); break;
                case 1: MB_TRY((launch_fm<32, 8, 80, 8, FM_IN_F32, FM_OUT_MAXOUT, 3>(a, 1, st))); break;
                case 2: MB_TRY((launch_fm<40, 4, 96, 8, FM_IN_F32, FM_OUT_MAXOUT, 2>(a, 1, st))); break;
                case 3: MB_TRY((launch_fm<48, 4, 112, 8, FM_IN_F32, FM_OUT_MAXOUT, 2>(a, 1, st))); break;
                default: MB_TRY((launch_fm<56, 4, 128, 8, FM_IN_F32, FM_OUT_MAXOUT, 2>(a, 1, st))); break;
            }
        }
        float* probs = probs_out ? probs_out + s * 3 * hw : prob_tmp;
        me_head<<<me_grid(hw), 256, 0, st>>>(act[4], (int)h, (int)w, head, probs);
        me_smooth_threshold<<<me_grid(hw), 256, 0, st>>>(probs, (int)h, (int)w, thr, masks_out + s * hw);
        count_launch(2);
        MB_CUDA(cudaGetLastError());
    }
    return MB_OK;
}

}  // namespace mb
