// fastmemb.cu - FastMemb in dense form on CUDA cores (FP32), one kernel per convolution.
//
// The network (Sec. 2.2, "A lightweight network architecture"): three [conv 4x4 -> max-out over
// 2 -> 2x2 stride-2 max-pool] stages, no transfer function, then conv 4x4 to two classes and a
// softmax. Dense computation (Sec. 2.2, "Accelerating dense computation") turns each stride-2
// pool into a stride-1 max-filter plus 2-factor sub-sampling; here that becomes a max-filter
// with dilation d and a conv with dilation 2d behind it (d = 1, 2, 4; the head has dilation 8).
//
// The convolution kernel (fm_conv.cuh) tiles each dilated conv by the paper's max-pooling
// fragments: a conv with dilation d restricted to one residue class (y mod d, x mod d) is a plain
// 4x4 conv on the d-strided sub-grid, so every CTA keeps the register reuse of an undilated conv.
// The previous stage's dilated max-filter is applied while staging; epilogues are max-out of
// adjacent channel pairs or the 2-class softmax p = 1 / (1 + exp(z0 - z1)).
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

#include "fm_conv.cuh"
#include "internal.h"

namespace mb {


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

// Tensor-core paths (BF16 or FP16): layer 1 on CUDA cores (FP32 arithmetic, 16-bit out); the two
// 32->64 dilated convs and the head on the tensor cores (fastmemb_tc.cu); activations between
// layers are 16-bit [slice][y][x][32] of the net's type.
mb_status tc_fastmemb_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
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
    uint16_t* act[kFmMaxConvs - 1];
    act[0] = static_cast<uint16_t*>(net->ws.ptr);
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
        if (net->prec == MB_PREC_FP16)
            MB_TRY((launch_fm<1, 1, 64, 8, FM_IN_U8, FM_OUT_MAXOUT_F16>(a, nz, st)));
        else
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
