// noalloc.cu - mb_infer_volume_noalloc: the FP32 CUDA-core teacher path with its layer-1 and
// layer-2 activations in a fixed, file-scope device array instead of a cudaMalloc'd workspace.
//
// Who needs it: callers that must not allocate device memory once they are running, for example
// a streaming service that fixes its memory budget at start-up, or a pipeline that cannot afford
// the device-wide synchronisation that cudaMalloc/cudaFree may cause while other streams work.
// This call allocates nothing: the scratch is the static array below, which every GPU that loads
// the library holds until the process exits.
//
// The array is shared by all calls on a device and keeps the last call's contents; every
// activation a call reads was written earlier in the same call, so nothing needs clearing.
// Calls whose work overlaps on the GPU (different streams, or host threads) race on the array.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "simt_conv.cuh"

namespace mb {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;  // 64 MiB per device
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float)];

static std::mutex g_noalloc_mu;
static float* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once per device. In host
// code the array's name stands for a host-side shadow, not a device address, so the address must
// come from cudaGetSymbolAddress with this device current.
static mb_status noalloc_scratch(int dev, float** out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("mb_infer_volume_noalloc: device %d beyond the %d supported", dev, kNoAllocMaxDevices);
        return MB_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return MB_OK;
}

// Scratch floats for `nz` slices of a band of `rows` output rows and `cols` columns: the layer-1
// activations (rows + 10) x (cols + 10) and the layer-2 activations (rows + 5) x (cols + 5), 32
// channels each. A call uses the largest band of a slice that fits (all h rows if they do), then
// as many slices of that band per launch as fit.
static size_t band_floats(int64_t nz, int64_t rows, int64_t cols) {
    return (size_t)nz * (size_t)((rows + 10) * (cols + 10) + (rows + 5) * (cols + 5)) * 32;
}

// The three layer launches of the FP32 path for output rows [y0, y0+rows) of nz slices, with the
// activations in `scratch`.
static mb_status noalloc_band(const mb_net* net, const uint8_t* in, int nz, int64_t h, int64_t w, int64_t y0,
                              int64_t rows, void* out, mb_out_type ot, float* scratch, cudaStream_t st) {
    const int64_t cols = w, r1 = rows + 10, c1 = cols + 10, r2 = rows + 5, c2 = cols + 5;
    float* act1 = scratch;
    float* act2 = act1 + (size_t)nz * r1 * c1 * 32;
    const float* w1 = net->d_simt;
    const float* b1 = w1 + 25 * 32;
    const float* w2 = b1 + 32;
    const float* b2 = w2 + 25 * 32 * 32;
    const float* w3 = b2 + 32;
    const float* b3 = w3 + 25 * 32 * 32;
    const float* hw = b3 + 32;
    ConvArgs a{};
    a.in = in;
    a.in_slice = h * w;
    a.in_pitch = w;
    a.in_rows = (int)(r1 + 4);
    a.in_cols = (int)(c1 + 4);
    a.src_h = (int)h;
    a.src_w = (int)w;
    a.off_y = (int)(y0 - 7);
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
    ConvArgs c{};
    c.in = act2;
    c.in_slice = r2 * c2 * 32;
    c.in_pitch = c2;
    c.in_rows = (int)(rows + 4);
    c.in_cols = (int)(cols + 4);
    c.out_h = (int)rows;
    c.out_w = (int)cols;
    c.out_slice = h * w;
    c.out_pitch = w;
    c.wt = w3;
    c.bias = b3;
    c.head_w = hw;
    if (ot == MB_OUT_F32) {
        c.out = static_cast<float*>(out) + y0 * w;
        MB_TRY((launch_conv<5, 32, 32, 8, IN_F32_MAXF, OUT_HEAD_F32>(c, nz, st)));
    } else {
        c.out = static_cast<uint8_t*>(out) + y0 * w;
        MB_TRY((launch_conv<5, 32, 32, 8, IN_F32_MAXF, OUT_HEAD_U8>(c, nz, st)));
    }
    return MB_OK;
}

}  // namespace mb

using namespace mb;

extern "C" mb_status mb_infer_volume_noalloc(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w,
                                             void* out, mb_out_type out_type, void* stream) {
    clear_error();
    if (!net || ((!in || !out) && z > 0)) {
        set_error("mb_infer_volume_noalloc: null argument");
        return MB_ERR_INVALID_ARG;
    }
    if (out_type != MB_OUT_F32 && out_type != MB_OUT_U8) {
        set_error("mb_infer_volume_noalloc: unknown output type %d", (int)out_type);
        return MB_ERR_INVALID_ARG;
    }
    if (!net->loaded) {
        set_error("mb_infer_volume_noalloc: weights not loaded");
        return MB_ERR_NOT_READY;
    }
    if (net->family != FAMILY_TEACHER || net->prec != MB_PREC_FP32) {
        set_error("mb_infer_volume_noalloc: FP32 teacher nets only");
        return MB_ERR_UNSUPPORTED;
    }
    if (z < 0 || h < 8 || w < 8) {
        set_error("mb_infer_volume_noalloc: bad volume %lldx%lldx%lld (slices need h, w >= 8)", (long long)z,
                  (long long)h, (long long)w);
        return z < 0 ? MB_ERR_INVALID_ARG : MB_ERR_SHAPE;
    }
    if (h > (1 << 20) || w > (1 << 20)) {
        set_error("mb_infer_volume_noalloc: slice %lldx%lld exceeds 2^20 per side", (long long)h, (long long)w);
        return MB_ERR_SHAPE;
    }
    const size_t cap = kNoAllocScratchBytes / sizeof(float);
    if (band_floats(1, 1, w) > cap) {
        set_error("mb_infer_volume_noalloc: slice width %lld needs %zu bytes of scratch for one row, beyond the "
                  "%zu-byte maximum",
                  (long long)w, band_floats(1, 1, w) * sizeof(float), kNoAllocScratchBytes);
        return MB_ERR_SHAPE;
    }
    if (z == 0) return MB_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != net->device) {
        cudaError_t e = cudaSetDevice(net->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice", __FILE__, __LINE__);
    }
    float* scratch = nullptr;
    mb_status rc = noalloc_scratch(net->device, &scratch);
    if (rc == MB_OK) {
        // largest row band of one slice that fits, then as many slices of that band as fit
        int64_t rows = std::min<int64_t>(h, 1);
        while (rows < h && band_floats(1, std::min<int64_t>(h, rows * 2), w) <= cap) rows = std::min<int64_t>(h, rows * 2);
        while (rows < h && band_floats(1, rows + 1, w) <= cap) ++rows;
        const int64_t nz = std::max<int64_t>(1, std::min<int64_t>({z, 65535, (int64_t)(cap / band_floats(1, rows, w))}));
        const size_t osz = out_type == MB_OUT_F32 ? 4 : 1;
        for (int64_t z0 = 0; z0 < z && rc == MB_OK; z0 += nz) {
            const int n = (int)std::min<int64_t>(nz, z - z0);
            for (int64_t y0 = 0; y0 < h && rc == MB_OK; y0 += rows) {
                const int64_t r = std::min<int64_t>(rows, h - y0);
                rc = noalloc_band(net, in + z0 * h * w, n, h, w, y0, r,
                                  static_cast<uint8_t*>(out) + (size_t)(z0 * h * w) * osz, out_type, scratch,
                                  (cudaStream_t)stream);
            }
        }
    }
    if (prev >= 0 && prev != net->device) cudaSetDevice(prev);
    return rc;
}
