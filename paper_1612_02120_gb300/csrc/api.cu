// api.cu - the extern "C" boundary of libmembrane: argument checks, net lifecycle, dispatch to
// the FP32 CUDA-core path or the tensor-core path, and host-memory slab streaming.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace mb {

static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

void clear_error() { g_err.clear(); }

mb_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    const char* base = strrchr(file, '/');
    set_error("%s:%d: %s: %s (%s)", base ? base + 1 : file, line, what, cudaGetErrorString(e),
              cudaGetErrorName(e));
    if (e == cudaErrorMemoryAllocation) return MB_ERR_OOM;
    return MB_ERR_CUDA;
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool fault_oom() {
    const char* v = getenv("MB_FAULT_OOM");
    return v && v[0] == '1';
}

mb_status dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (fault_oom()) {
        set_error("allocation of %zu bytes failed (MB_FAULT_OOM injected)", bytes);
        return MB_ERR_OOM;
    }
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MB_ERR_OOM : MB_ERR_CUDA;
    }
    return MB_OK;
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

mb_status Workspace::ensure(size_t need) {
    if (need <= bytes && ptr) return MB_OK;
    if (ptr) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize", __FILE__, __LINE__);
        dev_free(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    MB_TRY(dev_alloc(&ptr, need));
    bytes = need;
    return MB_OK;
}

void Workspace::release() {
    dev_free(ptr);
    ptr = nullptr;
    bytes = 0;
}

// Makes `dev` current for the scope of an API call and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static bool same_layer(const mb_layer_desc& a, int kind, int k, int cin, int cout, int relu) {
    const int dil = a.dilation == 0 ? 1 : a.dilation;
    const int mo = a.maxout_groups == 0 ? 1 : a.maxout_groups;
    return a.kind == kind && a.ksize == k && a.cin == cin && a.cout == cout && (a.relu != 0) == (relu != 0) &&
           dil == 1 && mo == 1;
}

static bool same_layer_dm(const mb_layer_desc& a, int kind, int k, int cin, int cout, int dil, int groups) {
    const int d = a.dilation == 0 ? 1 : a.dilation;
    const int mo = a.maxout_groups == 0 ? 1 : a.maxout_groups;
    return a.kind == kind && a.ksize == k && a.cin == cin && a.cout == cout && a.relu == 0 && d == dil &&
           mo == groups;
}

static int detect_family(const mb_layer_desc* L, int n) {
    if (n == 7 && same_layer_dm(L[0], MB_CONV, 4, 1, 32, 1, 2) && same_layer_dm(L[1], MB_MAXFILTER, 2, 32, 32, 1, 1) &&
        same_layer_dm(L[2], MB_CONV, 4, 32, 32, 2, 2) && same_layer_dm(L[3], MB_MAXFILTER, 2, 32, 32, 2, 1) &&
        same_layer_dm(L[4], MB_CONV, 4, 32, 32, 4, 2) && same_layer_dm(L[5], MB_MAXFILTER, 2, 32, 32, 4, 1) &&
        same_layer_dm(L[6], MB_HEAD_SOFTMAX2, 4, 32, 2, 8, 1))
        return FAMILY_FASTMEMB;
    if (n == 9 && same_layer_dm(L[0], MB_CONV, 4, 1, 32, 1, 2) && same_layer_dm(L[1], MB_MAXFILTER, 2, 32, 32, 1, 1) &&
        same_layer_dm(L[2], MB_CONV, 4, 32, 32, 2, 2) && same_layer_dm(L[3], MB_MAXFILTER, 2, 32, 32, 2, 1) &&
        same_layer_dm(L[4], MB_CONV, 4, 32, 32, 4, 2) && same_layer_dm(L[5], MB_MAXFILTER, 2, 32, 32, 4, 1) &&
        same_layer_dm(L[6], MB_CONV, 4, 32, 32, 8, 2) && same_layer_dm(L[7], MB_MAXFILTER, 2, 32, 32, 8, 1) &&
        same_layer_dm(L[8], MB_HEAD_SOFTMAX2, 4, 32, 2, 16, 1))
        return FAMILY_FASTMEMB_3NM;
    if (n == 10 && same_layer_dm(L[0], MB_CONV, 4, 12, 32, 1, 2) && same_layer_dm(L[1], MB_MAXFILTER, 2, 32, 32, 1, 1) &&
        same_layer_dm(L[2], MB_CONV, 4, 32, 40, 2, 2) && same_layer_dm(L[3], MB_MAXFILTER, 2, 40, 40, 2, 1) &&
        same_layer_dm(L[4], MB_CONV, 4, 40, 48, 4, 2) && same_layer_dm(L[5], MB_MAXFILTER, 2, 48, 48, 4, 1) &&
        same_layer_dm(L[6], MB_CONV, 4, 48, 56, 8, 2) && same_layer_dm(L[7], MB_MAXFILTER, 2, 56, 56, 8, 1) &&
        same_layer_dm(L[8], MB_CONV, 4, 56, 64, 16, 2) && same_layer_dm(L[9], MB_HEAD_SOFTMAX, 1, 64, 3, 1, 1))
        return FAMILY_MASKEXTEND;
    if (n == 6 && same_layer(L[0], MB_CONV, 5, 1, 32, 1) && same_layer(L[1], MB_MAXFILTER, 2, 32, 32, 0) &&
        same_layer(L[2], MB_CONV, 5, 32, 32, 1) && same_layer(L[3], MB_MAXFILTER, 2, 32, 32, 0) &&
        same_layer(L[4], MB_CONV, 5, 32, 32, 1) && same_layer(L[5], MB_HEAD_SIGMOID, 1, 32, 1, 0))
        return FAMILY_TEACHER;
    if (n == 3 && same_layer(L[0], MB_CONV, 3, 1, 16, 1) && same_layer(L[1], MB_CONV, 3, 16, 16, 1) &&
        same_layer(L[2], MB_HEAD_SIGMOID, 1, 16, 1, 0))
        return FAMILY_STUDENT;
    return 0;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of page-locked, mapped host memory at p (cudaHostAlloc / cudaHostRegister), or
// nullptr for any other memory.
static void* mapped_host_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    // the attributes describe the queried address; the offset term only matters if they name
    // the allocation's start instead
    const char* hp = a.hostPointer ? static_cast<const char*>(a.hostPointer) : static_cast<const char*>(p);
    return static_cast<char*>(a.devicePointer) + (static_cast<const char*>(p) - hp);
}

// Whether the device reads host memory through the host's own page tables: a coherent CPU-GPU
// link (NVLink-C2C), over which kernels stream host buffers at the rate this path needs.
static bool coherent_host_link(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return v != 0;
}

static mb_status check_ready(const mb_net* net) {
    if (!net) {
        set_error("net is NULL");
        return MB_ERR_INVALID_ARG;
    }
    if (!net->loaded) {
        set_error("weights not loaded (call mb_load_weights first)");
        return MB_ERR_NOT_READY;
    }
    if (net->prec == MB_PREC_FP8 && !net->calibrated) {
        set_error("FP8 net not calibrated (call mb_calibrate_fp8 first)");
        return MB_ERR_NOT_READY;
    }
    return MB_OK;
}

static int net_radius(const mb_net* net) {
    if (!net) return kTeacherRadius;
    switch (net->family) {
        case FAMILY_STUDENT: return kStudentRadius;
        case FAMILY_FASTMEMB: return kFastMembRadius;
        case FAMILY_FASTMEMB_3NM: return kFastMemb3nmRadius;
        case FAMILY_MASKEXTEND: return kFastMemb3nmRadius;
        default: return kTeacherRadius;
    }
}

// A slice must be larger than the net's radius for reflect-101 padding.
static mb_status check_net_slice(const mb_net* net, int64_t h, int64_t w) {
    const int R = net_radius(net);
    if (h <= R || w <= R) {
        set_error("slice %lldx%lld: this net's radius is %d, so h and w must be >= %d", (long long)h, (long long)w,
                  R, R + 1);
        return MB_ERR_SHAPE;
    }
    return MB_OK;
}

// MaskExtend reads a 12-map stack, not one uint8 slice: only mb_mask_extend runs it.
static mb_status check_map_net(const mb_net* net, const char* call) {
    if (net && net->family == FAMILY_MASKEXTEND) {
        set_error("%s: MaskExtend nets run through mb_mask_extend", call);
        return MB_ERR_UNSUPPORTED;
    }
    return MB_OK;
}

static mb_status check_slice(int64_t z, int64_t h, int64_t w) {
    if (z < 0) {
        set_error("negative slice count %lld", (long long)z);
        return MB_ERR_INVALID_ARG;
    }
    if (h < 8 || w < 8) {
        set_error("slice %lldx%lld: h and w must be >= 8 for reflect-101 padding by 7", (long long)h,
                  (long long)w);
        return MB_ERR_SHAPE;
    }
    if (h > (1 << 20) || w > (1 << 20)) {
        set_error("slice %lldx%lld exceeds 2^20 per side", (long long)h, (long long)w);
        return MB_ERR_SHAPE;
    }
    return MB_OK;
}

mb_status teacher_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                         int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                         int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st) {
    if (z == 0 || rows == 0 || cols == 0) return MB_OK;
    if (net->prec == MB_PREC_FP32)
        return simt_teacher_region(net, in, z, h, w, in_pitch, in_slice, y0, x0, rows, cols, out, out_pitch,
                                   out_slice, ot, st);
    mb_block b;
    b.in = in;
    b.z = z;
    b.h = h;
    b.w = w;
    b.in_pitch = in_pitch;
    b.in_slice_pitch = in_slice;
    b.out = out;
    b.out_pitch = out_pitch;
    b.out_slice_pitch = out_slice;
    return tc_infer_blocks(net, &b, 1, &y0, &x0, &rows, &cols, ot, st, false);
}

mb_status student_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                         int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                         int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st) {
    if (net->prec == MB_PREC_BF16)
        return st_tc_region(net, in, z, h, w, in_pitch, in_slice, y0, x0, rows, cols, out, out_pitch, out_slice, ot,
                            st);
    return simt_student_region(net, in, z, h, w, in_pitch, in_slice, y0, x0, rows, cols, out, out_pitch, out_slice,
                               ot, st);
}

static mb_status fastmemb_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                                 int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                                 int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st, int sub = 1) {
    if (net->prec == MB_PREC_BF16 || net->prec == MB_PREC_FP16)
        return tc_fastmemb_region(net, in, z, h, w, in_pitch, in_slice, y0, x0, rows, cols, out, out_pitch,
                                  out_slice, ot, st, sub);
    return simt_fastmemb_region(net, in, z, h, w, in_pitch, in_slice, y0, x0, rows, cols, out, out_pitch, out_slice,
                                ot, st, sub);
}

static mb_status net_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t y0,
                            int64_t x0, int64_t rows, int64_t cols, void* out, mb_out_type ot, cudaStream_t st) {
    if (is_fastmemb(net->family))
        return fastmemb_region(net, in, z, h, w, w, h * w, y0, x0, rows, cols, out, cols, rows * cols, ot, st);
    if (net->family == FAMILY_TEACHER)
        return teacher_region(net, in, z, h, w, w, h * w, y0, x0, rows, cols, out, cols, rows * cols, ot, st);
    if (z == 0) return MB_OK;
    return student_region(net, in, z, h, w, w, h * w, y0, x0, rows, cols, out, cols, rows * cols, ot, st);
}

// Host-memory volumes. Mapped page-locked buffers on a coherent link: the kernels access them
// directly. Otherwise z-slabs through double-buffered device slabs, H2D / compute / D2H on their
// own streams so copies overlap compute (the tensor-core teacher computes on two alternating
// streams, so one slab's launch tail overlaps the next launch).
static mb_status infer_host_volume(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, void* out,
                                   mb_out_type ot) {
    const size_t osz = ot == MB_OUT_F32 ? 4 : 1;
    const size_t in_slice = (size_t)h * w, out_slice = (size_t)h * w * osz;
    cudaStream_t* s = net->slab_streams;
    // Direct: the kernels load the input bytes from and store the maps to the host buffers over
    // the link, in the launches of the device path. A call then moves exactly the input and
    // output bytes across the link, with no device buffer and no exposed copy at either end. The
    // student's kernel (tens of Gvox/s) outruns what it gets from host memory this way (measured
    // 28.6 against 37.1 Gvox/s in slabs on 1024x1024x32), so student nets always stream slabs.
    if (net->host_io == MB_HOST_IO_AUTO && net->family != FAMILY_STUDENT && coherent_host_link(net->device)) {
        const void* mi = mapped_host_ptr(in);
        void* mo = mi ? mapped_host_ptr(out) : nullptr;
        if (mi && mo) {
            if (!s[1]) MB_CUDA(cudaStreamCreateWithFlags(&s[1], cudaStreamNonBlocking));
            MB_TRY(net_region(net, static_cast<const uint8_t*>(mi), z, h, w, 0, 0, h, w, mo, ot, s[1]));
            MB_CUDA(cudaStreamSynchronize(s[1]));
            return MB_OK;
        }
    }
    // Slabs of about 8 Mvox: large enough that one launch fills every SM, small enough that the
    // copies of neighbouring slabs overlap the compute (a 1024x1024x32 volume becomes 4 slabs);
    // at most 256 MB of device buffers per slab.
    int64_t slab = std::max<int64_t>(1, (int64_t)((8ll << 20) + h * w - 1) / (h * w));
    slab = std::min<int64_t>(slab, std::max<int64_t>(1, (int64_t)((256ull << 20) / (in_slice + out_slice))));
    slab = std::min<int64_t>(slab, z);
    if (z == 0) return MB_OK;
    constexpr int NB = 2;
    // device slabs, streams and events live with the net and are reused by later calls
    const size_t slab_bytes = (in_slice + out_slice) * (size_t)slab;
    MB_TRY(net->slab_ws.ensure(NB * slab_bytes));
    for (int i = 0; i < 4; ++i)
        if (!s[i]) MB_CUDA(cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking));
    // The fused tensor-core teacher keeps no device state between launches, so consecutive slabs
    // may compute on two streams: the next slab's CTAs start on the SMs the previous launch's
    // tail leaves idle. Paths with a shared workspace compute their slabs in order on one stream.
    const bool overlap = net->family == FAMILY_TEACHER && net->prec != MB_PREC_FP32;
    cudaEvent_t* ev_in = net->slab_events;
    cudaEvent_t* ev_comp = ev_in + NB;
    cudaEvent_t* ev_out = ev_comp + NB;
    for (int i = 0; i < 3 * NB; ++i)
        if (!net->slab_events[i]) MB_CUDA(cudaEventCreateWithFlags(&net->slab_events[i], cudaEventDisableTiming));
    mb_status rc = MB_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        rc = cuda_fail(e, what, __FILE__, __LINE__);
    };
    // Slab boundaries: with three or more slabs the first and the last are halved, so less of the
    // first upload and of the last download stays outside the overlap.
    std::vector<int64_t> zb{0};
    {
        const int64_t full = (z + slab - 1) / slab;
        const int64_t half = (slab + 1) / 2;
        if (full >= 3 && slab >= 2) {
            zb.push_back(half);
            while (zb.back() + slab < z - half) zb.push_back(zb.back() + slab);
            if (z - zb.back() > slab) zb.push_back(z - half);
        } else {
            while (zb.back() + slab < z) zb.push_back(zb.back() + slab);
        }
        zb.push_back(z);
    }
    const int64_t nslab = (int64_t)zb.size() - 1;
    for (int64_t k = 0; k < nslab && rc == MB_OK; ++k) {
        const int b = (int)(k % NB);
        const int64_t z0 = zb[(size_t)k], nz = zb[(size_t)k + 1] - z0;
        uint8_t* din = static_cast<uint8_t*>(net->slab_ws.ptr) + b * slab_bytes;
        uint8_t* dout = din + in_slice * slab;
        cudaError_t e = cudaSuccess;
        if (k >= NB) e = cudaStreamWaitEvent(s[0], ev_comp[b], 0);  // input buffer free
        if (e == cudaSuccess) e = cudaMemcpyAsync(din, in + z0 * in_slice, in_slice * nz, cudaMemcpyHostToDevice, s[0]);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[b], s[0]);
        cudaStream_t cs = overlap && (k & 1) ? s[3] : s[1];
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in[b], 0);
        if (e == cudaSuccess && k >= NB) e = cudaStreamWaitEvent(cs, ev_out[b], 0);  // output buffer free
        if (e != cudaSuccess) {
            fail(e, "slab H2D");
            break;
        }
        rc = net_region(net, din, nz, h, w, 0, 0, h, w, dout, ot, cs);
        if (rc != MB_OK) break;
        e = cudaEventRecord(ev_comp[b], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s[2], ev_comp[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<uint8_t*>(out) + z0 * out_slice, dout, out_slice * nz,
                                cudaMemcpyDeviceToHost, s[2]);
        if (e == cudaSuccess) e = cudaEventRecord(ev_out[b], s[2]);
        if (e != cudaSuccess) fail(e, "slab D2H");
    }
    for (int i = 0; i < 4; ++i) {
        cudaError_t e = cudaStreamSynchronize(s[i]);
        if (e != cudaSuccess && rc == MB_OK) fail(e, "cudaStreamSynchronize");
    }
    return rc;
}

static uint16_t f32_to_bf16_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);  // inf / nan passthrough
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;  // round to nearest even
    return (uint16_t)(u >> 16);
}

float bf16_round(float f) {
    uint32_t u = (uint32_t)f32_to_bf16_bits(f) << 16;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

}  // namespace mb

using namespace mb;

#define API_BEGIN clear_error();
#define API_GUARD(net)                                                  \
    DeviceGuard guard_((net)->device);                                  \
    if (guard_.err != cudaSuccess) return cuda_fail(guard_.err, "cudaSetDevice", __FILE__, __LINE__);

extern "C" {

const char* mb_status_string(mb_status s) {
    switch (s) {
        case MB_OK: return "MB_OK";
        case MB_ERR_INVALID_ARG: return "MB_ERR_INVALID_ARG";
        case MB_ERR_SHAPE: return "MB_ERR_SHAPE";
        case MB_ERR_OOM: return "MB_ERR_OOM";
        case MB_ERR_CUDA: return "MB_ERR_CUDA";
        case MB_ERR_TIMEOUT: return "MB_ERR_TIMEOUT";
        case MB_ERR_NOT_READY: return "MB_ERR_NOT_READY";
        case MB_ERR_UNSUPPORTED: return "MB_ERR_UNSUPPORTED";
    }
    return "MB_ERR_UNKNOWN";
}

const char* mb_last_error(void) { return g_err.c_str(); }

int64_t mb_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

mb_status mb_net_create(const mb_layer_desc* layers, int32_t n_layers, mb_precision prec, int32_t device,
                        mb_net** out_net) {
    API_BEGIN
    if (!out_net || !layers || n_layers <= 0) {
        set_error("mb_net_create: null argument or n_layers <= 0");
        return MB_ERR_INVALID_ARG;
    }
    *out_net = nullptr;
    if (prec != MB_PREC_FP32 && prec != MB_PREC_BF16 && prec != MB_PREC_FP8 && prec != MB_PREC_FP16) {
        set_error("mb_net_create: unknown precision %d", (int)prec);
        return MB_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n_layers; ++i) {
        const mb_layer_desc& L = layers[i];
        if (L.kind < MB_CONV || L.kind > MB_HEAD_SOFTMAX || L.ksize <= 0 || L.cin <= 0 || L.cout <= 0 ||
            L.dilation < 0 || L.maxout_groups < 0) {
            set_error("mb_net_create: layer %d is malformed", i);
            return MB_ERR_INVALID_ARG;
        }
    }
    const int fam = detect_family(layers, n_layers);
    if (!fam) {
        set_error("mb_net_create: no kernel for this layer stack (teacher 5x5/32, student 3x3/16, FastMemb, "
                  "FastMemb_3nm or MaskExtend only)");
        return MB_ERR_UNSUPPORTED;
    }
    if (fam == FAMILY_STUDENT && prec == MB_PREC_FP8) {
        set_error("mb_net_create: the student runs in FP32 or BF16");
        return MB_ERR_UNSUPPORTED;
    }
    if (fam == FAMILY_MASKEXTEND && prec != MB_PREC_FP32 && prec != MB_PREC_FP16) {
        set_error("mb_net_create: MaskExtend runs in FP32 or FP16");
        return MB_ERR_UNSUPPORTED;
    }
    if (fam != FAMILY_MASKEXTEND && !is_fastmemb(fam) && prec == MB_PREC_FP16) {
        set_error("mb_net_create: FP16 is a precision of the MaskExtend and FastMemb nets only");
        return MB_ERR_UNSUPPORTED;
    }
    if (is_fastmemb(fam) && prec == MB_PREC_FP8) {
        set_error("mb_net_create: FastMemb runs in FP32, BF16 or FP16");
        return MB_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    MB_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
        set_error("mb_net_create: device %d out of range (%d devices)", device, ndev);
        return MB_ERR_INVALID_ARG;
    }
    mb_net* net = new (std::nothrow) mb_net();
    if (!net) {
        set_error("mb_net_create: host allocation failed");
        return MB_ERR_OOM;
    }
    net->device = device;
    net->family = fam;
    net->prec = prec;
    net->layers.assign(layers, layers + n_layers);
    int64_t np = 0;
    for (const auto& L : net->layers)
        if (L.kind != MB_MAXFILTER) {
            const int64_t co = (int64_t)L.cout * (L.maxout_groups > 1 ? L.maxout_groups : 1);
            np += co * L.cin * L.ksize * L.ksize + co;
        }
    net->n_params = np;
    {
        DeviceGuard g(device);
        mb_status s = g.err == cudaSuccess ? MB_OK : cuda_fail(g.err, "cudaSetDevice", __FILE__, __LINE__);
        if (s == MB_OK) s = dev_alloc((void**)&net->d_queue, 64 * sizeof(int));
        if (s == MB_OK) {
            cudaError_t e = cudaMemset(net->d_queue, 0, 64 * sizeof(int));
            if (e != cudaSuccess) s = cuda_fail(e, "cudaMemset", __FILE__, __LINE__);
        }
        if (s != MB_OK) {
            dev_free(net->d_queue);
            delete net;
            return s;
        }
    }
    *out_net = net;
    return MB_OK;
}

mb_status mb_net_destroy(mb_net* net) {
    API_BEGIN
    if (!net) return MB_OK;
    {
        DeviceGuard g(net->device);
        cudaDeviceSynchronize();
        tc_release(net);
        fm_tc_release(net);
        me_tc_release(net);
        st_tc_release(net);
        dev_free(net->d_params);
        dev_free(net->d_simt);
        dev_free(net->d_queue);
        net->ws.release();
        net->ws2.release();
        net->slab_ws.release();
        for (cudaStream_t& st : net->slab_streams)
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t& ev : net->slab_events)
            if (ev) cudaEventDestroy(ev);
    }
    delete net;
    return MB_OK;
}

mb_status mb_net_param_count(const mb_net* net, int64_t* n_params) {
    API_BEGIN
    if (!net || !n_params) {
        set_error("mb_net_param_count: null argument");
        return MB_ERR_INVALID_ARG;
    }
    *n_params = net->n_params;
    return MB_OK;
}

mb_status mb_load_weights(mb_net* net, const float* params, int64_t n_params) {
    API_BEGIN
    if (!net || !params) {
        set_error("mb_load_weights: null argument");
        return MB_ERR_INVALID_ARG;
    }
    if (n_params != net->n_params) {
        set_error("mb_load_weights: got %lld parameters, the net has %lld", (long long)n_params,
                  (long long)net->n_params);
        return MB_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < n_params; ++i)
        if (!(params[i] == params[i]) || params[i] > 3.0e38f || params[i] < -3.0e38f) {
            set_error("mb_load_weights: parameter %lld is not finite", (long long)i);
            return MB_ERR_INVALID_ARG;
        }
    API_GUARD(net)
    net->host_params.assign(params, params + n_params);
    std::vector<float> fwd(params, params + n_params);
    if (net->family == FAMILY_STUDENT && net->prec == MB_PREC_BF16)
        for (auto& v : fwd) v = bf16_round(v);
    std::vector<float> packed;
    if (net->family == FAMILY_MASKEXTEND)
        me_pack(net, fwd.data(), packed);
    else
        simt_pack(net, fwd.data(), packed);
    if (!net->d_params) MB_TRY(dev_alloc((void**)&net->d_params, sizeof(float) * n_params));
    if (!net->d_simt) MB_TRY(dev_alloc((void**)&net->d_simt, sizeof(float) * packed.size()));
    net->simt_floats = packed.size();
    MB_CUDA(cudaMemcpy(net->d_params, params, sizeof(float) * n_params, cudaMemcpyHostToDevice));
    MB_CUDA(cudaMemcpy(net->d_simt, packed.data(), sizeof(float) * packed.size(), cudaMemcpyHostToDevice));
    net->calibrated = false;
    net->loaded = true;
    if (net->family == FAMILY_TEACHER && net->prec == MB_PREC_BF16) MB_TRY(tc_prepare(net));
    if (is_fastmemb(net->family) && (net->prec == MB_PREC_BF16 || net->prec == MB_PREC_FP16))
        MB_TRY(fm_tc_prepare(net));
    if (net->family == FAMILY_MASKEXTEND && net->prec == MB_PREC_FP16) MB_TRY(me_tc_prepare(net));
    return MB_OK;
}

mb_status mb_get_weights(const mb_net* net, float* params, int64_t n_params) {
    API_BEGIN
    if (!net || !params) {
        set_error("mb_get_weights: null argument");
        return MB_ERR_INVALID_ARG;
    }
    if (n_params != net->n_params) {
        set_error("mb_get_weights: got %lld parameters, the net has %lld", (long long)n_params,
                  (long long)net->n_params);
        return MB_ERR_INVALID_ARG;
    }
    if (!net->loaded) {
        set_error("mb_get_weights: weights not loaded");
        return MB_ERR_NOT_READY;
    }
    API_GUARD(net)
    MB_CUDA(cudaMemcpy(params, net->d_params, sizeof(float) * n_params, cudaMemcpyDeviceToHost));
    return MB_OK;
}

mb_status mb_calibrate_fp8(mb_net* net, const uint8_t* slices, int64_t n, int64_t h, int64_t w, float* amax_out,
                           void* stream) {
    API_BEGIN
    if (!net || !slices || n <= 0) {
        set_error("mb_calibrate_fp8: null argument or n <= 0");
        return MB_ERR_INVALID_ARG;
    }
    if (net->family != FAMILY_TEACHER || net->prec != MB_PREC_FP8) {
        set_error("mb_calibrate_fp8: only FP8 teacher nets are calibrated");
        return MB_ERR_UNSUPPORTED;
    }
    if (!net->loaded) {
        set_error("mb_calibrate_fp8: weights not loaded");
        return MB_ERR_NOT_READY;
    }
    MB_TRY(check_slice(n, h, w));
    API_GUARD(net)
    if (!is_device_ptr(slices)) {
        set_error("mb_calibrate_fp8: slices must be device memory");
        return MB_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    float* d_amax = nullptr;
    MB_TRY(dev_alloc((void**)&d_amax, 64 * sizeof(float)));
    mb_status s = simt_teacher_amax(net, slices, n, h, w, d_amax, st);
    float host[64];
    if (s == MB_OK) {
        cudaError_t e = cudaMemcpyAsync(host, d_amax, sizeof(host), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "amax readback", __FILE__, __LINE__);
    }
    dev_free(d_amax);
    if (s != MB_OK) return s;
    for (int m = 0; m < 2; ++m)
        for (int c = 0; c < 32; ++c) net->fp8_amax[m][c] = host[m * 32 + c];
    if (amax_out) memcpy(amax_out, host, sizeof(host));
    MB_TRY(tc_prepare(net));
    net->calibrated = true;
    return MB_OK;
}

mb_status mb_infer_volume(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, void* out,
                          mb_out_type out_type, void* stream) {
    API_BEGIN
    MB_TRY(check_ready(net));
    MB_TRY(check_map_net(net, "mb_infer_volume"));
    if ((!in || !out) && z > 0) {
        set_error("mb_infer_volume: null buffer");
        return MB_ERR_INVALID_ARG;
    }
    if (out_type != MB_OUT_F32 && out_type != MB_OUT_U8) {
        set_error("mb_infer_volume: unknown output type %d", (int)out_type);
        return MB_ERR_INVALID_ARG;
    }
    MB_TRY(check_slice(z, h, w));
    MB_TRY(check_net_slice(net, h, w));
    if (z == 0) return MB_OK;
    API_GUARD(net)
    const bool din = is_device_ptr(in), dout = is_device_ptr(out);
    if (din != dout) {
        set_error("mb_infer_volume: in and out must both be device or both host memory");
        return MB_ERR_INVALID_ARG;
    }
    if (!din) return infer_host_volume(net, in, z, h, w, out, out_type);
    return net_region(net, in, z, h, w, 0, 0, h, w, out, out_type, (cudaStream_t)stream);
}

mb_status mb_set_host_io(mb_net* net, int32_t mode) {
    API_BEGIN
    if (!net) {
        set_error("mb_set_host_io: net is NULL");
        return MB_ERR_INVALID_ARG;
    }
    if (mode != MB_HOST_IO_AUTO && mode != MB_HOST_IO_SLABS) {
        set_error("mb_set_host_io: unknown mode %d", (int)mode);
        return MB_ERR_INVALID_ARG;
    }
    net->host_io = mode;
    return MB_OK;
}

mb_status mb_infer_volume_subsampled(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int32_t factor,
                                     void* out, mb_out_type out_type, void* stream) {
    API_BEGIN
    MB_TRY(check_ready(net));
    MB_TRY(check_map_net(net, "mb_infer_volume_subsampled"));
    if ((!in || !out) && z > 0) {
        set_error("mb_infer_volume_subsampled: null buffer");
        return MB_ERR_INVALID_ARG;
    }
    if (out_type != MB_OUT_F32 && out_type != MB_OUT_U8) {
        set_error("mb_infer_volume_subsampled: unknown output type %d", (int)out_type);
        return MB_ERR_INVALID_ARG;
    }
    if (!is_fastmemb(net->family) || factor != 2) {
        set_error("mb_infer_volume_subsampled: only FastMemb nets with factor 2 (got factor %d)", (int)factor);
        return MB_ERR_UNSUPPORTED;
    }
    MB_TRY(check_slice(z, h, w));
    MB_TRY(check_net_slice(net, h, w));
    if (z == 0) return MB_OK;
    API_GUARD(net)
    if (!is_device_ptr(in) || !is_device_ptr(out)) {
        set_error("mb_infer_volume_subsampled: device pointers only");
        return MB_ERR_INVALID_ARG;
    }
    const int64_t h2 = (h + 1) / 2, w2 = (w + 1) / 2;
    return fastmemb_region(net, in, z, h, w, w, h * w, 0, 0, h, w, out, w2, h2 * w2, out_type, (cudaStream_t)stream,
                           2);
}

mb_status mb_infer_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t y0,
                          int64_t x0, int64_t rows, int64_t cols, void* out, mb_out_type out_type, void* stream) {
    API_BEGIN
    MB_TRY(check_ready(net));
    MB_TRY(check_map_net(net, "mb_infer_region"));
    if ((!in || !out) && z > 0) {
        set_error("mb_infer_region: null buffer");
        return MB_ERR_INVALID_ARG;
    }
    if (out_type != MB_OUT_F32 && out_type != MB_OUT_U8) {
        set_error("mb_infer_region: unknown output type");
        return MB_ERR_INVALID_ARG;
    }
    MB_TRY(check_slice(z, h, w));
    MB_TRY(check_net_slice(net, h, w));
    if (y0 < 0 || x0 < 0 || rows < 0 || cols < 0 || y0 + rows > h || x0 + cols > w) {
        set_error("mb_infer_region: region [%lld,+%lld) x [%lld,+%lld) outside the %lldx%lld slice",
                  (long long)y0, (long long)rows, (long long)x0, (long long)cols, (long long)h, (long long)w);
        return MB_ERR_SHAPE;
    }
    if (z == 0 || rows == 0 || cols == 0) return MB_OK;
    API_GUARD(net)
    if (!is_device_ptr(in) || !is_device_ptr(out)) {
        set_error("mb_infer_region: device pointers only");
        return MB_ERR_INVALID_ARG;
    }
    return net_region(net, in, z, h, w, y0, x0, rows, cols, out, out_type, (cudaStream_t)stream);
}

static mb_status check_blocks(const mb_net* net, const mb_block* blocks, int32_t n, mb_out_type ot) {
    MB_TRY(check_map_net(net, "mb_infer_batch"));
    if (!blocks && n > 0) {
        set_error("blocks is NULL");
        return MB_ERR_INVALID_ARG;
    }
    if (n < 0) {
        set_error("n_blocks < 0");
        return MB_ERR_INVALID_ARG;
    }
    if (ot != MB_OUT_F32 && ot != MB_OUT_U8) {
        set_error("unknown output type");
        return MB_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
        const mb_block& b = blocks[i];
        mb_status s = check_slice(b.z, b.h, b.w);
        if (s == MB_OK) s = check_net_slice(net, b.h, b.w);
        if (s != MB_OK) {
            set_error("block %d: %s", i, mb_last_error());
            return s;
        }
        if (b.z > 0 && (!b.in || !b.out)) {
            set_error("block %d: null buffer", i);
            return MB_ERR_INVALID_ARG;
        }
        if (b.in_pitch < b.w || b.in_slice_pitch < b.in_pitch * b.h || b.out_pitch < b.w ||
            b.out_slice_pitch < b.out_pitch * b.h) {
            set_error("block %d: pitches smaller than the block", i);
            return MB_ERR_INVALID_ARG;
        }
    }
    return MB_OK;
}

mb_status mb_infer_batch_per_block(mb_net* net, const mb_block* blocks, int32_t n_blocks, mb_out_type out_type,
                                   void* stream) {
    API_BEGIN
    MB_TRY(check_ready(net));
    MB_TRY(check_blocks(net, blocks, n_blocks, out_type));
    API_GUARD(net)
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n_blocks; ++i) {
        const mb_block& b = blocks[i];
        if (net->family == FAMILY_TEACHER) {
            MB_TRY(teacher_region(net, b.in, b.z, b.h, b.w, b.in_pitch, b.in_slice_pitch, 0, 0, b.h, b.w, b.out,
                                  b.out_pitch, b.out_slice_pitch, out_type, st));
        } else if (is_fastmemb(net->family)) {
            MB_TRY(fastmemb_region(net, b.in, b.z, b.h, b.w, b.in_pitch, b.in_slice_pitch, 0, 0, b.h, b.w, b.out,
                                   b.out_pitch, b.out_slice_pitch, out_type, st));
        } else if (b.z > 0) {
            MB_TRY(student_region(net, b.in, b.z, b.h, b.w, b.in_pitch, b.in_slice_pitch, 0, 0, b.h, b.w,
                                       b.out, b.out_pitch, b.out_slice_pitch, out_type, st));
        }
    }
    return MB_OK;
}

mb_status mb_infer_batch(mb_net* net, const mb_block* blocks, int32_t n_blocks, mb_out_type out_type,
                         void* stream) {
    API_BEGIN
    MB_TRY(check_ready(net));
    MB_TRY(check_blocks(net, blocks, n_blocks, out_type));
    if (n_blocks == 0) return MB_OK;
    if (net->family != FAMILY_TEACHER || net->prec == MB_PREC_FP32)
        return mb_infer_batch_per_block(net, blocks, n_blocks, out_type, stream);
    API_GUARD(net)
    std::vector<int64_t> y0(n_blocks, 0), x0(n_blocks, 0), rows(n_blocks), cols(n_blocks);
    for (int i = 0; i < n_blocks; ++i) {
        rows[i] = blocks[i].h;
        cols[i] = blocks[i].w;
    }
    return tc_infer_blocks(net, blocks, n_blocks, y0.data(), x0.data(), rows.data(), cols.data(), out_type,
                           (cudaStream_t)stream, true);
}

mb_status mb_autotune_batch(mb_net* net, const mb_block* blocks, int32_t n_blocks, mb_out_type out_type,
                            const char* cache_path, int32_t* choice_out, void* stream) {
    API_BEGIN
    MB_TRY(check_ready(net));
    MB_TRY(check_blocks(net, blocks, n_blocks, out_type));
    if (net->family != FAMILY_TEACHER || net->prec == MB_PREC_FP32) {
        set_error("mb_autotune_batch: only the tensor-core teacher (BF16/FP8) has tunables");
        return MB_ERR_UNSUPPORTED;
    }
    int64_t vox = 0;
    for (int i = 0; i < n_blocks; ++i) vox += blocks[i].z * blocks[i].h * blocks[i].w;
    if (vox == 0) {
        set_error("mb_autotune_batch: the batch has no voxels to time");
        return MB_ERR_INVALID_ARG;
    }
    API_GUARD(net)
    return tc_autotune_batch(net, blocks, n_blocks, out_type, cache_path, choice_out, (cudaStream_t)stream);
}

mb_status mb_student_loss_grad(mb_net* student, const uint8_t* in, const float* target, int64_t n, int64_t h,
                               int64_t w, double* loss, float* grad, void* stream) {
    API_BEGIN
    MB_TRY(check_ready(student));
    if (student->family != FAMILY_STUDENT) {
        set_error("mb_student_loss_grad: not a student net");
        return MB_ERR_UNSUPPORTED;
    }
    if (!in || !target || !loss || !grad || n <= 0) {
        set_error("mb_student_loss_grad: null argument or n <= 0");
        return MB_ERR_INVALID_ARG;
    }
    MB_TRY(check_slice(n, h, w));
    API_GUARD(student)
    return student_loss_grad(student, in, target, n, h, w, loss, grad, (cudaStream_t)stream);
}

mb_status mb_student_train(mb_net* student, const uint8_t* in, const float* target, int64_t n, int64_t h,
                           int64_t w, const mb_train_cfg* cfg, const char* ckpt_path, float* loss_curve,
                           void* stream) {
    API_BEGIN
    MB_TRY(check_ready(student));
    if (student->family != FAMILY_STUDENT) {
        set_error("mb_student_train: not a student net");
        return MB_ERR_UNSUPPORTED;
    }
    if (!in || !target || !cfg || n <= 0 || cfg->batch <= 0 || cfg->steps < 0 || cfg->ckpt_every < 0 ||
        !(cfg->lr > 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) || !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) ||
        !(cfg->eps > 0.f)) {
        set_error("mb_student_train: bad arguments");
        return MB_ERR_INVALID_ARG;
    }
    MB_TRY(check_slice(n, h, w));
    API_GUARD(student)
    return student_train(student, in, target, n, h, w, cfg, ckpt_path, loss_curve, (cudaStream_t)stream);
}

mb_status mb_infer_cascade(mb_net* student, mb_net* teacher, const uint8_t* in, int64_t z, int64_t h, int64_t w,
                           float* out, int32_t tile, float lo, float hi, float max_frac, double* fallback_rate,
                           uint8_t* tile_flags, void* stream) {
    API_BEGIN
    MB_TRY(check_ready(student));
    MB_TRY(check_ready(teacher));
    if (student->family != FAMILY_STUDENT || teacher->family != FAMILY_TEACHER) {
        set_error("mb_infer_cascade: needs a student net and a teacher net");
        return MB_ERR_INVALID_ARG;
    }
    if (student->device != teacher->device) {
        set_error("mb_infer_cascade: student and teacher on different devices");
        return MB_ERR_INVALID_ARG;
    }
    if (!in || !out || !fallback_rate || tile < 8 || !(lo <= hi) || !(max_frac >= 0.f)) {
        set_error("mb_infer_cascade: bad arguments");
        return MB_ERR_INVALID_ARG;
    }
    MB_TRY(check_slice(z, h, w));
    API_GUARD(student)
    return cascade(student, teacher, in, z, h, w, out, tile, lo, hi, max_frac, fallback_rate, tile_flags,
                   (cudaStream_t)stream);
}

mb_status mb_mask_extend_dir(mb_net* net, const uint8_t* em, const float* membrane, int64_t z, int64_t h, int64_t w,
                             const uint8_t* seed_masks, int64_t z0, int64_t n_steps, int32_t direction, float threshold,
                             uint8_t* masks_out, float* probs_out, void* stream) {
    API_BEGIN
    MB_TRY(check_ready(net));
    if (net->family != FAMILY_MASKEXTEND) {
        set_error("mb_mask_extend: not a MaskExtend net");
        return MB_ERR_UNSUPPORTED;
    }
    if (!em || !membrane || !seed_masks || (!masks_out && n_steps > 0) || n_steps < 0 || !(threshold == threshold) ||
        (direction != 1 && direction != -1)) {
        set_error("mb_mask_extend: null buffer or bad arguments (direction must be +1 or -1)");
        return MB_ERR_INVALID_ARG;
    }
    MB_TRY(check_slice(z, h, w));
    MB_TRY(check_net_slice(net, h, w));
    // sections read: membrane maps 2 before z0 .. 2 after the last step, along the direction
    const int64_t lo = direction > 0 ? z0 - 2 : z0 - n_steps - 1;
    const int64_t hi = direction > 0 ? z0 + n_steps + 1 : z0 + 2;
    if (n_steps > 0 && (lo < 0 || hi >= z)) {
        set_error("mb_mask_extend: sections %lld .. %lld must lie in the stack of %lld (z0 %lld, %lld steps, "
                  "direction %d)",
                  (long long)lo, (long long)hi, (long long)z, (long long)z0, (long long)n_steps, (int)direction);
        return MB_ERR_SHAPE;
    }
    if (n_steps == 0) return MB_OK;
    API_GUARD(net)
    if (!is_device_ptr(em) || !is_device_ptr(membrane) || !is_device_ptr(seed_masks) || !is_device_ptr(masks_out) ||
        (probs_out && !is_device_ptr(probs_out))) {
        set_error("mb_mask_extend: device pointers only");
        return MB_ERR_INVALID_ARG;
    }
    return maskextend_run(net, em, membrane, z, h, w, seed_masks, z0, n_steps, (int)direction, threshold, masks_out,
                          probs_out, (cudaStream_t)stream);
}

mb_status mb_mask_extend(mb_net* net, const uint8_t* em, const float* membrane, int64_t z, int64_t h, int64_t w,
                         const uint8_t* seed_masks, int64_t z0, int64_t n_steps, float threshold, uint8_t* masks_out,
                         float* probs_out, void* stream) {
    return mb_mask_extend_dir(net, em, membrane, z, h, w, seed_masks, z0, n_steps, 1, threshold, masks_out,
                              probs_out, stream);
}

}  // extern "C"
