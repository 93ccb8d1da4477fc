// internal.h - host-side internals shared by the translation units of libmembrane.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/membrane.h"

namespace mb {

enum Family { FAMILY_TEACHER = 1, FAMILY_STUDENT = 2, FAMILY_FASTMEMB = 3, FAMILY_FASTMEMB_3NM = 4, FAMILY_MASKEXTEND = 5 };

// Teacher geometry: conv5x5 x3 with two 2x2 max-filters -> receptive radius 7.
constexpr int kTeacherRadius = 7;
constexpr int kTeacherC = 32;
// Student geometry: conv3x3 x2 -> radius 2.
constexpr int kStudentRadius = 2;
constexpr int kStudentC = 16;
// FastMemb dense form: conv4x4 (dilation 1, 2, 4) with max-out 2, max-filters (1, 2, 4), conv4x4
// dilation 8 -> radius 26 (53x53 field of view).
constexpr int kFastMembRadius = 26;
// FastMemb_3nm: one more stage (dilation 8 conv and max-filter, head at 16) -> radius 54 (109x109).
constexpr int kFastMemb3nmRadius = 54;
inline bool is_fastmemb(int family) { return family == FAMILY_FASTMEMB || family == FAMILY_FASTMEMB_3NM; }
// convolutions of a FastMemb family (conv1, the 32->64 middle convs, the head)
inline int fastmemb_convs(int family) { return family == FAMILY_FASTMEMB_3NM ? 5 : 4; }

void set_error(const char* fmt, ...);
void clear_error();
mb_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);
void count_launch(int n = 1);
bool fault_oom();

#define MB_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ::mb::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define MB_TRY(call)                      \
    do {                                  \
        mb_status s_ = (call);            \
        if (s_ != MB_OK) return s_;       \
    } while (0)

mb_status dev_alloc(void** p, size_t bytes);
void dev_free(void* p);

// A growable device scratch buffer owned by a net.
struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
    mb_status ensure(size_t need);
    void release();
};

struct GraphCacheEntry;

}  // namespace mb

struct mb_net {
    int device = 0;
    int family = 0;
    mb_precision prec = MB_PREC_FP32;
    std::vector<mb_layer_desc> layers;
    int64_t n_params = 0;
    std::vector<float> host_params;  // FP32 master copy on the host
    bool loaded = false;
    bool calibrated = false;
    float* d_params = nullptr;   // FP32 parameters, API layout (student: the master copy)
    float* d_simt = nullptr;     // SIMT layout: per conv layer Wt[ci][ky][kx][co], b[co]; head w, b
    size_t simt_floats = 0;
    void* tc_state = nullptr;    // tensor-core path state (packed operands, constants), tc_conv.cu
    void* fm_state = nullptr;    // FastMemb tensor-core state (packed operands, error word), fastmemb_tc.cu
    void* me_state = nullptr;    // MaskExtend tensor-core state (packed operands, error word), maskextend_tc.cu
    void* st_state = nullptr;    // student tensor-core state (packed operands, error word), student_tc.cu
    float fp8_amax[2][32] = {};
    mb::Workspace ws;            // layered FP32 path activations
    mb::Workspace ws2;           // student training / cascade scratch
    mb::Workspace slab_ws;       // host-buffer streaming: double-buffered device slabs
    cudaStream_t slab_streams[4] = {};  // H2D, compute, D2H, second compute stream (overlapping slabs)
    int host_io = 0;             // mb_host_io: 0 direct host access where possible, 1 always slabs
    cudaEvent_t slab_events[6] = {};                              // per buffer: in, comp, out
    // persistent kernel tuning
    int rows_per_item = 64;
    int stages = 6;  // teacher A-ring depth (a compiled candidate; set by the autotuner or mb_set_tuning)
    bool tuned = false;
    // batch graph cache
    std::vector<mb::GraphCacheEntry*> graphs;
    int* d_queue = nullptr;      // work-queue counter + error word (device)
};

namespace mb {

// SIMT (FP32 arithmetic) layered path: conv kernels with activations in a workspace.
mb_status simt_teacher_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w,
                              int64_t in_pitch, int64_t in_slice, int64_t y0, int64_t x0, int64_t rows,
                              int64_t cols, void* out, int64_t out_pitch, int64_t out_slice,
                              mb_out_type ot, cudaStream_t st);
mb_status simt_student_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w,
                              int64_t in_pitch, int64_t in_slice, int64_t y0, int64_t x0, int64_t rows,
                              int64_t cols, void* out, int64_t out_pitch, int64_t out_slice,
                              mb_out_type ot, cudaStream_t st);
// FastMemb region (FP32 / BF16); sub = 1: the dense map, sub = 2: the map at even rows and columns
// of the region (out is ceil(rows/2) x ceil(cols/2)).
mb_status simt_fastmemb_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w,
                               int64_t in_pitch, int64_t in_slice, int64_t y0, int64_t x0, int64_t rows,
                               int64_t cols, void* out, int64_t out_pitch, int64_t out_slice,
                               mb_out_type ot, cudaStream_t st, int sub);
mb_status tc_fastmemb_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w,
                             int64_t in_pitch, int64_t in_slice, int64_t y0, int64_t x0, int64_t rows,
                             int64_t cols, void* out, int64_t out_pitch, int64_t out_slice,
                             mb_out_type ot, cudaStream_t st, int sub);
// FastMemb tensor-core layers (fastmemb_tc.cu): pack the B operands of the 32->64 convs and the
// head (split BF16, or FP16 for FP16 nets), launch one (the head ends with the softmax, FP32 or
// uint8 out), poll the device-side wait error word.
mb_status fm_tc_prepare(mb_net* net);
void fm_tc_release(mb_net* net);
mb_status fm_tc_poll_error(mb_net* net);
// in: [slice][src_rows][src_cols(pitch)][32] BF16 or FP16 (the net's type); the conv reads input
// (r, c) = 2x2 max (dilation dm) at source (stride r, stride c), for r < in_rows, c < in_cols.
// layer: 0-based index of the conv after conv1; the last one is the head.
mb_status fm_tc_layer(mb_net* net, int layer, const void* in, int64_t in_slice, int64_t in_pitch, int64_t src_rows,
                      int64_t src_cols, int in_rows, int in_cols, int dm, int stride, void* out, int64_t out_slice,
                      int64_t out_pitch, int out_h, int out_w, int d, int nz, int out_u8, cudaStream_t st);
// MaskExtend (maskextend.cu): SIMT weight layout, and the +z transfer recursion (device pointers).
void me_pack(const mb_net* net, const float* params, std::vector<float>& out);
// MaskExtend FP16 tensor-core convs (maskextend_tc.cu). layer 0..4; in: [src rows][in_pitch][cs] FP16;
// the conv reads input (r, c) = 2x2 max (dilation dm) at source (r, c), r < in_rows, c < in_cols;
// layers 0-3 write FP16 features [out_h][out_pitch][N/2]; layer 4 writes the 3 class probabilities
// [3][out_h][out_pitch] (planes probs_plane apart).
mb_status me_tc_prepare(mb_net* net);
void me_tc_release(mb_net* net);
mb_status me_tc_poll_error(mb_net* net);
mb_status me_tc_layer(mb_net* net, int layer, const void* in, int64_t in_pitch, int cs, int in_rows, int in_cols,
                      int dm, void* out, int64_t out_pitch, int out_h, int out_w, float* probs, int64_t probs_plane,
                      cudaStream_t st);
mb_status maskextend_run(mb_net* net, const uint8_t* em, const float* memb, int64_t zt, int64_t h, int64_t w,
                         const uint8_t* seeds, int64_t z0, int64_t n_steps, int dz, float thr, uint8_t* masks_out,
                         float* probs_out, cudaStream_t st);
// BF16 student inference on the tensor cores (student_tc.cu), same arguments as simt_student_region;
// student_region picks it for BF16 nets and the CUDA-core path for FP32 nets.
mb_status st_tc_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                       int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                       int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st);
void st_tc_release(mb_net* net);
mb_status student_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                         int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                         int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st);
// FP32 teacher activations after the two max-filters: per-channel amax over n slices (device out[64]).
mb_status simt_teacher_amax(mb_net* net, const uint8_t* in, int64_t n, int64_t h, int64_t w, float* d_amax,
                            cudaStream_t st);
// Pack the SIMT weight layout from the FP32 API layout (host side).
void simt_pack(const mb_net* net, const float* params, std::vector<float>& out);

// Tensor-core fused path.
mb_status tc_prepare(mb_net* net);   // pack BF16 / FP8 weights from host_params (+ calibration)
void tc_release(mb_net* net);
mb_status tc_poll_error(mb_net* net);  // MB_ERR_TIMEOUT if a launch recorded a timed-out wait
struct TcItem;                       // work item (device layout in tc_conv.cu)
mb_status tc_infer_blocks(mb_net* net, const mb_block* blocks, int n_blocks, const int64_t* y0,
                          const int64_t* x0, const int64_t* rows, const int64_t* cols, mb_out_type ot,
                          cudaStream_t st, bool use_graph);
// Autotuner timed on the caller's own batch (its outputs are written by every candidate).
mb_status tc_autotune_batch(mb_net* net, const mb_block* blocks, int n_blocks, mb_out_type ot, const char* cache_path,
                            int32_t* choice, cudaStream_t st);

// Student training and cascade.
mb_status student_loss_grad(mb_net* s, const uint8_t* in, const float* tgt, int64_t n, int64_t h, int64_t w,
                            double* loss, float* grad, cudaStream_t st);
mb_status student_train(mb_net* s, const uint8_t* in, const float* tgt, int64_t n, int64_t h, int64_t w,
                        const mb_train_cfg* cfg, const char* ckpt, float* curve, cudaStream_t st);
mb_status cascade(mb_net* s, mb_net* t, const uint8_t* in, int64_t z, int64_t h, int64_t w, float* out,
                  int tile, float lo, float hi, float max_frac, double* rate, uint8_t* flags,
                  cudaStream_t st);

// Teacher dispatch used by the API, the batch comparison path and the cascade.
mb_status teacher_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t in_pitch,
                         int64_t in_slice, int64_t y0, int64_t x0, int64_t rows, int64_t cols, void* out,
                         int64_t out_pitch, int64_t out_slice, mb_out_type ot, cudaStream_t st);

}  // namespace mb
