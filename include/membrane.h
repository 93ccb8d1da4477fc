/*
 * membrane.h - C ABI of libmembrane: dense per-pixel membrane-probability inference by a
 * shallow CNN over uint8 EM image stacks, on one GB300 (sm_103a).
 *
 * The operation (Sec. 2.1 "Membrane classification"; Sec. 2.2 "A lightweight network
 * architecture" and "Accelerating dense computation"): every pixel of every slice gets the
 * probability that it lies on a neuronal membrane, computed densely (all pixels in one pass,
 * max-pooling replaced by stride-1 max-filtering) by a stack of valid cross-correlations with
 * bias and ReLU, 2x2 stride-1 max-filters, and a 1x1 head with a sigmoid (for two classes the
 * softmax of Sec. 2.2 equals the sigmoid of the logit difference). Each slice is mirror-padded
 * (reflect-101: index -t for t < 0 and 2(n-1)-t for t > n-1) by the network's radius so the map
 * has the slice's size; the input pixel value is u/255. Slices and blocks are independent
 * (Sec. 2 "Block merging": the stack is split into blocks processed independently).
 *
 * Conventions of every call:
 *  - Every call returns an mb_status; no C++ exception crosses this boundary. On failure,
 *    mb_last_error() returns a thread-local message with the detail.
 *  - The caller owns all input and output buffers. The library owns its weights, plans and
 *    workspaces (released by mb_net_destroy).
 *  - Pointers are device pointers unless a call says otherwise. Calls on device pointers are
 *    asynchronous on `stream` (a cudaStream_t; NULL = the legacy default stream). Calls given
 *    host pointers are synchronous on return.
 *  - Sizes are element counts; pitches are in elements of the buffer's type.
 *  - Slices need h and w above the net's radius so reflect-101 padding is defined (>= 8 for the
 *    teacher and student, >= 27 for FastMemb, >= 55 for FastMemb_3nm); else MB_ERR_SHAPE.
 *  - A net/precision combination without a kernel returns MB_ERR_UNSUPPORTED.
 *  - Host-side fault injection for tests: environment MB_FAULT_OOM=1 makes every library
 *    allocation fail with MB_ERR_OOM.
 */
#ifndef MEMBRANE_H
#define MEMBRANE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mb_net mb_net; /* opaque, library-owned */

typedef enum {
    MB_OK = 0,
    MB_ERR_INVALID_ARG = 1, /* null pointer, bad enum, inconsistent sizes */
    MB_ERR_SHAPE = 2,       /* h or w below 8, or a size beyond a stated maximum */
    MB_ERR_OOM = 3,         /* device or pinned-host allocation failed */
    MB_ERR_CUDA = 4,        /* a CUDA runtime/driver call failed (detail in mb_last_error) */
    MB_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    MB_ERR_NOT_READY = 6,   /* weights not loaded, or FP8 net not calibrated */
    MB_ERR_UNSUPPORTED = 7  /* no kernel for this net / precision / option */
} mb_status;

typedef enum { MB_PREC_FP32 = 0, MB_PREC_BF16 = 1, MB_PREC_FP8 = 2, MB_PREC_FP16 = 3 } mb_precision;
typedef enum { MB_OUT_F32 = 0, MB_OUT_U8 = 1 } mb_out_type;
/* How mb_infer_volume moves a volume whose buffers are both in host memory (mb_set_host_io). */
typedef enum { MB_HOST_IO_AUTO = 0, MB_HOST_IO_SLABS = 1 } mb_host_io;
typedef enum {
    MB_CONV = 0,
    MB_MAXFILTER = 1,
    MB_HEAD_SIGMOID = 2,
    MB_HEAD_SOFTMAX2 = 3,
    MB_HEAD_SOFTMAX = 4
} mb_layer_kind;

/*
 * One layer of a network description (Sec. 2.2 describes the networks in prose as alternating
 * convolution / max-pooling layers, which dense computation turns into max-filters).
 *   MB_CONV:          ksize x ksize valid cross-correlation cin -> cout*G with dilation d
 *                     (y[i][j] = b + sum W[ky][kx] x[i + d ky][j + d kx]), + bias, ReLU if relu,
 *                     then max-out over G = maxout_groups adjacent channels (channel c of the
 *                     output is the max of conv channels c*G .. c*G + G-1). Parameters
 *                     W[cout*G][cin][k][k] then b[cout*G].
 *   MB_MAXFILTER:     2x2 stride-1 max over each channel at offsets {0, d} x {0, d} (cin == cout).
 *   MB_HEAD_SIGMOID:  1x1 cin -> 1, + bias, sigmoid; must be the last layer.
 *   MB_HEAD_SOFTMAX2: ksize x ksize cross-correlation with dilation d, cin -> 2, + bias, then the
 *                     2-class softmax's class-1 probability 1 / (1 + exp(z0 - z1)); last layer.
 *   MB_HEAD_SOFTMAX:  1x1 cin -> cout classes, + bias, softmax; every class probability is an
 *                     output; last layer (MaskExtend).
 * dilation and maxout_groups 0 are read as 1.
 * Supported networks: the teacher (conv5x5 1->32 ReLU, maxfilter 2, conv5x5 32->32 ReLU,
 * maxfilter 2, conv5x5 32->32 ReLU, head 32->1) in FP32, BF16 and FP8; the student (conv3x3
 * 1->16 ReLU, conv3x3 16->16 ReLU, head 16->1) in FP32 and BF16 (BF16 weights; its inference runs
 * on the tensor cores with BF16 layer-1 features and FP32 accumulation, its training forward in
 * FP32 arithmetic); and FastMemb in dense form
 * (Sec. 2.2: conv4x4 1->32 G=2 d=1, maxfilter d=1, conv4x4 32->32 G=2 d=2, maxfilter d=2,
 * conv4x4 32->32 G=2 d=4, maxfilter d=4, softmax head conv4x4 32->2 d=8; no ReLU; radius 26,
 * so its slices need h, w >= 27) and FastMemb_3nm (Sec. 2.2, "A subsampling CNN for 3 nm data":
 * one more stage, conv4x4 32->32 G=2 d=8 and maxfilter d=8, then the head at d=16; radius 54,
 * slices h, w >= 55), both in FP32, BF16 and FP16 (the 16-bit nets: layer 1 on CUDA cores in
 * FP32 stored as 16-bit, the later convs and the head on the tensor cores with FP32 accumulation;
 * BF16 weights are split into two BF16 parts, FP16 weights are one FP16 value except the head's;
 * FP16 activations are finite below 65504); and MaskExtend (Sec. 3.2: conv4x4 12->32 G=2 d=1,
 * maxfilter d=1, conv4x4 32->40 G=2 d=2, maxfilter d=2, conv4x4 40->48 G=2 d=4, maxfilter d=4,
 * conv4x4 48->56 G=2 d=8, maxfilter d=8, conv4x4 56->64 G=2 d=16, head 1x1 64->3 softmax; radius
 * 54) in FP32 (CUDA cores) and FP16 (tensor cores: FP16 operands, FP32 accumulation), run only
 * through mb_mask_extend (the map calls return MB_ERR_UNSUPPORTED). MB_PREC_FP16 is accepted for
 * FastMemb and MaskExtend nets only.
 */
typedef struct {
    int32_t kind, ksize, dilation, cin, cout, relu, maxout_groups;
} mb_layer_desc;

/* One block of a batch: z slices of h x w. in[zi*in_slice_pitch + y*in_pitch + x] (uint8),
 * out likewise with out_pitch / out_slice_pitch in elements of the output type. Device memory. */
typedef struct {
    const uint8_t* in;
    int64_t z, h, w, in_pitch, in_slice_pitch;
    void* out;
    int64_t out_pitch, out_slice_pitch;
} mb_block;

/* Student training settings (Adam: Kingma and Ba, 2014). */
typedef struct {
    int32_t batch;      /* slices per step, sampled with replacement */
    int32_t steps;      /* total optimiser steps of the run */
    int32_t ckpt_every; /* write a checkpoint every this many steps (0: never) */
    int32_t resume;     /* 1: continue from ckpt_path if it exists */
    float lr, beta1, beta2, eps;
    uint64_t seed; /* batch sampling */
} mb_train_cfg;

/* Create a net for `device` (a CUDA ordinal) from n_layers descriptions. Weights start
 * unloaded. Errors: MB_ERR_INVALID_ARG (null out_net, bad enum), MB_ERR_UNSUPPORTED (layer
 * stack or precision without a kernel), MB_ERR_CUDA, MB_ERR_OOM. */
mb_status mb_net_create(const mb_layer_desc* layers, int32_t n_layers, mb_precision prec, int32_t device,
                        mb_net** out_net);

/* Release everything the net owns. NULL is a no-op. Synchronises the net's device. */
mb_status mb_net_destroy(mb_net* net);

/* Number of FP32 parameters of the net (layout of mb_load_weights). */
mb_status mb_net_param_count(const mb_net* net, int64_t* n_params);

/* Copy FP32 parameters from HOST memory (caller keeps ownership). Layout: for each
 * parameterised layer in order, W[cout][cin][k][k] then b[cout]. BF16/FP8 nets round their
 * own copies from these. An FP8 net needs mb_calibrate_fp8 afterwards. Synchronous.
 * Errors: MB_ERR_INVALID_ARG when n_params differs from mb_net_param_count. */
mb_status mb_load_weights(mb_net* net, const float* params, int64_t n_params);

/* Copy the net's FP32 parameters (the master copy; after training, the trained ones) to HOST
 * memory. Synchronous. */
mb_status mb_get_weights(const mb_net* net, float* params, int64_t n_params);

/*
 * FP8 E4M3 calibration of a teacher net created with MB_PREC_FP8 (no counterpart in the
 * paper, which states no number format): runs the FP32 path on n calibration slices (device,
 * contiguous n x h x w uint8), takes the per-channel maximum of the activations entering the
 * 2nd and 3rd convolutions, folds those activation scales into the next layer's weights, then
 * quantises every output channel of those weights with its own scale (amax / 448) to E4M3
 * (round to nearest even, saturating). Synchronises `stream` before returning.
 * amax_out (HOST, may be NULL) receives the 2 x 32 activation maxima.
 */
mb_status mb_calibrate_fp8(mb_net* net, const uint8_t* slices, int64_t n, int64_t h, int64_t w,
                           float* amax_out, void* stream);

/*
 * Probability maps of a contiguous volume in[z][h][w] (uint8) into out[z][h][w] (float32 or
 * uint8 q = min(255, floor(255 p + 0.5))). Device pointers: asynchronous on `stream`.
 * HOST pointers (both in and out on the host; synchronous, `stream` unused):
 *   - both page-locked and mapped (cudaHostAlloc / cudaHostRegister, e.g. torch pin_memory), on
 *     a GPU that reads host memory through the host's page tables (a coherent CPU-GPU link such
 *     as NVLink-C2C; cudaDevAttrPageableMemoryAccessUsesHostPageTables), the net's host I/O
 *     mode MB_HOST_IO_AUTO (the default) and a teacher or FastMemb net: the kernels read the
 *     input from and write the maps to the host buffers themselves, in the same launches as for
 *     device buffers; no device buffer and no copy;
 *   - otherwise (pageable memory, another link, MB_HOST_IO_SLABS, or a student net, whose kernel
 *     outruns direct host access): the volume is streamed through device buffers in z-slabs,
 *     copies overlapped with compute.
 * Both give the device path's maps bitwise. Mixed host/device pointers: MB_ERR_INVALID_ARG.
 */
mb_status mb_infer_volume(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, void* out,
                          mb_out_type out_type, void* stream);

/*
 * Sub-sampled probability maps (Sec. 2.2, "Accelerating dense computation": the recursion tree of
 * max-pooling fragments can be pruned to sub-sample the image). For factor 2, out[z][h2][w2] with
 * h2 = ceil(h/2), w2 = ceil(w/2) holds the map of mb_infer_volume at rows 2i and columns 2j:
 * only the branch of the first stride-2 pool's offset (0, 0) is evaluated (a real 2x2 stride-2
 * max-pool after the first convolution, the later stages on the half grid), about a quarter of
 * the dense work. FastMemb nets (FP32, BF16) and factor 2 only, else MB_ERR_UNSUPPORTED. out is
 * float32 or uint8 as in mb_infer_volume. Device pointers only; asynchronous on `stream`.
 */
mb_status mb_infer_volume_subsampled(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w,
                                     int32_t factor, void* out, mb_out_type out_type, void* stream);

/*
 * Output rows [y0, y0 + rows) and columns [x0, x0 + cols) of every slice of the volume
 * in[z][h][w] into out[z][rows][cols], computed with the slice's true context (mirror padding
 * only at the slice borders). Values equal the corresponding pixels of mb_infer_volume.
 * Device pointers only.
 */
mb_status mb_infer_region(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, int64_t y0,
                          int64_t x0, int64_t rows, int64_t cols, void* out, mb_out_type out_type,
                          void* stream);

/*
 * A batch of independent blocks of uneven size (Sec. 2: blocks are segmented independently).
 * BF16/FP8 teacher nets: one persistent launch drains a device work queue of (block, slice,
 * strip) items; the first call for a new batch geometry captures the launch in a CUDA graph
 * that later calls with the same geometry replay. Other nets: one launch per block.
 * Device pointers; asynchronous. Output of each block equals mb_infer_volume of that block.
 */
mb_status mb_infer_batch(mb_net* net, const mb_block* blocks, int32_t n_blocks, mb_out_type out_type,
                         void* stream);

/* The comparison path of mb_infer_batch: one mb_infer_volume-style launch per block. */
mb_status mb_infer_batch_per_block(mb_net* net, const mb_block* blocks, int32_t n_blocks,
                                   mb_out_type out_type, void* stream);

/*
 * Autotuner of the persistent tensor-core teacher kernel (BF16/FP8 teacher nets). Its knobs:
 *  - stages: the depth of the kernel's two A-operand rings (staged layer-2 and layer-3 input rows)
 *    and so how far the layer-1 producers and the layer-2 epilogue may run ahead of the MMAs;
 *    compiled depths BF16 4, 5, 6 and FP8 4, 6, 8 (FP8 rows take half the bytes);
 *  - rows_per_item (BF16): output rows per work item taken round-robin by the CTAs, 64 .. 1024
 *    (each item restarts the row pipeline: 9 extra rows), or 0: the launch's strip-rows split into
 *    one equal contiguous range per CTA (no tail wave; items are the runs of a range within one
 *    strip). FP8 launches always split evenly (measured faster for FP8), reported as 0.
 * The strip width (118 output columns per 128-pixel MMA) is not a knob: a narrower strip costs the
 * same MMAs for fewer columns. Every candidate gives bitwise the same maps.
 * Times every candidate on a synthetic h x w x z workload on `stream` (median of 4 launches after
 * one), keeps the fastest in the net and records it in the JSON cache at cache_path (HOST string,
 * may be NULL) keyed on GPU name, precision and shape; a cached entry is reused without timing.
 * choice_out (HOST, may be NULL) receives {rows_per_item, stages, from_cache}. Synchronous.
 */
mb_status mb_autotune(mb_net* net, int64_t z, int64_t h, int64_t w, const char* cache_path,
                      int32_t* choice_out, void* stream);

/*
 * The same autotuner timed on the caller's own batch (configs of uneven blocks whose best schedule
 * a single-volume shape does not predict): every candidate runs the whole batch as mb_infer_batch
 * would (without its captured graph), so the blocks' outputs are written with valid maps; inputs are
 * only read. blocks, n_blocks and out_type as for mb_infer_batch (same checks and errors). The cache
 * key holds the GPU name, precision, output type and a hash of the blocks' shapes (z, h, w), not
 * their addresses. A batch with no voxels returns MB_ERR_INVALID_ARG; nets without the tensor-core
 * teacher kernel MB_ERR_UNSUPPORTED. choice_out as for mb_autotune. Synchronous.
 */
mb_status mb_autotune_batch(mb_net* net, const mb_block* blocks, int32_t n_blocks, mb_out_type out_type,
                            const char* cache_path, int32_t* choice_out, void* stream);

/*
 * Apply a known tuning choice (for example one recorded by mb_autotune on the same GPU) without
 * timing: rows_per_item 0, 64, 128, 256, 512 or 1024 for BF16 (0 for FP8) and stages among the
 * compiled depths of the net's precision (BF16 4, 5, 6; FP8 4, 6, 8). Other values return
 * MB_ERR_INVALID_ARG; nets without the tensor-core teacher kernel MB_ERR_UNSUPPORTED. Drops the
 * net's captured batch graphs (they hold the previous choice).
 */
mb_status mb_set_tuning(mb_net* net, int32_t rows_per_item, int32_t stages);

/*
 * Host I/O mode of mb_infer_volume for host buffers: MB_HOST_IO_AUTO (default: direct access
 * where the buffers and the link allow it, else slabs) or MB_HOST_IO_SLABS (always slabs through
 * device buffers). Other values: MB_ERR_INVALID_ARG. Results do not depend on the mode.
 */
mb_status mb_set_host_io(mb_net* net, int32_t mode);

/*
 * Student loss and gradient on n slices (device, in[n][h][w] uint8; target[n][h][w] float32):
 * loss = mean over all n*h*w pixels of (p - t)^2 (written to HOST *loss), gradient (device,
 * float32, parameter layout) of that mean. Student nets only. Synchronous.
 */
mb_status mb_student_loss_grad(mb_net* student, const uint8_t* in, const float* target, int64_t n,
                               int64_t h, int64_t w, double* loss, float* grad, void* stream);

/*
 * Train a student net in place on n slices (device in[n][h][w], target[n][h][w] float32 teacher
 * maps): cfg->steps Adam steps on batches of cfg->batch slices sampled with replacement
 * (seeded); FP32 master weights, m and v; the forward copy is rounded to BF16 for BF16 nets.
 * Layer 1 is optimised in centred-input coordinates: Adam updates W1 and c1 = b1 + sum(W1)/2
 * (the same network written for the input x - 1/2, a standard preconditioning of gradient
 * training); the weights stay stored for x = u/255, and m, v hold the centred moments.
 * loss_curve (HOST, may be NULL) receives one loss per step run. With ckpt_path (HOST string,
 * may be NULL), a checkpoint {step, master weights, m, v, sampler state} (format version 2: m and
 * v of the centred coordinates) is written every
 * cfg->ckpt_every steps; with cfg->resume the run continues from it, bitwise as if never
 * interrupted. With cfg->resume and no file at ckpt_path the run starts fresh; a file there that
 * is not a complete format-2 checkpoint of this student returns MB_ERR_INVALID_ARG before any
 * step and leaves the file unchanged. Synchronous.
 */
mb_status mb_student_train(mb_net* student, const uint8_t* in, const float* target, int64_t n, int64_t h,
                           int64_t w, const mb_train_cfg* cfg, const char* ckpt_path, float* loss_curve,
                           void* stream);

/*
 * Multi-pass inference (Sec. 1: a fast pass everywhere, a slower pass only where errors are
 * likely): the student maps the volume in[z][h][w] into out (float32); each tile x tile square
 * (aligned at multiples of tile, clipped at the edges) whose count of student outputs with
 * lo <= p <= hi exceeds max_frac of its pixels is recomputed by the teacher with its true
 * context and overwritten. *fallback_rate (HOST) receives flagged tiles / all tiles;
 * tile_flags (device, may be NULL) receives one byte per tile in [z][ty][tx] order.
 * Device pointers; synchronous (the flag count is read back).
 */
mb_status mb_infer_cascade(mb_net* student, mb_net* teacher, const uint8_t* in, int64_t z, int64_t h,
                           int64_t w, float* out, int32_t tile, float lo, float hi, float max_frac,
                           double* fallback_rate, uint8_t* tile_flags, void* stream);

/*
 * mb_infer_volume without any device allocation (the paper has no counterpart: it is a service
 * for callers of this library). For callers that must not allocate device memory once running:
 * a service whose memory budget is fixed at start-up, or a pipeline that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree may cause while other streams are busy.
 * FP32 teacher nets only; device pointers in[z][h][w] -> out[z][h][w] (float32 or uint8 as in
 * mb_infer_volume); asynchronous on `stream`.
 * Scratch: a fixed 64 MiB array in the library's device memory, held by every GPU that loads the
 * library until exit. A band of r output rows of n slices needs
 * n * ((r + 10)(w + 10) + (r + 5)(w + 5)) * 32 floats of it; slices are processed in the largest
 * row band that fits (all h rows if they fit), as many slices of that band per launch sequence as
 * fit, three kernel launches per band. A width needing more than 64 MiB for a single-row band
 * (w > 30,832), or h or w above 2^20, returns MB_ERR_SHAPE. The first call on each
 * device looks up the array's device address; make that first call before any stream capture.
 * All calls on a device share the array: calls that overlap on the GPU (other streams or host
 * threads) race and must be serialised by the caller. Nothing in the array needs clearing.
 * This call makes no cudaMalloc/cudaFree and calls no allocating library routine.
 */
mb_status mb_infer_volume_noalloc(mb_net* net, const uint8_t* in, int64_t z, int64_t h, int64_t w, void* out,
                                  mb_out_type out_type, void* stream);

/* Static string for a status code. */
const char* mb_status_string(mb_status s);

/* Thread-local detail of the last failing call on this thread ("" if none). */
const char* mb_last_error(void);

/* Number of kernel launches this library has issued since load (for launch accounting). */
int64_t mb_launch_count(void);

/*
 * MaskExtend transfer (Sec. 3.2), recursed in +z: for z = z0 .. z0 + n_steps - 1,
 *   Mask_z = J(CNN(Mask_{z-4..z-1}, EM_{z-1..z+1}, FastMemb_{z-2..z+2}))
 * where CNN is the dense inference of a MaskExtend net over the whole h x w section (12 input maps:
 * EM u/255, the object's binary masks, membrane probabilities; each mirror-padded reflect-101 by
 * 54), and J is the 3x3 mean of the object-class probability (reflect-101 borders) followed by
 * >= threshold. Each new mask feeds the next step.
 *   em:         uint8 [z][h][w] EM stack            membrane: float [z][h][w] membrane maps
 *   seed_masks: uint8 [4][h][w] masks of z0-4 .. z0-1 (0 or 1)
 *   masks_out:  uint8 [n_steps][h][w] (0/1)        probs_out: float [n_steps][3][h][w] or NULL
 *               (classes: object, other neurons, membrane)
 * Needs 2 <= z0 and z0 + n_steps + 1 < z (else MB_ERR_SHAPE). MaskExtend nets in FP32 or FP16 (an
 * FP16 net rounds the 12 maps, its weights and every layer's features to FP16 and accumulates in
 * FP32; a timed-out device-side wait returns MB_ERR_TIMEOUT). Device pointers; asynchronous on
 * `stream`. The net's workspace is shared by its calls: calls on one
 * net must not overlap on the GPU.
 */
mb_status mb_mask_extend(mb_net* net, const uint8_t* em, const float* membrane, int64_t z, int64_t h, int64_t w,
                         const uint8_t* seed_masks, int64_t z0, int64_t n_steps, float threshold, uint8_t* masks_out,
                         float* probs_out, void* stream);

/*
 * The MaskExtend recursion in either direction (Sec. 3.2: the algorithm continues iteratively in
 * z+ or z-). direction = +1 is mb_mask_extend. direction = -1 mirrors every offset of the transfer
 * equation: for z = z0, z0-1, .., z0-n_steps+1,
 *   Mask_z = J(CNN(Mask_{z+4..z+1}, EM_{z+1..z-1}, FastMemb_{z+2..z-2}))
 * (the same 12-channel order, each map taken at the mirrored section), which is the z+ recursion of
 * the stack read backwards. seed_masks[i] is the mask of section z0 + direction (i - 4), i.e. the
 * four sections before z0 along the direction of travel (z0+4 .. z0+1 for -1). masks_out[s] and
 * probs_out[s] belong to step s, section z0 + direction s. Needs the sections read,
 * z0-2 .. z0+n_steps+1 (+1) or z0-n_steps-1 .. z0+2 (-1), inside the stack (else MB_ERR_SHAPE);
 * a direction other than +1 or -1 returns MB_ERR_INVALID_ARG. Otherwise as mb_mask_extend.
 */
mb_status mb_mask_extend_dir(mb_net* net, const uint8_t* em, const float* membrane, int64_t z, int64_t h, int64_t w,
                             const uint8_t* seed_masks, int64_t z0, int64_t n_steps, int32_t direction, float threshold,
                             uint8_t* masks_out, float* probs_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MEMBRANE_H */
