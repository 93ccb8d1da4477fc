"""ctypes binding of libmembrane (include/membrane.h): same names, argument marshalling only.

Every computation runs in the library's CUDA kernels. Buffers are passed as raw pointers:
torch tensors (device or pinned host) or numpy arrays (host). The library must have been built
(``paper_1612_02120_gb300.build.build()``); importing this module without it raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmembrane.so")

MB_OK, MB_ERR_INVALID_ARG, MB_ERR_SHAPE, MB_ERR_OOM, MB_ERR_CUDA, MB_ERR_TIMEOUT, MB_ERR_NOT_READY, \
    MB_ERR_UNSUPPORTED = range(8)
MB_PREC_FP32, MB_PREC_BF16, MB_PREC_FP8, MB_PREC_FP16 = 0, 1, 2, 3
MB_OUT_F32, MB_OUT_U8 = 0, 1
MB_HOST_IO_AUTO, MB_HOST_IO_SLABS = 0, 1
MB_CONV, MB_MAXFILTER, MB_HEAD_SIGMOID, MB_HEAD_SOFTMAX2, MB_HEAD_SOFTMAX = 0, 1, 2, 3, 4

EXPORTED = (
    "mb_net_create", "mb_net_destroy", "mb_net_param_count", "mb_load_weights", "mb_get_weights",
    "mb_calibrate_fp8", "mb_infer_volume", "mb_infer_region", "mb_infer_batch", "mb_infer_batch_per_block",
    "mb_autotune", "mb_student_loss_grad", "mb_student_train", "mb_infer_cascade", "mb_status_string",
    "mb_last_error", "mb_launch_count", "mb_infer_volume_noalloc", "mb_infer_volume_subsampled", "mb_mask_extend",
    "mb_mask_extend_dir", "mb_set_tuning", "mb_autotune_batch", "mb_set_host_io",
)


class mb_layer_desc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("kind", "ksize", "dilation", "cin", "cout", "relu",
                                                "maxout_groups")]


class mb_block(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("z", ctypes.c_int64), ("h", ctypes.c_int64), ("w", ctypes.c_int64),
                ("in_pitch", ctypes.c_int64), ("in_slice_pitch", ctypes.c_int64), ("out", ctypes.c_void_p),
                ("out_pitch", ctypes.c_int64), ("out_slice_pitch", ctypes.c_int64)]


class mb_train_cfg(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("steps", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
                ("resume", ctypes.c_int32), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("seed", ctypes.c_uint64)]


class MembraneError(RuntimeError):
    def __init__(self, status: int, detail: str, call: str):
        self.status = status
        super().__init__(f"{call}: {status_name(status)}: {detail}")


_lib = None


def load() -> ctypes.CDLL:
    """Load libmembrane.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmembrane.so not built at {LIB_PATH}; run paper_1612_02120_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    p, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    st = ctypes.c_int
    sig = {
        "mb_net_create": ([p, i32, i32, i32, p], st),
        "mb_net_destroy": ([p], st),
        "mb_net_param_count": ([p, p], st),
        "mb_load_weights": ([p, p, i64], st),
        "mb_get_weights": ([p, p, i64], st),
        "mb_calibrate_fp8": ([p, p, i64, i64, i64, p, p], st),
        "mb_infer_volume": ([p, p, i64, i64, i64, p, i32, p], st),
        "mb_infer_region": ([p, p, i64, i64, i64, i64, i64, i64, i64, p, i32, p], st),
        "mb_infer_batch": ([p, p, i32, i32, p], st),
        "mb_infer_batch_per_block": ([p, p, i32, i32, p], st),
        "mb_autotune": ([p, i64, i64, i64, ctypes.c_char_p, p, p], st),
        "mb_set_tuning": ([p, i32, i32], st),
        "mb_set_host_io": ([p, i32], st),
        "mb_autotune_batch": ([p, p, i32, i32, ctypes.c_char_p, p, p], st),
        "mb_student_loss_grad": ([p, p, p, i64, i64, i64, p, p, p], st),
        "mb_student_train": ([p, p, p, i64, i64, i64, p, ctypes.c_char_p, p, p], st),
        "mb_infer_cascade": ([p, p, p, i64, i64, i64, p, i32, f32, f32, f32, p, p, p], st),
        "mb_status_string": ([st], ctypes.c_char_p),
        "mb_last_error": ([], ctypes.c_char_p),
        "mb_launch_count": ([], i64),
        "mb_infer_volume_noalloc": ([p, p, i64, i64, i64, p, i32, p], st),
        "mb_infer_volume_subsampled": ([p, p, i64, i64, i64, i32, p, i32, p], st),
        "mb_mask_extend": ([p, p, p, i64, i64, i64, p, i64, i64, ctypes.c_float, p, p, p], st),
        "mb_mask_extend_dir": ([p, p, p, i64, i64, i64, p, i64, i64, i32, ctypes.c_float, p, p, p], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def status_name(s: int) -> str:
    return load().mb_status_string(s).decode()


def last_error() -> str:
    return load().mb_last_error().decode()


def launch_count() -> int:
    return int(load().mb_launch_count())


def check(status: int, call: str) -> None:
    if status != MB_OK:
        raise MembraneError(status, last_error(), call)


def ptr(x) -> int | None:
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return int(x)


def stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def layer_array(layers):
    """layers: iterable of (kind, ksize, cin, cout, relu[, dilation[, maxout groups]]) tuples."""
    arr = (mb_layer_desc * len(layers))()
    for i, layer in enumerate(layers):
        kind, k, cin, cout, relu = layer[:5]
        dil = layer[5] if len(layer) > 5 else 1
        groups = layer[6] if len(layer) > 6 else 1
        arr[i] = mb_layer_desc(kind, k, dil, cin, cout, relu, groups)
    return arr


# --- the C calls, same names --------------------------------------------------------------------

def mb_net_create(layers, prec: int, device: int = 0) -> int:
    arr = layer_array(layers)
    out = ctypes.c_void_p()
    check(load().mb_net_create(arr, len(layers), prec, device, ctypes.byref(out)), "mb_net_create")
    return out.value


def mb_net_destroy(net) -> None:
    check(load().mb_net_destroy(net), "mb_net_destroy")


def mb_net_param_count(net) -> int:
    n = ctypes.c_int64()
    check(load().mb_net_param_count(net, ctypes.byref(n)), "mb_net_param_count")
    return n.value


def numel(x) -> int:
    return int(x.numel()) if hasattr(x, "numel") else int(x.size)


def mb_load_weights(net, params_f32_host) -> None:
    check(load().mb_load_weights(net, ptr(params_f32_host), numel(params_f32_host)), "mb_load_weights")


def mb_get_weights(net, out_f32_host) -> None:
    check(load().mb_get_weights(net, ptr(out_f32_host), numel(out_f32_host)), "mb_get_weights")


def mb_calibrate_fp8(net, slices, n, h, w, amax_out=None, stream=None) -> None:
    check(load().mb_calibrate_fp8(net, ptr(slices), n, h, w, ptr(amax_out), stream_handle(stream)),
          "mb_calibrate_fp8")


def mb_infer_volume(net, inp, z, h, w, out, out_type=MB_OUT_F32, stream=None) -> None:
    check(load().mb_infer_volume(net, ptr(inp), z, h, w, ptr(out), out_type, stream_handle(stream)),
          "mb_infer_volume")


def mb_infer_volume_subsampled(net, inp, z, h, w, factor, out, out_type=MB_OUT_F32, stream=None) -> None:
    """FastMemb map at even rows and columns: out is z x ceil(h/2) x ceil(w/2)."""
    check(load().mb_infer_volume_subsampled(net, ptr(inp), z, h, w, factor, ptr(out), out_type,
                                            stream_handle(stream)), "mb_infer_volume_subsampled")


def mb_mask_extend(net, em, membrane, z, h, w, seed_masks, z0, n_steps, masks_out, probs_out=None,
                   threshold=0.5, stream=None) -> None:
    """MaskExtend transfer recursion in +z (device tensors)."""
    check(load().mb_mask_extend(net, ptr(em), ptr(membrane), z, h, w, ptr(seed_masks), z0, n_steps, float(threshold),
                                ptr(masks_out), ptr(probs_out), stream_handle(stream)), "mb_mask_extend")


def mb_mask_extend_dir(net, em, membrane, z, h, w, seed_masks, z0, n_steps, direction, masks_out, probs_out=None,
                       threshold=0.5, stream=None) -> None:
    """MaskExtend transfer recursion in z+ (direction 1) or z- (direction -1), device tensors."""
    check(load().mb_mask_extend_dir(net, ptr(em), ptr(membrane), z, h, w, ptr(seed_masks), z0, n_steps, direction,
                                    float(threshold), ptr(masks_out), ptr(probs_out), stream_handle(stream)),
          "mb_mask_extend_dir")


def mb_infer_volume_noalloc(net, inp, z, h, w, out, out_type=MB_OUT_F32, stream=None) -> None:
    """mb_infer_volume for callers that cannot allocate device memory (FP32 teacher nets)."""
    check(load().mb_infer_volume_noalloc(net, ptr(inp), z, h, w, ptr(out), out_type, stream_handle(stream)),
          "mb_infer_volume_noalloc")


def mb_infer_region(net, inp, z, h, w, y0, x0, rows, cols, out, out_type=MB_OUT_F32, stream=None) -> None:
    check(load().mb_infer_region(net, ptr(inp), z, h, w, y0, x0, rows, cols, ptr(out), out_type,
                                 stream_handle(stream)), "mb_infer_region")


def block_array(blocks):
    """blocks: iterable of dicts/tuples (in, z, h, w, in_pitch, in_slice_pitch, out, out_pitch,
    out_slice_pitch) with tensors or raw pointers."""
    arr = (mb_block * len(blocks))()
    for i, b in enumerate(blocks):
        inp, z, h, w, ip, isp, out, op, osp = b
        arr[i] = mb_block(ptr(inp), z, h, w, ip, isp, ptr(out), op, osp)
    return arr


def mb_infer_batch(net, blocks, out_type=MB_OUT_F32, stream=None) -> None:
    arr = block_array(blocks)
    check(load().mb_infer_batch(net, arr, len(blocks), out_type, stream_handle(stream)), "mb_infer_batch")


def mb_infer_batch_per_block(net, blocks, out_type=MB_OUT_F32, stream=None) -> None:
    arr = block_array(blocks)
    check(load().mb_infer_batch_per_block(net, arr, len(blocks), out_type, stream_handle(stream)),
          "mb_infer_batch_per_block")


def mb_autotune(net, z, h, w, cache_path=None, stream=None):
    choice = (ctypes.c_int32 * 3)()
    check(load().mb_autotune(net, z, h, w, cache_path.encode() if cache_path else None, choice,
                             stream_handle(stream)), "mb_autotune")
    return {"rows_per_item": choice[0], "stages": choice[1], "from_cache": bool(choice[2])}


def mb_autotune_batch(net, blocks, out_type=MB_OUT_F32, cache_path=None, stream=None):
    arr = block_array(blocks)
    choice = (ctypes.c_int32 * 3)()
    check(load().mb_autotune_batch(net, arr, len(blocks), out_type, cache_path.encode() if cache_path else None,
                                   choice, stream_handle(stream)), "mb_autotune_batch")
    return {"rows_per_item": choice[0], "stages": choice[1], "from_cache": bool(choice[2])}


def mb_set_tuning(net, rows_per_item, stages) -> None:
    check(load().mb_set_tuning(net, rows_per_item, stages), "mb_set_tuning")


def mb_set_host_io(net, mode) -> None:
    check(load().mb_set_host_io(net, mode), "mb_set_host_io")


def mb_student_loss_grad(net, inp, target, n, h, w, grad, stream=None) -> float:
    loss = ctypes.c_double()
    check(load().mb_student_loss_grad(net, ptr(inp), ptr(target), n, h, w, ctypes.byref(loss), ptr(grad),
                                      stream_handle(stream)), "mb_student_loss_grad")
    return loss.value


def train_cfg(batch=32, steps=2000, ckpt_every=0, resume=0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
              seed=0) -> mb_train_cfg:
    return mb_train_cfg(batch, steps, ckpt_every, resume, lr, beta1, beta2, eps, seed)


def mb_student_train(net, inp, target, n, h, w, cfg: mb_train_cfg, ckpt_path=None, loss_curve=None,
                     stream=None) -> None:
    check(load().mb_student_train(net, ptr(inp), ptr(target), n, h, w, ctypes.byref(cfg),
                                  ckpt_path.encode() if ckpt_path else None, ptr(loss_curve),
                                  stream_handle(stream)), "mb_student_train")


def mb_infer_cascade(student, teacher, inp, z, h, w, out, tile=256, lo=0.3, hi=0.7, max_frac=0.05,
                     tile_flags=None, stream=None) -> float:
    rate = ctypes.c_double()
    check(load().mb_infer_cascade(student, teacher, ptr(inp), z, h, w, ptr(out), tile, lo, hi, max_frac,
                                  ctypes.byref(rate), ptr(tile_flags), stream_handle(stream)), "mb_infer_cascade")
    return rate.value


class Net:
    """Owning handle: Net(layers, prec, device) ... close()."""

    def __init__(self, layers, prec=MB_PREC_FP32, device=0, params=None):
        self.handle = mb_net_create(layers, prec, device)
        self.layers = tuple(layers)
        self.prec = prec
        if params is not None:
            self.load(params)

    def load(self, params):
        mb_load_weights(self.handle, params)

    @property
    def n_params(self) -> int:
        return mb_net_param_count(self.handle)

    def infer(self, inp, out, out_type=MB_OUT_F32, stream=None):
        z, h, w = inp.shape
        mb_infer_volume(self.handle, inp, z, h, w, out, out_type, stream)
        return out

    def close(self):
        if self.handle:
            mb_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
