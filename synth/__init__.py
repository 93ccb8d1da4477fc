"""Seeded synthetic inputs shared by the CUDA path's tests and bench and by the oracle tests.

Holds no arithmetic of the method: EM-like uint8 slices (stand-ins for the EM stacks of
Sec. 2 / Sec. 2.2), He-normal parameters, seeded integer draws, and the two workload network
descriptions as plain data (each side turns them into its own form).

The C library ``libsynth.so`` is compiled on first use (gcc, OpenMP, no FMA contraction).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

# Layer kinds of the workload descriptions (same numbering as the library's mb_layer_kind).
CONV, MAXFILTER, HEAD_SIGMOID, HEAD_SOFTMAX2, HEAD_SOFTMAX = 0, 1, 2, 3, 4

# (kind, ksize, cin, cout, relu[, dilation[, maxout groups]]); dilation and groups default to 1.
# The measured stand-in network: conv5x5 1->32 ReLU, 2x2 stride-1 max-filter, conv5x5 32->32
# ReLU, max-filter, conv5x5 32->32 ReLU, conv1x1 32->1 sigmoid (receptive field 15x15).
TEACHER = (
    (CONV, 5, 1, 32, 1),
    (MAXFILTER, 2, 32, 32, 0),
    (CONV, 5, 32, 32, 1),
    (MAXFILTER, 2, 32, 32, 0),
    (CONV, 5, 32, 32, 1),
    (HEAD_SIGMOID, 1, 32, 1, 0),
)
# The distilled student: conv3x3 1->16 ReLU, conv3x3 16->16 ReLU, conv1x1 16->1 sigmoid.
STUDENT = (
    (CONV, 3, 1, 16, 1),
    (CONV, 3, 16, 16, 1),
    (HEAD_SIGMOID, 1, 16, 1, 0),
)

# FastMemb (Sec. 2.2) in dense form: three [conv4x4 -> max-out over 2 -> 2x2 max-filter] stages
# whose stride-2 pooling has become dilation 1, 2, 4, then conv4x4 with dilation 8 to 2 classes
# and a softmax; no ReLU. Field of view 53x53, 67,778 parameters.
FASTMEMB = (
    (CONV, 4, 1, 32, 0, 1, 2),
    (MAXFILTER, 2, 32, 32, 0, 1, 1),
    (CONV, 4, 32, 32, 0, 2, 2),
    (MAXFILTER, 2, 32, 32, 0, 2, 1),
    (CONV, 4, 32, 32, 0, 4, 2),
    (MAXFILTER, 2, 32, 32, 0, 4, 1),
    (HEAD_SOFTMAX2, 4, 32, 2, 0, 8, 1),
)

# FastMemb_3nm (Sec. 2.2, "A subsampling CNN for 3 nm data"): FastMemb with one more [conv4x4 ->
# max-out 2 -> pool] stage, for 3 nm images: dilations 1, 2, 4, 8 and the head at 16. Field of view
# 109x109 (the four-pair structure Sec. 3.2 gives 109 for), 100,610 parameters.
FASTMEMB_3NM = (
    (CONV, 4, 1, 32, 0, 1, 2),
    (MAXFILTER, 2, 32, 32, 0, 1, 1),
    (CONV, 4, 32, 32, 0, 2, 2),
    (MAXFILTER, 2, 32, 32, 0, 2, 1),
    (CONV, 4, 32, 32, 0, 4, 2),
    (MAXFILTER, 2, 32, 32, 0, 4, 1),
    (CONV, 4, 32, 32, 0, 8, 2),
    (MAXFILTER, 2, 32, 32, 0, 8, 1),
    (HEAD_SOFTMAX2, 4, 32, 2, 0, 16, 1),
)

# MaskExtend (Sec. 3.2): 12 input maps, five [conv4x4 -> max-out 2] stages with 32, 40, 48, 56, 64
# features (the first four followed by pools: dilations 1, 2, 4, 8, 16 in dense form), then a 1x1
# head to 3 classes (object, other neurons, membrane) with a softmax. Field of view 109x109.
MASKEXTEND = (
    (CONV, 4, 12, 32, 0, 1, 2),
    (MAXFILTER, 2, 32, 32, 0, 1, 1),
    (CONV, 4, 32, 40, 0, 2, 2),
    (MAXFILTER, 2, 40, 40, 0, 2, 1),
    (CONV, 4, 40, 48, 0, 4, 2),
    (MAXFILTER, 2, 48, 48, 0, 4, 1),
    (CONV, 4, 48, 56, 0, 8, 2),
    (MAXFILTER, 2, 56, 56, 0, 8, 1),
    (CONV, 4, 56, 64, 0, 16, 2),
    (HEAD_SOFTMAX, 1, 64, 3, 0, 1, 1),
)

TEACHER_WEIGHT_SEED = 20161206
STUDENT_WEIGHT_SEED = 20161207
FASTMEMB_WEIGHT_SEED = 20161208
FASTMEMB_3NM_WEIGHT_SEED = 20161209
MASKEXTEND_WEIGHT_SEED = 20161210
BASE_SEED = 1612021200  # + workload index


def build(force: bool = False) -> str:
    """Compile libsynth.so next to this file; returns its path."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            u64, i64, p = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
            lib.synth_default_cells.argtypes = [i64, i64]
            lib.synth_default_cells.restype = i64
            lib.synth_slice_seed.argtypes = [u64, u64, u64]
            lib.synth_slice_seed.restype = u64
            lib.synth_em_slice.argtypes = [u64, i64, i64, i64, p, i64]
            lib.synth_em_slice_truth.argtypes = [u64, i64, i64, i64, p, i64, p]
            lib.synth_em_volume.argtypes = [u64, u64, i64, i64, i64, i64, p, i64, i64]
            lib.synth_he_normal.argtypes = [u64, i64, i64, p, i64, p, ctypes.c_double]
            lib.synth_uniform_ints.argtypes = [u64, i64, i64, i64, p]
            lib.synth_uniform_floats.argtypes = [u64, i64, ctypes.c_double, ctypes.c_double, p]
            for f in ("synth_em_slice", "synth_em_slice_truth", "synth_em_volume", "synth_he_normal", "synth_uniform_ints",
                      "synth_uniform_floats"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def default_cells(h: int, w: int) -> int:
    return int(_load().synth_default_cells(h, w))


def slice_seed(base: int, block: int, z: int) -> int:
    return int(_load().synth_slice_seed(base, block, z))


def em_slice(seed: int, h: int, w: int, n_cells: int = 0) -> np.ndarray:
    out = np.empty((h, w), dtype=np.uint8)
    _check(_load().synth_em_slice(seed, h, w, n_cells, out.ctypes.data, w), "synth_em_slice")
    return out


def em_slice_truth(seed: int, h: int, w: int, n_cells: int = 0):
    """(slice, truth): em_slice(seed, h, w) and the generator's membrane flag per pixel (0/1)."""
    out = np.empty((h, w), dtype=np.uint8)
    truth = np.empty((h, w), dtype=np.uint8)
    _check(_load().synth_em_slice_truth(seed, h, w, n_cells, out.ctypes.data, w, truth.ctypes.data),
           "synth_em_slice_truth")
    return out, truth


def em_volume(base: int, z: int, h: int, w: int, block: int = 0, n_cells: int = 0,
              out: np.ndarray | None = None) -> np.ndarray:
    """z independent slices [z][h][w]; `out` may be a preallocated (pinned) uint8 array."""
    if out is None:
        out = np.empty((z, h, w), dtype=np.uint8)
    assert out.dtype == np.uint8 and out.shape == (z, h, w) and out.flags.c_contiguous
    _check(_load().synth_em_volume(base, block, z, h, w, n_cells, out.ctypes.data, w, h * w),
           "synth_em_volume")
    return out


def he_normal(seed: int, fan_in: int, n_w: int, n_b: int, bias_std: float):
    w = np.empty(n_w, dtype=np.float32)
    b = np.empty(n_b, dtype=np.float32)
    _check(_load().synth_he_normal(seed, fan_in, n_w, w.ctypes.data, n_b, b.ctypes.data, bias_std),
           "synth_he_normal")
    return w, b


def uniform_ints(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int64)
    _check(_load().synth_uniform_ints(seed, n, lo, hi, out.ctypes.data), "synth_uniform_ints")
    return out


def uniform_floats(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    out = np.empty(n, dtype=np.float32)
    _check(_load().synth_uniform_floats(seed, n, lo, hi, out.ctypes.data), "synth_uniform_floats")
    return out


def _groups(layer) -> int:
    return int(layer[6]) if len(layer) > 6 else 1


def param_count(layers) -> int:
    n = 0
    for layer in layers:
        kind, k, cin, cout = layer[:4]
        if kind in (CONV, HEAD_SIGMOID, HEAD_SOFTMAX2, HEAD_SOFTMAX):
            co = cout * _groups(layer)
            n += co * cin * k * k + co
    return n


def init_params(layers, seed: int, bias_std: float = 0.01, center_head: bool = False,
                centred_input: bool = False) -> np.ndarray:
    """He-normal FP32 parameters for `layers`, packed per parameterised layer as
    W[cout*G][cin][k][k] then b[cout*G] (G max-out groups); parameterised layer number l draws
    from seed + l. bias_std 0 gives zero biases. center_head: the last layer's filters are
    shifted to zero mean over their input channels at every tap (a distribution choice that keeps
    a deep max-out stack's map away from saturation). centred_input: the first layer's biases are
    drawn for the input x - 1/2 instead of x and stored for x, i.e. each becomes
    b - (1/2) sum of its filter, so that mid-grey input puts every first-layer unit at its bias
    rather than far on one side of its ReLU."""
    parts = []
    l = 0
    n_par = sum(1 for layer in layers if layer[0] in (CONV, HEAD_SIGMOID, HEAD_SOFTMAX2, HEAD_SOFTMAX))
    for layer in layers:
        kind, k, cin, cout = layer[:4]
        if kind in (CONV, HEAD_SIGMOID, HEAD_SOFTMAX2, HEAD_SOFTMAX):
            co = cout * _groups(layer)
            w, b = he_normal(seed + l, cin * k * k, co * cin * k * k, co, bias_std)
            if center_head and l == n_par - 1:
                w4 = w.reshape(co, cin, k * k)
                w = (w4 - w4.mean(axis=1, keepdims=True)).reshape(-1)
            if centred_input and l == 0:
                b = (b.astype(np.float64) - 0.5 * w.reshape(co, -1).astype(np.float64).sum(axis=1)).astype(np.float32)
            parts += [w, b]
            l += 1
    return np.concatenate(parts).astype(np.float32)


def block_shapes(seed: int, n_blocks: int, side_lo: int = 256, side_hi: int = 1536,
                 depth_lo: int = 1, depth_hi: int = 16):
    """Uneven block shapes (D, H, W): H and W independent integers in [side_lo, side_hi],
    D in [depth_lo, depth_hi]."""
    hs = uniform_ints(seed, n_blocks, side_lo, side_hi)
    ws = uniform_ints(seed + 1, n_blocks, side_lo, side_hi)
    ds = uniform_ints(seed + 2, n_blocks, depth_lo, depth_hi)
    return [(int(d), int(h), int(w)) for d, h, w in zip(ds, hs, ws)]


def disk_masks(n: int, h: int, w: int, cy: float, cx: float, r: float, dy: float = 0.0, dx: float = 0.0):
    """n binary object masks [n][h][w] (uint8 0/1): disks of radius r centred at (cy + i dy,
    cx + i dx) in section i: a seeded stand-in for an object followed across sections."""
    yy, xx = np.mgrid[0:h, 0:w]
    out = np.empty((n, h, w), dtype=np.uint8)
    for i in range(n):
        out[i] = ((yy - (cy + i * dy)) ** 2 + (xx - (cx + i * dx)) ** 2 <= r * r).astype(np.uint8)
    return out


def membrane_maps(em_u8) -> np.ndarray:
    """Stand-in membrane probability maps for an EM stack: 1 - u/255 (membranes are dark), FP32."""
    return (1.0 - np.asarray(em_u8, dtype=np.float32) / np.float32(255.0)).astype(np.float32)
