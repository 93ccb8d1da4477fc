"""FP64 CPU oracle of dense membrane-probability inference (Sec. 2.1, Sec. 2.2).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``; never by the library. It shares no code with the CUDA path; the
only shared module is ``synth`` (seeded inputs).

``liboracle.so`` is compiled on first use from ``oracle.c`` (gcc, OpenMP over output channels,
no FMA contraction). Every function here marshals numpy arrays into that library, except the
student's change of coordinates for its training update (a few lines of numpy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CONV, MAXF, HEAD, SOFTMAX, SOFTMAXN = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
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
            i64, p, d = ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
            ci = ctypes.c_int
            sig = {
                "oracle_reflect101": ([i64, i64], i64),
                "oracle_conv": ([p, i64, i64, i64, p, p, i64, i64, ci, p], ci),
                "oracle_conv_dil": ([p, i64, i64, i64, p, p, i64, i64, i64, ci, p], ci),
                "oracle_maxfilter2": ([p, i64, i64, i64, p], ci),
                "oracle_maxfilter2_dil": ([p, i64, i64, i64, i64, p], ci),
                "oracle_maxout": ([p, i64, i64, i64, p], ci),
                "oracle_head_sigmoid": ([p, i64, i64, i64, p, d, p], ci),
                "oracle_net_radius": ([p, ci], i64),
                "oracle_param_count": ([p, ci], i64),
                "oracle_pad_region": ([p, i64, i64, i64, i64, i64, i64, i64, i64, p], ci),
                "oracle_run_layers": ([p, ci, p, p, i64, i64, p], ci),
                "oracle_run_layers_mc": ([p, ci, p, p, i64, i64, i64, p], ci),
                "oracle_smooth_threshold": ([p, i64, i64, d, p], ci),
                "oracle_forward_region": ([p, ci, p, p, i64, i64, i64, i64, i64, i64, i64, p], ci),
                "oracle_patch_pixel": ([p, ci, p, p, i64, i64, i64, i64, i64, p], ci),
                "oracle_maxfilter_amax": ([p, ci, p, p, i64, i64, i64, i64, i64, i64, i64, p, i64], ci),
                "oracle_student_loss_grad": ([p, ci, p, p, i64, i64, i64, i64, i64, p, p, p], ci),
                "oracle_adam_step": ([p, p, p, p, i64, i64, d, d, d, d], ci),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _chk(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle: {what} failed with code {rc}")


def _desc(layers) -> np.ndarray:
    """Layer tuples (kind, k, cin, cout, relu[, dilation[, maxout groups]]) as n x 7 int32."""
    rows = []
    for t in layers:
        t = tuple(int(v) for v in t)
        assert 5 <= len(t) <= 7, t
        rows.append(t + (1, 1)[len(t) - 5:])
    return np.ascontiguousarray(np.array(rows, dtype=np.int32).reshape(-1, 7))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def reflect101(t: int, n: int) -> int:
    return int(_load().oracle_reflect101(t, n))


def conv(x, W, b, relu: bool) -> np.ndarray:
    """Valid cross-correlation of x [cin][h][w] with W [cout][cin][k][k] plus b, optional ReLU."""
    x, W, b = _f64(x), _f64(W), _f64(b)
    cin, h, w = x.shape
    cout, cin2, k, k2 = W.shape
    assert cin2 == cin and k == k2 and b.shape == (cout,)
    y = np.empty((cout, h - k + 1, w - k + 1), dtype=np.float64)
    _chk(_load().oracle_conv(x.ctypes.data, cin, h, w, W.ctypes.data, b.ctypes.data, cout, k, int(relu),
                             y.ctypes.data), "conv")
    return y


def conv_dil(x, W, b, dilation: int, relu: bool) -> np.ndarray:
    """Dilated valid cross-correlation: y[i][j] = b + sum W[ky][kx] x[i + d ky][j + d kx]."""
    x, W, b = _f64(x), _f64(W), _f64(b)
    cin, h, w = x.shape
    cout, cin2, k, k2 = W.shape
    assert cin2 == cin and k == k2 and b.shape == (cout,)
    s = (k - 1) * dilation
    y = np.empty((cout, h - s, w - s), dtype=np.float64)
    _chk(_load().oracle_conv_dil(x.ctypes.data, cin, h, w, W.ctypes.data, b.ctypes.data, cout, k, dilation,
                                 int(relu), y.ctypes.data), "conv_dil")
    return y


def maxfilter2_dil(x, dilation: int) -> np.ndarray:
    x = _f64(x)
    c, h, w = x.shape
    y = np.empty((c, h - dilation, w - dilation), dtype=np.float64)
    _chk(_load().oracle_maxfilter2_dil(x.ctypes.data, c, h, w, dilation, y.ctypes.data), "maxfilter2_dil")
    return y


def maxout(x, groups: int) -> np.ndarray:
    """Max-out over consecutive channel groups: y[c] = max_g x[c*G + g]."""
    x = _f64(x)
    cg, h, w = x.shape
    assert cg % groups == 0
    y = np.empty((cg // groups, h, w), dtype=np.float64)
    _chk(_load().oracle_maxout(x.ctypes.data, cg // groups, groups, h * w, y.ctypes.data), "maxout")
    return y


def maxfilter2(x) -> np.ndarray:
    x = _f64(x)
    c, h, w = x.shape
    y = np.empty((c, h - 1, w - 1), dtype=np.float64)
    _chk(_load().oracle_maxfilter2(x.ctypes.data, c, h, w, y.ctypes.data), "maxfilter2")
    return y


def head_sigmoid(x, wv, b: float) -> np.ndarray:
    x, wv = _f64(x), _f64(wv)
    c, h, w = x.shape
    p = np.empty((h, w), dtype=np.float64)
    _chk(_load().oracle_head_sigmoid(x.ctypes.data, c, h, w, wv.ctypes.data, float(b), p.ctypes.data),
         "head_sigmoid")
    return p


def net_radius(layers) -> int:
    d = _desc(layers)
    return int(_load().oracle_net_radius(d.ctypes.data, len(d)))


def param_count(layers) -> int:
    d = _desc(layers)
    return int(_load().oracle_param_count(d.ctypes.data, len(d)))


def pad_region(slice_u8, y0, x0, h, w, R) -> np.ndarray:
    s = _u8(slice_u8)
    H, W = s.shape
    out = np.empty((h + 2 * R, w + 2 * R), dtype=np.float64)
    _chk(_load().oracle_pad_region(s.ctypes.data, H, W, W, y0, x0, h, w, R, out.ctypes.data), "pad_region")
    return out


def run_layers(layers, params, xp) -> np.ndarray:
    d, prm, xp = _desc(layers), _f64(params), _f64(xp)
    s = sum((int(row[1]) - 1) * int(row[5]) for row in d)
    ph, pw = xp.shape
    p = np.empty((ph - s, pw - s), dtype=np.float64)
    _chk(_load().oracle_run_layers(d.ctypes.data, len(d), prm.ctypes.data, xp.ctypes.data, ph, pw,
                                   p.ctypes.data), "run_layers")
    return p


def run_layers_mc(layers, params, xp) -> np.ndarray:
    """Layers on a multi-channel padded input xp [c][ph][pw]; the output is [classes][h][w] for an
    N-class softmax head, else [h][w]."""
    d, prm, xp = _desc(layers), _f64(params), _f64(xp)
    c, ph, pw = xp.shape
    s = sum((int(row[1]) - 1) * int(row[5]) for row in d)
    last = d[-1]
    nout = int(last[3]) if int(last[0]) == SOFTMAXN else 1
    p = np.empty((nout, ph - s, pw - s), dtype=np.float64)
    _chk(_load().oracle_run_layers_mc(d.ctypes.data, len(d), prm.ctypes.data, xp.ctypes.data, c, ph, pw,
                                      p.ctypes.data), "run_layers_mc")
    return p if nout > 1 else p[0]


def smooth_threshold(p, thr=0.5) -> np.ndarray:
    """J of the MaskExtend transfer: 3x3 mean (reflect-101) then >= thr, as uint8 0/1."""
    p = _f64(p)
    h, w = p.shape
    m = np.empty((h, w), dtype=np.uint8)
    _chk(_load().oracle_smooth_threshold(p.ctypes.data, h, w, float(thr), m.ctypes.data), "smooth_threshold")
    return m


def maskextend_input(em_u8, memb, masks, z, R, direction=1):
    """The 12-map input stack of MaskExtend at section z (Sec. 3.2), mirror-padded (reflect-101)
    by R. The maps sit at offsets k along the direction of travel s = +1 (z+) or -1 (z-), i.e. at
    sections z + s k: EM k = -1, 0, 1 (u/255), the object masks k = -4 .. -1 (0/1, the sections
    already extended), membrane maps k = -2 .. 2. For z+ that is EM z-1..z+1, masks z-4..z-1,
    membrane z-2..z+2; extending in z- mirrors the offsets (masks z+4..z+1).
    em_u8, memb: [Z][H][W]; masks: dict section -> [H][W] 0/1."""
    s = 1 if direction >= 0 else -1
    maps = [em_u8[z + s * k].astype(np.float64) / 255.0 for k in (-1, 0, 1)]
    maps += [np.asarray(masks[z + s * k], dtype=np.float64) for k in (-4, -3, -2, -1)]
    maps += [np.asarray(memb[z + s * k], dtype=np.float64) for k in (-2, -1, 0, 1, 2)]
    return np.stack([np.pad(m, R, mode="reflect") for m in maps])


def mask_extend(layers, params, em_u8, memb, seed_masks, z0, n_steps, thr=0.5, direction=1):
    """The MaskExtend recursion (Sec. 3.2, transfer equation), in z+ (direction 1) or z- (-1):
    with s the direction, Mask_z = J(CNN(masks at z + s k for k = -4..-1, EM at z + s k for
    k = -1..1, membrane at z + s k for k = -2..2)) for z = z0, z0 + s, ..., z0 + s (n_steps - 1).
    seed_masks[i] is the mask of section z0 + s (i - 4), i.e. the four sections before z0 in the
    direction of travel (z0-4 .. z0-1 for z+, z0+4 .. z0+1 for z-).
    Returns (masks [n][H][W] uint8, class probabilities [n][3][H][W]) in the order computed."""
    s = 1 if direction >= 0 else -1
    R = net_radius(layers)
    masks = {z0 + s * (i - 4): np.asarray(seed_masks[i]) for i in range(4)}
    out_m, out_p = [], []
    for t in range(n_steps):
        z = z0 + s * t
        p = run_layers_mc(layers, params, maskextend_input(em_u8, memb, masks, z, R, s))
        masks[z] = smooth_threshold(p[0], thr)
        out_m.append(masks[z])
        out_p.append(p)
    return np.stack(out_m), np.stack(out_p)


def forward_region(layers, params, slice_u8, y0=0, x0=0, h=None, w=None) -> np.ndarray:
    """Dense probabilities of the region [y0, y0+h) x [x0, x0+w) of one slice (FP64)."""
    d, prm, s = _desc(layers), _f64(params), _u8(slice_u8)
    H, W = s.shape
    h = H - y0 if h is None else h
    w = W - x0 if w is None else w
    p = np.empty((h, w), dtype=np.float64)
    _chk(_load().oracle_forward_region(d.ctypes.data, len(d), prm.ctypes.data, s.ctypes.data, H, W, W,
                                       y0, x0, h, w, p.ctypes.data), "forward_region")
    return p


def forward_volume(layers, params, vol_u8) -> np.ndarray:
    return np.stack([forward_region(layers, params, s) for s in vol_u8])


def patch_pixel(layers, params, slice_u8, i, j) -> float:
    d, prm, s = _desc(layers), _f64(params), _u8(slice_u8)
    H, W = s.shape
    out = np.empty(1, dtype=np.float64)
    _chk(_load().oracle_patch_pixel(d.ctypes.data, len(d), prm.ctypes.data, s.ctypes.data, H, W, W, i, j,
                                    out.ctypes.data), "patch_pixel")
    return float(out[0])


def features(layers, params, slice_u8, y0=0, x0=0, h=None, w=None) -> np.ndarray:
    """Activations entering the head of a conv / max-filter stack ([C][h][w], FP64) for the region
    [y0, y0+h) x [x0, x0+w) of one slice: the mirror-padded input through every layer but the
    last, composed from this module's conv and max-filter (dilation 1, no max-out)."""
    s = _u8(slice_u8)
    H, W = s.shape
    h = H - y0 if h is None else h
    w = W - x0 if w is None else w
    R = net_radius(layers)
    x = pad_region(s, y0, x0, h, w, R)[None]
    prm = _f64(params)
    o = 0
    for layer in layers[:-1]:
        kind, k, cin, cout = (int(v) for v in layer[:4])
        assert (len(layer) < 6 or int(layer[5]) == 1) and (len(layer) < 7 or int(layer[6]) == 1), layer
        if kind == CONV:
            nw = cout * cin * k * k
            x = conv(x, prm[o:o + nw].reshape(cout, cin, k, k), prm[o + nw:o + nw + cout], bool(layer[4]))
            o += nw + cout
        elif kind == MAXF:
            x = maxfilter2(x)
        else:
            raise ValueError(f"features: layer kind {kind} before the head")
    return x


def maxfilter_amax(layers, params, slice_u8, y0=0, x0=0, h=None, w=None, n_maxf=2, channels=32):
    d, prm, s = _desc(layers), _f64(params), _u8(slice_u8)
    H, W = s.shape
    h = H - y0 if h is None else h
    w = W - x0 if w is None else w
    out = np.zeros(n_maxf * channels, dtype=np.float64)
    _chk(_load().oracle_maxfilter_amax(d.ctypes.data, len(d), prm.ctypes.data, s.ctypes.data, H, W, W,
                                       y0, x0, h, w, out.ctypes.data, out.size), "maxfilter_amax")
    return out.reshape(n_maxf, channels)


def student_loss_grad(layers, params, slices_u8, targets):
    """Mean-squared-error loss of the student on n slices against target maps, and its gradient."""
    d, prm = _desc(layers), _f64(params)
    s = _u8(slices_u8)
    t = _f64(targets)
    n, H, W = s.shape
    assert t.shape == (n, H, W)
    grad = np.empty(prm.size, dtype=np.float64)
    loss = np.empty(1, dtype=np.float64)
    _chk(_load().oracle_student_loss_grad(d.ctypes.data, len(d), prm.ctypes.data, s.ctypes.data, n, H, W,
                                          W, H * W, t.ctypes.data, loss.ctypes.data, grad.ctypes.data),
         "student_loss_grad")
    return float(loss[0]), grad


def adam_step(w, m, v, g, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on FP64 arrays; returns (w, m, v)."""
    w, m, v, g = _f64(w).copy(), _f64(m).copy(), _f64(v).copy(), _f64(g)
    _chk(_load().oracle_adam_step(w.ctypes.data, m.ctypes.data, v.ctypes.data, g.ctypes.data, w.size, step,
                                  lr, b1, b2, eps), "adam_step")
    return w, m, v


def centred_layer1(layers, w):
    """Map student parameters to the coordinates in which layer 1 is optimised: the network
    rewritten for the zero-centred input x - 1/2. Correlating the mirror-padded input shifted by
    -1/2 with W1 shifts every output by -(1/2) sum W1, so the same map has bias
    c1 = b1 + (1/2) sum_k W1[co][k]; every other parameter is unchanged."""
    _, k, cin, cout = layers[0][:4]
    nw = cout * cin * k * k
    th = _f64(w).copy()
    th[nw:nw + cout] += 0.5 * th[:nw].reshape(cout, -1).sum(axis=1)
    return th


def plain_layer1(layers, th):
    """Inverse of centred_layer1: b1 = c1 - (1/2) sum_k W1[co][k]."""
    _, k, cin, cout = layers[0][:4]
    nw = cout * cin * k * k
    w = _f64(th).copy()
    w[nw:nw + cout] -= 0.5 * w[:nw].reshape(cout, -1).sum(axis=1)
    return w


def centred_grad(layers, g):
    """Gradient in the centred coordinates by the chain rule through b1 = c1 - (1/2) sum W1:
    dL/dW1[co][k] - (1/2) dL/db1[co] for the weights, dL/db1 for c1, the rest unchanged."""
    _, k, cin, cout = layers[0][:4]
    nw = cout * cin * k * k
    gc = _f64(g).copy()
    gc[:nw] = (gc[:nw].reshape(cout, -1) - 0.5 * gc[nw:nw + cout, None]).reshape(-1)
    return gc


def student_adam_step(layers, w, m, v, g, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One student training update: Adam (Kingma & Ba 2014) in the coordinates of centred_layer1,
    i.e. the step of training the same network on the centred input x - 1/2, mapped back to the
    stored form (input u/255). m and v are the moments of the centred gradients. Returns
    (w, m, v)."""
    th, m, v = adam_step(centred_layer1(layers, w), m, v, centred_grad(layers, g), step, lr, b1, b2, eps)
    return plain_layer1(layers, th), m, v


def metrics(p_gpu, p_ref) -> dict:
    """max-abs, mean-abs (FP64 sum), binarised agreement at 0.5 (p >= 0.5 is membrane), and the
    near-threshold mass: fraction of reference pixels with |p - 0.5| < max-abs."""
    a = np.asarray(p_gpu, dtype=np.float64)
    r = np.asarray(p_ref, dtype=np.float64)
    diff = np.abs(a - r)
    mx = float(diff.max()) if diff.size else 0.0
    return {
        "max_abs": mx,
        "mean_abs": float(diff.sum() / max(diff.size, 1)),
        "agreement": float(((a >= 0.5) == (r >= 0.5)).mean()) if diff.size else 1.0,
        "near_threshold": float((np.abs(r - 0.5) < mx).mean()) if diff.size else 0.0,
        "n": int(diff.size),
    }
