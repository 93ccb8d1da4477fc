"""Writes truth_head.json: the head (1x1 conv 32 -> 1 + sigmoid) of the stand-in teacher fitted to
the synthetic generator's own membrane truth, for the second teacher workload.

The stand-in teacher's layers 1-3 keep their seeded He-normal weights; only the head changes. With
random weights the stand-in's map sits in a narrow band around 0.58, so binarised agreement and
the stated fallback band [0.3, 0.7] say little about it. A trained membrane classifier's head maps
its last features to a calibrated membrane probability: here that is L2-regularised logistic
regression (maximum likelihood of the generator's membrane flag given the layer-3 features) on
standardised features, solved by Newton's method. The regularisation strength is chosen on
held-out slices: the largest lambda of a decade grid whose held-out accuracy is within 0.1
percentage point of the best (prefer the smoother head when accuracy is the same).

Calls only the oracle (FP64 layer-3 features) and the seeded generator:
    python tests/golden/fit_truth_head.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

SIDE = 256
TRAIN = (synth.BASE_SEED + 20, 8)      # (base seed, slices)
HELD_OUT = (synth.BASE_SEED + 22, 4)
LAMBDAS = (1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1)


def slices(base, n):
    feats, truth = [], []
    params = synth.init_params(synth.TEACHER, synth.TEACHER_WEIGHT_SEED)
    for i in range(n):
        s, t = synth.em_slice_truth(synth.slice_seed(base, 0, i), SIDE, SIDE)
        feats.append(oracle.features(synth.TEACHER, params, s).reshape(32, -1).T)
        truth.append(t.reshape(-1))
    return np.concatenate(feats), np.concatenate(truth).astype(np.float64)


def fit(a, y, lam, iters=60):
    """Minimise mean log-loss + lam/2 |w|^2 (bias unpenalised) over [a, 1] by Newton's method."""
    a1 = np.hstack([a, np.ones((a.shape[0], 1))])
    pen = lam * np.eye(a1.shape[1])
    pen[-1, -1] = 0.0
    w = np.zeros(a1.shape[1])
    n = len(y)
    for _ in range(iters):
        p = 1.0 / (1.0 + np.exp(-(a1 @ w)))
        g = a1.T @ (p - y) / n + pen @ w
        hess = (a1 * (p * (1.0 - p))[:, None]).T @ a1 / n + pen
        w -= np.linalg.solve(hess, g)
    return w


def main():
    xt, yt = slices(*TRAIN)
    xv, yv = slices(*HELD_OUT)
    mu, sd = xt.mean(axis=0), xt.std(axis=0)
    sd[sd == 0] = 1.0
    cands = []
    for lam in LAMBDAS:
        ws = fit((xt - mu) / sd, yt, lam)
        w = ws[:32] / sd                       # back to the raw features
        b = ws[32] - float((mu / sd) @ ws[:32])
        acc = float((((xv @ w + b) >= 0) == (yv > 0.5)).mean())
        cands.append((lam, acc, w, b))
    best = max(c[1] for c in cands)
    lam, acc, w, b = max((c for c in cands if c[1] >= best - 1e-3), key=lambda c: c[0])
    w32 = np.asarray(w, dtype=np.float32)
    out = {"what": "stand-in teacher head fitted to the generator's membrane truth (second teacher workload)",
           "head_w": [float(v) for v in w32], "head_b": float(np.float32(b)), "lambda": lam,
           "held_out_accuracy": acc, "held_out_accuracy_by_lambda": {f"{c[0]:g}": c[1] for c in cands},
           "train": {"base_seed": TRAIN[0], "slices": TRAIN[1], "side": SIDE},
           "held_out": {"base_seed": HELD_OUT[0], "slices": HELD_OUT[1], "side": SIDE},
           "membrane_fraction_held_out": float(yv.mean())}
    with open(os.path.join(HERE, "truth_head.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"lambda {lam:g}, held-out accuracy {acc:.4f}")


if __name__ == "__main__":
    main()
