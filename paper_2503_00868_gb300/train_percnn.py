"""Fit the kernel of the recurrent convolutional pressure solver (Sec. 3.4.1).

The paper validates its PeRCNN layer on (right-hand side, pressure) pairs recorded
from an implicit solver and then uses the fitted kernel to solve the pressure in
the optimisation. Here the pairs come from the library (divergence of seeded MAC
fields, pressure from MIC(0)-PCG; `train_precond.make_pairs`), the loss is the
energy norm of the K-sub-step pressure error, and Adam runs on the 14 free taps
of the point-symmetric 3x3x3 kernel (the library stores it symmetric), from the
under-relaxed Jacobi kernel (center 1/6).

    python -m paper_2503_00868_gb300.train_percnn --n 48 --masks 8 --rhs 6 \\
        --K 100 --steps 200 --out percnn_k100.npy --eval-n 128
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import fluidstep as F
from . import workloads as W
from .train_precond import make_mask
from .train_precond import make_pairs as _make_pairs

DEFAULT_KERNEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "percnn_k100.npy")


def jacobi_kernel() -> np.ndarray:
    """The starting kernel: center tap 1/6 (under-relaxed Jacobi sub-steps)."""
    w = np.zeros(27)
    w[13] = 1.0 / 6.0
    return w


def default_kernel() -> np.ndarray:
    """The fitted kernel shipped with the package (27 taps, K = 100)."""
    return np.load(DEFAULT_KERNEL).astype(np.float64)


def expand(theta: np.ndarray) -> np.ndarray:
    """14 free taps (t = 0..12 and the center) -> the point-symmetric 27-tap kernel."""
    w = np.empty(27)
    w[:14] = theta
    w[14:] = theta[12::-1]
    return w


def reduce_grad(dw: np.ndarray) -> np.ndarray:
    """Gradient w.r.t. the 27 taps -> w.r.t. the 14 free taps."""
    g = np.empty(14)
    g[:13] = dw[:13] + dw[26:13:-1]
    g[13] = dw[13]
    return g


def make_pairs(n: int, masks, rhs: int, seed: int):
    return _make_pairs(n, masks, rhs, seed)


def fit(n: int, data, w0: np.ndarray, K: int = 100, steps: int = 200, lr: float = 2e-3, log_every: int = 25):
    """Adam (on the host: 14 numbers) with the library's loss and gradient."""
    g = F.Grid(n, n, n, dx=1.0 / n)
    g.set_mask(data[0][0])
    theta = np.concatenate([np.asarray(w0, float)[:13], [float(w0[13])]])
    m = np.zeros(14)
    v = np.zeros(14)
    b1, b2, eps = 0.9, 0.999, 1e-12
    npairs = sum(len(p) for _, p in data)
    hist = []
    for step in range(1, steps + 1):
        F.fs_percnn_load(g.ctx, expand(theta), K)
        total, grad = 0.0, np.zeros(27)
        for types, pairs in data:
            g.set_mask(types)
            for b, q in pairs:
                l, dw = F.fs_percnn_grad(g.ctx, b, q)
                total += l
                grad += dw
        hist.append(total / npairs)
        gt = reduce_grad(grad / npairs)
        m = b1 * m + (1 - b1) * gt
        v = b2 * v + (1 - b2) * gt * gt
        lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * (step - 1) / steps))
        theta -= lr_t * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
        if log_every and (step % log_every == 0 or step == 1):
            print(f"step {step:4d} loss {hist[-1]:.5f}", flush=True)
    g.close()
    return expand(theta), hist


def energy_error(n: int, w: np.ndarray, K: int, seeds=(0,)):
    """Energy-norm relative error of K sub-steps on unseen sphere unions at n^3."""
    out = []
    for seed in seeds:
        types, info = W.sphere_union(n, n, n, seed + 50)
        data = _make_pairs(n, [types], 2, 900 + seed)
        g = F.Grid(n, n, n, dx=1.0 / n)
        g.set_mask(types)
        F.fs_percnn_load(g.ctx, w, K)
        errs = [F.fs_percnn_grad(g.ctx, b, q)[0] for b, q in data[0][1][:2]]
        g.close()
        out.append(float(np.mean(errs)))
    return float(np.mean(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--masks", type=int, default=8)
    ap.add_argument("--rhs", type=int, default=6)
    ap.add_argument("--K", type=int, default=100)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="percnn_k100.npy")
    ap.add_argument("--eval-n", type=int, nargs="*", default=[128])
    a = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.time()
    masks = [make_mask(a.n, k, a.seed + k) for k in range(a.masks)]
    data = make_pairs(a.n, masks, a.rhs, a.seed)
    t1 = time.time()
    w, hist = fit(a.n, data, jacobi_kernel(), a.K, a.steps, a.lr)
    t2 = time.time()
    np.save(a.out, w.astype(np.float32))
    rep = {"n": a.n, "pairs": sum(len(p) for _, p in data), "K": a.K, "loss_first": hist[0],
           "loss_last": hist[-1], "data_s": t1 - t0, "fit_s": t2 - t1, "kernel": [round(x, 6) for x in w],
           "eval": []}
    for n in a.eval_n:
        rep["eval"].append({"n": n, "jacobi_like": energy_error(n, jacobi_kernel(), a.K),
                            "fitted": energy_error(n, w, a.K)})
    print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()
