"""Train and evaluate the learned pressure preconditioner.

The paper fits a convolutional network to (right-hand side, pressure) pairs
recorded from an implicit solver and then uses it for the pressure solve
(Sec. 3.4.1, Fig. percnn_str_fit). Here the pairs come from the library itself:
b = -dx div(u) for seeded N(0, 1) MAC fields u (unblurred, the projection
right-hand side of the stress workload, and blurred) on liquid-blob and
sphere-union masks, q from MIC(0)-PCG to a tight tolerance, plus residual/error
pairs of truncated CG runs. The network (five 3x3x3 convolutions)
is trained with Adam through the library's own forward/backward kernels, then
used as the preconditioner of flexible CG and compared, by iterations and wall
time to relative residual 1e-6, with Jacobi and MIC(0) PCG.

    python -m paper_2503_00868_gb300.train_precond --n 64 --masks 8 --rhs 4 \
        --steps 300 --out weights.npy --eval-n 128

The shipped weights (weights/precond_n48.npy) come from
    python -m paper_2503_00868_gb300.train_precond --n 48 --masks 8 --rhs 6 \
        --steps 300 --lr 2e-3 --seed 0 --out precond_n48.npy
(192 pairs at 48^3, energy-norm loss 1.02 -> 0.168).
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

CH = (2, 16, 16, 16, 16, 1)
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "precond_n48.npy")


def default_weights() -> np.ndarray:
    """The trained network shipped with the package (flat FP32, fs_net_load order)."""
    return np.load(DEFAULT_WEIGHTS).astype(np.float32)


def init_params(seed: int) -> np.ndarray:
    """He-initialised conv weights, a small last layer; zero biases and zero
    weights on the cell-type channel. Training keeps those offsets at zero, so the
    network stays positively homogeneous in the residual (Net(a x) = a Net(x),
    a >= 0), which flexible CG needs as the residual shrinks."""
    rng = np.random.default_rng(seed)
    flat = []
    for l in range(5):
        fan = CH[l] * 27
        w = rng.standard_normal((CH[l + 1], CH[l], 3, 3, 3)) * np.sqrt(2.0 / fan)
        if l == 0:
            w[:, 1] = 0.0
        if l == 4:
            w *= 0.1
        flat += [w.ravel(), np.zeros(CH[l + 1])]
    return np.concatenate(flat).astype(np.float32)


def make_mask(n: int, k: int, seed: int) -> np.ndarray:
    """Alternate liquid blobs on the floor and unions of spheres."""
    if k % 2 == 0:
        return W.ellipsoid_blob(n, n, n, seed)[0]
    return W.sphere_union(n, n, n, seed)[0]


def make_pairs(n: int, masks, rhs: int, seed: int, tol: float = 1e-7, cg_iters=(2, 8, 32)):
    """[(types, [(b, q), ...])] with L_p q = b.

    Base pairs: b = -dx div(u) for seeded MAC fields u, q from MIC(0)-PCG to
    `tol`. Each base pair also yields one pair per k in `cg_iters` taken from
    Jacobi-PCG stopped after k iterations at x_k: the residual r_k = b - L_p x_k
    (the divergence left in u after subtracting grad x_k) and the error
    q - x_k. These are the smoother right-hand sides the preconditioner meets
    inside flexible CG."""
    g = F.Grid(n, n, n, dx=1.0 / n, tol_p=tol, maxit_p=20000, precond=F.FS_PRECOND_MIC0)
    gj = F.Grid(n, n, n, dx=1.0 / n, tol_p=1e-12, maxit_p=1, precond=F.FS_PRECOND_JACOBI)
    out = []
    for mi, types in enumerate(masks):
        g.set_mask(types)
        gj.set_mask(types)
        pairs = []
        for k in range(rhs):
            # rough and smooth right-hand sides (blur sigma 0, 1, 2 cells)
            sigma = k % 3
            sd = seed + 1000 * mi + k
            field = (W.random_mac(n, n, n, sd) if sigma == 0
                     else W.blurred_noise_mac(n, n, n, sd, sigma_cells=float(sigma), radius=3 * sigma))
            u = g.pack(field)
            b = g.empty_cell()
            F.fs_divergence(g.ctx, u, b)
            q = g.empty_cell()
            g.project(F.Mac(*(t.clone() for t in u)), q)
            pairs.append((b, q))
            for it in cg_iters:
                gj.set_params(maxit_p=it)
                uk = F.Mac(*(t.clone() for t in u))
                xk = gj.empty_cell()
                gj.project(uk, xk)  # stops at the iteration cap (FS_ENOCONV)
                rk = gj.empty_cell()
                F.fs_divergence(gj.ctx, uk, rk)
                pairs.append((rk, q - xk))
        out.append((types, pairs))
    g.close()
    gj.close()
    return out


def train(n: int, data, params: np.ndarray, steps: int, lr: float, log_every: int = 25):
    g = F.Grid(n, n, n, dx=1.0 / n)
    g.set_mask(data[0][0])
    F.fs_net_load(g.ctx, params)
    npairs = sum(len(p) for _, p in data)
    history = []
    for step in range(1, steps + 1):
        lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * (step - 1) / steps)) + 1e-5
        total = 0.0
        for types, pairs in data:
            g.set_mask(types)
            for b, q in pairs:
                total += F.fs_net_grad(g.ctx, b, q)
        F.fs_net_adam(g.ctx, lr_t, step, grad_scale=1.0 / npairs)
        history.append(total / npairs)
        if log_every and (step % log_every == 0 or step == 1):
            print(f"step {step:5d} lr {lr_t:.2e} loss {history[-1]:.5f}", flush=True)
    out = F.fs_net_read(g.ctx)
    g.close()
    return out, history


def timed_project(g: F.Grid, u0: F.Mac):
    u = F.Mac(*(t.clone() for t in u0))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rc, st = g.project(u)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, rc, st


def compare(n: int, params: np.ndarray, seeds=(0,), tol: float = 1e-6, warm: bool = True):
    """Wall time and iterations of the projection to relative residual `tol`
    with Jacobi, MIC(0) and the learned preconditioner (flexible CG)."""
    rows = []
    grids = {name: F.Grid(n, n, n, dx=1.0 / n, tol_p=tol, maxit_p=20000, precond=pc)
             for name, pc in (("jacobi", F.FS_PRECOND_JACOBI), ("mic0", F.FS_PRECOND_MIC0),
                              ("learned", F.FS_PRECOND_LEARNED))}
    F.fs_net_load(grids["learned"].ctx, params)
    for seed in seeds:
        types, info = W.sphere_union(n, n, n, seed)
        row = {"n": n, "seed": seed, "occupancy": info["occupancy"]}
        for name, g in grids.items():
            g.set_mask(types)
            u0 = g.pack(W.random_mac(n, n, n, 500 + seed))
            if warm:
                timed_project(g, u0)  # the MIC(0) factor and first-touch costs
            t, rc, st = timed_project(g, u0)
            row[name] = {"seconds": t, "iters": st["iters_p"], "true_relres": st["true_relres_p"],
                         "fallbacks": st["fallbacks"], "status": rc}
        rows.append(row)
    for g in grids.values():
        g.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--masks", type=int, default=8)
    ap.add_argument("--rhs", type=int, default=6)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="precond_weights.npy")
    ap.add_argument("--eval-n", type=int, nargs="*", default=[128])
    a = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.time()
    masks = [make_mask(a.n, k, a.seed + k) for k in range(a.masks)]
    data = make_pairs(a.n, masks, a.rhs, a.seed)
    t1 = time.time()
    params, hist = train(a.n, data, init_params(a.seed), a.steps, a.lr)
    t2 = time.time()
    np.save(a.out, params)
    report = {"pairs": a.masks * a.rhs, "n": a.n, "steps": a.steps, "loss_first": hist[0], "loss_last": hist[-1],
              "data_seconds": t1 - t0, "train_seconds": t2 - t1, "compare": []}
    for n in a.eval_n:
        report["compare"] += compare(n, params)
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()
