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

The data set of the learned-preconditioner configuration (``--c4``): 4000 pairs,
3000 at 64^3 and 1000 at 128^3, on ellipsoid blobs and sphere unions (radii
scaled by n/256) in equal numbers, split 3600 / 400 for training and validation.
``--role net_mg`` trains the network for FS_PRECOND_LEARNED_MG, where one V-cycle
follows it: the loss is then the energy-norm error left after the network and
the V-cycle together, so the network learns what the V-cycle misses.
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


def role_weights(role: str) -> np.ndarray:
    """The network trained for a role on the 4000-pair data set (``--c4``):
    "net" (FS_PRECOND_LEARNED) or "net_mg" (FS_PRECOND_LEARNED_MG)."""
    path = os.path.join(os.path.dirname(DEFAULT_WEIGHTS), f"precond_{role}_c4.npy")
    return np.load(path).astype(np.float32)


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


ROLES = {"net": F.FS_PRECOND_LEARNED, "net_mg": F.FS_PRECOND_LEARNED_MG}


def c4_data(seed: int = 0, n64: int = 3000, n128: int = 1000, per_mask: int = 50):
    """The pairs of the learned-preconditioner configuration: n64 pairs at 64^3
    and n128 at 128^3, `per_mask` per mask (ten right-hand sides, each with the
    residual/error pairs of Jacobi-PCG stopped after 2, 8, 32 and 128
    iterations), blobs and sphere unions alternating. Returns {n: [(types,
    pairs)]}."""
    rhs = per_mask // 5
    out = {}
    for n, count, base in ((64, n64, 0), (128, n128, 10000)):
        nmask = max(1, count // per_mask)
        masks = [make_mask(n, k, seed + base + k) for k in range(nmask)]
        out[n] = make_pairs(n, masks, rhs, seed + base, cg_iters=(2, 8, 32, 128))
    return out


def split(data, val_every: int = 10):
    """Every val_every-th pair of each mask goes to validation (3600 / 400)."""
    tr, va = {}, {}
    for n, items in data.items():
        tr[n] = [(t, [p for i, p in enumerate(ps) if i % val_every != val_every - 1]) for t, ps in items]
        va[n] = [(t, [p for i, p in enumerate(ps) if i % val_every == val_every - 1]) for t, ps in items]
    return tr, va


def train_batched(data, params: np.ndarray, role: str, epochs: int, batch: int, lr: float, seed: int = 0,
                  val=None, log=True):
    """Adam over minibatches of `batch` pairs of one mask (in shuffled order),
    `epochs` passes over the training pairs, cosine learning rate; the loss
    follows the role (FS_PRECOND_LEARNED or FS_PRECOND_LEARNED_MG). Returns the
    parameters and per-epoch (train loss, validation loss)."""
    rng = np.random.default_rng(seed)
    # one context per grid size, each with its own Adam moments and step count;
    # the parameters move between them when the size changes (once per epoch:
    # the minibatches of each size run together, in shuffled order)
    grids = {n: F.Grid(n, n, n, dx=1.0 / n, precond=ROLES[role]) for n in data}
    cur = params
    batches = {n: [] for n in data}
    for n, items in data.items():
        for mi, (types, pairs) in enumerate(items):
            idx = np.arange(len(pairs))
            for k in range(0, len(idx), batch):
                batches[n].append((mi, list(idx[k:k + batch])))
    total_steps = epochs * sum(len(v) for v in batches.values())
    hist, step = [], 0
    steps_of = {n: 0 for n in data}
    last_n = None
    for ep in range(epochs):
        tl, tc = 0.0, 0
        for n in rng.permutation(sorted(data)):
            n = int(n)
            g = grids[n]
            if last_n != n:
                if last_n is not None:
                    cur = F.fs_net_read(grids[last_n].ctx)
                F.fs_net_load(g.ctx, cur)
                last_n = n
            for bi in rng.permutation(len(batches[n])):
                mi, idx = batches[n][bi]
                types, pairs = data[n][mi]
                g.set_mask(types)
                for j in idx:
                    b, q = pairs[j]
                    tl += F.fs_net_grad(g.ctx, b, q)
                    tc += 1
                step += 1
                steps_of[n] += 1
                lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * (step - 1) / total_steps)) + 1e-5
                F.fs_net_adam(g.ctx, lr_t, steps_of[n], grad_scale=1.0 / len(idx))
        cur = F.fs_net_read(grids[last_n].ctx)
        vl = evaluate_loss(val, cur, role) if val else None
        hist.append((tl / max(tc, 1), vl))
        if log:
            print(f"epoch {ep + 1}: train loss {hist[-1][0]:.4f} validation {vl}", flush=True)
    for g in grids.values():
        g.close()
    return cur, hist


def evaluate_loss(data, params: np.ndarray, role: str) -> float:
    """Mean loss over the pairs of `data`, on contexts of its own (the gradients
    they accumulate are dropped with them)."""
    tot, cnt = 0.0, 0
    for n, items in data.items():
        g = F.Grid(n, n, n, dx=1.0 / n, precond=ROLES[role])
        F.fs_net_load(g.ctx, params)
        for types, pairs in items:
            g.set_mask(types)
            for b, q in pairs:
                tot += F.fs_net_grad(g.ctx, b, q)
                cnt += 1
        g.close()
    return tot / max(cnt, 1)


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


def compare(n: int, nets, seeds=(0,), tol: float = 1e-6, warm: bool = True):
    """Wall time and iterations of the projection to relative residual `tol`
    with Jacobi, MIC(0), the multigrid V-cycle and each learned preconditioner of
    `nets` ({name: (params, FS_PRECOND_LEARNED or FS_PRECOND_LEARNED_MG)}, in
    flexible CG), on sphere unions at n^3."""
    rows = []
    spec = [("jacobi", F.FS_PRECOND_JACOBI, None), ("mic0", F.FS_PRECOND_MIC0, None), ("mg", F.FS_PRECOND_MG, None)]
    spec += [(name, pc, params) for name, (params, pc) in nets.items()]
    for seed in seeds:
        types, info = W.sphere_union(n, n, n, seed)
        row = {"n": n, "seed": seed, "occupancy": info["occupancy"]}
        for name, pc, params in spec:
            g = F.Grid(n, n, n, dx=1.0 / n, tol_p=tol, maxit_p=20000, precond=pc)
            g.set_mask(types)
            if params is not None:
                F.fs_net_load(g.ctx, params)
            u0 = g.pack(W.random_mac(n, n, n, 500 + seed))
            if warm:
                timed_project(g, u0)  # the MIC(0) factor, the hierarchy and first-touch costs
            t, rc, st = timed_project(g, u0)
            row[name] = {"ms": round(1e3 * t, 3), "iters": st["iters_p"], "true_relres": st["true_relres_p"],
                         "fallbacks": st["fallbacks"], "status": rc}
            g.close()
        rows.append(row)
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
    ap.add_argument("--c4", action="store_true",
                    help="train on the 4000-pair data set (3000 at 64^3, 1000 at 128^3), minibatched")
    ap.add_argument("--roles", nargs="*", default=["net", "net_mg"], choices=list(ROLES))
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--out-dir", default=".")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.time()
    if a.c4:
        data = c4_data(a.seed)
        tr, va = split(data)
        t1 = time.time()
        nets, report = {}, {"pairs": {n: sum(len(p) for _, p in items) for n, items in data.items()},
                            "train_pairs": {n: sum(len(p) for _, p in items) for n, items in tr.items()},
                            "data_seconds": t1 - t0, "roles": {}}
        for role in a.roles:
            t2 = time.time()
            init = init_params(a.seed)
            v0 = evaluate_loss(va, init, role)
            params, hist = train_batched(tr, init, role, a.epochs, a.batch, a.lr, a.seed, val=va)
            out = os.path.join(a.out_dir, f"precond_{role}_c4.npy")
            np.save(out, params)
            nets["learned" if role == "net" else "learned_mg"] = (params, ROLES[role])
            report["roles"][role] = {"validation_loss_init": v0, "epochs": hist, "train_seconds": time.time() - t2,
                                     "weights": out}
        report["compare"] = []
        for n in a.eval_n:
            report["compare"] += compare(n, nets)
        print(json.dumps(report), flush=True)
        return
    masks = [make_mask(a.n, k, a.seed + k) for k in range(a.masks)]
    data = make_pairs(a.n, masks, a.rhs, a.seed)
    t1 = time.time()
    params, hist = train(a.n, data, init_params(a.seed), a.steps, a.lr)
    t2 = time.time()
    np.save(a.out, params)
    report = {"pairs": a.masks * a.rhs, "n": a.n, "steps": a.steps, "loss_first": hist[0], "loss_last": hist[-1],
              "data_seconds": t1 - t0, "train_seconds": t2 - t1, "compare": []}
    for n in a.eval_n:
        report["compare"] += compare(n, {"learned": (params, F.FS_PRECOND_LEARNED)})
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()
