"""Parameter fit through the differentiable step (Sec. 3.4.2).

The paper fits simulation parameters (among them the viscosity) and a correction of
the initial velocity by minimising the masked loss of Eq. eq::optLoss between
simulated and observed surface velocities over the frames, with each parameter
mapped to its physical scale through exp or a sigmoid (Sec. 3.4.2). This module
runs that fit on the library:
  * theta = log nu and a per-face correction delta of the initial velocity;
  * the loss at every frame on the surface band, its gradient w.r.t. nu and the
    initial velocity from the checkpointed rollout's hand-written adjoint;
  * Adam on both, by the library's device kernel (fs_adam_update); every step,
    adjoint and optimiser update runs in the library's kernels.
The scene is a liquid blob on the floor with a shallow liquid layer fed by an
inflow patch on the x = 0 wall, gravity along -y. Targets are synthetic: a
forward run with nu_true and a seeded smooth delta_true, observed every frame.

    python -m paper_2503_00868_gb300.fit --nx 192 --ny 128 --nz 192 --frames 60 \\
        --iters 50 --precond learned
"""
from __future__ import annotations

import argparse
import json
import math
import time
from typing import Callable, Dict, Optional

import numpy as np
import torch

from . import fluidstep as F
from .clocks import ClockSampler
from . import workloads as W
from .rollout import forward_states, rollout_loss

PRECONDS = {"jacobi": F.FS_PRECOND_JACOBI, "mic0": F.FS_PRECOND_MIC0, "learned": F.FS_PRECOND_LEARNED,
            "mg": F.FS_PRECOND_MG, "learned_mg": F.FS_PRECOND_LEARNED_MG}
ADVECT_GRADS = {"exact": F.FS_ADVECT_GRAD_EXACT, "upwind": F.FS_ADVECT_GRAD_UPWIND}


def river_scene(nx: int, ny: int, nz: int, seed: int, inflow_speed: float = 0.5, depth: float = 0.25):
    """Cell types, prescribed face values (inflow on the x = 0 wall faces of liquid
    cells below `depth` m, zero on the other fixed faces) and scene info."""
    types, inflow, info = W.river_with_blob(nx, ny, nz, seed, depth)
    bc = [np.zeros(s) for s in W.face_shapes(nx, ny, nz)]
    bc[0] = np.where(inflow == 1, inflow_speed, 0.0)
    return types, bc, info


def make_grid(nx: int, ny: int, nz: int, types, bc, precond: str = "jacobi", nu: float = 1e-2,
              weights: Optional[np.ndarray] = None, percnn_kernel: Optional[np.ndarray] = None,
              percnn_k: int = 100, **kw) -> F.Grid:
    """A grid for the scene. With `percnn_kernel` every projection solves the
    pressure by `percnn_k` recurrent sub-steps of that kernel (Sec. 3.4.1)
    instead of PCG."""
    solver = F.FS_SOLVER_PERCNN if percnn_kernel is not None else F.FS_SOLVER_PCG
    g = F.Grid(nx, ny, nz, dx=1.0 / ny, dt=1.0 / 30.0, nu=nu, g=(0.0, -9.81, 0.0), precond=PRECONDS[precond],
               pressure_solver=solver, **kw)
    g.set_mask(types, g.pack(bc))
    if percnn_kernel is not None:
        F.fs_percnn_load(g.ctx, percnn_kernel, percnn_k)
    if precond in ("learned", "learned_mg"):
        if weights is None:
            from .train_precond import default_weights, role_weights
            weights = default_weights() if precond == "learned" else role_weights("net_mg")
        F.fs_net_load(g.ctx, weights)
    return g


def synthetic_targets(grid: F.Grid, u_base: F.Mac, delta_true: F.Mac, nu_true: float, frames: int):
    """Band observations of a forward run from u_base + delta_true with nu_true:
    {frame: state} for frames 1..frames."""
    grid.set_params(nu=nu_true)
    u0 = F.Mac(*(b + d for b, d in zip(u_base, delta_true)))
    states = forward_states(grid, u0, frames)
    return {n: states[n] for n in range(1, frames + 1)}


def fit(grid: F.Grid, u_base: F.Mac, targets: Dict[int, F.Mac], frames: int, iters: int = 50,
        nu0: float = 1e-3, lr_theta: float = 0.05, lr_delta: float = 1e-3, checkpoint_every: int = 4,
        fit_delta: bool = True, cosine: bool = False, betas=(0.9, 0.999),
        callback: Optional[Callable[[int, float, float], None]] = None) -> dict:
    """Adam on theta = log nu (and delta when `fit_delta`) against `targets`, with
    the learning rates decayed to zero along a cosine when `cosine`. The Adam step
    is the library's (fs_adam_update, on the device, one call per parameter
    tensor). Returns the fitted nu, delta and the (loss, nu) history before each
    update."""
    dev = u_base[0].device
    theta = torch.full((1,), math.log(nu0), dtype=torch.float32, device=dev, requires_grad=True)
    delta = [torch.zeros_like(t, requires_grad=fit_delta) for t in u_base]
    params = [(theta, lr_theta)] + ([(d, lr_delta) for d in delta] if fit_delta else [])
    moments = [(torch.zeros_like(t), torch.zeros_like(t)) for t, _ in params]
    history = []
    for it in range(iters):
        for t, _ in params:
            t.grad = None
        u0 = F.Mac(*(b + d for b, d in zip(u_base, delta)))
        nu = torch.exp(theta[0])
        loss = rollout_loss(grid, u0, nu, frames, targets, checkpoint_every)
        loss.backward()
        history.append((float(loss.detach()), float(nu.detach())))
        if callback:
            callback(it, history[-1][0], history[-1][1])
        decay = 0.5 * (1.0 + math.cos(math.pi * it / iters)) if cosine else 1.0
        with torch.no_grad():
            for (t, lr), (m, v) in zip(params, moments):
                g = t.grad if t.grad is not None else torch.zeros_like(t)
                F.fs_adam_update(grid.ctx, t, g.contiguous(), m, v, lr * decay, it + 1, betas[0], betas[1])
    return {"nu": float(torch.exp(theta[0]).detach()), "delta": [d.detach() for d in delta], "history": history}


def compare_pressure_solvers(nx: int = 64, ny: int = 48, nz: int = 64, frames: int = 12, iters: int = 30,
                             K: int = 100, seed: int = 0) -> dict:
    """The optimisation with the pressure from the fitted recurrent solver, from K
    Jacobi-like sub-steps (the same recurrence from its starting kernel) and from
    PCG to 1e-6, against targets made with PCG (the analogue of the paper's
    comparison of PeRCNN with Jacobi iterations in the optimisation): the loss
    after each update and the fitted nu."""
    from .train_percnn import default_kernel, jacobi_kernel
    types, bc, info = river_scene(nx, ny, nz, seed)
    ref = make_grid(nx, ny, nz, types, bc, "jacobi", tol_p=1e-6, maxit_p=20000)
    u_base = ref.pack(bc)
    d = W.blurred_noise_mac(nx, ny, nz, seed + 7)
    sc = 0.05 / max(float(np.std(np.concatenate([x.ravel() for x in d]))), 1e-12)
    targets = synthetic_targets(ref, u_base, ref.pack([x * sc for x in d]), 1e-2, frames)
    out = {"grid": [nx, ny, nz], "frames": frames, "iters": iters, "K": K, "runs": {}}
    for name, kern in (("pcg", None), ("percnn_fitted", default_kernel()), ("jacobi_substeps", jacobi_kernel())):
        g = ref if kern is None else make_grid(nx, ny, nz, types, bc, "jacobi", percnn_kernel=kern, percnn_k=K)
        t0 = time.time()
        res = fit(g, u_base, targets, frames, iters, 1e-3)
        torch.cuda.synchronize()
        out["runs"][name] = {"loss": [round(h[0], 6) for h in res["history"]], "nu_fit": res["nu"],
                             "s_per_iter": (time.time() - t0) / iters}
    return out


def compare_gradient_paths(nx: int = 64, ny: int = 48, nz: int = 64, frames: int = 12, iters: int = 30,
                           seed: int = 0) -> dict:
    """The fit with the reverse of convection by the exact discrete adjoint and by
    the paper's upwind surrogate (Sec. 3.4.1), against the same targets: the
    loss after each update and the fitted nu of each, and at the starting point
    the agreement of the two gradients (cosine of dL/du0, ratio of dL/dnu)."""
    types, bc, info = river_scene(nx, ny, nz, seed)
    ref = make_grid(nx, ny, nz, types, bc, "mg", tol_p=1e-6, maxit_p=20000)
    u_base = ref.pack(bc)
    d = W.blurred_noise_mac(nx, ny, nz, seed + 7)
    sc = 0.05 / max(float(np.std(np.concatenate([x.ravel() for x in d]))), 1e-12)
    targets = synthetic_targets(ref, u_base, ref.pack([x * sc for x in d]), 1e-2, frames)
    out = {"grid": [nx, ny, nz], "frames": frames, "iters": iters, "runs": {}, "start": {}}
    grads = {}
    for name, ag in ADVECT_GRADS.items():
        g = make_grid(nx, ny, nz, types, bc, "mg", tol_p=1e-6, maxit_p=20000, advect_grad=ag)
        leaves = [t.clone().requires_grad_(True) for t in u_base]
        nu = torch.tensor(1e-3, requires_grad=True)
        loss = rollout_loss(g, F.Mac(*leaves), nu, frames, targets, 4)
        loss.backward()
        grads[name] = (torch.cat([t.grad.reshape(-1).double() for t in leaves]), float(nu.grad))
        t0 = time.time()
        res = fit(g, u_base, targets, frames, iters, 1e-3)
        torch.cuda.synchronize()
        out["runs"][name] = {"loss": [round(h[0], 8) for h in res["history"]], "nu_fit": res["nu"],
                             "s_per_iter": (time.time() - t0) / iters}
        g.close()
    ge, gu = grads["exact"], grads["upwind"]
    out["start"] = {"cosine_dL_du0": float((ge[0] @ gu[0]) / (ge[0].norm() * gu[0].norm())),
                    "dL_dnu_exact": ge[1], "dL_dnu_upwind": gu[1]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=192)
    ap.add_argument("--ny", type=int, default=128)
    ap.add_argument("--nz", type=int, default=192)
    ap.add_argument("--frames", type=int, default=60)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--precond", default="learned", choices=sorted(PRECONDS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--nu-true", type=float, default=1e-2)
    ap.add_argument("--nu0", type=float, default=1e-3)
    ap.add_argument("--delta-sigma", type=float, default=0.05, help="std of the true correction, m/s")
    ap.add_argument("--advect-grad", default="exact", choices=sorted(ADVECT_GRADS))
    ap.add_argument("--compare-pressure-solvers", action="store_true",
                    help="run the PCG / fitted recurrent solver / Jacobi sub-step comparison instead")
    ap.add_argument("--compare-gradient-paths", action="store_true",
                    help="run the exact-adjoint / upwind-surrogate comparison instead")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    if a.compare_pressure_solvers:
        print(json.dumps(compare_pressure_solvers(seed=a.seed)), flush=True)
        return
    if a.compare_gradient_paths:
        print(json.dumps(compare_gradient_paths(seed=a.seed)), flush=True)
        return
    types, bc, info = river_scene(a.nx, a.ny, a.nz, a.seed)
    grid = make_grid(a.nx, a.ny, a.nz, types, bc, a.precond, maxit_p=20000, advect_grad=ADVECT_GRADS[a.advect_grad])
    u_base = grid.pack(bc)
    dt_np = W.blurred_noise_mac(a.nx, a.ny, a.nz, a.seed + 7)
    scale = a.delta_sigma / max(float(np.std(np.concatenate([x.ravel() for x in dt_np]))), 1e-12)
    delta_true = grid.pack([x * scale for x in dt_np])
    t0 = time.time()
    targets = synthetic_targets(grid, u_base, delta_true, a.nu_true, a.frames)
    torch.cuda.synchronize()
    t1 = time.time()
    log = []
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    res = fit(grid, u_base, targets, a.frames, a.iters, a.nu0,
              callback=lambda it, l, nu: (log.append((it, l, nu)), print(f"iter {it:3d} loss {l:.6e} nu {nu:.5e}",
                                                                          flush=True)))
    torch.cuda.synchronize()
    t2 = time.time()
    clocks = sampler.stop()
    cells = a.nx * a.ny * a.nz
    steps = a.iters * a.frames * 3  # forward, recompute, adjoint
    print(json.dumps({"metric": "fit iterations/s", "value": a.iters / (t2 - t1), "unit": "iter/s",
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "parameter fit (nu and the initial-velocity correction) on the river "
                                             "scene", "grid": [a.nx, a.ny, a.nz], "frames": a.frames,
                                 "iters": a.iters, "precond": a.precond, "advect_grad": a.advect_grad,
                                 "checkpoint_every": 4},
                      "clocks": clocks,
                      "occupancy": info["occupancy"], "nu_true": a.nu_true, "nu_fit": res["nu"],
                      "loss_first": res["history"][0][0], "loss_last": res["history"][-1][0],
                      "targets_s": t1 - t0, "fit_s": t2 - t1, "s_per_iter": (t2 - t1) / max(a.iters, 1),
                      "cell_steps_per_s": cells * steps / (t2 - t1)}), flush=True)
    grid.close()


if __name__ == "__main__":
    main()

