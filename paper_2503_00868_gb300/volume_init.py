"""Volumetric-velocity initialisation (Sec. 3.3.3) on the library.

The paper builds the initial volumetric velocity from the observed surface
velocity: a laminar wall-function profile damps the base velocity towards the
riverbed, then the constrained projection of Eq. eq::divProj makes the field
divergence-free while the enclosure (the observed free surface and the walls)
keeps its values. Here the surface speed per cell column is an input (the video
is not available; synthetic columns stand in for it).

    python -m paper_2503_00868_gb300.volume_init --n 256 --iters 200
prints the time per projection iteration and its algorithmic bandwidth.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import fluidstep as F
from . import workloads as W


def volume_init(grid: F.Grid, direction, vinf: torch.Tensor, delta: float, iters: int, eps: float,
                hold_surface: bool = True):
    """Base profile then `iters` constrained-projection iterations; returns the
    field and |div|_2 before and after the projection."""
    u = grid.zeros()
    F.fs_wall_profile(grid.ctx, direction, vinf, delta, u)
    n0 = F.fs_pbd_project(grid.ctx, u, hold_surface, 0, eps)
    n1 = F.fs_pbd_project(grid.ctx, u, hold_surface, iters, eps)
    return u, n0, n1


def synthetic_surface_speed(nx: int, nz: int, seed: int, mean: float = 0.5) -> np.ndarray:
    """Smooth positive column speeds (nz, nx) around `mean`."""
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 2 * np.pi, nx)[None, :]
    z = np.linspace(0, 2 * np.pi, nz)[:, None]
    a, b = rng.uniform(0, 2 * np.pi, 2)
    return mean * (1.0 + 0.3 * np.sin(x + a) * np.cos(z + b))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    n = a.n
    types, inflow, info = W.river_with_blob(n, n, n, a.seed)
    bc = [np.zeros(s) for s in W.face_shapes(n, n, n)]
    bc[0] = np.where(inflow == 1, 0.5, 0.0)
    g = F.Grid(n, n, n, dx=1.0 / n)
    g.set_mask(types, g.pack(bc))
    vinf = torch.tensor(synthetic_surface_speed(n, n, a.seed), dtype=torch.float32, device="cuda").contiguous()
    eps = 0.5 * n * n
    volume_init(g, (1.0, 0.0, 0.0), vinf, 0.1, 5, eps)  # warm-up
    u = g.zeros()
    F.fs_wall_profile(g.ctx, (1.0, 0.0, 0.0), vinf, 0.1, u)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    norm = F.fs_pbd_project(g.ctx, u, True, a.iters, eps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lay = F.fs_layout(g.ctx)
    S = lay.nelems
    # per iteration and element of the public layout: read 3 face arrays + cell flag,
    # write lambda (17 B); read lambda, 3 face flags, 3 face arrays, write them (31 B)
    bytes_iter = 48.0 * S
    per_it = ms / (a.iters + 1) * 1e-3
    print(json.dumps({"grid": [n, n, n], "occupancy": info["occupancy"], "iters": a.iters,
                      "ms": ms, "us_per_iteration": per_it * 1e6, "div_norm_after": norm,
                      "algorithmic_bytes_per_iteration": bytes_iter, "achieved_GBps": bytes_iter / per_it / 1e9}))


if __name__ == "__main__":
    main()
