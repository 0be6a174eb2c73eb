"""APIC re-simulation of particles (Gaussians) through the grid step (Sec. 3.2.2,
Sec. 3.4.3): P2G with the affine matrices, the library's grid step (advection,
viscosity, projection), G2P with the C update, then advection of the particles and
the deformation gradient / covariance update of the Gaussians.

    python -m paper_2503_00868_gb300.apic --n 256 --ppc 4 --steps 3
times P2G, G2P and one APIC step on the ellipsoid-blob scene (the mask is held
fixed: cells are not re-marked from particle occupancy here).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import fluidstep as F
from . import workloads as W


class Particles:
    """Arrays of structures on the device: x, v (np, 3); C, F, A0, A (np, 9); m (np,)."""

    def __init__(self, x: torch.Tensor, m: torch.Tensor, A0: torch.Tensor):
        n = x.shape[0]
        dev = x.device
        self.x = x.contiguous()
        self.m = m.contiguous()
        self.v = torch.zeros(n, 3, device=dev)
        self.C = torch.zeros(n, 9, device=dev)
        self.F = torch.eye(3, device=dev).reshape(1, 9).repeat(n, 1).contiguous()
        self.A0 = A0.contiguous()
        self.A = A0.clone()


def seed_particles(types: np.ndarray, dx: float, ppc: int, seed: int, sigma: float = 0.3) -> Particles:
    """`ppc` jittered particles per liquid cell, unit mass per cell, isotropic
    covariance (sigma dx)^2."""
    rng = np.random.default_rng(seed)
    k, j, i = np.nonzero(types == W.LIQUID)
    cells = np.stack([i, j, k], axis=1).astype(np.float64)
    x = (np.repeat(cells, ppc, axis=0) + rng.random((cells.shape[0] * ppc, 3))) * dx
    n = x.shape[0]
    A0 = np.tile((np.eye(3) * (sigma * dx) ** 2).ravel(), (n, 1))
    return Particles(torch.tensor(x, dtype=torch.float32, device="cuda"),
                     torch.full((n,), 1.0 / ppc, device="cuda"),
                     torch.tensor(A0, dtype=torch.float32, device="cuda"))


def apic_step(grid: F.Grid, parts: Particles, u: F.Mac, u_next: F.Mac, lo: float, hi: float):
    """One re-simulation step: P2G -> grid step -> G2P + particle update."""
    F.fs_p2g(grid.ctx, parts.x, parts.v, parts.C, parts.m, u)
    rc, st = grid.step(u, u_next)
    F.fs_g2p(grid.ctx, parts.x, parts.v, parts.C, u_next, F=parts.F, A0=parts.A0, A_out=parts.A,
             dt=grid.params.dt, advance=True, lo=lo, hi=hi)
    return rc, st


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--ppc", type=int, default=4)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    n = a.n
    dx = 1.0 / n
    types, info = W.ellipsoid_blob(n, n, n, a.seed)
    g = F.Grid(n, n, n, dx=dx, dt=1.0 / 30.0, nu=0.01, g=(0.0, -9.81, 0.0), maxit_p=20000)
    g.set_mask(types)
    parts = seed_particles(types, dx, a.ppc, a.seed)
    npart = parts.x.shape[0]
    rng = np.random.default_rng(a.seed + 1)
    parts.v = torch.tensor(0.2 * rng.standard_normal((npart, 3)), dtype=torch.float32, device="cuda")
    u, u2 = g.zeros(), g.zeros()
    lo, hi = 1.5 * dx, (n - 1.5) * dx
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for _ in range(2):  # warm-up
        F.fs_p2g(g.ctx, parts.x, parts.v, parts.C, parts.m, u)
        F.fs_g2p(g.ctx, parts.x, parts.v, parts.C, u)
    torch.cuda.synchronize()
    e0, e1, e2 = ev(), ev(), ev()
    e0.record()
    F.fs_p2g(g.ctx, parts.x, parts.v, parts.C, parts.m, u)
    e1.record()
    F.fs_g2p(g.ctx, parts.x.clone(), parts.v, parts.C, u)
    e2.record()
    torch.cuda.synchronize()
    p2g_ms, g2p_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    s0, s1 = ev(), ev()
    s0.record()
    iters = []
    for _ in range(a.steps):
        rc, st = apic_step(g, parts, u, u2, lo, hi)
        iters.append(st["iters_p"])
    s1.record()
    torch.cuda.synchronize()
    step_ms = s0.elapsed_time(s1) / a.steps
    print(json.dumps({"grid": [n, n, n], "particles": npart, "ppc": a.ppc, "occupancy": info["occupancy"],
                      "p2g_ms": p2g_ms, "g2p_ms": g2p_ms,
                      "p2g_particles_per_s": npart / (p2g_ms * 1e-3), "g2p_particles_per_s": npart / (g2p_ms * 1e-3),
                      "apic_step_ms": step_ms, "pressure_iters": iters,
                      "finite": bool(torch.isfinite(parts.x).all() and torch.isfinite(parts.A).all())}))


if __name__ == "__main__":
    main()
