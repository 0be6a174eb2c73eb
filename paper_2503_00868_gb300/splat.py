"""Splatting render of the fluid's Gaussians into a headless image (Sec. 3.2.1,
Sec. 3.5): one Gaussian per liquid cell of an ellipsoid blob on an n^3 grid,
seen by a pinhole camera on a sphere around the blob.

    python -m paper_2503_00868_gb300.splat --n 128 --width 1920 --height 1080
times fs_splat_render (projection, tile binning, sorts, compositing, and the one
host synchronisation that sizes the key buffer) with CUDA events, after warm-up.
`--out file.npy` saves the image.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import fluidstep as F
from . import workloads as W


def scene(n: int, seed: int):
    types, info = W.ellipsoid_blob(n, n, n, seed)
    x, op, A, col = W.gaussian_cloud(types, 1.0 / n, seed)
    dev = lambda a, k: torch.tensor(np.asarray(a, np.float32).reshape(-1, k), device="cuda").contiguous()
    return dev(x, 3), dev(op, 1).reshape(-1), dev(A, 9), dev(col, 3), info


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    x, op, A, col, info = scene(a.n, a.seed)
    R, t, fx, fy, cx, cy = W.look_at([0.5, 0.2, 0.5], 1.6, 0.6, 0.35, a.width, a.height)
    cam = F.make_camera(R, t, fx, fy, cx, cy, a.width, a.height, 0.01, (0.1, 0.2, 0.3))
    grid = F.Grid(8, 8, 8)
    rgb = torch.empty(a.height, a.width, 3, device="cuda")
    T = torch.empty(a.height, a.width, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        F.fs_splat_render(grid.ctx, x, op, A, col, cam, rgb, T)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.reps + 1)]
    ev[0].record(stream)
    for r in range(a.reps):
        F.fs_splat_render(grid.ctx, x, op, A, col, cam, rgb, T)
        ev[r + 1].record(stream)
    torch.cuda.synchronize()
    ms = [ev[r].elapsed_time(ev[r + 1]) for r in range(a.reps)]
    med = float(np.median(ms))
    if a.out:
        np.save(a.out, rgb.cpu().numpy())
    print(json.dumps({"grid": [a.n] * 3, "gaussians": int(x.shape[0]), "image": [a.width, a.height],
                      "ms_per_frame_median": med, "ms_per_frame_min": float(min(ms)),
                      "frames_per_s": 1e3 / med, "gaussians_per_s": x.shape[0] / (med * 1e-3),
                      "covered_pixel_share": float((T < 1).float().mean()),
                      "tile_entries": F.fs_splat_stats(grid.ctx)["entries"],
                      "max_tile_entries": F.fs_splat_stats(grid.ctx)["max_tile"],
                      "finite": bool(torch.isfinite(rgb).all())}))


if __name__ == "__main__":
    main()
