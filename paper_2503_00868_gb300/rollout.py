"""Checkpointed differentiable rollout over the C ABI (arXiv 2503.00868, Sec. 3.4.2).

The paper optimises v_sim^{i+n} = DiffSim^n(v^i; nu, ...) under the masked loss of
Eq. eq::optLoss over deep graphs (up to 25 steps, Sec. 3.4.2). ``rollout_loss``
runs n steps, adds the loss at the requested frames, and differentiates w.r.t.
the initial velocity and the viscosity through the library's hand-written
adjoint. Only every k-th state is stored on the way forward; the backward pass
recomputes one segment at a time (keeping that segment's states and the fields
after viscosity), so memory is O(n/k + k) fields instead of O(n).

torch is used for memory, streams and autograd plumbing only; every step, loss
and adjoint runs in the library's kernels.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import torch

from . import fluidstep as F


def _clone(m: F.Mac) -> F.Mac:
    return F.Mac(*(t.clone() for t in m))


class _RolloutLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, grid: F.Grid, nsteps: int, k: int, targets: Dict[int, F.Mac], alpha: float,
                beta: float, mask_kind: int, stats: Optional[list], nu: torch.Tensor, u0: torch.Tensor,
                v0: torch.Tensor, w0: torch.Tensor):
        grid.set_params(nu=float(nu.detach().cpu()))
        cur = F.Mac(u0.detach().contiguous(), v0.detach().contiguous(), w0.detach().contiguous())
        checkpoints = {0: _clone(cur)}
        loss = 0.0
        if 0 in targets:
            loss += grid.loss_grad(cur, targets[0], mask_kind, alpha, beta)
        a, b = _clone(cur), grid.zeros()
        for n in range(1, nsteps + 1):
            rc, st = grid.step(a, b)
            if stats is not None:
                stats.append(("fwd", n, st))
            a, b = b, a
            if n % k == 0 and n < nsteps:
                checkpoints[n] = _clone(a)
            if n in targets:
                loss += grid.loss_grad(a, targets[n], mask_kind, alpha, beta)
        ctx.grid, ctx.nsteps, ctx.k = grid, nsteps, k
        ctx.targets, ctx.alpha, ctx.beta, ctx.mask_kind = targets, alpha, beta, mask_kind
        ctx.checkpoints, ctx.stats = checkpoints, stats
        ctx.nu_value = float(nu.detach().cpu())
        return torch.tensor(loss, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gloss):
        grid, nsteps, k = ctx.grid, ctx.nsteps, ctx.k
        grid.set_params(nu=ctx.nu_value)
        g = grid.zeros()
        gnu = 0.0
        seg_starts = list(range(0, nsteps, k))
        for start in reversed(seg_starts):
            end = min(start + k, nsteps)
            # recompute the segment, keeping its states and fields after viscosity
            states = [ctx.checkpoints[start]]
            viscs = [None]
            for n in range(start + 1, end + 1):
                out, uv = grid.zeros(), grid.zeros()
                rc, st = grid.step(states[-1], out, uv)
                if ctx.stats is not None:
                    ctx.stats.append(("recompute", n, st))
                states.append(out)
                viscs.append(uv)
            for n in range(end, start, -1):
                if n in ctx.targets:
                    grid.loss_grad(states[n - start], ctx.targets[n], ctx.mask_kind, ctx.alpha, ctx.beta, g)
                g_in = grid.zeros()
                rc, dnu, st = grid.adjoint_step(states[n - 1 - start], g, g_in, viscs[n - start])
                if ctx.stats is not None:
                    ctx.stats.append(("adjoint", n, st))
                gnu += dnu
                g = g_in
            del states, viscs
        if 0 in ctx.targets:
            grid.loss_grad(ctx.checkpoints[0], ctx.targets[0], ctx.mask_kind, ctx.alpha, ctx.beta, g)
        s = gloss.to(torch.float64)
        dnu = (s * gnu).to(torch.float32).reshape(())
        gu = [(t * s.to(t.dtype)) for t in g]
        return (None, None, None, None, None, None, None, None, dnu, gu[0], gu[1], gu[2])


def rollout_loss(grid: F.Grid, u0: F.Mac, nu: torch.Tensor, nsteps: int, targets: Dict[int, F.Mac],
                 checkpoint_every: int = 4, alpha: float = 0.0, beta: float = 1.0,
                 mask_kind: int = F.FS_MASK_SURFACE, stats: Optional[list] = None) -> torch.Tensor:
    """Sum over frames n in `targets` of the Eq. eq::optLoss loss at v_sim^n, where
    v_sim^0 = u0 and v_sim^{n+1} = step(v_sim^n). Differentiable w.r.t. `nu` (a
    0-d tensor) and the three tensors of `u0`."""
    if nsteps < 0 or checkpoint_every < 1:
        raise ValueError("nsteps >= 0 and checkpoint_every >= 1 required")
    return _RolloutLoss.apply(grid, nsteps, checkpoint_every, targets, alpha, beta, mask_kind, stats, nu,
                              u0.u, u0.v, u0.w)


def forward_states(grid: F.Grid, u0: F.Mac, nsteps: int) -> Sequence[F.Mac]:
    """All states of a plain forward rollout (no gradient), for generating targets."""
    out = [_clone(u0)]
    for _ in range(nsteps):
        nxt = grid.zeros()
        grid.step(out[-1], nxt)
        out.append(nxt)
    return out
