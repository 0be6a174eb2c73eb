"""GPU: the network followed by one multigrid V-cycle (FS_PRECOND_LEARNED_MG).

* The training loss of that role, w.L_p w / (q/s).L_p (q/s) with
  w = q/s - y - M(b/s - L_p y), recomputed here from public calls (the network's
  output z = s y from fs_net_forward, the V-cycle M from fs_precond_apply on a
  multigrid context of the same mask) and the oracle's FP64 operator.
* Its gradient: the loss is quadratic in the network output y, and the output
  bias b5 shifts y by the same amount on every cell, so the central difference
  of the loss in b5 is exact; the library's dloss/db5 must match it.
* Training in that role lowers the loss, and flexible CG with the result
  reaches the tolerance in no more iterations than the V-cycle alone."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_00868_gb300 import fluidstep as F
from paper_2503_00868_gb300 import train_precond as T
from paper_2503_00868_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_PARAM_B5 = -1   # the output bias is the last parameter


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def pair(n, seed):
    types, _ = W.sphere_union(n, n, n, seed)
    gm = F.Grid(n, n, n, dx=1.0 / n, tol_p=1e-7, precond=F.FS_PRECOND_MIC0)
    gm.set_mask(types)
    u = gm.pack(W.random_mac(n, n, n, 40 + seed))
    b = gm.empty_cell()
    F.fs_divergence(gm.ctx, u, b)
    q = gm.empty_cell()
    gm.project(u, q)
    gm.close()
    return types, b, q


def test_learned_mg_loss_matches_its_definition():
    n = 40
    types, b, q = pair(n, 3)
    params = T.init_params(5)
    gl = F.Grid(n, n, n, dx=1.0 / n, precond=F.FS_PRECOND_LEARNED_MG)
    gl.set_mask(types)
    F.fs_net_load(gl.ctx, params)
    loss = F.fs_net_grad(gl.ctx, b, q)
    # the same quantity from public calls
    og = O.Grid(types, 1.0 / n, 1 / 30, 0.01)
    liq = types == 1
    b64, q64 = gl.unpack_cell(b), gl.unpack_cell(q)
    s = float(np.abs(b64[liq]).max())
    z = gl.empty_cell()
    F.fs_net_forward(gl.ctx, b, z)
    y = gl.unpack_cell(z) / s
    gm = F.Grid(n, n, n, dx=1.0 / n, precond=F.FS_PRECOND_MG)
    gm.set_mask(types)
    t1 = np.where(liq, b64 / s - O.poisson_apply(og, y), 0.0)
    mt = gm.empty_cell()
    gm.precond_apply(gm.pack_cell(t1), mt)
    w = np.where(liq, q64 / s - y - gm.unpack_cell(mt), 0.0)
    tq = np.where(liq, q64 / s, 0.0)
    ref = float((w * O.poisson_apply(og, w)).sum() / (tq * O.poisson_apply(og, tq)).sum())
    assert abs(loss - ref) <= 1e-4 * ref, (loss, ref)
    # the role changes the loss: the V-cycle removes most of what the network leaves
    gp = F.Grid(n, n, n, dx=1.0 / n, precond=F.FS_PRECOND_LEARNED)
    gp.set_mask(types)
    F.fs_net_load(gp.ctx, params)
    assert F.fs_net_grad(gp.ctx, b, q) > 2.0 * loss


def test_learned_mg_output_bias_gradient_is_the_exact_difference():
    n = 36
    types, b, q = pair(n, 4)
    params = T.init_params(6)
    params[N_PARAM_B5] = 0.25
    g = F.Grid(n, n, n, dx=1.0 / n, precond=F.FS_PRECOND_LEARNED_MG)
    g.set_mask(types)
    F.fs_net_load(g.ctx, params)
    F.fs_net_grad(g.ctx, b, q)
    grad = F.fs_net_grad_read(g.ctx)[N_PARAM_B5]
    h = 1e-2
    lv = []
    for sgn in (1.0, -1.0):
        p = params.copy()
        p[N_PARAM_B5] += sgn * h
        gg = F.Grid(n, n, n, dx=1.0 / n, precond=F.FS_PRECOND_LEARNED_MG)
        gg.set_mask(types)
        F.fs_net_load(gg.ctx, p)
        lv.append(F.fs_net_grad(gg.ctx, b, q))
        gg.close()
    fd = (lv[0] - lv[1]) / (2 * h)
    assert abs(grad - fd) <= 1e-3 * abs(fd) + 1e-7, (grad, fd)


def test_training_for_the_role_lowers_the_loss_and_fcg_converges():
    n = 32
    masks = [T.make_mask(n, k, 20 + k) for k in range(2)]
    data = {n: T.make_pairs(n, masks, 3, 7)}
    tr, va = T.split(data, val_every=4)
    init = T.init_params(1)
    v0 = T.evaluate_loss(va, init, "net_mg")
    params, hist = T.train_batched(tr, init, "net_mg", epochs=4, batch=4, lr=2e-3, val=va, log=False)
    assert hist[-1][1] < 0.8 * v0, (v0, hist)
    types = T.make_mask(n, 1, 99)
    res = {}
    for name, pc in (("mg", F.FS_PRECOND_MG), ("learned_mg", F.FS_PRECOND_LEARNED_MG)):
        g = F.Grid(n, n, n, dx=1.0 / n, tol_p=1e-6, maxit_p=2000, precond=pc)
        g.set_mask(types)
        if pc == F.FS_PRECOND_LEARNED_MG:
            F.fs_net_load(g.ctx, params)
        u = g.pack(W.random_mac(n, n, n, 123))
        rc, st = g.project(u)
        assert rc == F.FS_OK and st["fallbacks"] == 0 and st["true_relres_p"] <= 1e-6, (name, st)
        res[name] = (st["iters_p"], g.unpack(u))
        g.close()
    assert res["learned_mg"][0] <= res["mg"][0] + 1, (res["learned_mg"][0], res["mg"][0])
    num = sum(float(((a - b) ** 2).sum()) for a, b in zip(res["learned_mg"][1], res["mg"][1]))
    den = sum(float((b ** 2).sum()) for b in res["mg"][1])
    assert (num / den) ** 0.5 < 1e-5
