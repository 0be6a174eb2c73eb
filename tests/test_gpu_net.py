"""GPU learned preconditioner: the BF16 tensor-core network against the FP64
oracle (which rounds weights, the input and every hidden activation to bf16
like the GPU stores them), its gradients against the oracle's backpropagation,
training reducing the loss, and flexible CG with the network."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_00868_gb300 import fluidstep as F
from paper_2503_00868_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CH = (2, 16, 16, 16, 16, 1)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def rand_params(seed, scale=1.0):
    """Flat FP32 parameters (PyTorch Conv3d order) with bf16-representable values,
    and the same as per-layer float64 arrays for the oracle."""
    rng = np.random.default_rng(seed)
    Ws, Bs, flat = [], [], []
    for l in range(5):
        fan = CH[l] * 27
        w = rng.standard_normal((CH[l + 1], CH[l], 3, 3, 3)) * np.sqrt(2.0 / fan) * scale
        w = torch.from_numpy(w).to(torch.bfloat16).to(torch.float64).numpy()
        b = rng.standard_normal(CH[l + 1]) * 0.05
        b = torch.from_numpy(b).to(torch.float32).to(torch.float64).numpy()
        Ws.append(w)
        Bs.append(b)
        flat += [w.ravel(), b.ravel()]
    return np.concatenate(flat).astype(np.float32), Ws, Bs


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def setup(nx, ny, nz, seed=2):
    types, _ = W.ellipsoid_blob(nx, ny, nz, seed)
    types[0, 0, :3] = 2  # a few solid cells: the type channel takes all three codes
    og = O.Grid(types, 1.0 / ny, 1 / 30, 0.01)
    gg = F.Grid(nx, ny, nz, dx=1.0 / ny, tol_p=1e-6, maxit_p=3000)
    gg.set_mask(types)
    return types, og, gg


def test_param_count_matches_layout():
    assert F.fs_net_param_count() == sum(CH[l] * CH[l + 1] * 27 + CH[l + 1] for l in range(5))


def test_forward_matches_oracle():
    types, og, gg = setup(37, 21, 26)   # ragged against the 32 x 8 conv tiles
    flat, Ws, Bs = rand_params(1)
    F.fs_net_load(gg.ctx, flat)
    r = np.where(types == 1, np.random.default_rng(5).standard_normal(types.shape), 0.0)
    z = gg.empty_cell()
    F.fs_net_forward(gg.ctx, gg.pack_cell(r), z)
    zo = O.net_forward(og, Ws, Bs, r)
    e = rel(gg.unpack_cell(z), zo)
    assert e < 1e-3, e
    assert np.all(gg.unpack_cell(z)[types != 1] == 0.0)
    np.testing.assert_allclose(F.fs_net_read(gg.ctx), flat, rtol=0, atol=0)


def test_gradients_match_oracle():
    types, og, gg = setup(30, 17, 19, seed=5)
    flat, Ws, Bs = rand_params(3)
    F.fs_net_load(gg.ctx, flat)
    rng = np.random.default_rng(7)
    b = np.where(types == 1, rng.standard_normal(types.shape), 0.0)
    q = np.where(types == 1, rng.standard_normal(types.shape), 0.0)
    loss = F.fs_net_grad(gg.ctx, gg.pack_cell(b), gg.pack_cell(q))
    g = F.fs_net_grad_read(gg.ctx)
    lo, gW, gB = O.net_loss_grad(og, Ws, Bs, b, q)
    assert abs(loss - lo) <= 1e-3 * abs(lo), (loss, lo)
    off = 0
    for l in range(5):
        nw, nb = gW[l].size, gB[l].size
        ew, eb = rel(g[off:off + nw], gW[l].ravel()), rel(g[off + nw:off + nw + nb], gB[l].ravel())
        assert ew < 1e-2, f"layer {l + 1} weights: {ew:.3e}"
        off += nw
        assert eb < 1e-2, f"layer {l + 1} bias: {eb:.3e}"
        off += nb


def test_training_reduces_loss_and_fcg_converges():
    types, og, gg = setup(24, 24, 24, seed=8)
    flat, _, _ = rand_params(11, scale=0.5)
    F.fs_net_load(gg.ctx, flat)
    # training pairs: random right-hand sides, labels from the solver (MIC(0)-PCG)
    gm = F.Grid(24, 24, 24, dx=1 / 24, tol_p=1e-7, precond=F.FS_PRECOND_MIC0)
    gm.set_mask(types)
    pairs = []
    for s in range(6):
        u = gm.pack(W.random_mac(24, 24, 24, 100 + s))
        q = gm.empty_cell()
        gm.project(u, q)                       # L_p q = b, b = -dx div(u) on liquid cells
        bn = O.divergence(og, W.random_mac(24, 24, 24, 100 + s))
        pairs.append((gm.pack_cell(bn), q))
    losses = []
    for step in range(1, 41):
        l = 0.0
        for b, q in pairs:
            l += F.fs_net_grad(gg.ctx, b, q)
        F.fs_net_adam(gg.ctx, 2e-3, step, grad_scale=1.0 / len(pairs))
        losses.append(l / len(pairs))
    assert losses[-1] < 0.8 * losses[0], losses[::8]
    # flexible CG with the trained network reaches the tolerance (true residual)
    gg.set_params(precond=F.FS_PRECOND_LEARNED)
    u = gg.pack(W.random_mac(24, 24, 24, 999))
    rc, st = gg.project(u)
    assert rc == F.FS_OK and st["true_relres_p"] < 1e-5, st


def jacobi_like_params():
    """Weights that make the network y = x0 / 6 (x0 = r/s): layer 1 splits x0 into
    relu(x0), relu(-x0); layers 2-4 pass both through (centre tap 1); layer 5
    recombines them / 6. With them flexible CG must behave like Jacobi PCG."""
    flat = []
    ws = []
    w1 = np.zeros((16, 2, 3, 3, 3)); w1[0, 0, 1, 1, 1] = 1.0; w1[1, 0, 1, 1, 1] = -1.0
    ws.append(w1)
    for _ in range(3):
        w = np.zeros((16, 16, 3, 3, 3)); w[0, 0, 1, 1, 1] = 1.0; w[1, 1, 1, 1, 1] = 1.0
        ws.append(w)
    w5 = np.zeros((1, 16, 3, 3, 3)); w5[0, 0, 1, 1, 1] = 0.1666666; w5[0, 1, 1, 1, 1] = -0.1666666
    ws.append(w5)
    for l, w in enumerate(ws):
        flat += [w.ravel(), np.zeros(CH[l + 1])]
    return np.concatenate(flat).astype(np.float32)


def test_fcg_with_a_jacobi_like_network_matches_jacobi_pcg():
    n = 40
    types, _ = W.sphere_union(n, n, n, 3)
    gj = F.Grid(n, n, n, dx=1 / n, tol_p=1e-6)
    gl = F.Grid(n, n, n, dx=1 / n, tol_p=1e-6, maxit_p=2000, precond=F.FS_PRECOND_LEARNED)
    gj.set_mask(types)
    gl.set_mask(types)
    F.fs_net_load(gl.ctx, jacobi_like_params())
    u0 = W.random_mac(n, n, n, 4)
    uj, ul = gj.pack(u0), gl.pack(u0)
    _, sj = gj.project(uj)
    rc, sl = gl.project(ul)
    assert rc == F.FS_OK and sl["fallbacks"] == 0, (sj, sl)
    assert sl["iters_p"] <= 1.5 * sj["iters_p"] + 5, (sj["iters_p"], sl["iters_p"])
    assert rel(np.concatenate([a.ravel() for a in gl.unpack(ul)]),
               np.concatenate([a.ravel() for a in gj.unpack(uj)])) < 1e-5


def test_shipped_network_beats_jacobi_and_the_untrained_network():
    """The trained weights shipped with the package (trained at 48^3) used by
    flexible CG on unseen 64^3 sphere unions: no fallback to MIC(0), the true
    residual at the tolerance, fewer iterations than Jacobi PCG and than the
    untrained initialisation, and the same projected velocity as MIC(0)-PCG."""
    from paper_2503_00868_gb300 import train_precond as T
    n = 64
    types, _ = W.sphere_union(n, n, n, 1)
    grids = {}
    for name, pc in (("jacobi", F.FS_PRECOND_JACOBI), ("mic0", F.FS_PRECOND_MIC0),
                     ("trained", F.FS_PRECOND_LEARNED), ("untrained", F.FS_PRECOND_LEARNED)):
        g = F.Grid(n, n, n, dx=1 / n, tol_p=1e-6, maxit_p=5000, precond=pc)
        g.set_mask(types)
        grids[name] = g
    F.fs_net_load(grids["trained"].ctx, T.default_weights())
    F.fs_net_load(grids["untrained"].ctx, T.init_params(0))
    u0 = W.random_mac(n, n, n, 500)
    res = {}
    for name, g in grids.items():
        u = g.pack(u0)
        rc, st = g.project(u)
        res[name] = (rc, st, np.concatenate([a.ravel() for a in g.unpack(u)]))
    rc, st, ut = res["trained"]
    assert rc == F.FS_OK and st["fallbacks"] == 0, st
    assert st["true_relres_p"] < 1.2e-6, st
    assert st["iters_p"] < res["jacobi"][1]["iters_p"], (st["iters_p"], res["jacobi"][1]["iters_p"])
    su = res["untrained"][1]
    assert su["fallbacks"] > 0 or su["iters_p"] > st["iters_p"], (su, st)
    assert rel(ut, res["mic0"][2]) < 1e-4
