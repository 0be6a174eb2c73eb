"""Pins of the oracle's preconditioner network against torch's own conv3d,
bf16 conversion and autograd on the CPU (library routines, float64)."""
import numpy as np
import torch

from paper_2503_00868_gb300 import workloads as W

CH = (2, 16, 16, 16, 16, 1)


def rand_net(seed):
    rng = np.random.default_rng(seed)
    Ws, Bs = [], []
    for l in range(5):
        fan = CH[l] * 27
        w = rng.standard_normal((CH[l + 1], CH[l], 3, 3, 3)) * np.sqrt(2.0 / fan)
        w = torch.from_numpy(w).to(torch.bfloat16).to(torch.float64).numpy()
        Ws.append(w)
        Bs.append(rng.standard_normal(CH[l + 1]) * 0.1)
    return Ws, Bs


def _round_st(x):
    """bf16 rounding with a straight-through derivative."""
    return x + (x.to(torch.bfloat16).to(torch.float64) - x).detach()


def torch_net(types, Ws, Bs, r):
    liq = torch.from_numpy(types == 1)
    code = torch.from_numpy(np.where(types == 1, 1.0, np.where(types == 2, -1.0, 0.0)))
    rt = torch.from_numpy(r)
    s = rt[liq].abs().max()
    x0 = torch.where(liq, rt / s, torch.zeros_like(rt))
    x = torch.stack([_round_st(x0), code])[None]
    Wt = [torch.from_numpy(w).requires_grad_(True) for w in Ws]
    Bt = [torch.from_numpy(b).requires_grad_(True) for b in Bs]
    for l in range(5):
        x = torch.nn.functional.conv3d(x, Wt[l], Bt[l], padding=1)
        if l < 4:
            x = _round_st(torch.relu(x))
    y = x[0, 0]
    return y, s, liq, Wt, Bt


def test_bf16_rounding_matches_torch(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-8, 8, 2000),
                        [0.0, -0.0, 1.0, 65504.0, 1e-30]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.bf16_round(x), ref)


def test_net_forward_matches_torch_conv3d(oracle_mod):
    O = oracle_mod
    types, _ = W.ellipsoid_blob(9, 8, 7, 1)
    types[0, 0, 0] = 2
    g = O.Grid(types, 0.1, 0.03, 0.0)
    Ws, Bs = rand_net(3)
    r = np.random.default_rng(4).standard_normal(types.shape)
    z = O.net_forward(g, Ws, Bs, r)
    y, s, liq, _, _ = torch_net(types, Ws, Bs, r)
    ref = torch.where(liq, s * y, torch.zeros_like(y)).detach().numpy()
    np.testing.assert_allclose(z, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_net_loss_gradient_matches_torch_autograd(oracle_mod):
    O = oracle_mod
    types, _ = W.ellipsoid_blob(8, 8, 8, 2)
    g = O.Grid(types, 0.1, 0.03, 0.0)
    Ws, Bs = rand_net(5)
    rng = np.random.default_rng(6)
    b = np.where(types == 1, rng.standard_normal(types.shape), 0.0)
    q = np.where(types == 1, rng.standard_normal(types.shape), 0.0)
    loss, gW, gB = O.net_loss_grad(g, Ws, Bs, b, q)
    y, s, liq, Wt, Bt = torch_net(types, Ws, Bs, b)
    # the pressure operator as a dense matrix on the liquid cells, by applying it
    # to unit vectors (it is pinned separately by its eigenvectors)
    idx = np.flatnonzero(types.ravel() == 1)
    A = np.zeros((idx.size, idx.size))
    for col, t in enumerate(idx):
        e = np.zeros(types.size)
        e[t] = 1.0
        A[:, col] = O.poisson_apply(g, e.reshape(types.shape)).ravel()[idx]
    At = torch.from_numpy(A)
    tq = (torch.from_numpy(q) / s).reshape(-1)[idx]
    ev = y.reshape(-1)[idx] - tq
    lt = (ev @ (At @ ev)) / (tq @ (At @ tq))
    lt.backward()
    assert abs(loss - lt.item()) <= 1e-10 * abs(loss)
    for l in range(5):
        np.testing.assert_allclose(gW[l], Wt[l].grad.numpy(), rtol=1e-8,
                                   atol=1e-9 * np.abs(Wt[l].grad.numpy()).max())
        np.testing.assert_allclose(gB[l], Bt[l].grad.numpy(), rtol=1e-8,
                                   atol=1e-9 * np.abs(Bt[l].grad.numpy()).max())
