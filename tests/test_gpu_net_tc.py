"""GPU: the network's inference layers on the tcgen05 tensor cores (fs_net_kernel
1: M = 128 cells x N = 16 channels x K = 16 per tap, accumulators in tensor
memory) against the FP64 oracle (which rounds the weights, the input and every
hidden activation to bf16 like the GPU stores them) and against the mma.sync
layers, on grids whose rows span a full and a partial 128-cell tile; and flexible
CG with it, which must land on the same projection."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_00868_gb300 import fluidstep as F
from paper_2503_00868_gb300 import train_precond as T
from paper_2503_00868_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def bf16_params(seed):
    """random parameters with bf16-representable weights, and the oracle's arrays"""
    rng = np.random.default_rng(seed)
    Ws, Bs, flat = [], [], []
    ch = T.CH
    for l in range(5):
        w = rng.standard_normal((ch[l + 1], ch[l], 3, 3, 3)) * np.sqrt(2.0 / (ch[l] * 27))
        w = torch.from_numpy(w).to(torch.bfloat16).to(torch.float64).numpy()
        b = torch.from_numpy(rng.standard_normal(ch[l + 1]) * 0.05).to(torch.float32).to(torch.float64).numpy()
        Ws.append(w)
        Bs.append(b)
        flat += [w.ravel(), b.ravel()]
    return np.concatenate(flat).astype(np.float32), Ws, Bs


@pytest.mark.parametrize("shape", [(150, 21, 26), (37, 20, 19)])
def test_tc_forward_matches_oracle_and_mma(shape):
    nx, ny, nz = shape
    types, _ = W.ellipsoid_blob(nx, ny, nz, 2)
    types[0, 0, :3] = 2
    og = O.Grid(types, 1.0 / ny, 1 / 30, 0.01)
    flat, Ws, Bs = bf16_params(1)
    r = np.where(types == 1, np.random.default_rng(5).standard_normal(types.shape), 0.0)
    zo = O.net_forward(og, Ws, Bs, r)
    out = {}
    for k in (0, 1):
        g = F.Grid(nx, ny, nz, dx=1.0 / ny)
        g.set_mask(types)
        F.fs_net_load(g.ctx, flat)
        F.fs_net_kernel(g.ctx, k)
        z = g.empty_cell()
        F.fs_net_forward(g.ctx, g.pack_cell(r), z)
        out[k] = g.unpack_cell(z)
        assert np.all(out[k][types != 1] == 0.0)
        g.close()
    e_tc, e_mma, e_pair = rel(out[1], zo), rel(out[0], zo), rel(out[1], out[0])
    assert e_tc < 1e-3 and e_pair < 1e-3, (e_tc, e_mma, e_pair)


def test_tc_flexible_cg_matches_mma():
    n = 64
    types, _ = W.sphere_union(n, n, n, 1)
    u0 = W.random_mac(n, n, n, 500)
    res = {}
    for k in (0, 1):
        g = F.Grid(n, n, n, dx=1.0 / n, tol_p=1e-6, maxit_p=5000, precond=F.FS_PRECOND_LEARNED)
        g.set_mask(types)
        F.fs_net_load(g.ctx, T.default_weights())
        F.fs_net_kernel(g.ctx, k)
        u = g.pack(u0)
        rc, st = g.project(u)
        assert rc == F.FS_OK and st["fallbacks"] == 0 and st["true_relres_p"] <= 1e-6, (k, st)
        res[k] = (st["iters_p"], np.concatenate([a.ravel() for a in g.unpack(u)]))
        g.close()
    assert abs(res[1][0] - res[0][0]) <= max(2, 0.1 * res[0][0]), (res[0][0], res[1][0])
    assert rel(res[1][1], res[0][1]) < 1e-5


def test_net_kernel_is_validated():
    g = F.Grid(8, 8, 8, dx=1 / 8)
    with pytest.raises(F.FluidStepError) as e:
        F.fs_net_kernel(g.ctx, 2)
    assert e.value.status == F.FS_EINVAL
