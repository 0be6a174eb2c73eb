"""GPU: the fit's Adam step (fs_adam_update) against the update written out in
FP64 numpy (Kingma and Ba's bias-corrected Adam), over three steps, on an
aligned array (four elements per thread plus a ragged tail) and on a misaligned
view (one element per thread); a zero learning rate moves only the moments."""
import numpy as np
import pytest
import torch

from paper_2503_00868_gb300 import fluidstep as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grid():
    from paper_2503_00868_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    g = F.Grid(8, 8, 8, dx=1 / 8)
    yield g
    g.close()


def adam_ref(p, gs, lr, b1, b2, eps, scale):
    """p, m, v after the steps, and the sum of the magnitudes of m's terms (the
    scale of its rounding error where the terms cancel)"""
    p = p.astype(np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    mabs = np.zeros_like(p)
    for k, g in enumerate(gs, start=1):
        g = g.astype(np.float64) * scale
        m = b1 * m + (1 - b1) * g
        mabs = b1 * mabs + (1 - b1) * np.abs(g)
        v = b2 * v + (1 - b2) * g * g
        p -= lr * (m / (1 - b1 ** k)) / (np.sqrt(v / (1 - b2 ** k)) + eps)
    return p, m, v, mabs


@pytest.mark.parametrize("offset", [0, 1])
def test_adam_matches_the_formula(grid, offset):
    n = 4099
    rng = np.random.default_rng(offset)
    p0 = rng.standard_normal(n).astype(np.float32)
    gs = [rng.standard_normal(n).astype(np.float32) * 10.0 ** rng.uniform(-3, 1, n).astype(np.float32)
          for _ in range(3)]
    buf = [torch.zeros(n + offset, device="cuda") for _ in range(4)]
    p, g, m, v = (b[offset:] for b in buf)
    p.copy_(torch.from_numpy(p0))
    for k, gk in enumerate(gs, start=1):
        g.copy_(torch.from_numpy(gk))
        F.fs_adam_update(grid.ctx, p, g, m, v, 0.01, k, 0.9, 0.999, 1e-8, grad_scale=0.5)
    torch.cuda.synchronize()
    pr, mr, vr, mabs = adam_ref(p0, gs, 0.01, 0.9, 0.999, 1e-8, 0.5)
    # FP32 rounding: a few units in the last place of each term's magnitude
    np.testing.assert_allclose(p.cpu().numpy(), pr, rtol=1e-6, atol=1e-6)
    assert np.all(np.abs(m.cpu().numpy() - mr) <= 2e-6 * mabs)
    np.testing.assert_allclose(v.cpu().numpy(), vr, rtol=2e-6, atol=0)
    assert np.array_equal(g.cpu().numpy(), gs[-1])   # the gradient is read only


def test_zero_rate_moves_only_the_moments(grid):
    p = torch.arange(10, dtype=torch.float32, device="cuda")
    g = torch.ones(10, device="cuda")
    m, v = torch.zeros(10, device="cuda"), torch.zeros(10, device="cuda")
    F.fs_adam_update(grid.ctx, p, g, m, v, 0.0, 1)
    torch.cuda.synchronize()
    assert torch.equal(p, torch.arange(10, dtype=torch.float32, device="cuda"))
    assert torch.allclose(m, torch.full_like(m, 0.1)) and torch.allclose(v, torch.full_like(v, 1e-3))


def test_bad_arguments(grid):
    t = torch.zeros(4, device="cuda")
    with pytest.raises(F.FluidStepError):
        F.fs_adam_update(grid.ctx, t, t.clone(), t.clone(), t.clone(), 0.01, 0)     # step < 1
    with pytest.raises(F.FluidStepError):
        F.fs_adam_update(grid.ctx, t, t.clone(), t.clone(), t.clone(), 0.01, 1, beta1=1.0)
    with pytest.raises(ValueError):
        F.fs_adam_update(grid.ctx, t, torch.zeros(5, device="cuda"), t.clone(), t.clone(), 0.01, 1)
