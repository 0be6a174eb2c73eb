"""GPU parameter fit (Sec. 3.4.2): Adam on log nu through the checkpointed
rollout's adjoint recovers the viscosity that generated synthetic surface-band
targets, on the river scene (blob + inflow patch, gravity)."""
import numpy as np
import pytest
import torch

from paper_2503_00868_gb300 import fit as FT
from paper_2503_00868_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def test_fit_recovers_viscosity_from_band_targets():
    nx, ny, nz, frames = 24, 20, 22, 6
    types, bc, _ = FT.river_scene(nx, ny, nz, 3)
    g = FT.make_grid(nx, ny, nz, types, bc, "jacobi", tol_p=1e-7, tol_v=1e-7)
    u_base = g.pack([b + 0.3 * n for b, n in zip(bc, W.blurred_noise_mac(nx, ny, nz, 5, sigma_cells=1.5,
                                                                          radius=4))])
    zero = g.zeros()
    nu_true = 2e-2
    targets = FT.synthetic_targets(g, u_base, zero, nu_true, frames)
    # a short second-moment memory keeps Adam's steps from shrinking near the optimum
    res = FT.fit(g, u_base, targets, frames, iters=80, nu0=2e-3, lr_theta=0.1, checkpoint_every=2,
                 fit_delta=False, cosine=True, betas=(0.8, 0.9))
    losses = [h[0] for h in res["history"]]
    assert losses[-1] < 1e-2 * losses[0], losses[::10]
    assert abs(res["nu"] - nu_true) / nu_true < 0.05, res["history"][-5:]


def test_fit_with_initial_velocity_correction_reduces_the_loss():
    nx, ny, nz, frames = 20, 16, 18, 4
    types, bc, _ = FT.river_scene(nx, ny, nz, 4)
    g = FT.make_grid(nx, ny, nz, types, bc, "jacobi", tol_p=1e-7, tol_v=1e-7)
    u_base = g.pack(bc)
    d = W.blurred_noise_mac(nx, ny, nz, 9, sigma_cells=1.5, radius=4)
    delta_true = g.pack([0.05 * x for x in d])
    targets = FT.synthetic_targets(g, u_base, delta_true, 1e-2, frames)
    res = FT.fit(g, u_base, targets, frames, iters=25, nu0=1e-3, lr_theta=0.05, lr_delta=5e-3,
                 checkpoint_every=2)
    losses = [h[0] for h in res["history"]]
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.3 * losses[0], losses[::5]
