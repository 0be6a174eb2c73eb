"""GPU APIC transfers and Gaussian deformation (Sec. 3.2.2, Sec. 3.4.3) against the
FP64 oracle, with particles spread over a ragged grid (some close to and outside
its faces), plus the affine-exactness property on the GPU."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_00868_gb300 import fluidstep as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def setup(nx=21, ny=17, nz=19, n=20000, seed=0):
    dx = 1.0 / ny
    types = np.ones((nz, ny, nx), np.uint8)
    og = O.Grid(types, dx, 1 / 30, 0.0)
    gg = F.Grid(nx, ny, nz, dx=dx)
    rng = np.random.default_rng(seed)
    ext = np.array([nx, ny, nz]) * dx
    x = (rng.random((n, 3)) * 1.1 - 0.05) * ext  # a few particles beyond the grid
    v = rng.standard_normal((n, 3))
    Cp = 0.5 * rng.standard_normal((n, 3, 3))
    m = rng.uniform(0.5, 2.0, n)
    # float32 inputs, and the oracle sees the same rounded values
    x, v, Cp, m = (a.astype(np.float32).astype(np.float64) for a in (x, v, Cp, m))
    return og, gg, x, v, Cp, m


def cuda(a, cols):
    return torch.tensor(np.asarray(a, np.float32).reshape(-1, cols), device="cuda").contiguous()


def rel(a, b):
    a = np.concatenate([np.ravel(x) for x in a])
    b = np.concatenate([np.ravel(x) for x in b])
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_p2g_matches_oracle():
    og, gg, x, v, Cp, m = setup()
    uo, mo = O.p2g(og, x, v, Cp, m, return_mass=True)
    u, mass = gg.zeros(), gg.zeros()
    F.fs_p2g(gg.ctx, cuda(x, 3), cuda(v, 3), cuda(Cp, 9), cuda(m, 1), u, mass)
    assert rel(gg.unpack(mass), mo) < 1e-5
    assert rel(gg.unpack(u), uo) < 1e-5


def test_g2p_and_particle_update_match_oracle():
    og, gg, x, v, Cp, m = setup(n=5000, seed=1)
    rng = np.random.default_rng(2)
    u = [rng.standard_normal(s) for s in og.shapes()]
    u = [a.astype(np.float32).astype(np.float64) for a in u]
    Fm = (np.eye(3) + 0.1 * rng.standard_normal((5000, 3, 3))).astype(np.float32).astype(np.float64)
    L = rng.standard_normal((5000, 3, 3))
    A0 = (L @ np.transpose(L, (0, 2, 1))).astype(np.float32).astype(np.float64)
    hi = float(og.ny * og.dx)
    xo, vo, Co, Fo, Ao = O.g2p(og, x, u, F=Fm, A0=A0, dt=0.02, advance=True, lo=0.0, hi=hi)
    xt, vt, Ct = cuda(x, 3), torch.zeros(5000, 3, device="cuda"), torch.zeros(5000, 9, device="cuda")
    Ft, At = cuda(Fm, 9), torch.zeros(5000, 9, device="cuda")
    F.fs_g2p(gg.ctx, xt, vt, Ct, gg.pack(u), F=Ft, A0=cuda(A0, 9), A_out=At, dt=0.02, advance=True, lo=0.0, hi=hi)
    assert rel([vt.cpu().numpy()], [vo]) < 1e-5
    assert rel([Ct.cpu().numpy()], [Co.reshape(-1, 9)]) < 1e-4
    assert rel([xt.cpu().numpy()], [xo]) < 1e-6
    assert rel([Ft.cpu().numpy()], [Fo.reshape(-1, 9)]) < 1e-5
    assert rel([At.cpu().numpy()], [Ao.reshape(-1, 9)]) < 1e-5


def test_affine_field_round_trip_on_the_gpu():
    nx = ny = nz = 16
    dx = 1.0 / ny
    gg = F.Grid(nx, ny, nz, dx=dx)
    rng = np.random.default_rng(4)
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    n = 60000
    x = 2.5 * dx + rng.random((n, 3)) * (nx - 5) * dx
    v = a + x @ B.T
    xt = cuda(x, 3)
    u = gg.zeros()
    F.fs_p2g(gg.ctx, xt, cuda(v, 3), cuda(np.broadcast_to(B, (n, 3, 3)), 9), torch.ones(n, device="cuda"), u)
    vt, Ct = torch.zeros(512, 3, device="cuda"), torch.zeros(512, 9, device="cuda")
    F.fs_g2p(gg.ctx, xt[:512].clone(), vt, Ct, u)
    assert np.allclose(vt.cpu().numpy(), v[:512], atol=2e-4 * np.abs(v).max())
    assert np.allclose(Ct.cpu().numpy(), np.broadcast_to(B.ravel(), (512, 9)), atol=5e-3 * np.abs(B).max())


def test_apic_argument_errors():
    _, gg, *_ = setup(8, 7, 6, 10)
    u = gg.zeros()
    with pytest.raises(F.FluidStepError):
        F.fs_g2p(gg.ctx, torch.zeros(4, 3, device="cuda"), torch.zeros(4, 3, device="cuda"),
                 torch.zeros(4, 9, device="cuda"), u, dt=float("inf"))
