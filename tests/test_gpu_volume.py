"""GPU volumetric-velocity initialisation (Sec. 3.3.3) against the FP64 oracle:
the wall-function base profile and the constrained divergence projection of
Eq. eq::divProj, on a ragged river scene (blob + inflow layer, prescribed faces)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_00868_gb300 import fluidstep as F
from paper_2503_00868_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def scene(nx=29, ny=17, nz=23, seed=1):
    types, inflow, _ = W.river_with_blob(nx, ny, nz, seed)
    bc = [np.zeros(s) for s in W.face_shapes(nx, ny, nz)]
    bc[0] = np.where(inflow == 1, 0.5, 0.0)
    dx = 1.0 / ny
    og = O.Grid(types, dx, 1 / 30, 0.01, bc=bc)
    gg = F.Grid(nx, ny, nz, dx=dx)
    gg.set_mask(types, gg.pack(bc))
    return types, bc, og, gg


def rel(a, b):
    a = np.concatenate([x.ravel() for x in a])
    b = np.concatenate([x.ravel() for x in b])
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_wall_profile_matches_oracle():
    types, bc, og, gg = scene()
    nz, ny, nx = types.shape
    vinf = np.random.default_rng(3).uniform(0.2, 0.8, (nz, nx))
    d = (0.8, 0.0, -0.6)
    uo = O.wall_profile(og, d, vinf, 0.3)
    u = gg.zeros()
    F.fs_wall_profile(gg.ctx, d, torch.tensor(vinf, dtype=torch.float32, device="cuda"), 0.3, u)
    ug = gg.unpack(u)
    assert rel(ug, uo) < 1e-6
    for a, b in zip(ug, uo):  # prescribed and air faces exactly
        mask = (b == 0) | (b == 0.5)
        assert np.array_equal(a[mask].astype(np.float32), b[mask].astype(np.float32))


@pytest.mark.parametrize("hold", [False, True])
def test_pbd_projection_matches_oracle(hold):
    types, bc, og, gg = scene()
    nz, ny, nx = types.shape
    u0 = [b + n for b, n in zip(bc, W.blurred_noise_mac(nx, ny, nz, 4, sigma_cells=1.5, radius=4))]
    # fixed faces carry their prescribed values in both
    cls = [np.zeros(s, np.uint8) for s in W.face_shapes(nx, ny, nz)]
    for c in range(3):
        O.lib().or_face_class(og.cstruct(), c, cls[c].ctypes.data_as(O.C.POINTER(O.C.c_uint8)))
        u0[c] = np.where(cls[c] == 2, bc[c], u0[c])
    eps = 0.5 * ny * ny
    uo, no = O.pbd_project(og, u0, hold_surface=hold, iters=40, eps=eps)
    u = gg.pack(u0)
    ng = F.fs_pbd_project(gg.ctx, u, hold_surface=hold, iters=40, eps=eps)
    ug = gg.unpack(u)
    assert rel(ug, uo) < 1e-5
    assert ng == pytest.approx(no, rel=1e-4)
    # held faces keep their (float32) values exactly
    u0f = [a.astype(np.float32) for a in u0]
    _, n0 = O.pbd_project(og, u0, hold_surface=hold, iters=0, eps=eps)
    assert no < n0
    for c in range(3):
        held = cls[c] != 1
        assert np.array_equal(ug[c][held].astype(np.float32), u0f[c][held])


def test_profile_then_projection_reduces_the_divergence():
    types, bc, og, gg = scene(33, 24, 27, 2)
    nz, ny, nx = types.shape
    u = gg.zeros()
    vinf = torch.full((nz * nx,), 0.5, device="cuda")
    F.fs_wall_profile(gg.ctx, (1.0, 0.0, 0.0), vinf, 0.1, u)
    n0 = F.fs_pbd_project(gg.ctx, u, hold_surface=False, iters=0, eps=0.0)
    n1 = F.fs_pbd_project(gg.ctx, u, hold_surface=False, iters=400, eps=0.5 * ny * ny)
    assert n0 > 0 and n1 < 0.05 * n0, (n0, n1)


def test_volume_init_argument_errors():
    types, bc, og, gg = scene(9, 8, 7, 0)
    u = gg.zeros()
    vinf = torch.ones(7 * 9, device="cuda")
    with pytest.raises(F.FluidStepError):
        F.fs_wall_profile(gg.ctx, (1, 0, 0), vinf, -1.0, u)
    with pytest.raises(F.FluidStepError):
        F.fs_pbd_project(gg.ctx, u, iters=-1)
    with pytest.raises(F.FluidStepError):
        F.fs_pbd_project(gg.ctx, u, eps=float("nan"))
