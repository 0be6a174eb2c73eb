"""GPU: the paper's upwind surrogate for the reverse of convection
(fs_params.advect_grad = FS_ADVECT_GRAD_UPWIND, Sec. 3.4.1) against the oracle's
surrogate (or_advect_adjoint_upwind inside or_adjoint_step), on a ragged blob
and on a river with prescribed inflow faces across two 128-wide tiles. The
adjoint step with the surrogate matches the oracle at the gradient tolerance
(1e-4), dL/dnu is unchanged by it (the viscosity gradient is formed before the
convection step is reversed), and it is a different gradient from the exact
adjoint's, though pointing the same way."""
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


def rel(a, b):
    num = sum(float(((np.asarray(x, np.float64) - y) ** 2).sum()) for x, y in zip(a, b))
    den = sum(float((np.asarray(y) ** 2).sum()) for y in b)
    return (num / den) ** 0.5


def case(name):
    if name == "blob_ragged":
        types, _ = W.ellipsoid_blob(37, 29, 33, 0)
        return types, None, (0.0, -9.81, 0.0)
    nx, ny, nz = 133, 40, 36
    types, inflow, _ = W.river_with_blob(nx, ny, nz, 2)
    bc = [np.zeros(s) for s in O.face_shapes(nx, ny, nz)]
    bc[0] = np.where(inflow == 1, 0.5, 0.0)
    return types, bc, (0.0, -9.81, 0.0)


@pytest.mark.parametrize("name", ["blob_ragged", "river_wide"])
@pytest.mark.parametrize("precond", [F.FS_PRECOND_JACOBI, F.FS_PRECOND_MG])
def test_upwind_surrogate_matches_oracle(name, precond):
    types, bc, g = case(name)
    nz, ny, nx = types.shape
    dx = 1.0 / ny
    og = O.Grid(types, dx, 1 / 30, 0.02, g=g, bc=bc, advect_grad=1)
    oe = O.Grid(types, dx, 1 / 30, 0.02, g=g, bc=bc, advect_grad=0)
    gg = F.Grid(nx, ny, nz, dx=dx, dt=1 / 30, nu=0.02, g=g, precond=precond, tol_p=1e-7, tol_v=1e-7,
                advect_grad=F.FS_ADVECT_GRAD_UPWIND)
    gg.set_mask(types, gg.pack(bc) if bc is not None else None)
    u0 = W.blurred_noise_mac(nx, ny, nz, 1)
    if bc is not None:
        for c in range(3):
            fc = O.face_class(og, c)
            u0[c][fc == 2] = bc[c][fc == 2]
    gout = W.blurred_noise_mac(nx, ny, nz, 7)
    ogin, ognu = O.adjoint_step(og, u0, gout)
    oex, oexnu = O.adjoint_step(oe, u0, gout)
    u = gg.pack(u0)
    uv, out = gg.zeros(), gg.zeros()
    gg.step(u, out, uv)
    gin = gg.zeros()
    rc, gnu, st = gg.adjoint_step(u, gg.pack(gout), gin, uv)
    assert rc == F.FS_OK, st
    gi = gg.unpack(gin)
    assert rel(gi, ogin) < 1e-4, rel(gi, ogin)
    assert abs(gnu - ognu) <= 1e-4 * abs(ognu)
    assert ognu == pytest.approx(oexnu, rel=1e-12)
    # a different gradient from the exact adjoint's, pointing the same way
    dot = sum(float((a * b).sum()) for a, b in zip(ogin, oex))
    na = sum(float((a * a).sum()) for a in ogin) ** 0.5
    nb = sum(float((b * b).sum()) for b in oex) ** 0.5
    assert rel(ogin, oex) > 1e-3 and dot / (na * nb) > 0.5, (rel(ogin, oex), dot / (na * nb))


def test_advect_grad_is_validated():
    with pytest.raises(F.FluidStepError) as e:
        F.Grid(8, 8, 8, dx=1 / 8, advect_grad=2)
    assert e.value.status == F.FS_EINVAL
