"""GPU MIC(0): the tile-wavefront schedule reproduces the oracle's lexicographic
factor and substitutions, and PCG with it matches the oracle's projection.
Also checks that a bounded device wait that runs out is reported as
FS_ETIMEOUT and leaves the context usable."""
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
    if name == "blob":
        return W.ellipsoid_blob(27, 22, 19, 4)[0]          # ragged: tiles of 8 do not divide
    if name == "spheres":
        return W.sphere_union(41, 35, 30, 2)[0]
    if name == "box":
        return W.all_liquid(17, 16, 20)                     # singular, closed
    raise KeyError(name)


@pytest.mark.parametrize("name", ["blob", "spheres", "box"])
def test_mic0_apply_matches_oracle(name):
    types = case(name)
    nz, ny, nx = types.shape
    og = O.Grid(types, 1.0 / ny, 1 / 30, 0.01)
    gg = F.Grid(nx, ny, nz, dx=1.0 / ny, precond=F.FS_PRECOND_MIC0)
    gg.set_mask(types)
    rng = np.random.default_rng(3)
    r = np.where(types == 1, rng.standard_normal(types.shape), 0.0)
    prec = O.mic0_factor(og)
    zo = O.mic0_apply(og, prec, r)
    z = gg.empty_cell()
    gg.precond_apply(gg.pack_cell(r), z)
    assert rel([gg.unpack_cell(z)], [zo]) < 1e-5


@pytest.mark.parametrize("name", ["blob", "spheres", "box"])
def test_mic0_pcg_projection_matches_oracle(name):
    types = case(name)
    nz, ny, nx = types.shape
    og = O.Grid(types, 1.0 / ny, 1 / 30, 0.01)
    gj = F.Grid(nx, ny, nz, dx=1.0 / ny, tol_p=1e-7)
    gm = F.Grid(nx, ny, nz, dx=1.0 / ny, tol_p=1e-7, precond=F.FS_PRECOND_MIC0)
    gj.set_mask(types)
    gm.set_mask(types)
    u0 = W.random_mac(nx, ny, nz, 5)
    ou, _, _ = O.project(og, u0)
    uj, um = gj.pack(u0), gm.pack(u0)
    _, sj = gj.project(uj)
    rc, sm = gm.project(um)
    assert rc == F.FS_OK
    assert rel(gm.unpack(um), ou) < 1e-5
    assert sm["iters_p"] < sj["iters_p"]  # the factor does its job


def test_mic0_step_plain_forward_box():
    """The plain-forward configuration (closed liquid box, MIC(0)), reduced size."""
    n = 24
    types = W.all_liquid(n, n, n)
    u0 = W.blurred_noise_mac(n, n, n, 0)
    og = O.Grid(types, 1.0 / n, 1 / 30, 0.01, precond=O.PC_MIC0)
    gg = F.Grid(n, n, n, dx=1.0 / n, tol_p=1e-7, tol_v=1e-7, precond=F.FS_PRECOND_MIC0)
    gg.set_mask(types)
    ou = u0
    a, b = gg.pack(u0), gg.zeros()
    for _ in range(3):
        ou, _ = O.step(og, ou)
        rc, _ = gg.step(a, b)
        assert rc == F.FS_OK
        a, b = b, a
    assert rel(gg.unpack(a), ou) < 1e-5


def test_wavefront_wait_that_runs_out_reports_timeout():
    """spin_limit = 1: the first tile that must wait for a predecessor gives up at
    once; the sweep aborts, the call returns FS_ETIMEOUT, and the next call on the
    same context (normal limit) succeeds."""
    n = 48
    types = W.all_liquid(n, n, n)
    gg = F.Grid(n, n, n, dx=1.0 / n, precond=F.FS_PRECOND_MIC0, spin_limit=1)
    gg.set_mask(types)
    r = gg.pack_cell(np.random.default_rng(0).standard_normal((n, n, n)))
    z = gg.empty_cell()
    with pytest.raises(F.FluidStepError) as e:
        gg.precond_apply(r, z)
    assert e.value.status == F.FS_ETIMEOUT
    gg.set_params(spin_limit=1 << 22)
    gg.set_mask(types)  # refactor from scratch
    gg.precond_apply(r, z)
    og = O.Grid(types, 1.0 / n, 1 / 30, 0.01)
    prec = O.mic0_factor(og)
    zo = O.mic0_apply(og, prec, gg.unpack_cell(r))
    assert rel([gg.unpack_cell(z)], [zo]) < 1e-5
