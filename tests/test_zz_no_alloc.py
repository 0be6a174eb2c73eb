"""GPU test of fs_project_noalloc, the projection for callers that cannot
allocate device memory (its scratch is a fixed static device array instead of a
context's buffers). It must give what fs_project gives, call after call: the
second call here uses a smaller grid, so anything the first call left in the
shared scratch that is not cleared would show up as a mismatch.

This file is named to be collected last, so a run that stops at the first
failure has run every other test before it."""
import pytest
import torch

from paper_2503_00868_gb300 import fluidstep as F
from paper_2503_00868_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_U = 1e-5   # the velocity tolerance of the other GPU parity tests
TOL_Q = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    F.load()
    torch.cuda.set_device(0)


def rel(a, b):
    a = [t.double() for t in a]
    b = [t.double() for t in b]
    num = sum(float(((x - y) ** 2).sum()) for x, y in zip(a, b))
    den = sum(float((y ** 2).sum()) for y in b)
    return (num / den) ** 0.5


def test_noalloc_projection_matches_fs_project_on_consecutive_calls():
    # the closed box full of liquid is the singular case: the liquid mean of the
    # right-hand side is removed and q is reported mean-free
    cases = [((44, 37, 41), "spheres", 1), ((23, 19, 26), "blob", 2), ((21, 18, 19), "closed_box", 3)]
    for (nx, ny, nz), kind, seed in cases:
        if kind == "spheres":
            types, _ = W.sphere_union(nx, ny, nz, seed)
        elif kind == "blob":
            types, _ = W.ellipsoid_blob(nx, ny, nz, seed)
        else:
            types = W.all_liquid(nx, ny, nz)
        u0 = W.random_mac(nx, ny, nz, seed + 10)
        dx = 1.0 / ny
        ref = F.Grid(nx, ny, nz, dx=dx, tol_p=1e-7)
        ref.set_mask(types)
        u_ref, q_ref = ref.pack(u0), ref.empty_cell()
        rc_ref, _ = ref.project(u_ref, q_ref)
        assert rc_ref == F.FS_OK

        u_new, q_new = ref.pack(u0), ref.empty_cell()
        t = torch.as_tensor(types).cuda().contiguous()
        torch.cuda.synchronize()
        rc, st = F.fs_project_noalloc(nx, ny, nz, t, u_new, q_new, dx=dx, tol=1e-7, maxit=20000)
        assert rc == F.FS_OK, st
        assert st["true_relres_p"] < 1e-6
        assert rel(u_new, u_ref) < TOL_U
        assert rel([q_new], [q_ref]) < TOL_Q

        # without q_out: the same velocity
        u_noq = ref.pack(u0)
        rc, st = F.fs_project_noalloc(nx, ny, nz, t, u_noq, None, dx=dx, tol=1e-7, maxit=20000)
        assert rc == F.FS_OK, st
        assert rel(u_noq, u_ref) < TOL_U
        ref.close()


def test_noalloc_rejects_a_grid_beyond_its_scratch():
    nx = ny = nz = 96
    types = torch.ones((nz, ny, nx), dtype=torch.uint8, device="cuda")
    z = torch.zeros(((nz + 1), (ny + 1), 100), dtype=torch.float32, device="cuda")
    u = F.Mac(z, z.clone(), z.clone())
    with pytest.raises(F.FluidStepError) as e:
        F.fs_project_noalloc(nx, ny, nz, types, u)
    assert e.value.status == F.FS_EINVAL and "static scratch" in str(e.value)
