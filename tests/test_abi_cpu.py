"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a,
loads, and exports every function include/fluidstep.h declares; the binding
expects no symbol the header lacks."""
import ctypes
import os
import re

import pytest

from paper_2503_00868_gb300 import build as B
from paper_2503_00868_gb300 import fluidstep as F

HEADER = os.path.join(B.ROOT, "include", "fluidstep.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ["fs_init_grid", "fs_set_mask", "fs_step", "fs_adjoint_step", "fs_project", "fs_loss_grad"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header():
    assert sorted(F.exported_symbols()) == declared_functions()


def test_default_params_without_gpu(lib):
    F.load(B.LIB)
    p = F.fs_default_params()
    assert p.tol_p == 1e-6 and p.precond == F.FS_PRECOND_JACOBI and p.check_every >= 1


def test_init_rejects_bad_sizes_before_touching_the_device(lib):
    F.load(B.LIB)
    p = F.fs_default_params()
    with pytest.raises(F.FluidStepError) as e:
        F.fs_init_grid(1, 8, 8, p)
    assert e.value.status == F.FS_EINVAL
    p.tol_p = -1.0
    with pytest.raises(F.FluidStepError) as e:
        F.fs_init_grid(8, 8, 8, p)
    assert e.value.status == F.FS_EINVAL
