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


def test_enum_values_match_the_header():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(FS_[A-Z0-9_]+)\s*=\s*(-?\d+)", text))
    assert {"FS_PRECOND_MG", "FS_SOLVER_PERCNN", "FS_OK", "FS_EINVAL"} <= set(consts)
    for name in ("FS_PRECOND_JACOBI", "FS_PRECOND_MIC0", "FS_PRECOND_LEARNED", "FS_PRECOND_MG",
                 "FS_SOLVER_PCG", "FS_SOLVER_PERCNN"):
        assert getattr(F, name) == consts[name], name
    mirrored = [k for k in consts if hasattr(F, k)]
    assert len(mirrored) >= 10
    for name in mirrored:
        assert getattr(F, name) == consts[name], name


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and every field's offset of the structs the binding mirrors, as the C
    compiler lays them out from the header."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [F.fs_params, F.fs_stats, F.fs_layout_t, F.fs_kernel_time, F.fs_mac, F.fs_camera]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fluidstep.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} %zu\\n", sizeof({n}));')
        for fname, _ in st._fields_:
            lines.append(f'printf("{n}.{fname} %zu\\n", offsetof({n}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(out[n]) == ctypes.sizeof(st), n
        for fname, _ in st._fields_:
            assert int(out[f"{n}.{fname}"]) == getattr(st, fname).offset, f"{n}.{fname}"


def _noalloc_args(nx, ny, nz):
    import torch
    shape = F.noalloc_layout(nx, ny, nz)
    types = torch.ones(nx * ny * nz, dtype=torch.uint8).reshape(nz, ny, nx)
    u = F.Mac(*(torch.zeros(shape, dtype=torch.float32) for _ in range(3)))
    q = torch.zeros(shape, dtype=torch.float32)
    return types, u, q


def test_noalloc_arguments_checked_against_the_grid():
    """fs_project_noalloc has no context to hold the layout, so the binding checks
    every tensor against the grid before the library sees a pointer."""
    import torch
    nx, ny, nz = 10, 7, 9
    assert F.noalloc_layout(nx, ny, nz) == (10, 8, 12)
    types, u, q = _noalloc_args(nx, ny, nz)
    F.check_noalloc_args(nx, ny, nz, types, u, q, device="cpu")       # consistent: accepted
    F.check_noalloc_args(nx, ny, nz, types, u, None, device="cpu")
    bad = [
        dict(types=types[:, :, :-1].contiguous()),                           # too few cell types
        dict(types=types.to(torch.int32)),                                   # wrong dtype
        dict(u=F.Mac(u.u[:, :, :-4].contiguous(), u.v, u.w)),                # pitch too small
        dict(u=F.Mac(u.u, u.v[:-1].contiguous(), u.w)),                      # a plane short
        dict(u=F.Mac(u.u, u.v, u.w.to(torch.float64))),                     # wrong dtype
        dict(u=F.Mac(u.u, u.v, u.w.transpose(1, 2).contiguous().transpose(1, 2))),  # not contiguous
        dict(q=q[:, :-1].contiguous()),                                      # q_out a row short
        dict(q=q.to(torch.float16)),
    ]
    for b in bad:
        with pytest.raises(ValueError):
            F.check_noalloc_args(nx, ny, nz, b.get("types", types), b.get("u", u), b.get("q", q), device="cpu")
    with pytest.raises(ValueError):      # a tensor on another device than the current one
        F.check_noalloc_args(nx, ny, nz, types, u, q, device="cuda:0")
    with pytest.raises(ValueError):
        F.check_noalloc_args(1, ny, nz, types, u, q, device="cpu")


def test_noalloc_wrong_shape_rejected_before_the_library_is_called(monkeypatch):
    import torch

    def no_library(*a, **k):
        raise AssertionError("the library must not be reached")

    monkeypatch.setattr(F, "load", no_library)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    nx, ny, nz = 10, 7, 9
    types, u, q = _noalloc_args(nx, ny, nz)
    with pytest.raises(ValueError):
        F.fs_project_noalloc(nx, ny, nz, types, F.Mac(u.u[:, :, :4].contiguous(), u.v, u.w), q)
    with pytest.raises(ValueError):   # right shapes, but host tensors, not on the current CUDA device
        F.fs_project_noalloc(nx, ny, nz, types, u, q)


def test_adam_arguments_checked_before_the_library_is_called(monkeypatch):
    import torch
    called = []
    monkeypatch.setattr(F, "load", lambda: called.append(1))
    t = torch.zeros(4)
    with pytest.raises(ValueError):
        F.fs_adam_update(0, t, t, t, t, 0.01, 1)   # host tensors
    assert not called
