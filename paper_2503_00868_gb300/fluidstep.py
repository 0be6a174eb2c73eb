"""Thin ctypes binding of libfluidstep.so, the C ABI of include/fluidstep.h.

Argument marshalling only: every step of the fluid step runs in the library's
CUDA kernels. PyTorch provides device memory and the stream. The functions
``fs_*`` mirror the C entry points one to one; ``Grid`` is a small convenience
wrapper used by the tests, the rollout and the benchmark.

Fields are ``Mac`` triples of float32 CUDA tensors of shape (planes, rows, pitch)
in the library layout; ``pack``/``unpack`` convert from/to the dense staggered
shapes (nz, ny, nx+1), (nz, ny+1, nx), (nz+1, ny, nx).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import NamedTuple, Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfluidstep.so")

FS_OK, FS_EINVAL, FS_ENOMEM, FS_ECUDA, FS_ENOCONV, FS_ENONFINITE, FS_ESTATE, FS_ETIMEOUT, FS_EBREAKDOWN = range(9)
STATUS_NAMES = {0: "FS_OK", 1: "FS_EINVAL", 2: "FS_ENOMEM", 3: "FS_ECUDA", 4: "FS_ENOCONV",
                5: "FS_ENONFINITE", 6: "FS_ESTATE", 7: "FS_ETIMEOUT", 8: "FS_EBREAKDOWN"}
FS_AIR, FS_LIQUID, FS_SOLID = 0, 1, 2
FS_PRECOND_JACOBI, FS_PRECOND_MIC0, FS_PRECOND_LEARNED, FS_PRECOND_MG, FS_PRECOND_LEARNED_MG = 0, 1, 2, 3, 4
FS_MASK_SURFACE, FS_MASK_OCCUPIED = 0, 1
FS_SOLVER_PCG, FS_SOLVER_PERCNN = 0, 1
FS_ADVECT_GRAD_EXACT, FS_ADVECT_GRAD_UPWIND = 0, 1
SOFT_STATUS = (FS_OK, FS_ENOCONV)


class FluidStepError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fs_params(C.Structure):
    _fields_ = [("dx", C.c_double), ("dt", C.c_double), ("nu", C.c_double), ("rho", C.c_double),
                ("g", C.c_double * 3), ("precond", C.c_int), ("maxit_p", C.c_int), ("maxit_v", C.c_int),
                ("tol_p", C.c_double), ("tol_v", C.c_double), ("check_every", C.c_int),
                ("spin_limit", C.c_int), ("mic_tau", C.c_double), ("mic_sigma", C.c_double),
                ("warm_start", C.c_int), ("pressure_solver", C.c_int), ("advect_grad", C.c_int)]


class fs_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iters_p", C.c_int), ("iters_v", C.c_int),
                ("relres_p", C.c_double), ("relres_v", C.c_double), ("true_relres_p", C.c_double),
                ("fallbacks", C.c_int), ("restarts_p", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fs_layout_t(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("pitch", C.c_int),
                ("rows", C.c_int), ("planes", C.c_int), ("nelems", C.c_longlong)]


class fs_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("total_ms", C.c_double),
                ("bytes", C.c_double), ("all_launches", C.c_longlong)]


class fs_mac(C.Structure):
    _fields_ = [("u", C.c_void_p), ("v", C.c_void_p), ("w", C.c_void_p)]


_lib = None

_SIGS = {
    "fs_default_params": ([C.POINTER(fs_params)], None),
    "fs_init_grid": ([C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.POINTER(fs_params), C.c_void_p], C.c_int),
    "fs_destroy": ([C.c_void_p], C.c_int),
    "fs_layout": ([C.c_void_p, C.POINTER(fs_layout_t)], C.c_int),
    "fs_set_stream": ([C.c_void_p, C.c_void_p], C.c_int),
    "fs_set_params": ([C.c_void_p, C.POINTER(fs_params)], C.c_int),
    "fs_set_mask": ([C.c_void_p, C.c_void_p, C.POINTER(fs_mac)], C.c_int),
    "fs_step": ([C.c_void_p, C.POINTER(fs_mac), C.POINTER(fs_mac), C.POINTER(fs_mac), C.POINTER(fs_stats)], C.c_int),
    "fs_project": ([C.c_void_p, C.POINTER(fs_mac), C.c_void_p, C.POINTER(fs_stats)], C.c_int),
    "fs_adjoint_step": ([C.c_void_p, C.POINTER(fs_mac), C.POINTER(fs_mac), C.POINTER(fs_mac), C.POINTER(fs_mac),
                         C.POINTER(C.c_double), C.POINTER(fs_stats)], C.c_int),
    "fs_loss_grad": ([C.c_void_p, C.POINTER(fs_mac), C.POINTER(fs_mac), C.c_int, C.c_double, C.c_double,
                      C.POINTER(C.c_double), C.POINTER(fs_mac)], C.c_int),
    "fs_profile": ([C.c_void_p, C.c_int], C.c_int),
    "fs_profile_read": ([C.c_void_p, C.POINTER(fs_kernel_time), C.c_int, C.POINTER(C.c_int)], C.c_int),
    "fs_precond_apply": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fs_divergence": ([C.c_void_p, C.POINTER(fs_mac), C.c_void_p], C.c_int),
    "fs_splat_render": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                         C.c_void_p, C.c_void_p], C.c_int),
    "fs_splat_render_sh": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                            C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fs_splat_stats": ([C.c_void_p, C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)], C.c_int),
    "fs_p2g": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(fs_mac),
                C.POINTER(fs_mac)], C.c_int),
    "fs_g2p": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                C.POINTER(fs_mac), C.c_double, C.c_int, C.c_double, C.c_double], C.c_int),
    "fs_percnn_load": ([C.c_void_p, C.POINTER(C.c_float), C.c_int], C.c_int),
    "fs_percnn_read": ([C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_int)], C.c_int),
    "fs_percnn_grad": ([C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float)],
                       C.c_int),
    "fs_wall_profile": ([C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_double, C.POINTER(fs_mac)], C.c_int),
    "fs_pbd_project": ([C.c_void_p, C.POINTER(fs_mac), C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double)],
                       C.c_int),
    "fs_net_param_count": ([], C.c_int),
    "fs_net_load": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int], C.c_int),
    "fs_net_read": ([C.c_void_p, C.c_void_p, C.c_int], C.c_int),
    "fs_net_forward": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fs_net_kernel": ([C.c_void_p, C.c_int], C.c_int),
    "fs_net_grad": ([C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)], C.c_int),
    "fs_net_grad_read": ([C.c_void_p, C.c_void_p, C.c_int], C.c_int),
    "fs_net_adam": ([C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int],
                    C.c_int),
    "fs_adam_update": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_double,
                        C.c_double, C.c_double, C.c_double, C.c_int, C.c_double], C.c_int),
    "fs_pressure_pair": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fs_net_train_step": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int,
                           C.POINTER(C.c_double)], C.c_int),
    "fs_project_noalloc": ([C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(fs_mac), C.c_void_p, C.c_double,
                            C.c_double, C.c_int, C.c_void_p, C.POINTER(fs_stats)], C.c_int),
    "fs_last_error": ([], C.c_char_p),
}


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return list(_SIGS)


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: build it with paper_2503_00868_gb300.build.build()")
    L = C.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc: int, soft=SOFT_STATUS) -> int:
    if rc not in soft:
        raise FluidStepError(rc, load().fs_last_error().decode())
    return rc


# ---- one-to-one wrappers of the C entry points ------------------------------

def fs_default_params() -> fs_params:
    p = fs_params()
    load().fs_default_params(C.byref(p))
    return p


def fs_init_grid(nx: int, ny: int, nz: int, params: fs_params, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().fs_init_grid(C.byref(h), nx, ny, nz, C.byref(params), C.c_void_p(stream)), (FS_OK,))
    return h.value


def fs_destroy(ctx: int) -> None:
    load().fs_destroy(C.c_void_p(ctx))


def fs_layout(ctx: int) -> fs_layout_t:
    out = fs_layout_t()
    _check(load().fs_layout(C.c_void_p(ctx), C.byref(out)), (FS_OK,))
    return out


def fs_set_stream(ctx: int, stream: int) -> None:
    _check(load().fs_set_stream(C.c_void_p(ctx), C.c_void_p(stream)), (FS_OK,))


def fs_set_params(ctx: int, params: fs_params) -> None:
    _check(load().fs_set_params(C.c_void_p(ctx), C.byref(params)), (FS_OK,))


class Mac(NamedTuple):
    u: torch.Tensor
    v: torch.Tensor
    w: torch.Tensor


def _mac(m: Optional[Mac]):
    if m is None:
        return None
    for t in m:
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("fields must be contiguous float32 CUDA tensors")
    return fs_mac(m.u.data_ptr(), m.v.data_ptr(), m.w.data_ptr())


def _ref(s):
    return C.byref(s) if s is not None else None


def fs_set_mask(ctx: int, cell_type_dense: torch.Tensor, bc: Optional[Mac] = None) -> None:
    if cell_type_dense.dtype != torch.uint8 or not cell_type_dense.is_cuda:
        raise ValueError("cell types must be a uint8 CUDA tensor")
    t = cell_type_dense.contiguous()
    _check(load().fs_set_mask(C.c_void_p(ctx), C.c_void_p(t.data_ptr()), _ref(_mac(bc))), (FS_OK,))


def fs_step(ctx: int, u_in: Mac, u_out: Mac, u_visc: Optional[Mac] = None):
    st = fs_stats()
    rc = _check(load().fs_step(C.c_void_p(ctx), _ref(_mac(u_in)), _ref(_mac(u_out)), _ref(_mac(u_visc)),
                               C.byref(st)))
    return rc, st.as_dict()


def fs_project(ctx: int, u: Mac, q_out: Optional[torch.Tensor] = None):
    st = fs_stats()
    q = C.c_void_p(q_out.data_ptr()) if q_out is not None else None
    rc = _check(load().fs_project(C.c_void_p(ctx), _ref(_mac(u)), q, C.byref(st)))
    return rc, st.as_dict()


def fs_pressure_pair(ctx: int, q_hi: torch.Tensor, q_lo: torch.Tensor) -> None:
    """The last projection's q as its two FP32 terms (cell arrays, library layout)."""
    _check(load().fs_pressure_pair(C.c_void_p(ctx), _cell(q_hi), _cell(q_lo)), (FS_OK,))


def fs_adjoint_step(ctx: int, u_in: Mac, u_visc: Optional[Mac], g_out: Mac, g_in: Mac):
    st = fs_stats()
    gnu = C.c_double(0.0)
    rc = _check(load().fs_adjoint_step(C.c_void_p(ctx), _ref(_mac(u_in)), _ref(_mac(u_visc)), _ref(_mac(g_out)),
                                       _ref(_mac(g_in)), C.byref(gnu), C.byref(st)))
    return rc, gnu.value, st.as_dict()


def fs_loss_grad(ctx: int, u: Mac, target: Mac, mask_kind: int = FS_MASK_SURFACE, alpha: float = 0.0,
                 beta: float = 1.0, g: Optional[Mac] = None) -> float:
    loss = C.c_double(0.0)
    _check(load().fs_loss_grad(C.c_void_p(ctx), _ref(_mac(u)), _ref(_mac(target)), mask_kind, alpha, beta,
                               C.byref(loss), _ref(_mac(g))), (FS_OK,))
    return loss.value


def fs_profile(ctx: int, period: int) -> None:
    """period >= 1: time every period-th CG iteration (and count launches); 0: off."""
    _check(load().fs_profile(C.c_void_p(ctx), int(period)), (FS_OK,))


def fs_profile_read(ctx: int):
    """Per-kernel timing since fs_profile(ctx, k): {name: (timed launches, total_ms,
    bytes, all launches)}."""
    buf = (fs_kernel_time * 32)()
    n = C.c_int(0)
    _check(load().fs_profile_read(C.c_void_p(ctx), buf, 32, C.byref(n)), (FS_OK,))
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms, buf[i].bytes, buf[i].all_launches)
            for i in range(n.value)}


def fs_precond_apply(ctx: int, r: torch.Tensor, z: torch.Tensor) -> None:
    for t in (r, z):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("r and z must be contiguous float32 CUDA tensors")
    _check(load().fs_precond_apply(C.c_void_p(ctx), C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr())), (FS_OK,))


def _cell(t: torch.Tensor) -> C.c_void_p:
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("cell arrays must be contiguous float32 CUDA tensors")
    return C.c_void_p(t.data_ptr())


def fs_divergence(ctx: int, u: Mac, b_out: torch.Tensor) -> None:
    _check(load().fs_divergence(C.c_void_p(ctx), _ref(_mac(u)), _cell(b_out)), (FS_OK,))


class fs_camera(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int), ("height", C.c_int),
                ("znear", C.c_double), ("bg", C.c_double * 3)]


def make_camera(R, t, fx, fy, cx, cy, width, height, znear=0.01, bg=(0.0, 0.0, 0.0)) -> fs_camera:
    cam = fs_camera()
    for k in range(9):
        cam.R[k] = float(np.asarray(R, float).ravel()[k])
    for k in range(3):
        cam.t[k] = float(t[k])
        cam.bg[k] = float(bg[k])
    cam.fx, cam.fy, cam.cx, cam.cy = float(fx), float(fy), float(cx), float(cy)
    cam.width, cam.height, cam.znear = int(width), int(height), float(znear)
    return cam


def fs_splat_render(ctx: int, x: torch.Tensor, opacity: torch.Tensor, A: torch.Tensor, color: torch.Tensor,
                    cam: fs_camera, rgb_out: torch.Tensor, T_out: Optional[torch.Tensor] = None) -> None:
    """x (n, 3), opacity (n,), A (n, 9), color (n, 3): float32 CUDA; rgb_out (h, w, 3), T_out (h, w)."""
    n = x.shape[0]
    for t, cols in ((x, 3), (A, 9), (color, 3), (opacity.reshape(-1, 1), 1)):
        _parts(t, cols)
        if t.shape[0] != n:
            raise ValueError("x, opacity, A and color must have the same number of rows")
    if T_out is not None and (T_out.shape != (cam.height, cam.width) or T_out.dtype != torch.float32
                              or not T_out.is_cuda):
        raise ValueError("T_out must be a float32 CUDA tensor of shape (height, width)")
    if rgb_out.shape != (cam.height, cam.width, 3) or rgb_out.dtype != torch.float32 or not rgb_out.is_cuda:
        raise ValueError("rgb_out must be a float32 CUDA tensor of shape (height, width, 3)")
    _check(load().fs_splat_render(C.c_void_p(ctx), int(n), C.c_void_p(x.data_ptr()),
                                  C.c_void_p(opacity.data_ptr()), C.c_void_p(A.data_ptr()),
                                  C.c_void_p(color.data_ptr()), C.byref(cam), C.c_void_p(rgb_out.data_ptr()),
                                  C.c_void_p(T_out.data_ptr()) if T_out is not None else None), (FS_OK,))


def fs_splat_render_sh(ctx: int, x: torch.Tensor, opacity: torch.Tensor, A: torch.Tensor, sh: torch.Tensor,
                       degree: int, cam: fs_camera, rgb_out: torch.Tensor, T_out: Optional[torch.Tensor] = None) -> None:
    """Like fs_splat_render with colours from spherical-harmonic coefficients sh
    (n, (degree+1)^2, 3) float32 CUDA, degree 0 .. 3."""
    n = x.shape[0]
    nb = (int(degree) + 1) ** 2
    if sh.dtype != torch.float32 or not sh.is_cuda or not sh.is_contiguous() or tuple(sh.shape) != (n, nb, 3):
        raise ValueError(f"sh must be a contiguous float32 CUDA tensor of shape ({n}, {nb}, 3)")
    for t, cols in ((x, 3), (A, 9), (opacity.reshape(-1, 1), 1)):
        _parts(t, cols)
        if t.shape[0] != n:
            raise ValueError("x, opacity, A and sh must have the same number of rows")
    if T_out is not None and (T_out.shape != (cam.height, cam.width) or T_out.dtype != torch.float32
                              or not T_out.is_cuda):
        raise ValueError("T_out must be a float32 CUDA tensor of shape (height, width)")
    if rgb_out.shape != (cam.height, cam.width, 3) or rgb_out.dtype != torch.float32 or not rgb_out.is_cuda:
        raise ValueError("rgb_out must be a float32 CUDA tensor of shape (height, width, 3)")
    _check(load().fs_splat_render_sh(C.c_void_p(ctx), int(n), C.c_void_p(x.data_ptr()),
                                     C.c_void_p(opacity.data_ptr()), C.c_void_p(A.data_ptr()),
                                     C.c_void_p(sh.data_ptr()), int(degree), C.byref(cam),
                                     C.c_void_p(rgb_out.data_ptr()),
                                     C.c_void_p(T_out.data_ptr()) if T_out is not None else None), (FS_OK,))


def fs_splat_stats(ctx: int) -> dict:
    """{"entries", "max_tile"} of the last fs_splat_render on this context."""
    e, m = C.c_ulonglong(0), C.c_ulonglong(0)
    _check(load().fs_splat_stats(C.c_void_p(ctx), C.byref(e), C.byref(m)), (FS_OK,))
    return {"entries": int(e.value), "max_tile": int(m.value)}


def _parts(t: Optional[torch.Tensor], cols: int):
    if t is None:
        return None
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.shape[-1] != cols:
        raise ValueError(f"particle arrays must be contiguous float32 CUDA tensors with {cols} columns")
    return C.c_void_p(t.data_ptr())


def fs_p2g(ctx: int, x: torch.Tensor, v: torch.Tensor, Cp: torch.Tensor, m: torch.Tensor, u_out: Mac,
           mass_out: Optional[Mac] = None) -> None:
    """x, v: (np, 3); Cp: (np, 9) (row-major 3x3); m: (np, 1) or (np,) -- float32 CUDA."""
    npart = x.shape[0]
    _check(load().fs_p2g(C.c_void_p(ctx), int(npart), _parts(x, 3), _parts(v, 3), _parts(Cp, 9),
                         _parts(m.reshape(-1, 1), 1), _ref(_mac(u_out)), _ref(_mac(mass_out))), (FS_OK,))


def fs_g2p(ctx: int, x: torch.Tensor, v_out: torch.Tensor, C_out: torch.Tensor, u: Mac,
           F: Optional[torch.Tensor] = None, A0: Optional[torch.Tensor] = None, A_out: Optional[torch.Tensor] = None,
           dt: float = 0.0, advance: bool = False, lo: float = 0.0, hi: float = 1e30) -> None:
    npart = x.shape[0]
    _check(load().fs_g2p(C.c_void_p(ctx), int(npart), _parts(x, 3), _parts(v_out, 3), _parts(C_out, 9),
                         _parts(F, 9), _parts(A0, 9), _parts(A_out, 9), _ref(_mac(u)), float(dt), int(bool(advance)),
                         float(lo), float(hi)), (FS_OK,))


def fs_percnn_load(ctx: int, w27, substeps: int) -> None:
    w = np.ascontiguousarray(np.asarray(w27, dtype=np.float32).ravel())
    if w.size != 27:
        raise ValueError("the recurrent-solver kernel has 27 taps")
    _check(load().fs_percnn_load(C.c_void_p(ctx), w.ctypes.data_as(C.POINTER(C.c_float)), int(substeps)),
           (FS_OK,))


def fs_percnn_read(ctx: int):
    w = np.zeros(27, np.float32)
    k = C.c_int(0)
    _check(load().fs_percnn_read(C.c_void_p(ctx), w.ctypes.data_as(C.POINTER(C.c_float)), C.byref(k)), (FS_OK,))
    return w, k.value


def fs_percnn_grad(ctx: int, b: torch.Tensor, q: torch.Tensor):
    """(loss, dloss/dW over the 27 stored taps) for one pair L_p q = b."""
    loss = C.c_double(0.0)
    dw = np.zeros(27, np.float32)
    _check(load().fs_percnn_grad(C.c_void_p(ctx), _cell(b), _cell(q), C.byref(loss),
                                 dw.ctypes.data_as(C.POINTER(C.c_float))), (FS_OK,))
    return loss.value, dw


def fs_wall_profile(ctx: int, direction, vinf: torch.Tensor, delta: float, u_out: Mac) -> None:
    """vinf: device float32 tensor of nz * nx column surface speeds ([k][i])."""
    if vinf.dtype != torch.float32 or not vinf.is_cuda or not vinf.is_contiguous():
        raise ValueError("vinf must be a contiguous float32 CUDA tensor")
    d = (C.c_double * 3)(*[float(x) for x in direction])
    _check(load().fs_wall_profile(C.c_void_p(ctx), d, C.c_void_p(vinf.data_ptr()), float(delta),
                                  _ref(_mac(u_out))), (FS_OK,))


def fs_pbd_project(ctx: int, u: Mac, hold_surface: bool = True, iters: int = 100, eps: float = 0.0) -> float:
    """In place; returns |div u|_2 over the liquid after the last iteration."""
    n = C.c_double(0.0)
    _check(load().fs_pbd_project(C.c_void_p(ctx), _ref(_mac(u)), int(bool(hold_surface)), int(iters),
                                 float(eps), C.byref(n)), (FS_OK,))
    return n.value


def fs_net_param_count() -> int:
    return load().fs_net_param_count()


def fs_net_load(ctx: int, params) -> None:
    """params: 1-D float32 array (numpy, CPU or CUDA tensor) in PyTorch Conv3d order."""
    if isinstance(params, torch.Tensor) and params.is_cuda:
        p = params.detach().to(torch.float32).contiguous()
        _check(load().fs_net_load(C.c_void_p(ctx), C.c_void_p(p.data_ptr()), p.numel(), 0), (FS_OK,))
    else:
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
        _check(load().fs_net_load(C.c_void_p(ctx), p.ctypes.data_as(C.c_void_p), p.size, 1), (FS_OK,))


def fs_net_read(ctx: int) -> np.ndarray:
    out = np.zeros(fs_net_param_count(), dtype=np.float32)
    _check(load().fs_net_read(C.c_void_p(ctx), out.ctypes.data_as(C.c_void_p), out.size), (FS_OK,))
    return out


def fs_net_forward(ctx: int, r: torch.Tensor, z: torch.Tensor) -> None:
    _check(load().fs_net_forward(C.c_void_p(ctx), _cell(r), _cell(z)), (FS_OK,))


def fs_net_kernel(ctx: int, which: int) -> None:
    """Inference layers: 0 mma.sync, 1 tcgen05 (tensor memory)."""
    _check(load().fs_net_kernel(C.c_void_p(ctx), int(which)), (FS_OK,))


def fs_net_grad(ctx: int, b: torch.Tensor, q: torch.Tensor) -> float:
    loss = C.c_double(0.0)
    _check(load().fs_net_grad(C.c_void_p(ctx), _cell(b), _cell(q), C.byref(loss)), (FS_OK,))
    return loss.value


def fs_net_grad_read(ctx: int) -> np.ndarray:
    out = np.zeros(fs_net_param_count(), dtype=np.float32)
    _check(load().fs_net_grad_read(C.c_void_p(ctx), out.ctypes.data_as(C.c_void_p), out.size), (FS_OK,))
    return out


def fs_net_adam(ctx: int, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0,
                fix_offsets=True) -> None:
    _check(load().fs_net_adam(C.c_void_p(ctx), lr, beta1, beta2, eps, step, grad_scale, 1 if fix_offsets else 0),
           (FS_OK,))


def fs_adam_update(ctx: int, p: torch.Tensor, g: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float,
                   step: int, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0) -> None:
    """One Adam step in place on p, m and v (contiguous float32 tensors of one size
    on the current CUDA device); g is read only."""
    n = p.numel()
    arrays = (("p", p), ("g", g), ("m", m), ("v", v))
    for name, t in arrays:
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    dev = torch.cuda.current_device()
    for name, t in arrays:
        if t.device.index != dev:
            raise ValueError(f"{name} is not on the current CUDA device")
        if t.numel() != n:
            raise ValueError(f"{name} has {t.numel()} elements, p has {n}")
    _check(load().fs_adam_update(C.c_void_p(ctx), C.c_void_p(p.data_ptr()), C.c_void_p(g.data_ptr()),
                                 C.c_void_p(m.data_ptr()), C.c_void_p(v.data_ptr()), n, lr, beta1, beta2, eps,
                                 step, grad_scale), (FS_OK,))


def fs_net_train_step(ctx: int, b_batch: torch.Tensor, q_batch: torch.Tensor, lr: float, step: int) -> float:
    loss = C.c_double(0.0)
    _check(load().fs_net_train_step(C.c_void_p(ctx), _cell(b_batch), _cell(q_batch), b_batch.shape[0], lr, step,
                                    C.byref(loss)), (FS_OK,))
    return loss.value


def noalloc_layout(nx: int, ny: int, nz: int):
    """(planes, rows, pitch) of a field of an nx x ny x nz grid: the layout
    fs_init_grid uses, which fs_project_noalloc assumes without a context."""
    return nz + 1, ny + 1, (nx + 1 + 3) // 4 * 4


def check_noalloc_args(nx, ny, nz, cell_type_dense, u, q_out=None, device=None):
    """Raises ValueError unless the arguments of fs_project_noalloc match the
    grid: cell types uint8 with nx*ny*nz elements, the three components of u and
    q_out (if given) contiguous float32 of shape noalloc_layout(nx, ny, nz), and
    every tensor on `device` (default: the current CUDA device)."""
    if min(int(nx), int(ny), int(nz)) < 2:
        raise ValueError(f"grid sizes must be >= 2 (got {nx} {ny} {nz})")
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    shape = noalloc_layout(nx, ny, nz)

    def on_device(t, what):
        if t.device != torch.device(device):
            raise ValueError(f"{what} is on {t.device}, not on the current device {device}")

    if not isinstance(cell_type_dense, torch.Tensor) or cell_type_dense.dtype != torch.uint8 \
            or not cell_type_dense.is_contiguous() or cell_type_dense.numel() != nx * ny * nz:
        raise ValueError(f"cell types must be a contiguous uint8 tensor of {nx}*{ny}*{nz} elements")
    on_device(cell_type_dense, "the cell-type tensor")
    if u is None or len(u) != 3:
        raise ValueError("u must be a Mac of three components")
    for name, t in zip("uvw", u):
        if t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shape:
            raise ValueError(f"u.{name} must be a contiguous float32 tensor of shape {shape}, "
                             f"got {tuple(t.shape)} {t.dtype}")
        on_device(t, f"u.{name}")
    if q_out is not None:
        if q_out.dtype != torch.float32 or not q_out.is_contiguous() or tuple(q_out.shape) != shape:
            raise ValueError(f"q_out must be a contiguous float32 tensor of shape {shape}, "
                             f"got {tuple(q_out.shape)} {q_out.dtype}")
        on_device(q_out, "q_out")


def fs_project_noalloc(nx: int, ny: int, nz: int, cell_type_dense: torch.Tensor, u: Mac,
                       q_out: Optional[torch.Tensor] = None, dx: float = 1.0, tol: float = 1e-6,
                       maxit: int = 20000, stream: Optional[int] = None):
    """Projection for callers that cannot allocate device memory: the library
    uses a fixed static scratch array (grids up to 64^3) instead of a context.
    The tensors passed in are the caller's; this wrapper allocates nothing.

    There is no context to hold the layout, so the library trusts the pointers:
    every tensor is checked here first (shape, dtype, contiguity, and that it
    sits on the current CUDA device) and ValueError is raised before any call."""
    check_noalloc_args(nx, ny, nz, cell_type_dense, u, q_out)
    st = fs_stats()
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    q = C.c_void_p(q_out.data_ptr()) if q_out is not None else None
    rc = _check(load().fs_project_noalloc(nx, ny, nz, C.c_void_p(cell_type_dense.data_ptr()), _ref(_mac(u)), q,
                                          dx, tol, maxit, C.c_void_p(s), C.byref(st)))
    return rc, st.as_dict()


def fs_last_error() -> str:
    return load().fs_last_error().decode()


# ---- convenience wrapper -----------------------------------------------------

def make_params(**kw) -> fs_params:
    p = fs_default_params()
    for k, v in kw.items():
        if k == "g":
            for c in range(3):
                p.g[c] = float(v[c])
        else:
            setattr(p, k, v)
    return p


class Grid:
    """A context plus layout helpers. Fields live on `device` in the library layout."""

    def __init__(self, nx, ny, nz, params: Optional[fs_params] = None, device="cuda", stream=None, **kw):
        self.device = torch.device(device)
        self.params = params if params is not None else make_params(**kw)
        with torch.cuda.device(self.device):
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.stream = s
            self.ctx = fs_init_grid(nx, ny, nz, self.params, s.cuda_stream)
        lay = fs_layout(self.ctx)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.pitch, self.rows, self.planes, self.nelems = lay.pitch, lay.rows, lay.planes, lay.nelems

    def close(self):
        if getattr(self, "ctx", None):
            fs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **kw):
        for k, v in kw.items():
            if k == "g":
                for c in range(3):
                    self.params.g[c] = float(v[c])
            else:
                setattr(self.params, k, v)
        fs_set_params(self.ctx, self.params)

    # layout
    def empty_cell(self):
        return torch.zeros((self.planes, self.rows, self.pitch), dtype=torch.float32, device=self.device)

    def zeros(self) -> Mac:
        return Mac(self.empty_cell(), self.empty_cell(), self.empty_cell())

    def dense_shapes(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        return (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)

    def pack(self, dense) -> Mac:
        out = self.zeros()
        for t, a, s in zip(out, dense, self.dense_shapes()):
            a = torch.as_tensor(np.ascontiguousarray(a) if isinstance(a, np.ndarray) else a)
            assert tuple(a.shape) == s, (tuple(a.shape), s)
            t[: s[0], : s[1], : s[2]] = a.to(device=self.device, dtype=torch.float32)
        return out

    def unpack(self, m: Mac, dtype=np.float64):
        return tuple(t[: s[0], : s[1], : s[2]].detach().cpu().numpy().astype(dtype)
                     for t, s in zip(m, self.dense_shapes()))

    def unpack_cell(self, q: torch.Tensor, dtype=np.float64):
        return q[: self.nz, : self.ny, : self.nx].detach().cpu().numpy().astype(dtype)

    # calls
    def set_mask(self, types, bc: Optional[Mac] = None):
        t = torch.as_tensor(np.ascontiguousarray(types, dtype=np.uint8)) if isinstance(types, np.ndarray) else types
        fs_set_mask(self.ctx, t.to(self.device), bc)

    def step(self, u_in: Mac, u_out: Mac, u_visc: Optional[Mac] = None):
        return fs_step(self.ctx, u_in, u_out, u_visc)

    def project(self, u: Mac, q: Optional[torch.Tensor] = None):
        return fs_project(self.ctx, u, q)

    def adjoint_step(self, u_in: Mac, g_out: Mac, g_in: Mac, u_visc: Optional[Mac] = None):
        return fs_adjoint_step(self.ctx, u_in, u_visc, g_out, g_in)

    def precond_apply(self, r: torch.Tensor, z: torch.Tensor):
        fs_precond_apply(self.ctx, r, z)

    def pack_cell(self, a) -> torch.Tensor:
        out = self.empty_cell()
        out[: self.nz, : self.ny, : self.nx] = torch.as_tensor(np.ascontiguousarray(a)).to(self.device, torch.float32)
        return out

    def profile(self, period: int = 1):
        fs_profile(self.ctx, period)

    def profile_read(self):
        return fs_profile_read(self.ctx)

    def loss_grad(self, u: Mac, target: Mac, mask_kind=FS_MASK_SURFACE, alpha=0.0, beta=1.0,
                  g: Optional[Mac] = None) -> float:
        return fs_loss_grad(self.ctx, u, target, mask_kind, alpha, beta, g)
