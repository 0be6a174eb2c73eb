"""FP64 CPU oracle for the differentiable MAC-grid fluid step (arXiv 2503.00868).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. The CUDA product path
never does, and the two share no code (this package is plain C in ``oracle.c``
behind ctypes, compiled with gcc).

Fields are tuples ``(u, v, w)`` of dense float64 arrays with shapes
``(nz, ny, nx+1)``, ``(nz, ny+1, nx)``, ``(nz+1, ny, nx)``; cell arrays have shape
``(nz, ny, nx)``; cell types are uint8 (0 air, 1 liquid, 2 solid).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PC_NONE, PC_JACOBI, PC_MIC0 = 0, 1, 2
NET_CH = (2, 16, 16, 16, 16, 1)


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, portable flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("type", C.POINTER(C.c_uint8)),
                ("bc", C.POINTER(C.c_double) * 3),
                ("dx", C.c_double), ("dt", C.c_double), ("nu", C.c_double),
                ("g", C.c_double * 3),
                ("tol_p", C.c_double), ("tol_v", C.c_double),
                ("maxit_p", C.c_int), ("maxit_v", C.c_int),
                ("precond", C.c_int),
                ("mic_tau", C.c_double), ("mic_sigma", C.c_double),
                ("percnn_w", C.POINTER(C.c_double)), ("percnn_k", C.c_int), ("advect_grad", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int),
                ("relres", C.c_double), ("true_relres", C.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "status": self.status, "relres": self.relres,
                "true_relres": self.true_relres}


_D = C.POINTER(C.c_double)
_P3 = _D * 3


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            G = C.POINTER(_Grid)
            sig = {
                "or_face_class": [G, C.c_int, C.POINTER(C.c_uint8)],
                "or_advect": [G, _P3, _P3],
                "or_advect_adjoint": [G, _P3, _P3, _P3],
                "or_advect_samples": [G, C.c_int, _P3, _D],
                "or_advect_adjoint_upwind": [G, _P3, _P3, _P3],
                "or_visc_apply": [G, _P3, _P3],
                "or_visc_solve": [G, _P3, _P3, C.POINTER(Stats)],
                "or_divergence": [G, _P3, _D],
                "or_poisson_apply": [G, _D, _D],
                "or_grad_subtract": [G, _D, _P3],
                "or_is_singular": [G],
                "or_mic0_factor": [G, C.c_double, C.c_double, _D],
                "or_mic0_apply": [G, _D, _D, _D],
                "or_pcg": [G, _D, _D, C.c_int, C.POINTER(Stats)],
                "or_project": [G, _P3, _D, C.POINTER(Stats)],
                "or_step": [G, _P3, _P3, C.c_void_p, C.POINTER(Stats)],
                "or_adjoint_step": [G, _P3, _P3, _P3, _D, C.POINTER(Stats)],
                "or_band_cells": [G, C.c_int, C.POINTER(C.c_uint8)],
                "or_loss_grad": [G, _P3, _P3, C.c_int, C.c_double, C.c_double, _D, _P3],
                "or_bf16_round": [C.c_double],
                "or_net_forward": [G, _D * 5, _D * 5, _D, _D, _D],
                "or_net_loss_grad": [G, _D * 5, _D * 5, _D, _D, _D * 5, _D * 5],
                "or_wall_profile": [G, _D, _D, C.c_double, _P3],
                "or_pbd_project": [G, _P3, C.c_int, C.c_int, C.c_double],
                "or_percnn_solve": [G, _D, C.c_int, _D, _D, C.POINTER(Stats)],
                "or_p2g": [G, C.c_int, _D, _D, _D, _D, _P3, C.c_void_p],
                "or_splat_render": [C.c_int, _D, _D, _D, _D, C.c_void_p, _D, _D],
                "or_splat_render_flags": [C.c_int, _D, _D, _D, _D, C.c_void_p, _D, _D, C.POINTER(C.c_uint8),
                                          C.c_double],
                "or_splat_render_sh": [C.c_int, _D, _D, _D, _D, C.c_int, C.c_void_p, _D, _D, C.POINTER(C.c_uint8),
                                       C.c_double],
                "or_sh_basis": [C.c_int, _D, _D],
                "or_g2p": [G, C.c_int, _D, _D, _D, _D, _D, _D, _P3, C.c_double, C.c_int, C.c_double, C.c_double],
                "or_percnn_loss_grad": [G, _D, C.c_int, _D, _D, _D],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = None
            L.or_is_singular.restype = C.c_int
            L.or_bf16_round.restype = C.c_double
            L.or_net_forward.restype = C.c_double
            L.or_net_loss_grad.restype = C.c_double
            L.or_pbd_project.restype = C.c_double
            L.or_percnn_loss_grad.restype = C.c_double
            _lib = L
    return _lib


def face_shapes(nx, ny, nz):
    return (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_D)


def _p3(arrs):
    return _P3(*[_ptr(a) for a in arrs])


class Grid:
    """A grid, its cell types, prescribed face values and step parameters."""

    def __init__(self, types, dx, dt, nu, g=(0.0, 0.0, 0.0), bc=None, tol_p=1e-13,
                 tol_v=1e-13, maxit_p=100000, maxit_v=100000, precond=PC_JACOBI,
                 mic_tau=0.97, mic_sigma=0.25, advect_grad=0):
        self.types = np.ascontiguousarray(types, dtype=np.uint8)
        self.nz, self.ny, self.nx = self.types.shape
        self.bc = None if bc is None else tuple(_f64(a) for a in bc)
        if self.bc is not None:
            for a, s in zip(self.bc, face_shapes(self.nx, self.ny, self.nz)):
                assert a.shape == s, (a.shape, s)
        self.dx, self.dt, self.nu = float(dx), float(dt), float(nu)
        self.g = tuple(float(x) for x in g)
        self.tol_p, self.tol_v = float(tol_p), float(tol_v)
        self.maxit_p, self.maxit_v = int(maxit_p), int(maxit_v)
        self.precond = int(precond)
        self.mic_tau, self.mic_sigma = float(mic_tau), float(mic_sigma)
        self.advect_grad = int(advect_grad)   # 0 exact adjoint of advection, 1 the upwind surrogate

    def shapes(self):
        return face_shapes(self.nx, self.ny, self.nz)

    def zeros(self):
        return tuple(np.zeros(s) for s in self.shapes())

    def cstruct(self):
        s = _Grid()
        s.nx, s.ny, s.nz = self.nx, self.ny, self.nz
        s.type = self.types.ctypes.data_as(C.POINTER(C.c_uint8))
        for c in range(3):
            s.bc[c] = _ptr(self.bc[c]) if self.bc is not None else _D()
        s.dx, s.dt, s.nu = self.dx, self.dt, self.nu
        for c in range(3):
            s.g[c] = self.g[c]
        s.tol_p, s.tol_v = self.tol_p, self.tol_v
        s.maxit_p, s.maxit_v = self.maxit_p, self.maxit_v
        s.precond = self.precond
        s.mic_tau, s.mic_sigma = self.mic_tau, self.mic_sigma
        pw = getattr(self, "percnn_w", None)
        s.percnn_w = _ptr(pw) if pw is not None else _D()
        s.percnn_k = int(getattr(self, "percnn_k", 0)) if pw is not None else 0
        s.advect_grad = self.advect_grad
        self._keep = s
        return C.byref(s)


def _field(g: Grid, u):
    out = tuple(_f64(a) for a in u)
    for a, s in zip(out, g.shapes()):
        assert a.shape == s, (a.shape, s)
    return out


def face_class(g: Grid, c: int):
    out = np.zeros(g.shapes()[c], dtype=np.uint8)
    lib().or_face_class(g.cstruct(), c, out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return out


def advect(g: Grid, u):
    u = _field(g, u)
    out = g.zeros()
    lib().or_advect(g.cstruct(), _p3(u), _p3(out))
    return out


def advect_adjoint_upwind(g: Grid, u, ga):
    """The upwind surrogate of the reverse of advection (Sec. 3.4.1): gu =
    ga + the transport terms -dt ga_c dv_c/de (upwind differences of the
    convected field v), routed to the velocity components seen at each face."""
    u, ga = _field(g, u), _field(g, ga)
    gu = g.zeros()
    lib().or_advect_adjoint_upwind(g.cstruct(), _p3(u), _p3(ga), _p3(gu))
    return gu


def advect_samples(g: Grid, u, c: int):
    """Back-traced sample points (index space, before clamping) of the fluid
    faces of component c, shape face_shapes[c] + (3,) in (x, y, z) order; NaN on
    faces that are not advected."""
    u = _field(g, u)
    out = np.zeros(g.shapes()[c] + (3,))
    lib().or_advect_samples(g.cstruct(), int(c), _p3(u), _ptr(out))
    return out


def kink_faces(g: Grid, u, eps: float = 3e-5, halo: int = 2):
    """Per component, the faces whose reverse-mode value is not unique under a
    perturbation of the sample point by eps: those within `halo` cells of a
    fluid face whose back-traced sample has a coordinate within eps of an
    integer (a kink of the trilinear interpolation). Boolean arrays of the face
    shapes. Used by tests that bound errors face by face."""
    from scipy.ndimage import binary_dilation
    cell = np.zeros((g.nz + 1, g.ny + 1, g.nx + 1), dtype=bool)
    for c in range(3):
        s = advect_samples(g, u, c)
        near = np.any(np.abs(s - np.round(s)) < eps, axis=-1)   # NaN compares False
        k, j, i = np.nonzero(near)
        cell[k, j, i] = True
    cell = binary_dilation(cell, iterations=halo)
    return tuple(cell[:sh[0], :sh[1], :sh[2]] for sh in g.shapes())


def advect_adjoint(g: Grid, u, ga):
    u, ga = _field(g, u), _field(g, ga)
    out = g.zeros()
    lib().or_advect_adjoint(g.cstruct(), _p3(u), _p3(ga), _p3(out))
    return out


def visc_apply(g: Grid, x):
    x = _field(g, x)
    out = g.zeros()
    lib().or_visc_apply(g.cstruct(), _p3(x), _p3(out))
    return out


def visc_solve(g: Grid, ub):
    ub = _field(g, ub)
    out = g.zeros()
    st = Stats()
    lib().or_visc_solve(g.cstruct(), _p3(ub), _p3(out), C.byref(st))
    return out, st.as_dict()


def divergence(g: Grid, u):
    u = _field(g, u)
    b = np.zeros((g.nz, g.ny, g.nx))
    lib().or_divergence(g.cstruct(), _p3(u), _ptr(b))
    return b


def poisson_apply(g: Grid, x):
    x = _f64(x)
    y = np.zeros_like(x)
    lib().or_poisson_apply(g.cstruct(), _ptr(x), _ptr(y))
    return y


def grad_subtract(g: Grid, q, u):
    q = _f64(q)
    u = tuple(a.copy() for a in _field(g, u))
    lib().or_grad_subtract(g.cstruct(), _ptr(q), _p3(u))
    return u


def is_singular(g: Grid) -> bool:
    return bool(lib().or_is_singular(g.cstruct()))


def mic0_factor(g: Grid, tau=None, sigma=None):
    prec = np.zeros((g.nz, g.ny, g.nx))
    lib().or_mic0_factor(g.cstruct(), g.mic_tau if tau is None else tau,
                         g.mic_sigma if sigma is None else sigma, _ptr(prec))
    return prec


def mic0_apply(g: Grid, prec, r):
    prec, r = _f64(prec), _f64(r)
    z = np.zeros_like(r)
    lib().or_mic0_apply(g.cstruct(), _ptr(prec), _ptr(r), _ptr(z))
    return z


def pcg(g: Grid, b, precond=None):
    b = _f64(b)
    x = np.zeros_like(b)
    st = Stats()
    lib().or_pcg(g.cstruct(), _ptr(b), _ptr(x), g.precond if precond is None else precond,
                 C.byref(st))
    return x, st.as_dict()


def project(g: Grid, u):
    u = tuple(a.copy() for a in _field(g, u))
    q = np.zeros((g.nz, g.ny, g.nx))
    st = Stats()
    lib().or_project(g.cstruct(), _p3(u), _ptr(q), C.byref(st))
    return u, q, st.as_dict()


def step(g: Grid, u, save_visc=False):
    u = _field(g, u)
    out = g.zeros()
    st = (Stats * 2)()
    uv = g.zeros() if save_visc else None
    uv_ptrs = _p3(uv) if save_visc else None
    lib().or_step(g.cstruct(), _p3(u), _p3(out),
                  C.cast(uv_ptrs, C.c_void_p) if save_visc else None, st)
    stats = {"visc": st[0].as_dict(), "pressure": st[1].as_dict()}
    return (out, uv, stats) if save_visc else (out, stats)


def adjoint_step(g: Grid, u, g_out):
    u, g_out = _field(g, u), _field(g, g_out)
    g_in = g.zeros()
    gnu = C.c_double(0.0)
    st = (Stats * 3)()
    lib().or_adjoint_step(g.cstruct(), _p3(u), _p3(g_out), _p3(g_in), C.byref(gnu), st)
    return g_in, gnu.value


def band_cells(g: Grid, kind=0):
    out = np.zeros((g.nz, g.ny, g.nx), dtype=np.uint8)
    lib().or_band_cells(g.cstruct(), kind, out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return out


def loss_grad(g: Grid, u, target, kind=0, alpha=0.0, beta=1.0):
    u, target = _field(g, u), _field(g, target)
    grad = g.zeros()
    loss = C.c_double(0.0)
    lib().or_loss_grad(g.cstruct(), _p3(u), _p3(target), kind, alpha, beta, C.byref(loss),
                       _p3(grad))
    return loss.value, grad


def bf16_round(x):
    f = np.vectorize(lib().or_bf16_round, otypes=[np.float64])
    return f(np.asarray(x, dtype=np.float64))


def _net_ptrs(arrs):
    return (_D * 5)(*[_ptr(a) for a in arrs])


def net_forward(g: Grid, W, B, r, return_acts=False):
    """W: 5 arrays [co, ci, 3, 3, 3]; B: 5 arrays [co]. Returns z (and s, acts)."""
    W = [_f64(w) for w in W]
    B = [_f64(b) for b in B]
    r = _f64(r)
    z = np.zeros_like(r)
    n = r.size
    acts = np.zeros(sum(NET_CH) * n)
    s = lib().or_net_forward(g.cstruct(), _net_ptrs(W), _net_ptrs(B), _ptr(r), _ptr(z), _ptr(acts))
    if return_acts:
        return z, s, acts
    return z


def net_loss_grad(g: Grid, W, B, b, q):
    W = [_f64(w) for w in W]
    B = [_f64(x) for x in B]
    gW = [np.zeros_like(w) for w in W]
    gB = [np.zeros_like(x) for x in B]
    loss = lib().or_net_loss_grad(g.cstruct(), _net_ptrs(W), _net_ptrs(B), _ptr(_f64(b)),
                                  _ptr(_f64(q)), _net_ptrs(gW), _net_ptrs(gB))
    return loss, gW, gB


def wall_profile(g: Grid, direction, vinf, delta):
    """Base velocity of the volumetric initialisation (Sec. 3.3.3); vinf: (nz, nx)."""
    out = g.zeros()
    d = _f64(direction)
    v = _f64(vinf)
    assert v.shape == (g.nz, g.nx)
    lib().or_wall_profile(g.cstruct(), _ptr(d), _ptr(v), float(delta), _p3(out))
    return out


def pbd_project(g: Grid, u, hold_surface=True, iters=100, eps=0.0):
    """Constrained divergence projection (Eq. eq::divProj); returns (u, |div|_2)."""
    u = [a.copy() for a in _field(g, u)]
    norm = lib().or_pbd_project(g.cstruct(), _p3(u), int(bool(hold_surface)), int(iters), float(eps))
    return u, norm


def set_percnn(g: Grid, W, K: int):
    """Make the grid's projection (project, step, adjoint_step) solve the pressure by
    K recurrent sub-steps with the 27-tap kernel W (None: back to PCG)."""
    g.percnn_w = None if W is None else _f64(np.asarray(W).ravel())
    g.percnn_k = int(K)


def percnn_solve(g: Grid, W, K, b):
    p = np.zeros((g.nz, g.ny, g.nx))
    st = Stats()
    lib().or_percnn_solve(g.cstruct(), _ptr(_f64(np.asarray(W).ravel())), int(K), _ptr(_f64(b)), _ptr(p),
                          C.byref(st))
    return p, st.as_dict()


def percnn_loss_grad(g: Grid, W, K, b, q):
    dW = np.zeros(27)
    loss = lib().or_percnn_loss_grad(g.cstruct(), _ptr(_f64(np.asarray(W).ravel())), int(K), _ptr(_f64(b)),
                                     _ptr(_f64(q)), _ptr(dW))
    return loss, dW


def p2g(g: Grid, x, v, Cp, m, return_mass=False):
    """APIC particle -> MAC grid (Eq. eq::particle_map). x, v: (np, 3); Cp: (np, 3, 3); m: (np,)."""
    x, v, Cp, m = _f64(x), _f64(v), _f64(Cp), _f64(m)
    n = x.shape[0]
    u = g.zeros()
    mass = g.zeros()
    mp = _P3(*[_ptr(a) for a in mass])
    lib().or_p2g(g.cstruct(), n, _ptr(x), _ptr(v), _ptr(Cp), _ptr(m), _p3(u), C.cast(C.pointer(mp), C.c_void_p))
    return (u, mass) if return_mass else u


def g2p(g: Grid, x, u, F=None, A0=None, dt=0.0, advance=False, lo=0.0, hi=1e30):
    """MAC grid -> particles: returns (x, v, C, F, A) after the optional advance."""
    x = _f64(x).copy()
    n = x.shape[0]
    v = np.zeros((n, 3))
    Cm = np.zeros((n, 3, 3))
    Fm = None if F is None else _f64(F).copy()
    A = None if A0 is None else np.zeros((n, 3, 3))
    u = _field(g, u)
    lib().or_g2p(g.cstruct(), n, _ptr(x), _ptr(v), _ptr(Cm), _ptr(Fm) if Fm is not None else _D(),
                 _ptr(_f64(A0)) if A0 is not None else _D(), _ptr(A) if A is not None else _D(), _p3(u),
                 float(dt), int(bool(advance)), float(lo), float(hi))
    return x, v, Cm, Fm, A


class Camera(C.Structure):
    """Pinhole camera of the splatting renderer: x_c = R x + t; pixels (fx, fy, cx, cy)."""
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int), ("height", C.c_int),
                ("znear", C.c_double), ("bg", C.c_double * 3)]


def make_camera(R, t, fx, fy, cx, cy, width, height, znear=0.01, bg=(0.0, 0.0, 0.0)):
    cam = Camera()
    for k in range(9):
        cam.R[k] = float(np.asarray(R, float).ravel()[k])
    for k in range(3):
        cam.t[k] = float(t[k])
        cam.bg[k] = float(bg[k])
    cam.fx, cam.fy, cam.cx, cam.cy = float(fx), float(fy), float(cx), float(cy)
    cam.width, cam.height, cam.znear = int(width), int(height), float(znear)
    return cam


def splat_render(x, opacity, A, color, cam, near_rel=None):
    """Front-to-back splatting (Sec. 3.2.1); returns rgb (h, w, 3) and transmittance
    (h, w). With near_rel, also a uint8 (h, w) mask of the pixels whose value turns
    on a threshold decision within that relative distance, by enough to show (the
    3-sigma cutoff and the 1/255 alpha floor where the Gaussian's share there
    exceeds 2e-5, the 1e-4 transmittance floor, depths within 4e-6 of each
    other)."""
    x, o, A, c = _f64(x), _f64(opacity), _f64(A), _f64(color)
    n = x.shape[0]
    rgb = np.zeros((cam.height, cam.width, 3))
    T = np.zeros((cam.height, cam.width))
    cp = C.cast(C.pointer(cam), C.c_void_p)
    if near_rel is None:
        lib().or_splat_render(n, _ptr(x), _ptr(o), _ptr(A), _ptr(c), cp, _ptr(rgb), _ptr(T))
        return rgb, T
    near = np.zeros((cam.height, cam.width), dtype=np.uint8)
    lib().or_splat_render_flags(n, _ptr(x), _ptr(o), _ptr(A), _ptr(c), cp, _ptr(rgb), _ptr(T),
                                near.ctypes.data_as(C.POINTER(C.c_uint8)), float(near_rel))
    return rgb, T, near


def sh_basis(degree: int, d):
    """The real spherical harmonics Y_0 .. Y_{(degree+1)^2 - 1} at the unit vector d."""
    out = np.zeros(16)
    lib().or_sh_basis(int(degree), _ptr(_f64(d)), _ptr(out))
    return out[:(degree + 1) ** 2]


def splat_render_sh(x, opacity, A, sh, degree, cam, near_rel=None):
    """Splatting with view-dependent colours from spherical-harmonic coefficients
    sh (n, (degree+1)^2, 3); returns rgb, T and, with near_rel, the flag mask."""
    x, o, A, sh = _f64(x), _f64(opacity), _f64(A), _f64(sh)
    n = x.shape[0]
    rgb = np.zeros((cam.height, cam.width, 3))
    T = np.zeros((cam.height, cam.width))
    near = np.zeros((cam.height, cam.width), dtype=np.uint8)
    lib().or_splat_render_sh(n, _ptr(x), _ptr(o), _ptr(A), _ptr(sh), int(degree), C.cast(C.pointer(cam), C.c_void_p),
                             _ptr(rgb), _ptr(T), near.ctypes.data_as(C.POINTER(C.c_uint8)),
                             float(near_rel if near_rel is not None else 0.0))
    return (rgb, T, near) if near_rel is not None else (rgb, T)
