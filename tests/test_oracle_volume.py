"""Oracle pins of the volumetric-velocity initialisation (Sec. 3.3.3): the
laminar wall-function base profile and the constrained divergence projection of
Eq. eq::divProj. The projection is checked against a separate matrix form (face
/ cell incidence matrices assembled here with scipy), against its fixed points,
and against its limit: the least-norm correction that removes the divergence
using only the free faces (a direct sparse solve)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2503_00868_gb300 import workloads as W

AIR, LIQ, SOL = 0, 1, 2


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def small_scene(nx=7, ny=6, nz=5, seed=0):
    types, _ = W.ellipsoid_blob(nx, ny, nz, seed, occupancy=0.5)
    return types


# ---------------------------------------------------------------- wall profile

def test_wall_profile_closed_form_values():
    nx, ny, nz = 6, 10, 5
    types = np.full((nz, ny, nx), LIQ, np.uint8)
    dx = 0.1
    g = O.Grid(types, dx, 1 / 30, 0.0)
    vinf = np.full((nz, nx), 2.0)
    delta = 0.4  # four cells
    u, v, w = O.wall_profile(g, (1.0, 0.0, 0.0), vinf, delta)
    # u faces at row j sit at y = (j + 1/2) dx; interior x faces are fluid faces
    for j in range(ny):
        e = (j + 0.5) * dx / delta
        f = 1.5 * e - 0.5 * e ** 3 if e < 1 else 1.0
        assert u[2, j, 3] == pytest.approx(2.0 * f, rel=1e-14)
    assert u[2, 1, 3] == pytest.approx(2.0 * (1.5 * 0.375 - 0.5 * 0.375 ** 3))
    # wall-normal faces at the box walls are fixed (zero), other components zero
    assert np.all(u[:, :, 0] == 0) and np.all(u[:, :, -1] == 0)
    assert np.all(v == 0) and np.all(w == 0)


def test_wall_profile_joins_the_free_stream_smoothly():
    # 1 - f(1 - h) = 3/2 h^2 - 1/2 h^3: no kink at y = delta
    nx, ny, nz = 4, 40, 3
    types = np.full((nz, ny, nx), LIQ, np.uint8)
    dx = 1.0 / ny
    g = O.Grid(types, dx, 1 / 30, 0.0)
    delta = 20.5 * dx  # face row j = 20 sits at y = delta
    u, _, _ = O.wall_profile(g, (1.0, 0.0, 0.0), np.ones((nz, nx)), delta)
    for j, h in ((19, dx / delta), (18, 2 * dx / delta)):
        assert 1.0 - u[1, j, 2] == pytest.approx(1.5 * h ** 2 - 0.5 * h ** 3, rel=1e-12)
    assert u[1, 20, 2] == 1.0 and u[1, 25, 2] == 1.0


def test_wall_profile_column_means_direction_and_face_classes():
    types = small_scene()
    nz, ny, nx = types.shape
    rng = np.random.default_rng(1)
    vinf = rng.uniform(0.5, 1.5, (nz, nx))
    shapes = W.face_shapes(nx, ny, nz)
    bc = [np.zeros(s) for s in shapes]
    bc[0][:, :, 0] = 0.3  # prescribed values on the x = 0 wall faces
    g = O.Grid(types, 1.0 / ny, 1 / 30, 0.0, bc=bc)
    d = np.array([0.6, 0.0, 0.8])
    u = O.wall_profile(g, d, vinf, 10.0)  # delta beyond the grid: factor (y/delta) profile
    cls = [np.zeros(s, np.uint8) for s in shapes]
    for c in range(3):
        O.lib().or_face_class(g.cstruct(), c, cls[c].ctypes.data_as(O.C.POINTER(O.C.c_uint8)))
    for c in range(3):
        assert np.all(u[c][cls[c] == 2] == bc[c][cls[c] == 2])   # fixed faces: prescribed
        assert np.all(u[c][cls[c] == 0] == 0.0)                  # air faces: zero
    # an interior x face between columns i-1 and i takes the mean of both speeds
    k, j, i = np.argwhere(cls[0] == 1)[0]
    e = (j + 0.5) / ny / 10.0
    assert u[0][k, j, i] == pytest.approx(0.6 * 0.5 * (vinf[k, i - 1] + vinf[k, i]) * (1.5 * e - 0.5 * e ** 3))
    kk, jj, ii = np.argwhere(cls[1] == 1)[0]
    assert u[1][kk, jj, ii] == 0.0


# ------------------------------------------------------ constrained projection

def incidence(types, dx, hold_surface):
    """Divergence matrix D (cells x stacked faces, +-1/dx), the free-face mask and
    the liquid-cell mask, built from the cell types."""
    nz, ny, nx = types.shape
    shapes = W.face_shapes(nx, ny, nz)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in shapes])

    def ctype(i, j, k):
        if i < 0 or j < 0 or k < 0 or i >= nx or j >= ny or k >= nz:
            return SOL
        return types[k, j, i]

    rows, cols, vals = [], [], []
    free = np.zeros(offs[-1], bool)
    for c in range(3):
        d = shapes[c]
        o = np.zeros(3, int)
        o[c] = 1
        for k in range(d[0]):
            for j in range(d[1]):
                for i in range(d[2]):
                    f = offs[c] + (k * d[1] + j) * d[2] + i
                    lo = ctype(i - o[0], j - o[1], k - o[2])
                    hi = ctype(i, j, k)
                    fluid = SOL not in (lo, hi) and LIQ in (lo, hi)
                    surface = {lo, hi} == {LIQ, AIR}
                    free[f] = fluid and not (hold_surface and surface)
                    if lo == LIQ:   # the face is the high face of the low cell
                        rows.append(((k - o[2]) * ny + (j - o[1])) * nx + (i - o[0])); cols.append(f); vals.append(1 / dx)
                    if hi == LIQ:
                        rows.append((k * ny + j) * nx + i); cols.append(f); vals.append(-1 / dx)
    D = sp.csr_matrix((vals, (rows, cols)), shape=(nx * ny * nz, offs[-1]))
    return D, free, (types == LIQ).ravel(), offs


def stack(u):
    return np.concatenate([a.ravel() for a in u])


def test_pbd_iteration_equals_its_matrix_form():
    types = small_scene()
    nz, ny, nx = types.shape
    dx, eps = 1.0 / ny, 3.0 * ny * ny
    g = O.Grid(types, dx, 1 / 30, 0.0)
    u0 = W.random_mac(nx, ny, nz, 4)
    for hold in (False, True):
        D, free, liq, _ = incidence(types, dx, hold)
        Df = D[:, free]
        wdiag = np.asarray((Df.multiply(Df)).sum(axis=1)).ravel() + eps
        x = stack(u0)
        for _ in range(7):
            lam = np.where(liq, -(D @ x) / wdiag, 0.0)
            x[free] += Df.T @ lam
        u, norm = O.pbd_project(g, u0, hold_surface=hold, iters=7, eps=eps)
        assert np.allclose(stack(u), x, rtol=0, atol=1e-12 * np.abs(x).max())
        assert norm == pytest.approx(np.linalg.norm((D @ x)[liq]), rel=1e-10)


def test_pbd_fixed_points_and_held_faces():
    types = small_scene(seed=3)
    nz, ny, nx = types.shape
    dx = 1.0 / ny
    g = O.Grid(types, dx, 1 / 30, 0.0)
    # a divergence-free field (the oracle's exact projection) does not move
    u, _, _ = O.project(g, W.random_mac(nx, ny, nz, 2))
    out, norm = O.pbd_project(g, u, hold_surface=False, iters=20, eps=ny * ny)
    assert norm < 1e-9
    assert np.allclose(stack(out), stack(u), atol=1e-11)
    # held faces (fixed and free-surface faces) keep their values
    u0 = W.random_mac(nx, ny, nz, 5)
    out, _ = O.pbd_project(g, u0, hold_surface=True, iters=15, eps=ny * ny)
    _, free, _, _ = incidence(types, dx, True)
    assert np.array_equal(stack(out)[~free], stack(u0)[~free])


@pytest.mark.parametrize("hold", [False, True])
def test_pbd_converges_to_the_least_norm_correction(hold):
    """The limit is a least-norm change of the free faces. When the free surface
    may move it removes the divergence. With the surface held this blob is
    enclosed by held faces: the constant over the liquid is in the null space of
    the free-face divergence D_f, and the Jacobi iteration C <- (I - D_f D_f^T W^-1) C,
    W = diag(n_free/dx^2 + eps), keeps the component of C along W 1: the divergence
    tends to alpha W 1 with alpha = sum(C_0) / sum(W), and the faces take the
    least-norm step that removes the rest."""
    types = small_scene(6, 5, 4, seed=2)
    nz, ny, nx = types.shape
    dx, eps = 1.0 / ny, 0.5 * ny * ny
    g = O.Grid(types, dx, 1 / 30, 0.0)
    u0 = W.random_mac(nx, ny, nz, 6)
    D, free, liq, _ = incidence(types, dx, hold)
    Df = D[liq][:, free].toarray()
    x0 = stack(u0)
    c0 = (D @ x0)[liq]
    w = (Df ** 2).sum(axis=1) + eps
    c_inf = (c0.sum() / w.sum()) * w if hold else np.zeros_like(c0)
    delta, *_ = np.linalg.lstsq(Df, -(c0 - c_inf), rcond=None)
    x = x0.copy()
    x[free] += delta
    assert np.linalg.norm(c0 + Df @ delta - c_inf) < 1e-10 * np.linalg.norm(c0)
    out, norm = O.pbd_project(g, u0, hold_surface=hold, iters=6000, eps=eps)
    assert norm == pytest.approx(np.linalg.norm(c_inf), abs=1e-8 * np.linalg.norm(c0))
    assert np.allclose(stack(out), x, atol=1e-8 * np.abs(x0).max())
