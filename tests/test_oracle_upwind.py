"""Oracle pins of the upwind surrogate for the reverse of convection (Sec. 3.4.1:
the derivative of the convected velocity v with respect to the transporting
velocity component i is taken as -dt dv/di, with dv/di a first-order upwind
difference). The surrogate passes each fluid face's cotangent through to the
same face and routes -dt ga_c dv_c/de to the velocity component e seen there.

Pinned by hand on fields where every quantity has a closed form:
* a u-component linear in x, v and w constant: the convected u is u (1 - h s),
  so the surrogate is ga_u (1 - h s (1 - h s)) on interior x-faces and the
  identity on the other components (h = dt/dx, s the slope per cell);
* a V-shaped w-component across x transported by a constant u: the upwind
  difference at the kink takes the side the flow comes from, which flips with
  the sign of u, and the x-transport term of a w-face goes to the four u-faces
  averaged there, a quarter each;
* dt = 0: the identity on fluid faces, zero elsewhere."""
import numpy as np
import pytest

from paper_2503_00868_gb300 import workloads as W

LIQ = 1


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def test_linear_u_closed_form(O):
    nx, ny, nz = 12, 7, 6
    dx, dt = 0.1, 0.02
    h = dt / dx
    types = W.all_liquid(nx, ny, nz)
    g = O.Grid(types, dx, dt, 0.0)
    s_cell = 1.0                       # slope of u per cell: h s = 0.2
    U, V, Wc = (np.zeros(sh) for sh in g.shapes())
    ii = np.arange(nx + 1)[None, None, :]
    U[:] = 0.3 + s_cell * ii
    V[:] = 0.05
    Wc[:] = -0.07
    for c in range(3):                  # the wall-normal faces hold their prescribed 0
        fc = O.face_class(g, c)
        (U, V, Wc)[c][fc == 2] = 0.0
    rng = np.random.default_rng(3)
    ga = tuple(rng.standard_normal(sh) for sh in g.shapes())
    gu = O.advect_adjoint_upwind(g, (U, V, Wc), ga)
    # x-faces whose upwind stencil and back-traces stay off the wall faces (the
    # back-trace from face 1 samples the fixed face 0)
    sl = (slice(None), slice(None), slice(3, nx - 1))
    expect = ga[0] * (1.0 - h * s_cell * (1.0 - h * s_cell))
    np.testing.assert_allclose(gu[0][sl], expect[sl], rtol=1e-12, atol=1e-12)
    # v and w are constant and convect to themselves, except next to their wall
    # faces, whose prescribed 0 the back-trace samples (v transported by +0.05
    # in y reads the face below, w by -0.07 in z the face above): away from
    # those, the surrogate is the identity
    fv, fw = O.face_class(g, 1), O.face_class(g, 2)
    np.testing.assert_allclose(gu[1][:, 3:ny, :], ga[1][:, 3:ny, :], rtol=0, atol=1e-12)
    np.testing.assert_allclose(gu[2][1:nz - 2], ga[2][1:nz - 2], rtol=0, atol=1e-12)
    # (transport terms routed to the wall faces of v and w vanish: no slope along y or z)
    assert np.abs(gu[1][fv != 1]).max() < 1e-12 and np.abs(gu[2][fw != 1]).max() < 1e-12


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_upwind_side_and_routing_at_a_kink(O, sign):
    nx, ny, nz = 10, 5, 6
    dx, dt = 0.1, 0.02
    h = dt / dx
    types = W.all_liquid(nx, ny, nz)
    g = O.Grid(types, dx, dt, 0.0)
    Uc = 0.4 * sign                     # constant transport along x: h |U| = 0.08
    t = 0.5
    i0 = 5
    U, V, Wc = (np.zeros(sh) for sh in g.shapes())
    U[:] = Uc
    fc_u = O.face_class(g, 0)
    U[fc_u == 2] = 0.0
    ii = np.arange(nx)[None, None, :]
    Wc[:] = t * np.abs(ii - i0)         # w faces: shape (nz + 1, ny, nx)
    fc_w = O.face_class(g, 2)
    Wc[fc_w == 2] = 0.0
    ga = tuple(np.zeros(sh) for sh in g.shapes())
    k, j = 3, 2                          # an interior w-face at the kink
    ga[2][k, j, i0] = 1.0
    gu = O.advect_adjoint_upwind(g, (U, V, Wc), ga)
    # convected w near the kink: v(i) = w(i - h U); the upwind side is i0 - 1 for
    # U > 0 and i0 + 1 for U < 0; both differences equal -t and +t respectively
    dv = -t if sign > 0 else t
    gv = -h * dv * 1.0
    # w-face (k, j, i0) averages the u-faces of cells (i0, j, k - 1) and (i0, j, k):
    # u indices (k - 1, j, i0), (k - 1, j, i0 + 1), (k, j, i0), (k, j, i0 + 1)
    for kk in (k - 1, k):
        for ii_ in (i0, i0 + 1):
            assert gu[0][kk, j, ii_] == pytest.approx(0.25 * gv, rel=1e-12)
    # the value term, and nothing else on the w-faces
    assert gu[2][k, j, i0] == pytest.approx(1.0, rel=1e-12)
    mask = np.ones_like(gu[2], dtype=bool)
    mask[k, j, i0] = False
    assert np.all(gu[2][mask] == 0.0)


def test_zero_time_step_is_the_identity(O):
    nx, ny, nz = 9, 8, 7
    types, _ = W.ellipsoid_blob(nx, ny, nz, 1)
    g = O.Grid(types, 1.0 / ny, 0.0, 0.0)
    u = W.blurred_noise_mac(nx, ny, nz, 2)
    ga = W.random_mac(nx, ny, nz, 5)
    gu = O.advect_adjoint_upwind(g, u, ga)
    for c in range(3):
        fc = O.face_class(g, c)
        np.testing.assert_array_equal(gu[c][fc == 1], ga[c][fc == 1])
        assert np.all(gu[c][fc != 1] == 0.0)
