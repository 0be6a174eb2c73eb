"""Oracle pins of the APIC transfers and the Gaussian deformation (Sec. 3.2.2,
Sec. 3.4.3) on the MAC grid, per face component with quadratic B-splines.

Independent checks: the quadratic B-spline's partition of unity, zero first
moment and dx^2/4 second moment make P2G reproduce any affine velocity field
exactly when C_p is its gradient, and make G2P recover an affine grid field's
value and gradient exactly; P2G conserves linear momentum; a single particle
with C = 0 spreads its own velocity; the deformation and covariance updates
match their closed forms."""
import numpy as np
import pytest

import oracle as O

AIR, LIQ = 0, 1


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def grid(nx=10, ny=9, nz=8):
    return O.Grid(np.full((nz, ny, nx), LIQ, np.uint8), 0.1, 1 / 30, 0.0)


def interior_particles(g, n, seed, margin=2.0):
    rng = np.random.default_rng(seed)
    lo = margin * g.dx
    hi = np.array([g.nx, g.ny, g.nz]) * g.dx - margin * g.dx
    return lo + rng.random((n, 3)) * (hi - lo)


def face_positions(g, c):
    d = [g.nx, g.ny, g.nz]
    d[c] += 1
    k, j, i = np.meshgrid(np.arange(d[2]), np.arange(d[1]), np.arange(d[0]), indexing="ij")
    pos = [i * g.dx, j * g.dx, k * g.dx]
    for a in range(3):
        if a != c:
            pos[a] = pos[a] + 0.5 * g.dx
    return pos


def test_p2g_reproduces_affine_fields():
    g = grid()
    rng = np.random.default_rng(1)
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    x = interior_particles(g, 4000, 2)
    v = a + x @ B.T
    Cp = np.broadcast_to(B, (x.shape[0], 3, 3))
    m = rng.uniform(0.5, 2.0, x.shape[0])
    u, mass = O.p2g(g, x, v, Cp, m, return_mass=True)
    for c in range(3):
        pos = face_positions(g, c)
        exact = a[c] + sum(B[c, k] * pos[k] for k in range(3))
        got = mass[c] > 0
        assert got.sum() > 0.3 * got.size
        assert np.allclose(u[c][got], exact[got], atol=1e-11)
        assert np.all(u[c][~got] == 0.0)


def test_p2g_conserves_momentum_and_spreads_a_single_particle():
    g = grid()
    rng = np.random.default_rng(3)
    x = interior_particles(g, 500, 4)
    v = rng.standard_normal((500, 3))
    Cp = 0.3 * rng.standard_normal((500, 3, 3))
    m = rng.uniform(0.5, 2.0, 500)
    u, mass = O.p2g(g, x, v, Cp, m, return_mass=True)
    for c in range(3):
        # sum_i m_i v_i = sum_p m_p v_p: the weights sum to 1 and the affine part has zero mean
        assert (mass[c] * u[c]).sum() == pytest.approx((m * v[:, c]).sum(), rel=1e-12)
        assert mass[c].sum() == pytest.approx(m.sum(), rel=1e-12)
    one = O.p2g(g, x[:1], v[:1], np.zeros((1, 3, 3)), m[:1])
    for c in range(3):
        nz = one[c] != 0
        assert nz.sum() == 27 and np.allclose(one[c][nz], v[0, c])


def test_g2p_recovers_affine_value_and_gradient():
    g = grid()
    rng = np.random.default_rng(5)
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    u = []
    for c in range(3):
        pos = face_positions(g, c)
        u.append(a[c] + sum(B[c, k] * pos[k] for k in range(3)))
    x = interior_particles(g, 300, 6)
    _, v, Cp, _, _ = O.g2p(g, x, u)
    assert np.allclose(v, a + x @ B.T, atol=1e-11)
    assert np.allclose(Cp, np.broadcast_to(B, Cp.shape), atol=1e-9)


def test_particle_advance_deformation_and_covariance():
    g = grid()
    rng = np.random.default_rng(7)
    B = 0.5 * rng.standard_normal((3, 3))
    a = rng.standard_normal(3)
    u = []
    for c in range(3):
        pos = face_positions(g, c)
        u.append(a[c] + sum(B[c, k] * pos[k] for k in range(3)))
    x0 = interior_particles(g, 50, 8, margin=3.0)
    F0 = np.broadcast_to(np.eye(3) + 0.1 * rng.standard_normal((3, 3)), (50, 3, 3)).copy()
    L = rng.standard_normal((50, 3, 3))
    A0 = L @ np.transpose(L, (0, 2, 1))
    dt = 0.01
    x, v, Cp, F, A = O.g2p(g, x0, u, F=F0, A0=A0, dt=dt, advance=True, lo=0.0, hi=1.0)
    assert np.allclose(x, x0 + dt * (a + x0 @ B.T), atol=1e-12)
    Fx = (np.eye(3) + dt * B) @ F0
    assert np.allclose(F, Fx, atol=1e-10)
    assert np.allclose(A, Fx @ A0 @ np.transpose(Fx, (0, 2, 1)), atol=1e-9)
    # positions are clamped to [lo, hi]
    x2, *_ = O.g2p(g, x0, u, dt=100.0, advance=True, lo=0.2, hi=0.7)
    assert x2.min() >= 0.2 and x2.max() <= 0.7


def test_round_trip_keeps_affine_velocity():
    g = grid(12, 11, 10)
    rng = np.random.default_rng(9)
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    x = interior_particles(g, 6000, 10)
    u = O.p2g(g, x, a + x @ B.T, np.broadcast_to(B, (6000, 3, 3)), np.ones(6000))
    _, v, Cp, _, _ = O.g2p(g, x[:200], u)
    assert np.allclose(v, a + x[:200] @ B.T, atol=1e-10)
    assert np.allclose(Cp, np.broadcast_to(B, Cp.shape), atol=1e-8)
