"""Oracle pins of the recurrent convolutional pressure solver (Sec. 3.4.1, the
PeRCNN layer in this build's reading): K sub-steps p <- p + m (W * (b - L_p p)).

Pinned against: the same recurrence written as dense matrix products (the
masked 27-tap correlation assembled here tap by tap, L_p from the pinned
operator), its fixed point (the scheme's own solution), the symmetry of the map
b -> p_K for a point-symmetric kernel (so the projection built on it is
self-adjoint, and the step's adjoint reuses it), and central finite differences
of the fit loss w.r.t. the 27 taps."""
import numpy as np
import pytest

import oracle as O
from paper_2503_00868_gb300 import workloads as W

LIQ = 1


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def scene(nx=6, ny=5, nz=4, seed=1):
    types, _ = W.ellipsoid_blob(nx, ny, nz, seed, occupancy=0.5)
    return types, O.Grid(types, 1.0 / ny, 1 / 30, 0.01)


def dense_poisson(g):
    n = g.nx * g.ny * g.nz
    A = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        A[:, c] = O.poisson_apply(g, e.reshape(g.nz, g.ny, g.nx)).ravel()
    return A


def dense_conv(types, Wk):
    """Matrix of z = m (W * r): z_i = sum_t W[t] r_{i + o(t)} over liquid i and liquid
    in-grid neighbours; taps ordered [dz][dy][dx]."""
    nz, ny, nx = types.shape
    n = nx * ny * nz
    M = np.zeros((n, n))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if types[k, j, i] != LIQ:
                    continue
                for t in range(27):
                    dz, dy, dxo = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
                    a, b, c = i + dxo, j + dy, k + dz
                    if 0 <= a < nx and 0 <= b < ny and 0 <= c < nz and types[c, b, a] == LIQ:
                        M[(k * ny + j) * nx + i, (c * ny + b) * nx + a] += Wk[t]
    return M


def symmetric_kernel(seed, center=0.12):
    w = np.random.default_rng(seed).uniform(-0.01, 0.02, 27)
    w = 0.5 * (w + w[::-1])
    w[13] = center
    return w


def liquid_rhs(types, seed):
    b = np.random.default_rng(seed).standard_normal(types.shape)
    return np.where(types == LIQ, b, 0.0)


@pytest.mark.parametrize("K", [1, 3, 12])
def test_recurrence_equals_its_dense_matrix_form(K):
    types, g = scene()
    A = dense_poisson(g)
    w = np.random.default_rng(K).uniform(-0.02, 0.05, 27)  # not symmetric: the plain recurrence
    Wm = dense_conv(types, w)
    b = liquid_rhs(types, 3).ravel()
    p = np.zeros_like(b)
    for _ in range(K):
        p = p + Wm @ (b - A @ p)
    got, st = O.percnn_solve(g, w, K, b.reshape(types.shape))
    assert np.allclose(got.ravel(), p, rtol=0, atol=1e-12 * max(1.0, np.abs(p).max()))
    assert st["iters"] == K
    assert st["true_relres"] == pytest.approx(np.linalg.norm(b - A @ p) / np.linalg.norm(b), rel=1e-10)


def test_fixed_point_is_the_scheme_solution():
    types, g = scene(seed=2)
    A = dense_poisson(g)
    q = liquid_rhs(types, 4).ravel()
    b = A @ q
    w = np.zeros(27)
    w[13] = 1.0 / 6.0  # under-relaxed Jacobi: converges for any mask
    p, st = O.percnn_solve(g, w, 4000, b.reshape(types.shape))
    assert st["true_relres"] < 1e-10
    assert np.allclose(p.ravel(), q, atol=1e-9 * np.abs(q).max())


def test_point_symmetric_kernel_gives_a_symmetric_map():
    types, g = scene(7, 6, 5, seed=3)
    w = symmetric_kernel(5)
    b, c = liquid_rhs(types, 6), liquid_rhs(types, 7)
    pb, _ = O.percnn_solve(g, w, 9, b)
    pc, _ = O.percnn_solve(g, w, 9, c)
    lhs, rhs = float((pb * c).sum()), float((b * pc).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # a kernel without the symmetry does not give a symmetric map
    w2 = w.copy()
    w2[0] += 0.05
    pb, _ = O.percnn_solve(g, w2, 9, b)
    pc, _ = O.percnn_solve(g, w2, 9, c)
    assert abs(float((pb * c).sum()) - float((b * pc).sum())) > 1e-6 * abs(lhs)


def test_loss_gradient_matches_finite_differences():
    types, g = scene(seed=4)
    A = dense_poisson(g)
    q = liquid_rhs(types, 8)
    b = (A @ q.ravel()).reshape(types.shape)
    w = symmetric_kernel(9, 0.1)
    K = 7
    loss, dW = O.percnn_loss_grad(g, w, K, b, q)
    # the loss is the energy norm of p_K - q relative to that of q
    p, _ = O.percnn_solve(g, w, K, b)
    e = (p - q).ravel()
    assert loss == pytest.approx(e @ A @ e / (q.ravel() @ A @ q.ravel()), rel=1e-12)
    h = 1e-6
    for t in (0, 4, 13, 22, 26):
        wp, wm = w.copy(), w.copy()
        wp[t] += h
        wm[t] -= h
        fd = (O.percnn_loss_grad(g, wp, K, b, q)[0] - O.percnn_loss_grad(g, wm, K, b, q)[0]) / (2 * h)
        assert dW[t] == pytest.approx(fd, rel=1e-6, abs=1e-9), t


def test_projection_with_the_recurrent_solver_and_its_adjoint():
    types, g = scene(7, 6, 5, seed=5)
    nz, ny, nx = types.shape
    w = symmetric_kernel(11, 1.0 / 6.0)
    O.set_percnn(g, w, 30)
    u0 = W.random_mac(nx, ny, nz, 12)
    b0 = O.divergence(g, u0)
    u1, _, st = O.project(g, u0)
    b1 = O.divergence(g, u1)
    # 30 sub-steps reduce the divergence without removing it
    assert np.linalg.norm(b1) < 0.7 * np.linalg.norm(b0)
    assert st["iters"] == 30
    # on fields carried by the fluid faces (the adjoint step drops the cotangent of
    # fixed faces, which the divergence reads but the gradient never moves) the
    # projection is symmetric: dot-product test
    cls = [np.zeros(s, np.uint8) for s in W.face_shapes(nx, ny, nz)]
    for c in range(3):
        O.lib().or_face_class(g.cstruct(), c, cls[c].ctypes.data_as(O.C.POINTER(O.C.c_uint8)))
    u0 = [np.where(cl == 1, a, 0.0) for cl, a in zip(cls, u0)]
    v0 = [np.where(cl == 1, a, 0.0) for cl, a in zip(cls, W.random_mac(nx, ny, nz, 13))]
    pu, _, _ = O.project(g, u0)
    pv, _, _ = O.project(g, v0)
    dot = lambda a, b: sum(float((x * y).sum()) for x, y in zip(a, b))
    assert dot(pu, v0) == pytest.approx(dot(u0, pv), rel=1e-11)
