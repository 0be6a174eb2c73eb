"""Pins of the FP64 oracle's grid operators against mathematics that does not come
from the oracle itself: closed-form eigenvectors, exact identities of the MAC
discretisation, dense library solves and the defining properties of IC(0)/MIC(0).
"""
import numpy as np
import pytest

from paper_2503_00868_gb300 import workloads as W

AIR, LIQ, SOL = 0, 1, 2


def tg_field(nx, ny, nz, h):
    """Discrete Taylor-Green mode u = sin(pi x) cos(pi y), v = -cos(pi x) sin(pi y)
    sampled on the MAC faces of the box [0, nx h] x [0, ny h] (nx = ny = 1/h)."""
    i = np.arange(nx + 1)
    j = np.arange(ny)
    u = np.zeros((nz, ny, nx + 1))
    u[:] = np.sin(np.pi * i * h)[None, None, :] * np.cos(np.pi * (j + 0.5) * h)[None, :, None]
    ii = np.arange(nx)
    jj = np.arange(ny + 1)
    v = np.zeros((nz, ny + 1, nx))
    v[:] = -np.cos(np.pi * (ii + 0.5) * h)[None, None, :] * np.sin(np.pi * jj * h)[None, :, None]
    w = np.zeros((nz + 1, ny, nx))
    return u, v, w


def small_blob(n=12, seed=3):
    types, _ = W.ellipsoid_blob(n, n - 2, n + 1, seed)
    return types


def restrict_fluid(O, g, u):
    return tuple(np.where(O.face_class(g, c) == 1, u[c], 0.0) for c in range(3))


def test_face_classes_on_box_walls(oracle_mod):
    O = oracle_mod
    types = W.all_liquid(5, 4, 3)
    types[1, 1, 2] = AIR
    g = O.Grid(types, 0.2, 0.1, 0.0)
    fu = O.face_class(g, 0)
    assert (fu[:, :, 0] == 2).all() and (fu[:, :, -1] == 2).all()
    assert (fu[:, :, 1:-1] == 1).all()  # every interior face touches a liquid cell
    types2 = np.full((3, 3, 4), AIR, dtype=np.uint8)
    types2[1, 1, 1] = LIQ
    types2[1, 1, 3] = SOL
    g2 = O.Grid(types2, 1.0, 0.1, 0.0)
    fu2 = O.face_class(g2, 0)
    assert fu2[1, 1, 1] == 1 and fu2[1, 1, 2] == 1     # liquid-air both sides
    assert fu2[1, 1, 3] == 2 and fu2[1, 1, 4] == 2     # touching the solid cell / wall
    assert fu2[0, 0, 2] == 0                           # air-air


def test_divergence_of_linear_field(oracle_mod):
    """u = a x, v = b y, w = c z has exact divergence a + b + c on every cell."""
    O = oracle_mod
    nx, ny, nz, h = 6, 5, 7, 0.125
    a, b, c = 0.3, -1.7, 2.2
    u = np.broadcast_to(a * np.arange(nx + 1) * h, (nz, ny, nx + 1)).copy()
    v = np.broadcast_to((b * np.arange(ny + 1) * h)[:, None], (nz, ny + 1, nx)).copy()
    w = np.broadcast_to((c * np.arange(nz + 1) * h)[:, None, None], (nz + 1, ny, nx)).copy()
    types = W.all_liquid(nx, ny, nz)
    types[0, 0, 0] = AIR
    g = O.Grid(types, h, 0.1, 0.0)
    rhs = O.divergence(g, (u, v, w))
    expect = np.where(types == LIQ, -h * (a + b + c) * h, 0.0)
    np.testing.assert_allclose(rhs, expect, atol=1e-14)


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_divergence_single_face_signs(oracle_mod, comp):
    """A unit flow through one face leaves the low cell and enters the high cell."""
    O = oracle_mod
    nx, ny, nz, h = 4, 5, 3, 0.5
    g = O.Grid(W.all_liquid(nx, ny, nz), h, 0.1, 0.0)
    u = g.zeros()
    idx = [2, 2, 1]
    u[comp][idx[2], idx[1], idx[0]] = 1.0
    rhs = O.divergence(g, u)
    lo = list(idx)
    lo[comp] -= 1
    expect = np.zeros((nz, ny, nx))
    expect[lo[2], lo[1], lo[0]] = -h * 1.0      # outflow +1 from the low cell
    expect[idx[2], idx[1], idx[0]] = -h * -1.0  # inflow into the high cell
    np.testing.assert_allclose(rhs, expect, atol=0)


def test_poisson_neumann_cosine_eigenvectors(oracle_mod):
    """Closed liquid box: cos(pi m (i+1/2)/n) products are eigenvectors with
    eigenvalue sum_d 4 sin^2(pi m_d / (2 n_d))."""
    O = oracle_mod
    nx, ny, nz = 7, 6, 5
    g = O.Grid(W.all_liquid(nx, ny, nz), 1.0, 0.1, 0.0)
    for m in [(1, 0, 0), (2, 3, 1), (0, 1, 4)]:
        cx = np.cos(np.pi * m[0] * (np.arange(nx) + 0.5) / nx)
        cy = np.cos(np.pi * m[1] * (np.arange(ny) + 0.5) / ny)
        cz = np.cos(np.pi * m[2] * (np.arange(nz) + 0.5) / nz)
        q = cz[:, None, None] * cy[None, :, None] * cx[None, None, :]
        lam = sum(4 * np.sin(np.pi * md / (2 * nd)) ** 2 for md, nd in zip(m, (nx, ny, nz)))
        np.testing.assert_allclose(O.poisson_apply(g, q), lam * q, atol=1e-12)


def test_poisson_air_dirichlet_sine_eigenvectors(oracle_mod):
    """Liquid for 1 <= i <= nx-2 with air at i = 0 and i = nx-1 (p = 0 there):
    sin(pi m i/(nx-1)) x Neumann cosines in y, z are eigenvectors."""
    O = oracle_mod
    nx, ny, nz = 9, 4, 5
    types = W.all_liquid(nx, ny, nz)
    types[:, :, 0] = AIR
    types[:, :, -1] = AIR
    g = O.Grid(types, 1.0, 0.1, 0.0)
    L = nx - 1
    for m in [(1, 0, 0), (3, 1, 2)]:
        sx = np.sin(np.pi * m[0] * np.arange(nx) / L)
        sx[0] = sx[-1] = 0.0
        cy = np.cos(np.pi * m[1] * (np.arange(ny) + 0.5) / ny)
        cz = np.cos(np.pi * m[2] * (np.arange(nz) + 0.5) / nz)
        q = cz[:, None, None] * cy[None, :, None] * sx[None, None, :]
        lam = (4 * np.sin(np.pi * m[0] / (2 * L)) ** 2 + 4 * np.sin(np.pi * m[1] / (2 * ny)) ** 2
               + 4 * np.sin(np.pi * m[2] / (2 * nz)) ** 2)
        np.testing.assert_allclose(O.poisson_apply(g, q), lam * q, atol=1e-12)
        # p = 0 in air: whatever is stored in air cells must not enter
        junk = q + np.where(types == AIR, 1e3, 0.0)
        np.testing.assert_allclose(O.poisson_apply(g, junk), lam * q, atol=1e-12)


def test_projection_kills_gradients_and_keeps_divfree(oracle_mod):
    """P(G phi) = 0 for any phi on the liquid cells, and the discrete Taylor-Green
    mode (exactly divergence-free on the MAC grid) is left unchanged."""
    O = oracle_mod
    types = small_blob()
    nz, ny, nx = types.shape
    h = 1.0 / ny
    g = O.Grid(types, h, 1 / 30, 0.0)
    rng = np.random.default_rng(0)
    phi = np.where(types == LIQ, rng.standard_normal(types.shape), 0.0)
    # discrete gradient on fluid faces, written out from the face geometry
    u = list(g.zeros())
    for c in range(3):
        fc = O.face_class(g, c)
        pad = [(0, 0)] * 3
        pad[2 - c] = (1, 1)
        pp = np.pad(phi, pad)
        hi = [slice(None)] * 3
        lo = [slice(None)] * 3
        hi[2 - c] = slice(1, None)
        lo[2 - c] = slice(None, -1)
        grad = (pp[tuple(hi)] - pp[tuple(lo)]) / h
        u[c] = np.where(fc == 1, grad, 0.0)
    out, q, st = O.project(g, u)
    assert st["status"] == 0
    for c in range(3):
        assert np.abs(out[c]).max() < 1e-9 * max(1.0, np.abs(u[c]).max())
    np.testing.assert_allclose(q, phi, atol=1e-9)

    n = 16
    gtg = O.Grid(W.all_liquid(n, n, 3), 1.0 / n, 1 / 30, 0.0)
    tg = tg_field(n, n, 3, 1.0 / n)
    out, q, st = O.project(gtg, tg)
    for c in range(3):
        np.testing.assert_allclose(out[c], tg[c], atol=1e-12)


def test_projection_divfree_idempotent_symmetric(oracle_mod):
    O = oracle_mod
    types = small_blob(11, 5)
    nz, ny, nx = types.shape
    g = O.Grid(types, 1.0 / ny, 1 / 30, 0.0)
    x = restrict_fluid(O, g, W.random_mac(nx, ny, nz, 1))
    y = restrict_fluid(O, g, W.random_mac(nx, ny, nz, 2))
    px, _, _ = O.project(g, x)
    py, _, _ = O.project(g, y)
    assert np.abs(O.divergence(g, px)).max() < 1e-10
    ppx, _, _ = O.project(g, px)
    for c in range(3):
        np.testing.assert_allclose(ppx[c], px[c], atol=1e-10)
    lhs = sum((px[c] * y[c]).sum() for c in range(3))
    rhs = sum((x[c] * py[c]).sum() for c in range(3))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def dense_poisson(O, g):
    types = g.types
    liq = np.flatnonzero(types.ravel() == LIQ)
    A = np.zeros((liq.size, liq.size))
    for col, t in enumerate(liq):
        e = np.zeros(types.size)
        e[t] = 1.0
        A[:, col] = O.poisson_apply(g, e.reshape(types.shape)).ravel()[liq]
    return A, liq


@pytest.mark.parametrize("precond", [0, 1, 2])
def test_pcg_matches_dense_cholesky(oracle_mod, precond):
    """On a grid of at most 8^3 the solve equals a dense Cholesky solve."""
    O = oracle_mod
    types = small_blob(8, 7)[:, :8, :8].copy()
    g = O.Grid(types, 1.0 / 8, 1 / 30, 0.0, precond=precond)
    A, liq = dense_poisson(O, g)
    np.testing.assert_allclose(A, A.T, atol=0)
    Lc = np.linalg.cholesky(A)  # SPD (air present)
    rng = np.random.default_rng(4)
    b = np.zeros(types.size)
    b[liq] = rng.standard_normal(liq.size)
    x, st = O.pcg(g, b.reshape(types.shape))
    ref = np.linalg.solve(Lc.T, np.linalg.solve(Lc, b[liq]))
    np.testing.assert_allclose(x.ravel()[liq], ref, rtol=1e-10, atol=1e-10)


def test_pcg_singular_box_matches_pinned_cholesky(oracle_mod):
    """Closed liquid box: b is made mean-free, the solution is the mean-free one;
    check against a dense Cholesky with the first cell pinned to zero."""
    O = oracle_mod
    types = W.all_liquid(5, 4, 6)
    g = O.Grid(types, 0.25, 1 / 30, 0.0, precond=2)
    assert O.is_singular(g)
    A, liq = dense_poisson(O, g)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(liq.size)
    bm = b - b.mean()
    Ap = A[1:, 1:]
    xp = np.linalg.solve(Ap, bm[1:])
    ref = np.concatenate([[0.0], xp])
    ref -= ref.mean()
    x, st = O.pcg(g, b.reshape(types.shape))
    np.testing.assert_allclose(x.ravel(), ref, atol=1e-9)


def mic_dense_factor(O, g, prec):
    """Dense L with L_ii = 1/prec_i and L_im = A_im prec_m for lower neighbours m."""
    A, liq = dense_poisson(O, g)
    pos = {t: n for n, t in enumerate(liq)}
    Lm = np.zeros_like(A)
    pr = prec.ravel()
    for a, t in enumerate(liq):
        Lm[a, a] = 1.0 / pr[t]
        for b, t2 in enumerate(liq):
            if t2 < t and A[a, b] != 0.0:
                Lm[a, b] = A[a, b] * pr[t2]
    return A, Lm


def test_ic0_matches_matrix_on_pattern(oracle_mod):
    """tau = 0 is IC(0): L L^T equals A on A's sparsity pattern."""
    O = oracle_mod
    types = small_blob(7, 2)
    g = O.Grid(types, 1.0, 0.1, 0.0)
    prec = O.mic0_factor(g, tau=0.0, sigma=0.0)
    A, Lm = mic_dense_factor(O, g, prec)
    LLt = Lm @ Lm.T
    pattern = A != 0.0
    np.testing.assert_allclose(LLt[pattern], A[pattern], atol=1e-12)
    assert np.abs(LLt[~pattern]).max() > 1e-3  # fill was dropped


def test_mic_full_modification_preserves_row_sums(oracle_mod):
    """tau = 1 (full modification, no safety): L L^T has A's row sums and A's
    off-diagonal entries on the pattern."""
    O = oracle_mod
    types = small_blob(7, 2)
    g = O.Grid(types, 1.0, 0.1, 0.0)
    prec = O.mic0_factor(g, tau=1.0, sigma=0.0)
    A, Lm = mic_dense_factor(O, g, prec)
    LLt = Lm @ Lm.T
    np.testing.assert_allclose(LLt.sum(axis=1), A.sum(axis=1), atol=1e-11)
    off = (A != 0.0) & ~np.eye(A.shape[0], dtype=bool)
    np.testing.assert_allclose(LLt[off], A[off], atol=1e-12)


def test_mic0_on_a_line_is_exact(oracle_mod):
    """A one-cell-thick line of liquid has no fill: MIC(0) is the exact Cholesky
    factor for any tau, so PCG converges in one iteration."""
    O = oracle_mod
    types = np.full((3, 3, 12), SOL, dtype=np.uint8)
    types[1, 1, :] = LIQ
    types[1, 1, -1] = AIR
    g = O.Grid(types, 1.0, 0.1, 0.0, precond=2, mic_tau=0.97, mic_sigma=0.25)
    rng = np.random.default_rng(1)
    b = np.where(types == LIQ, rng.standard_normal(types.shape), 0.0)
    x, st = O.pcg(g, b)
    assert st["iters"] == 1 and st["true_relres"] < 1e-13
    prec = O.mic0_factor(g)
    A, Lm = mic_dense_factor(O, g, prec)
    np.testing.assert_allclose(Lm @ Lm.T, A, atol=1e-12)


def test_viscosity_taylor_green_exact_decay(oracle_mod):
    """The Taylor-Green mode is an exact eigenvector of the face Laplacian
    (Dirichlet normal faces, mirror tangential walls) with k^2 = 8 sin^2(pi h/2)/h^2,
    and exactly divergence-free: viscosity then projection scales it by
    1/(1 + nu dt k^2) per step."""
    O = oracle_mod
    n = 16
    h = 1.0 / n
    nu, dt = 0.05, 1 / 30
    g = O.Grid(W.all_liquid(n, n, 4), h, dt, nu)
    u = tg_field(n, n, 4, h)
    k2 = 8 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    fac = 1.0 / (1.0 + nu * dt * k2)
    cur = u
    for step in range(3):
        cur, st = O.visc_solve(g, cur)
        cur, q, st2 = O.project(g, cur)
    for c in range(3):
        np.testing.assert_allclose(cur[c], fac ** 3 * u[c], atol=1e-11)


def test_viscosity_air_is_mirror(oracle_mod):
    """Liquid layer j < J under air: u = sin(pi i/nx) cos(pi (j+1/2)/J) on the fluid
    u-faces is an eigenvector when air neighbours are zero-flux (mirror)."""
    O = oracle_mod
    nx, ny, nz, J = 10, 9, 3, 5
    h = 0.1
    types = W.all_liquid(nx, ny, nz)
    types[:, J:, :] = AIR
    nu, dt = 0.3, 0.02
    g = O.Grid(types, h, dt, nu)
    u = np.zeros((nz, ny, nx + 1))
    prof = np.sin(np.pi * np.arange(nx + 1) / nx)[None, :] * \
        np.cos(np.pi * (np.arange(J) + 0.5) / J)[:, None]
    u[:, :J, :] = prof[None]
    zero = g.zeros()
    x = (u, zero[1], zero[2])
    y = O.visc_apply(g, x)
    lam = (4 * np.sin(np.pi / (2 * nx)) ** 2 + 4 * np.sin(np.pi / (2 * J)) ** 2) / h ** 2
    fluid = O.face_class(g, 0) == 1
    np.testing.assert_allclose(y[0][fluid], ((1 + nu * dt * lam) * u)[fluid], atol=1e-12)


def test_viscosity_solve_is_symmetric_and_dirichlet_enters(oracle_mod):
    O = oracle_mod
    types = small_blob(9, 1)
    nz, ny, nx = types.shape
    bc = tuple(0.3 * a for a in W.random_mac(nx, ny, nz, 9))
    g = O.Grid(types, 1.0 / ny, 1 / 30, 0.2, bc=bc)
    g0 = O.Grid(types, 1.0 / ny, 1 / 30, 0.2)
    x = restrict_fluid(O, g0, W.random_mac(nx, ny, nz, 1))
    y = restrict_fluid(O, g0, W.random_mac(nx, ny, nz, 2))
    ax, _ = O.visc_solve(g0, x)
    ay, _ = O.visc_solve(g0, y)
    lhs = sum((ax[c] * y[c]).sum() for c in range(3))
    rhs = sum((x[c] * ay[c]).sum() for c in range(3))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    # with prescribed values: A u = rhs + Dirichlet; check through the operator
    out, _ = O.visc_solve(g, x)
    for c in range(3):
        fc = O.face_class(g, c)
        assert np.all(out[c][fc == 2] == bc[c][fc == 2])
        assert np.all(out[c][fc == 0] == 0.0)
    # the Dirichlet part is linear in bc: out(bc) - out(0) = A^{-1} D(bc) must be
    # nonzero near walls and vanish when bc = 0
    diff = sum(np.abs(out[c] - ax[c]).max() for c in range(3))
    assert diff > 1e-6


def test_mic0_safety_branch_by_hand(oracle_mod):
    """The safety branch of MIC(0) (a pivot e below sigma * diag is replaced by
    diag, Bridson's recipe cited for the projection), on the closed 2 x 2 x 2 box
    of liquid, where every cell has diag 3 and the pivots follow by hand in
    lexicographic order (x fastest), with A's off-diagonals -1:
      e0 = 3;  e1 = e2 = e4 = 3 - 1/3 - tau * 2/3 = 2.02 (tau = 0.97);
      e3 = e5 = e6 = 3 - 2 (1 + tau) / 2.02 = 3 - 3.94/2.02 (two lower neighbours,
           each with one further coupling);
      e7 = 3 - 3 / e3 (three lower neighbours, no further couplings) = 0.14150...
    With sigma = 0.25, e7 < 0.75 is replaced by diag = 3. With sigma = 0.36,
    e3, e5, e6 (1.0495 < 1.08) are replaced by 3 first, which makes
    e7 = 3 - 3/3 = 2 >= 1.08, kept."""
    O = oracle_mod
    g = O.Grid(np.full((2, 2, 2), LIQ, dtype=np.uint8), 1.0, 0.1, 0.0)
    tau = 0.97
    e12 = 3.0 - 1.0 / 3.0 - tau * 2.0 / 3.0
    e3 = 3.0 - 2.0 * (1.0 + tau) / e12
    # order of prec.ravel(): (k, j, i) C order = lexicographic with x fastest
    expect = {
        0.0: [3.0, e12, e12, e3, e12, e3, e3, 3.0 - 3.0 / e3],
        0.25: [3.0, e12, e12, e3, e12, e3, e3, 3.0],
        0.36: [3.0, e12, e12, 3.0, e12, 3.0, 3.0, 2.0],
    }
    assert abs(e12 - 2.02) < 1e-15 and abs(3.0 - 3.0 / e3 - 0.14150943396) < 1e-10
    for sigma, e in expect.items():
        prec = O.mic0_factor(g, tau=tau, sigma=sigma).ravel()
        np.testing.assert_allclose(prec, 1.0 / np.sqrt(e), rtol=1e-14, atol=0)
