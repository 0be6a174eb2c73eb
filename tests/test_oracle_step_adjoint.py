"""Pins of the oracle's advection, step, loss and reverse pass: exactness on
linear fields, agreement with scipy's independent trilinear interpolator,
closed-form loss values, and central finite differences of the forward."""
import numpy as np
import pytest

from paper_2503_00868_gb300 import workloads as W

AIR, LIQ, SOL = 0, 1, 2


def face_positions(c, nx, ny, nz, h):
    """World coordinates of the faces of component c (each (nz', ny', nx'))."""
    d = [nx, ny, nz]
    d[c] += 1
    off = [0.5, 0.5, 0.5]
    off[c] = 0.0
    z, y, x = np.meshgrid((np.arange(d[2]) + off[2]) * h, (np.arange(d[1]) + off[1]) * h,
                          (np.arange(d[0]) + off[0]) * h, indexing="ij")
    return x, y, z


def test_advection_exact_for_linear_fields(oracle_mod):
    """A linear velocity field is reproduced exactly by the 4-face averages and by
    trilinear interpolation, so an unclamped back-trace lands on the closed form
    u_c(X - dt u(X)) + dt g_c."""
    O = oracle_mod
    nx, ny, nz, h, dt = 9, 8, 7, 0.1, 0.05
    a = np.array([0.4, -0.3, 0.2])
    B = np.array([[0.5, -0.2, 0.3], [0.1, 0.4, -0.6], [-0.3, 0.2, 0.1]])
    gvec = (0.7, -9.81, 0.25)
    u = []
    for c in range(3):
        x, y, z = face_positions(c, nx, ny, nz, h)
        u.append(a[c] + B[c, 0] * x + B[c, 1] * y + B[c, 2] * z)
    types = W.all_liquid(nx, ny, nz)
    types[5, 6, 7] = AIR
    g = O.Grid(types, h, dt, 0.0, g=gvec)
    ua = O.advect(g, u)
    checked = 0
    for c in range(3):
        x, y, z = face_positions(c, nx, ny, nz, h)
        X = np.stack([x, y, z])
        vel = np.stack([a[d] + B[d, 0] * x + B[d, 1] * y + B[d, 2] * z for d in range(3)])
        Xb = X - dt * vel
        expect = a[c] + sum(B[c, d] * Xb[d] for d in range(3)) + dt * gvec[c]
        # index coordinates of the trace on this component's grid
        dims = [nx, ny, nz]
        dims[c] += 1
        off = [0.5, 0.5, 0.5]
        off[c] = 0.0
        s = [Xb[d] / h - off[d] for d in range(3)]
        inside = np.ones_like(x, dtype=bool)
        for d in range(3):
            inside &= (s[d] >= 0) & (s[d] <= dims[d] - 1)
        fc = O.face_class(g, c)
        sel = inside & (fc == 1)
        checked += sel.sum()
        np.testing.assert_allclose(ua[c][sel], expect[sel], atol=1e-12)
        assert np.all(ua[c][fc == 2] == 0.0)
        assert np.all(ua[c][fc == 0] == 0.0)
    assert checked > 500


def test_advection_matches_scipy_trilinear(oracle_mod):
    """Random fields: every fluid face equals scipy's RegularGridInterpolator at the
    back-traced, clamped index position (own component; others 4-face means)."""
    from scipy.interpolate import RegularGridInterpolator
    O = oracle_mod
    types, _ = W.ellipsoid_blob(10, 9, 11, 4)
    nz, ny, nx = types.shape
    h, dt = 1.0 / ny, 0.03
    u = W.random_mac(nx, ny, nz, 7, scale=2.0)
    g = O.Grid(types, h, dt, 0.0)
    ua = O.advect(g, u)
    U, V, Wc = u
    for c in range(3):
        arr = u[c]
        dims = arr.shape[::-1]
        interp = RegularGridInterpolator((np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0])),
                                         arr, method="linear")
        fc = O.face_class(g, c)
        ks, js, is_ = np.nonzero(fc == 1)
        vel = np.zeros((3, ks.size))
        vel[c] = arr[ks, js, is_]
        for e in range(3):
            if e == c:
                continue
            lo = [is_.copy(), js.copy(), ks.copy()]
            lo[c] -= 1
            hi_l = [lo[0].copy(), lo[1].copy(), lo[2].copy()]
            hi_l[e] += 1
            hi_r = [is_.copy(), js.copy(), ks.copy()]
            hi_r[e] += 1
            ue = u[e]
            vel[e] = 0.25 * (ue[lo[2], lo[1], lo[0]] + ue[hi_l[2], hi_l[1], hi_l[0]] +
                             ue[ks, js, is_] + ue[hi_r[2], hi_r[1], hi_r[0]])
        idx = np.stack([is_, js, ks]).astype(float)
        s = idx - dt / h * vel
        for d in range(3):
            s[d] = np.clip(s[d], 0, dims[d] - 1)
        ref = interp(np.stack([s[2], s[1], s[0]], axis=1))
        np.testing.assert_allclose(ua[c][ks, js, is_], ref, atol=1e-12)


def _rand_dir(shape_list, seed):
    rng = np.random.default_rng(seed)
    return tuple(rng.standard_normal(s) for s in shape_list)


def _inner(a, b):
    return sum(float((x * y).sum()) for x, y in zip(a, b))


def test_advection_adjoint_against_central_differences(oracle_mod):
    O = oracle_mod
    types, _ = W.ellipsoid_blob(9, 8, 10, 2)
    nz, ny, nx = types.shape
    g = O.Grid(types, 1.0 / ny, 0.04, 0.0, g=(0.0, -9.81, 0.0))
    u = W.random_mac(nx, ny, nz, 3, scale=1.5)
    d = _rand_dir(g.shapes(), 11)
    ybar = _rand_dir(g.shapes(), 12)
    adj = _inner(d, O.advect_adjoint(g, u, ybar))
    fds = []
    for eps in (1e-5, 1e-6):
        up = tuple(a + eps * b for a, b in zip(u, d))
        um = tuple(a - eps * b for a, b in zip(u, d))
        fp, fm = O.advect(g, up), O.advect(g, um)
        fds.append(_inner(ybar, tuple((p - m) / (2 * eps) for p, m in zip(fp, fm))))
    assert abs(fds[0] - fds[1]) <= 1e-6 * abs(fds[0])  # no kink crossed
    assert abs(adj - fds[1]) <= 1e-7 * abs(adj)


def test_loss_closed_forms(oracle_mod):
    O = oracle_mod
    types, _ = W.ellipsoid_blob(10, 10, 10, 1)
    g = O.Grid(types, 0.1, 0.03, 0.0)
    t = W.random_mac(10, 10, 10, 5)
    loss, _ = O.loss_grad(g, t, t, alpha=1.0, beta=1.0)
    assert abs(loss) < 1e-15
    # constant offset c on every face: L2 term = beta c^2 / 2
    c0 = 0.37
    u = tuple(a + c0 for a in t)
    loss, _ = O.loss_grad(g, u, t, alpha=0.0, beta=2.0)
    assert abs(loss - 2.0 * c0 ** 2 / 2) < 1e-14
    # parallel fields: cosine term vanishes; antiparallel: 2 alpha
    u2 = tuple(3.0 * a for a in t)
    loss, _ = O.loss_grad(g, u2, t, alpha=1.5, beta=0.0)
    assert abs(loss) < 1e-12
    loss, _ = O.loss_grad(g, tuple(-a for a in t), t, alpha=1.5, beta=0.0)
    assert abs(loss - 3.0) < 1e-12
    # surface band: liquid cells with an air neighbour, none of them deep inside
    band = O.band_cells(g, 0)
    assert band.sum() > 0 and np.all(types[band == 1] == LIQ)
    assert O.band_cells(g, 1).sum() == (types == LIQ).sum()


@pytest.mark.parametrize("kind", [0, 1])
def test_loss_gradient_against_central_differences(oracle_mod, kind):
    O = oracle_mod
    types, _ = W.ellipsoid_blob(8, 9, 10, 6)
    nz, ny, nx = types.shape
    g = O.Grid(types, 0.1, 0.03, 0.0)
    u = W.random_mac(nx, ny, nz, 1)
    t = W.random_mac(nx, ny, nz, 2)
    d = _rand_dir(g.shapes(), 3)
    _, grad = O.loss_grad(g, u, t, kind=kind, alpha=0.7, beta=1.3)
    eps = 1e-6
    lp, _ = O.loss_grad(g, tuple(a + eps * b for a, b in zip(u, d)), t, kind=kind, alpha=0.7, beta=1.3)
    lm, _ = O.loss_grad(g, tuple(a - eps * b for a, b in zip(u, d)), t, kind=kind, alpha=0.7, beta=1.3)
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - _inner(grad, d)) <= 1e-7 * abs(fd)


def test_step_invariants(oracle_mod):
    """After a step: zero divergence on liquid cells, prescribed values on fixed
    faces, zero on air faces; the mask is untouched."""
    O = oracle_mod
    types, inflow, _ = W.river_with_blob(12, 8, 10, 3)
    nz, ny, nx = types.shape
    bc = [np.zeros(s) for s in O.face_shapes(nx, ny, nz)]
    bc[0] = np.where(inflow == 1, 0.5, 0.0)
    types0 = types.copy()
    g = O.Grid(types, 1.0 / ny, 1 / 30, 0.01, g=(0.0, -9.81, 0.0), bc=bc)
    u = W.blurred_noise_mac(nx, ny, nz, 1)
    out, uv, st = O.step(g, u, save_visc=True)
    assert st["pressure"]["status"] == 0 and st["visc"]["status"] == 0
    assert np.abs(O.divergence(g, out)).max() < 1e-10
    for c in range(3):
        fc = O.face_class(g, c)
        assert np.all(out[c][fc == 2] == bc[c][fc == 2])
        assert np.all(out[c][fc == 0] == 0.0)
        assert np.all(uv[c][fc == 2] == bc[c][fc == 2])
    assert np.abs(out[0][:, :, 0]).max() == 0.5
    assert np.array_equal(types, types0)


def _rollout_loss(O, g, u0, target, nsteps):
    u = u0
    for _ in range(nsteps):
        u, _ = O.step(g, u)
    loss, grad = O.loss_grad(g, u, target)
    return loss, grad


def test_adjoint_step_against_central_differences(oracle_mod):
    """Two steps then the band loss: the reverse pass matches central differences
    along a random initial-velocity direction and along log(nu)."""
    O = oracle_mod
    types, _ = W.ellipsoid_blob(9, 8, 9, 5)
    nz, ny, nx = types.shape
    nu = 0.02
    mk = lambda v: O.Grid(types, 1.0 / ny, 1 / 30, v, g=(0.0, -9.81, 0.0))
    g = mk(nu)
    u0 = W.blurred_noise_mac(nx, ny, nz, 2, scale=20.0)
    target = W.blurred_noise_mac(nx, ny, nz, 102, scale=20.0)
    nsteps = 2
    # forward with saved states
    states = [u0]
    for _ in range(nsteps):
        states.append(O.step(g, states[-1])[0])
    loss, gbar = O.loss_grad(g, states[-1], target)
    gnu = 0.0
    for n in range(nsteps - 1, -1, -1):
        gbar, dnu = O.adjoint_step(g, states[n], gbar)
        gnu += dnu
    d = _rand_dir(g.shapes(), 8)
    eps = 1e-5
    lp, _ = _rollout_loss(O, g, tuple(a + eps * b for a, b in zip(u0, d)), target, nsteps)
    lm, _ = _rollout_loss(O, g, tuple(a - eps * b for a, b in zip(u0, d)), target, nsteps)
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - _inner(gbar, d)) <= 1e-6 * abs(fd)
    th = 1e-4
    lp, _ = _rollout_loss(O, mk(nu * np.exp(th)), u0, target, nsteps)
    lm, _ = _rollout_loss(O, mk(nu * np.exp(-th)), u0, target, nsteps)
    fd_theta = (lp - lm) / (2 * th)
    assert abs(fd_theta - nu * gnu) <= 1e-5 * abs(fd_theta)
