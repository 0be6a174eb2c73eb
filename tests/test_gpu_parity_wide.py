"""GPU parity on grids whose rows span several 128-wide tiles, on the
benchmark's own path, against the FP64 oracle.

At 133 cells across, a row of the library layout (pitch 136) covers two
128 x 8 tiles, the operator apply's TMA boxes straddle the tile seam and the
multigrid hierarchy has odd sizes at every level. The liquid spans the seam
(a liquid layer on the floor under a blob, with an inflow patch), so every
solver (Jacobi, MIC(0), the multigrid V-cycle) works across it.

Every field is compared twice: a global relative L2 error (velocity 1e-5,
gradients 1e-4, the tolerances of the fluid-step parity tests) and a per-face
bound, max |gpu - oracle| <= TOL * max |oracle|, so that an error confined to a
few hundred faces (a tile edge) cannot hide in the global norm. For gradients
the per-face bound leaves out the neighbourhoods (2 cells) of faces whose
back-traced sample point lies within 3e-5 of a grid line in some axis, a few
FP32 roundings of the index-space coordinate: trilinear interpolation has a kink
there, the discrete adjoint jumps, and either one-sided value is correct, so
the GPU (FP32 sample) and the oracle (FP64 sample) may take different sides.
The faces left out are fewer than one in ten.

The rollout test runs the benchmark's configuration: multigrid in both solves,
warm-started pressure solves, tolerance 1e-6, a checkpointed rollout and its
reverse pass."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_00868_gb300 import fluidstep as F
from paper_2503_00868_gb300 import workloads as W
from paper_2503_00868_gb300.rollout import rollout_loss

pytestmark = pytest.mark.gpu

NX, NY, NZ = 133, 40, 36
TOL_U, MAX_U = 1e-5, 2e-5
TOL_G, MAX_G = 1e-4, 2e-4
PRECONDS = {"jacobi": F.FS_PRECOND_JACOBI, "mic0": F.FS_PRECOND_MIC0, "mg": F.FS_PRECOND_MG}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def rel(a, b):
    num = sum(float(((np.asarray(x, np.float64) - y) ** 2).sum()) for x, y in zip(a, b))
    den = sum(float((np.asarray(y) ** 2).sum()) for y in b)
    return (num / max(den, 1e-300)) ** 0.5


def maxrel(a, b):
    """max over all faces of |a - b|, over max |b|"""
    num = max(float(np.abs(np.asarray(x, np.float64) - y).max()) for x, y in zip(a, b))
    den = max(float(np.abs(y).max()) for y in b)
    return num / max(den, 1e-300)


def check(a, b, tol, tol_max, what, skip=None):
    """rel-L2 over all faces; the per-face max over the faces not in `skip`"""
    e2 = rel(a, b)
    if skip is None:
        em = maxrel(a, b)
    else:
        assert sum(int(k.sum()) for k in skip) < 0.1 * sum(k.size for k in skip)
        num = max(float(np.abs(np.asarray(x, np.float64) - y)[~k].max()) for x, y, k in zip(a, b, skip))
        em = num / max(float(np.abs(y).max()) for y in b)
    assert e2 < tol and em < tol_max, f"{what}: rel-L2 {e2:.3e} (bound {tol}), max {em:.3e} (bound {tol_max})"


def scene(kind):
    """(types, prescribed face values or None, gravity)"""
    if kind == "river":
        types, inflow, _ = W.river_with_blob(NX, NY, NZ, 2)
        bc = [np.zeros(s) for s in O.face_shapes(NX, NY, NZ)]
        bc[0] = np.where(inflow == 1, 0.5, 0.0)
        return types, bc, (0.0, -9.81, 0.0)
    if kind == "spheres":      # small spheres spread over the whole width
        types, _ = W.sphere_union(NX, NY, NZ, 4, count=24, occ_range=(0.05, 0.5))
        return types, None, (0.0, 0.0, 0.0)
    if kind == "closed_box":   # all liquid: the singular operator, 133 x 20 x 18
        return W.all_liquid(NX, 20, 18), None, (0.0, 0.0, 0.0)
    raise KeyError(kind)


def grids(types, bc, g, precond, nu=0.01, tol=1e-7, **kw):
    nz, ny, nx = types.shape
    dx = 1.0 / ny
    og = O.Grid(types, dx, 1 / 30, nu, g=g, bc=bc)
    gg = F.Grid(nx, ny, nz, dx=dx, dt=1 / 30, nu=nu, g=g, precond=PRECONDS[precond], tol_p=tol, tol_v=tol,
                maxit_p=20000, maxit_v=4000, **kw)
    gg.set_mask(types, gg.pack(bc) if bc is not None else None)
    return og, gg


def test_rows_span_several_tiles():
    types, _, _ = scene("river")
    gg = F.Grid(NX, NY, NZ, dx=1.0 / NY)
    assert gg.pitch == 136 and gg.pitch > 128
    liq_x = np.nonzero((types == 1).any(axis=(0, 1)))[0]
    assert liq_x.min() == 0 and liq_x.max() == NX - 1   # liquid on both sides of the x = 128 seam


@pytest.mark.parametrize("precond", list(PRECONDS))
@pytest.mark.parametrize("kind", ["river", "spheres", "closed_box"])
def test_wide_projection(kind, precond):
    types, bc, g = scene(kind)
    og, gg = grids(types, bc, g, precond)
    nz, ny, nx = types.shape
    u0 = W.random_mac(nx, ny, nz, 31)
    if bc is not None:
        for c in range(3):
            fc = O.face_class(og, c)
            u0[c][fc == 2] = bc[c][fc == 2]
    ou, oq, _ = O.project(og, u0)
    u, q = gg.pack(u0), gg.empty_cell()
    rc, st = gg.project(u, q)
    assert rc == F.FS_OK and st["true_relres_p"] < 1e-6, st
    check(gg.unpack(u), ou, TOL_U, MAX_U, "velocity")
    check([gg.unpack_cell(q)], [oq], 1e-4, 2e-4, "pressure")


@pytest.mark.parametrize("precond", list(PRECONDS))
def test_wide_step_and_adjoint(precond):
    types, bc, g = scene("river")
    og, gg = grids(types, bc, g, precond, nu=0.02)
    nz, ny, nx = types.shape
    u0 = W.blurred_noise_mac(nx, ny, nz, 1)
    oout, ouv, _ = O.step(og, u0, save_visc=True)
    u, out, uv = gg.pack(u0), gg.zeros(), gg.zeros()
    rc, st = gg.step(u, out, uv)
    assert rc == F.FS_OK, st
    check(gg.unpack(uv), ouv, TOL_U, MAX_U, "after viscosity")
    check(gg.unpack(out), oout, TOL_U, MAX_U, "step output")
    for c, arr in enumerate(gg.unpack(out)):     # fixed faces exact, air-air faces zero
        fc = O.face_class(og, c)
        assert np.array_equal(arr[fc == 2], bc[c][fc == 2].astype(np.float32).astype(np.float64))
        assert np.all(arr[fc == 0] == 0.0)
    gout = W.blurred_noise_mac(nx, ny, nz, 7)
    ogin, ognu = O.adjoint_step(og, u0, gout)
    gin = gg.zeros()
    rc, gnu, st = gg.adjoint_step(u, gg.pack(gout), gin, uv)
    assert rc == F.FS_OK, st
    check(gg.unpack(gin), ogin, TOL_G, MAX_G, "adjoint", skip=O.kink_faces(og, u0))
    assert abs(gnu - ognu) <= TOL_G * abs(ognu), (gnu, ognu)


def oracle_rollout(og, u0, targets, nsteps):
    """(loss, dL/du0, dL/dnu, the states of the forward pass)"""
    states = [u0]
    for _ in range(nsteps):
        states.append(O.step(og, states[-1])[0])
    loss = sum(O.loss_grad(og, states[n], targets[n])[0] for n in sorted(targets))
    g = og.zeros()
    gnu = 0.0
    for n in range(nsteps, 0, -1):
        if n in targets:
            g = tuple(a + b for a, b in zip(g, O.loss_grad(og, states[n], targets[n])[1]))
        g, dnu = O.adjoint_step(og, states[n - 1], g)
        gnu += dnu
    return loss, g, gnu, states


def test_wide_rollout_benchmark_configuration():
    """Three frames with the multigrid preconditioner in both solves, warm-started
    pressure solves and tolerance 1e-6 (the benchmark's settings), checkpoint
    every 2 frames, losses at frames 1 and 3: loss, dL/du0 and dL/dnu against
    the oracle's forward and reverse pass."""
    types, bc, g = scene("river")
    nu = 0.01
    og, gg = grids(types, bc, g, "mg", nu=nu, tol=1e-6, warm_start=1, check_every=16)
    nz, ny, nx = types.shape
    u0 = W.blurred_noise_mac(nx, ny, nz, 3)
    for c in range(3):
        fc = O.face_class(og, c)
        u0[c][fc == 2] = bc[c][fc == 2]
    tg = {1: W.blurred_noise_mac(nx, ny, nz, 101), 3: W.blurred_noise_mac(nx, ny, nz, 103)}
    oloss, og_u0, ognu, states = oracle_rollout(og, u0, tg, 3)
    kinks = [O.kink_faces(og, st) for st in states[:3]]
    skip = tuple(np.logical_or.reduce([k[c] for k in kinks]) for c in range(3))

    stats = []
    leaves = [t.requires_grad_(True) for t in gg.pack(u0)]
    nu_t = torch.tensor(nu, requires_grad=True)
    loss = rollout_loss(gg, F.Mac(*leaves), nu_t, 3, {n: gg.pack(t) for n, t in tg.items()},
                        checkpoint_every=2, stats=stats)
    loss.backward()
    assert all(s[2]["status"] == F.FS_OK for s in stats), stats
    assert abs(float(loss.detach()) - oloss) <= 1e-5 * abs(oloss), (float(loss.detach()), oloss)
    gu = gg.unpack(F.Mac(*(t.grad for t in leaves)))
    # fixed faces are inputs the step overwrites: their gradient is zero on both sides
    check(gu, og_u0, TOL_G, MAX_G, "dL/du0", skip=skip)
    assert abs(float(nu_t.grad) - ognu) <= TOL_G * abs(ognu), (float(nu_t.grad), ognu)


# ---- the benchmark's full size: properties that hold at any size -------------

def full_grid(n=256):
    types, _ = W.ellipsoid_blob(n, n, n, 0)
    gg = F.Grid(n, n, n, dx=1.0 / n, dt=1 / 30, nu=0.01, precond=F.FS_PRECOND_MG, tol_p=1e-6, tol_v=1e-6,
                maxit_p=20000, maxit_v=4000, check_every=16, warm_start=1)
    gg.set_mask(types)
    return types, gg


def torch_div(m: F.Mac, nx, ny, nz):
    """Cell divergence of a field in the library layout, computed with torch ops
    (independent of the library's divergence kernel), float64."""
    u = m.u[:nz, :ny, :nx + 1].double()
    v = m.v[:nz, :ny + 1, :nx].double()
    w = m.w[:nz + 1, :ny, :nx].double()
    return (u[:, :, 1:] - u[:, :, :-1]) + (v[:, 1:, :] - v[:, :-1, :]) + (w[1:] - w[:-1])


def test_full_size_step_is_divergence_free_and_keeps_the_mask():
    """One step of the benchmark's 256^3 scene in its configuration: the output is
    divergence-free on the liquid to the solve tolerance, air-air faces are zero,
    and a second step (warm-started) does the same."""
    n = 256
    types, gg = full_grid(n)
    u0 = W.blurred_noise_mac(n, n, n, 0)
    a, b = gg.pack(u0), gg.zeros()
    liq = torch.as_tensor(types == 1, device="cuda")
    div0 = torch_div(a, n, n, n)[liq].norm()
    for _ in range(2):
        rc, st = gg.step(a, b)
        # the FP64 residual of the pressure the velocity was corrected with
        assert rc == F.FS_OK and st["true_relres_p"] <= 1e-6, st
        # the divergence left in the FP32 output: the solve's residual plus the
        # rounding of the output faces
        d = torch_div(b, n, n, n)[liq].norm()
        assert float(d / div0) < 2e-6, float(d / div0)
        # no liquid cell next to a face: the face holds 0
        nb = torch.zeros((n, n, n + 1), dtype=torch.bool, device="cuda")
        nb[:, :, 1:] |= liq
        nb[:, :, :-1] |= liq
        assert float(b.u[:n, :n, :n + 1][~nb].abs().max()) == 0.0
        a, b = b, a


def test_full_size_projection_is_a_symmetric_projector():
    """At 256^3 with the multigrid preconditioner: <P x, y> = <x, P y> and
    P(P x) = P x, to the solve tolerance (the adjoint reuses P as its own
    transpose, so this is what the reverse pass rests on at full size)."""
    n = 256
    types, gg = full_grid(n)
    gg.set_params(tol_p=1e-7)
    x, y = gg.pack(W.random_mac(n, n, n, 1)), gg.pack(W.random_mac(n, n, n, 2))
    x0 = F.Mac(*(t.clone() for t in x))
    y0 = F.Mac(*(t.clone() for t in y))
    for m in (x, y):
        rc, st = gg.project(m)
        assert rc == F.FS_OK, st

    def dot(a, b):
        return sum(float((s.double() * t.double()).sum()) for s, t in zip(a, b))

    def nrm(a):
        return dot(a, a) ** 0.5

    lhs, rhs = dot(x, y0), dot(x0, y)
    assert abs(lhs - rhs) <= 1e-5 * nrm(x0) * nrm(y0), (lhs, rhs)
    px = F.Mac(*(t.clone() for t in x))
    rc, st = gg.project(px)
    assert rc == F.FS_OK
    num = sum(float((s.double() - t.double()).pow(2).sum()) for s, t in zip(px, x)) ** 0.5
    assert num <= 1e-5 * nrm(x), num / nrm(x)


def test_full_size_gradient_along_a_direction():
    """The benchmark's rollout (256^3, 2 frames, checkpoint 1, multigrid, warm
    start, tolerance 1e-6): <dL/du0, d> against the central difference of the
    loss along a smooth direction d. The forward solves are only converged to
    1e-6, so agreement to 1e-3 is the bar."""
    n = 256
    types, gg = full_grid(n)
    u0 = gg.pack(W.blurred_noise_mac(n, n, n, 0))
    tgt = {2: gg.pack(W.blurred_noise_mac(n, n, n, 100))}
    d = gg.pack(W.blurred_noise_mac(n, n, n, 55))
    nu = torch.tensor(0.01, requires_grad=True)
    leaves = [t.clone().requires_grad_(True) for t in u0]
    loss = rollout_loss(gg, F.Mac(*leaves), nu, 2, tgt, checkpoint_every=1)
    loss.backward()
    gd = sum(float((t.grad.double() * s.double()).sum()) for t, s in zip(leaves, d))
    h = 1e-2
    lp = float(rollout_loss(gg, F.Mac(*(a + h * s for a, s in zip(u0, d))), torch.tensor(0.01), 2, tgt, 1))
    lm = float(rollout_loss(gg, F.Mac(*(a - h * s for a, s in zip(u0, d))), torch.tensor(0.01), 2, tgt, 1))
    fd = (lp - lm) / (2 * h)
    assert abs(fd - gd) <= 1e-3 * abs(gd), (fd, gd)
