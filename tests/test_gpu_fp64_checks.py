"""GPU: precision of the pressure solve's reductions, pinned against FP64
recomputations of the same device vectors.

The CG scalars of each iteration (r.z, p.Ap, r.r) are sums of FP32 products
carried in compensated FP32 pairs; the final convergence check |b - A q| / |b|
is evaluated in FP64. Both are checked here on right-hand sides whose entries
span eight decades (a divergent field scaled face by face by 10^U(-4, 4)):

* the reported true relative residual equals |b - A q|_2 / |b|_2 recomputed in
  FP64 from the solver's own b (fs_divergence) and q, the pair of FP32 terms the
  solver keeps it in after a refinement (fs_pressure_pair, summed in FP64; the
  second term is zero without one), with A the oracle's FP64 operator, to 1e-10
  relative; q_out is that pair rounded to FP32;
* the first iteration's step length alpha = r.z / p.Ap (Jacobi: z = p =
  D^-1 b) read back from q = alpha p agrees with alpha recomputed in FP64 to
  the FP32 resolution of q (2e-6 relative)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_00868_gb300 import fluidstep as F
from paper_2503_00868_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def wide_range_field(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    u = W.random_mac(nx, ny, nz, seed)
    return tuple(a * 10.0 ** rng.uniform(-4.0, 4.0, a.shape) for a in u)


@pytest.mark.parametrize("precond", [F.FS_PRECOND_JACOBI, F.FS_PRECOND_MIC0, F.FS_PRECOND_MG])
@pytest.mark.parametrize("field", ["wide_range", "plain"])
def test_true_residual_matches_fp64_recomputation(precond, field):
    n = 48
    types, _ = W.sphere_union(n, n, n, 6)
    og = O.Grid(types, 1.0 / n, 1 / 30, 0.01)
    gg = F.Grid(n, n, n, dx=1.0 / n, tol_p=1e-5, maxit_p=5000, precond=precond)
    gg.set_mask(types)
    u0 = wide_range_field(n, n, n, 3) if field == "wide_range" else W.random_mac(n, n, n, 3)
    u = gg.pack(u0)
    b = gg.empty_cell()
    F.fs_divergence(gg.ctx, u, b)
    q = gg.empty_cell()
    rc, st = gg.project(u, q)
    assert rc == F.FS_OK, st
    qh, ql = gg.empty_cell(), gg.empty_cell()
    F.fs_pressure_pair(gg.ctx, qh, ql)
    b64 = gg.unpack_cell(b)
    q64 = gg.unpack_cell(qh).astype(np.float64) + gg.unpack_cell(ql).astype(np.float64)
    assert np.array_equal(gg.unpack_cell(q), (gg.unpack_cell(qh) + gg.unpack_cell(ql)).astype(np.float32))
    liq = types == 1
    e = np.where(liq, b64 - O.poisson_apply(og, q64), 0.0)
    ref = float(np.sqrt(np.sum(e * e)) / np.sqrt(np.sum(np.where(liq, b64, 0.0) ** 2)))
    assert ref > 0.0
    assert abs(st["true_relres_p"] - ref) <= 1e-10 * ref, (st["true_relres_p"], ref)
    # the solver's b is the divergence the oracle computes (FP32 rounding only)
    ob = O.divergence(og, u0)
    assert np.abs(b64 - ob).max() <= 1e-6 * np.abs(ob).max()


def test_first_step_length_matches_fp64():
    n = 40
    types, _ = W.sphere_union(n, n, n, 2)
    og = O.Grid(types, 1.0 / n, 1 / 30, 0.01)
    gg = F.Grid(n, n, n, dx=1.0 / n, tol_p=1e-12, maxit_p=1, check_every=1)
    gg.set_mask(types)
    u = gg.pack(wide_range_field(n, n, n, 8))
    b = gg.empty_cell()
    F.fs_divergence(gg.ctx, u, b)
    q = gg.empty_cell()
    rc, st = gg.project(u, q)
    assert rc == F.FS_ENOCONV and st["iters_p"] == 1, st
    liq = types == 1
    bf = gg.unpack_cell(b, np.float32)
    # the Jacobi diagonal: the count of non-solid neighbours (walls are solid)
    d = np.zeros(types.shape)
    pad = np.pad(types != 2, 1, constant_values=False)
    for ax in range(3):
        for s in (-1, 1):
            d += np.roll(pad, s, axis=ax)[1:-1, 1:-1, 1:-1]
    inv = np.where(liq, np.float32(1.0) / d.astype(np.float32), np.float32(0.0)).astype(np.float32)
    z = (bf * inv).astype(np.float32)               # z = D^-1 b as the solver forms it in FP32
    z64, b64 = z.astype(np.float64), bf.astype(np.float64)
    alpha = float(np.sum(b64 * z64) / np.sum(z64 * O.poisson_apply(og, z64)))
    qg = gg.unpack_cell(q)
    sel = liq & (np.abs(z64) > 1e-3 * np.abs(z64).max())
    ratio = np.median(qg[sel] / z64[sel])
    assert abs(ratio - alpha) <= 2e-6 * abs(alpha), (ratio, alpha)
