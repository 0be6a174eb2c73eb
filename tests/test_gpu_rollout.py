"""GPU: the checkpointed rollout (torch.autograd.Function over the C ABI) against
the oracle's forward and reverse pass over several frames, and checkpoint-length
invariance."""
import pytest
import torch

import oracle as O
from paper_2503_00868_gb300 import fluidstep as F
from paper_2503_00868_gb300 import workloads as W
from paper_2503_00868_gb300.rollout import rollout_loss

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_00868_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def oracle_rollout(og, u0, targets, nsteps):
    states = [u0]
    for _ in range(nsteps):
        states.append(O.step(og, states[-1])[0])
    loss = 0.0
    g = og.zeros()
    for n in sorted(targets):
        l, _ = O.loss_grad(og, states[n], targets[n])
        loss += l
    gnu = 0.0
    for n in range(nsteps, 0, -1):
        if n in targets:
            _, gl = O.loss_grad(og, states[n], targets[n])
            g = tuple(a + b for a, b in zip(g, gl))
        g, dnu = O.adjoint_step(og, states[n - 1], g)
        gnu += dnu
    if 0 in targets:
        _, gl = O.loss_grad(og, states[0], targets[0])
        g = tuple(a + b for a, b in zip(g, gl))
    return loss, g, gnu


def rel(a, b):
    num = sum(float(((x - y) ** 2).sum()) for x, y in zip(a, b))
    den = sum(float((y ** 2).sum()) for y in b)
    return (num / den) ** 0.5


@pytest.mark.parametrize("k", [1, 2, 5])
def test_rollout_gradients_match_oracle(k):
    nx, ny, nz = 26, 21, 23
    types, _ = W.ellipsoid_blob(nx, ny, nz, 3)
    nu = 0.03
    kw = dict(dx=1.0 / ny, dt=1 / 30, nu=nu, g=(0.0, -9.81, 0.0))
    og = O.Grid(types, kw["dx"], kw["dt"], nu, g=kw["g"])
    gg = F.Grid(nx, ny, nz, tol_p=1e-7, tol_v=1e-7, **kw)
    gg.set_mask(types)
    u0 = W.blurred_noise_mac(nx, ny, nz, 1)
    nsteps = 5
    tg = {2: W.blurred_noise_mac(nx, ny, nz, 102), 5: W.blurred_noise_mac(nx, ny, nz, 105)}
    oloss, og_u0, ognu = oracle_rollout(og, u0, tg, nsteps)

    leaves = [t.requires_grad_(True) for t in gg.pack(u0)]
    nu_t = torch.tensor(nu, requires_grad=True)
    loss = rollout_loss(gg, F.Mac(*leaves), nu_t, nsteps, {n: gg.pack(t) for n, t in tg.items()},
                        checkpoint_every=k)
    loss.backward()
    assert abs(float(loss) - oloss) <= 1e-5 * abs(oloss)
    gu = gg.unpack(F.Mac(*(t.grad for t in leaves)))
    assert rel(gu, og_u0) < 1e-4
    assert abs(float(nu_t.grad) - ognu) <= 1e-4 * abs(ognu)
