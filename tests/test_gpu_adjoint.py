"""GPU adjoint (acs_grad and the autograd Function) against the FP64 oracle adjoint
and central finite differences.

Tolerances: FP64 GPU vs FP64 oracle, relative 1e-10 (both are the same transpose
chain, differently ordered); FP32 GPU vs FP64 oracle, max-abs error <= 2e-3 of
max |grad| (the FP32 forward differs from FP64 by up to 2e-5 and the adjoint
inherits that).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import BC_DIRICHLET, BC_NEUMANN, BC_PERIODIC, cfg5, dt_rule, uniform_field, tanh_disc

pytestmark = pytest.mark.gpu

BCS = [BC_PERIODIC, BC_NEUMANN, BC_DIRICHLET]


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


def _setup(shape, bc, seed):
    d = len(shape)
    h = 1.0 / max(shape)
    eps = 0.03
    dt = dt_rule(d, eps, h)
    phi0 = uniform_field(shape, -0.5, 0.5, seed)
    target = uniform_field(shape, -1, 1, seed + 1000)
    return h, eps, dt, phi0, target


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape", [(37,), (12, 9), (6, 5, 7)], ids=str)
def test_grad_fp64_vs_oracle(acs, shape, bc):
    h, eps, dt, phi0, target = _setup(shape, bc, 3 + bc)
    steps, C = 30, 7
    s = acs.AllenCahn(shape, eps, dt, h, bc, "f64")
    s.set_state(phi0)
    s.record_for_grad(steps, C)
    s.step(steps)
    pT = s.numpy()
    gT = 2 * (pT - target) / pT.size
    g0, ge = s.grad(torch.from_numpy(gT).cuda())
    rg0, rge = oracle.grad(phi0, eps, dt, h, bc, steps, gT, checkpoint_every=C)
    g0 = g0.cpu().numpy()
    assert np.abs(g0 - rg0).max() <= 1e-10 * np.abs(rg0).max()
    assert ge == pytest.approx(rge, rel=1e-10)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape", [(40, 70), (33, 130), (16, 64)], ids=str)
def test_grad_fp64_streamed_2d_vs_oracle(acs, shape, bc):
    """Rows a multiple of 16 bytes take the TMA-streamed 2D adjoint kernel: several
    column strips, a ragged last strip and a ragged last block of rows."""
    h, eps, dt, phi0, target = _setup(shape, bc, 20 + bc)
    steps, C = 23, 6
    s = acs.AllenCahn(shape, eps, dt, h, bc, "f64")
    s.set_state(phi0)
    s.record_for_grad(steps, C)
    s.step(steps)
    pT = s.numpy()
    gT = 2 * (pT - target) / pT.size
    for _ in range(2):  # the second call replays the recorded sweep
        g0, ge = s.grad(torch.from_numpy(gT).cuda())
        rg0, rge = oracle.grad(phi0, eps, dt, h, bc, steps, gT, checkpoint_every=C)
        g0 = g0.cpu().numpy()
        assert np.abs(g0 - rg0).max() <= 1e-10 * np.abs(rg0).max()
        assert ge == pytest.approx(rge, rel=1e-10)


@pytest.mark.parametrize("bc", BCS)
def test_grad_fp32_vs_fp64_oracle(acs, bc):
    shape = (64, 48)
    h, eps, dt, phi0, target = _setup(shape, bc, 10 + bc)
    steps = 60
    p32 = phi0.astype(np.float32)
    s = acs.AllenCahn(shape, eps, dt, h, bc, "f32")
    s.set_state(p32)
    s.record_for_grad(steps, 25)
    s.step(steps)
    pT = s.numpy().astype(np.float64)
    gT = 2 * (pT - target) / pT.size
    g0, ge = s.grad(torch.from_numpy(gT.astype(np.float32)).cuda())
    rg0, rge = oracle.grad(p32.astype(np.float64), eps, dt, h, bc, steps, gT, checkpoint_every=25)
    assert np.abs(g0.cpu().numpy() - rg0).max() <= 2e-3 * np.abs(rg0).max()
    assert ge == pytest.approx(rge, rel=2e-3)


def test_autograd_function_and_finite_differences(acs):
    """Scaled version of the 1024^2 periodic workload: loss = mean((phi_T - disc)^2)."""
    w = cfg5()
    n = 128
    h = 1.0 / n
    dt = dt_rule(2, w.eps, h)
    steps = 100
    phi0 = uniform_field((n, n), -0.5, 0.5, w.seed)
    target = torch.from_numpy(tanh_disc(n, h, w.eps)).cuda()
    p = torch.from_numpy(phi0).cuda().requires_grad_(True)
    e2 = torch.tensor(w.eps ** 2, dtype=torch.float64, requires_grad=True)
    out = acs.allen_cahn(p, e2, steps, dt, h, BC_PERIODIC, 50)
    loss = torch.mean((out - target) ** 2)
    loss.backward()
    g0 = p.grad.cpu().numpy()
    ge = float(e2.grad)

    def L(ph, eps2):
        s = acs.AllenCahn((n, n), math.sqrt(eps2), dt, h, BC_PERIODIC, "f64")
        s.set_state(ph)
        s.step(steps)
        return float(np.mean((s.numpy() - target.cpu().numpy()) ** 2))

    v = uniform_field((n, n), -1, 1, 77)
    st = 1e-6
    fd = (L(phi0 + st * v, w.eps ** 2) - L(phi0 - st * v, w.eps ** 2)) / (2 * st)
    assert float(np.sum(g0 * v)) == pytest.approx(fd, rel=1e-6)
    se = 1e-7
    fde = (L(phi0, w.eps ** 2 + se) - L(phi0, w.eps ** 2 - se)) / (2 * se)
    assert ge == pytest.approx(fde, rel=1e-5)
    # and the oracle adjoint
    pT = out.detach().cpu().numpy()
    gT = 2 * (pT - target.cpu().numpy()) / pT.size
    rg0, rge = oracle.grad(phi0, w.eps, dt, h, BC_PERIODIC, steps, gT, checkpoint_every=50)
    assert np.abs(g0 - rg0).max() <= 1e-10 * np.abs(rg0).max()
    assert ge == pytest.approx(rge, rel=1e-10)


def test_grad_requires_recording(acs):
    s = acs.AllenCahn((8, 8), 0.02, 0.01, 1 / 8, BC_PERIODIC, "f32")
    s.set_state(np.zeros((8, 8), np.float32))
    s.step(2)
    with pytest.raises(acs.AcsError) as e:
        s.grad(torch.zeros((8, 8), device="cuda"))
    assert e.value.status == -6
    s.record_for_grad(4, 2)
    s.step(4)
    with pytest.raises(acs.AcsError) as e:
        s.step(1)
    assert e.value.status == -3


def test_adjoint_full_size_fp64_dot_product(acs):
    """The 1024^2 periodic adjoint workload (500 steps, checkpoints every 50) in FP64:
    the gradient against central differences of the loss along a random direction of
    phi0 and along eps^2."""
    w = cfg5()
    n = w.n[0]
    phi0 = w.phi0()
    target = tanh_disc(n, w.h, w.eps)
    s = acs.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f64")
    s.set_state(phi0)
    s.record_for_grad(w.steps, 50)
    s.step(w.steps)
    pT = s.numpy()
    g0, ge = s.grad(torch.from_numpy(2 * (pT - target) / pT.size).cuda())
    g0 = g0.cpu().numpy()

    def L(ph, eps2):
        t = acs.AllenCahn(w.n, math.sqrt(eps2), w.dt, w.h, w.bc, "f64")
        t.set_state(ph)
        t.step(w.steps)
        v = float(np.mean((t.numpy() - target) ** 2))
        t.close()
        return v

    v = uniform_field((n, n), -1, 1, 91)
    st = 1e-6
    fd = (L(phi0 + st * v, w.eps ** 2) - L(phi0 - st * v, w.eps ** 2)) / (2 * st)
    assert float(np.sum(g0 * v)) == pytest.approx(fd, rel=1e-6)
    se = 1e-7
    fde = (L(phi0, w.eps ** 2 + se) - L(phi0, w.eps ** 2 - se)) / (2 * se)
    assert ge == pytest.approx(fde, rel=1e-5)


@pytest.mark.parametrize("shape,bc", [((40, 64), BCS[0]), ((33, 17, 12), BCS[1]), ((257,), BCS[2])], ids=str)
def test_store_every_state_equals_checkpointed(acs, shape, bc):
    """Checkpoints after every step (no recompute in the backward sweep) give the same
    bits as checkpoints every 7 steps, and the state after the recording is the run's."""
    h, eps, dt, phi0, target = _setup(shape, bc, 11 + bc)
    steps = 23
    out = []
    for every in (1, 7):
        s = acs.AllenCahn(shape, eps, dt, h, bc, "f64")
        s.set_state(phi0)
        s.record_for_grad(steps, every)
        s.step(10)
        s.step(13)
        pT = s.numpy()
        gT = 2 * (pT - target) / pT.size
        g0, ge = s.grad(torch.from_numpy(gT).cuda())
        out.append((pT, g0.cpu().numpy(), ge))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    assert np.abs(out[0][0] - oracle.run_fd(phi0, eps, dt, h, bc, steps)).max() <= 1e-12 * np.abs(out[0][0]).max()
