"""The benchmark workloads at their full sizes and step counts, against the FP64 oracle.

Each test runs one workload through the C ABI exactly as stated (grid, boundary, eps,
step count, logging interval) and compares the final state element by element with the
oracle's run of Eq. (IE-FD) from the same initial field (the FP32-rounded field for
FP32 runs), and the logged E_h (Theorem 3, Eq. proof2-eq0) with the oracle's E_h.

Tolerances:
  FP64 state: max |gpu - oracle| / max |oracle| <= 1e-12; logged E_h relative 1e-12.
  FP32 state: max |gpu - oracle| <= 2e-5 and max |phi| <= 1 (Theorem 2).  Its logged
    E_h is compared (a) with the oracle's E_h of the GPU's own final state at 1e-12
    (the reduction is FP64 whatever the state's precision) and (b) with the oracle
    trajectory's E_h at relative 1e-3: with |delta phi| <= 2e-5 the bulk term moves by
    at most h^d sum |(phi^2 - 1) phi| 2e-5 <= 0.385 * 2e-5 |Omega|, about 1e-4 of the
    energies these runs reach, and the link term by less.
  Adjoint (1024^2 periodic FP32, 500 steps, checkpoints every 50) against the oracle
    adjoint of the FP64 run from the FP32-rounded phi0: max-abs 2e-3 of max |grad|, and
    dL/d(eps^2) relative 2e-3 (the FP32 forward differs from FP64 by up to 2e-5 and the
    adjoint inherits that).
  Batched FP32 instances: as FP32 states.

The oracle runs on every host core (OpenMP over points); its results are computed once
per module.  The worst error of each case is printed (pytest -rA shows it).
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import BATCH_STEPS, adjoint_target, batched_instances, cfg2, cfg3, cfg5

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


_ORACLE = {}


def _oracle_logged(w, phi0, key):
    """Oracle state after w.steps steps and its E_h every w.log_every steps (cached)."""
    if key not in _ORACLE:
        ref = np.ascontiguousarray(phi0, dtype=np.float64)
        E = [oracle.energy(ref, w.eps, w.dt, w.h, w.bc)]
        for _ in range(w.steps // w.log_every):
            ref = oracle.run_fd(ref, w.eps, w.dt, w.h, w.bc, w.log_every)
            E.append(oracle.energy(ref, w.eps, w.dt, w.h, w.bc))
        _ORACLE[key] = (ref, np.array(E))
    return _ORACLE[key]


def _check_logged_run(acs, w, dtype):
    nd = np.float32 if dtype == "f32" else np.float64
    phi0 = w.phi0().astype(nd)
    s = acs.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, dtype)
    s.set_state(phi0)
    E, M = s.run_logged(w.steps, w.log_every)
    got = s.numpy()
    kernel = s.get_kernel()
    s.close()
    ref, Eref = _oracle_logged(w, phi0, (w.name, dtype))
    assert np.all(np.diff(E) <= 0)                       # Theorem 3
    if dtype == "f64":
        err = relerr(got, ref)
        eerr = float(np.max(np.abs(E - Eref) / np.abs(Eref)))
        print(f"{w.name} f64 kernel {kernel}: state rel err {err:.3e}, E_h rel err {eerr:.3e}")
        assert err <= 1e-12
        assert eerr <= 1e-12
    else:
        g64 = got.astype(np.float64)
        err = float(np.abs(g64 - ref).max())
        eown = abs(E[-1] - oracle.energy(g64, w.eps, w.dt, w.h, w.bc)) / abs(E[-1])
        eerr = float(np.max(np.abs(E - Eref) / np.abs(Eref)))
        print(f"{w.name} f32 kernel {kernel}: state max-abs err {err:.3e}, max|phi| {np.abs(got).max():.9f}, "
              f"E_h(own state) rel {eown:.3e}, E_h vs oracle trajectory rel {eerr:.3e}")
        assert err <= 2e-5
        assert float(np.abs(got).max()) <= 1.0 and np.all(M <= 1.0)
        assert eown <= 1e-12
        assert eerr <= 1e-3


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_cfg2_3d_neumann_512_200_steps(acs, dtype):
    """512^3 homogeneous Neumann, eps = 0.01, phi0 ~ U[-1, 1] (seed 1), 200 steps, E_h
    logged every 50 steps."""
    _check_logged_run(acs, cfg2(dtype), dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_cfg3_2d_dirichlet_4096_2000_steps(acs, dtype):
    """4096^2 homogeneous Dirichlet star interface, eps = 0.005, 2000 steps, E_h logged
    every 50 steps."""
    _check_logged_run(acs, cfg3(dtype), dtype)


def test_cfg5_adjoint_fp32_vs_oracle_adjoint(acs):
    """1024^2 periodic FP32 forward of 500 steps, checkpoints every 50; the gradients of
    mean((phi_T - disc)^2) with respect to phi0 and eps^2 against the FP64 oracle adjoint."""
    w = cfg5()
    C = w.extra["checkpoint_every"]
    p32 = w.phi0().astype(np.float32)
    target = adjoint_target(w)
    s = acs.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")
    s.set_state(p32)
    s.record_for_grad(w.steps, C)
    s.step(w.steps)
    pT = s.numpy().astype(np.float64)
    gT = 2 * (pT - target) / pT.size
    g0, ge = s.grad(torch.from_numpy(gT.astype(np.float32)).cuda())
    g0 = g0.cpu().numpy().astype(np.float64)
    s.close()
    rg0, rge = oracle.grad(p32.astype(np.float64), w.eps, w.dt, w.h, w.bc, w.steps, gT, checkpoint_every=C)
    gerr = float(np.abs(g0 - rg0).max() / np.abs(rg0).max())
    eerr = abs(ge - rge) / abs(rge)
    print(f"cfg5 adjoint f32: dL/dphi0 max-abs err / max|grad| {gerr:.3e}, dL/deps2 rel err {eerr:.3e}")
    assert gerr <= 2e-3
    assert eerr <= 2e-3


def test_cfg4_batched_sample_vs_oracle(acs):
    """The 256-instance batched FP32 workload, 500 steps in one call; a sample of twelve
    instances (every boundary, the smallest and the largest sides) against the oracle."""
    inst = batched_instances()
    b = acs.Batch([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
                  [i.bc for i in inst], "f32")
    phi0 = [i.phi0().astype(np.float32) for i in inst]
    b.set_states(phi0)
    b.step(BATCH_STEPS)
    got = b.states()
    b.close()
    order = sorted(range(len(inst)), key=lambda k: inst[k].n)
    sample = set(order[:2] + order[-2:])
    for bc in (0, 1, 2):
        ks = [k for k in order if inst[k].bc == bc]
        sample.update([ks[0], ks[len(ks) // 2], ks[-1]])
    worst = 0.0
    for k in sorted(sample):
        i = inst[k]
        ref = oracle.run_fd(phi0[k].astype(np.float64), i.eps, i.dt, i.h, i.bc, BATCH_STEPS)
        err = float(np.abs(got[k].astype(np.float64) - ref).max())
        worst = max(worst, err)
        assert err <= 2e-5, (k, i.n, i.bc, err)
        assert float(np.abs(got[k]).max()) <= 1.0
    print(f"cfg4 batched f32: {len(sample)} instances (sides {min(inst[k].n for k in sample)}.."
          f"{max(inst[k].n for k in sample)}), worst max-abs err {worst:.3e}")
