"""The collide-and-stream (population) form on the GPU (ACS_KERNEL_LB).

FP64: each step matches the oracle's own collide-and-stream form (Sec. II) within
1e-12 relative, for d = 1, 2, 3 and every boundary; and it stays within rounding of
the finite-difference path (Eq. IE-FD), for the paper's weights and others (the sum
over populations does not depend on w_1).  FP32: within 2e-5 of the FD path.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


# odd rows take the one-value-per-thread kernels, rows of a multiple of four values the
# vectorised ones
SHAPES = {1: (301,), 2: (37, 45), 3: (13, 17, 19)}
VSHAPES = {1: (300,), 2: (37, 44), 3: (13, 17, 20)}


def _problem(dims, bc, seed=0, vec=False):
    rng = np.random.default_rng(seed + 10 * dims + bc)
    shape = (VSHAPES if vec else SHAPES)[dims]
    n = shape[-1]
    h = 1.0 / (n + 1) if bc == 2 else 1.0 / n
    eps = 0.03
    import paper_2312_07010_gb300 as P
    dt = 0.9 * P.dt_max(dims, eps, h)[0]
    return rng.uniform(-1, 1, size=shape), eps, dt, h


@pytest.mark.parametrize("vec", [False, True], ids=["scalar", "vector"])
@pytest.mark.parametrize("dims", [1, 2, 3])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_lb_fp64_matches_oracle_lb(acs, dims, bc, vec):
    phi0, eps, dt, h = _problem(dims, bc, vec=vec)
    s = acs.AllenCahn(phi0.shape, eps, dt, h, bc, "f64")
    s.use_lb_form()
    s.set_state(phi0)
    ref = phi0.copy()
    for _ in range(6):
        ref = oracle.step_lb(ref, eps, dt, h, bc)
    s.step(6)
    got = s.numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("vec", [False, True], ids=["scalar", "vector"])
@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("omega1", [0.0, 0.05, 0.11])
def test_lb_equals_fd_to_rounding(acs, dims, omega1, vec):
    bc = 1
    phi0, eps, dt, h = _problem(dims, bc, seed=3, vec=vec)
    a = acs.AllenCahn(phi0.shape, eps, dt, h, bc, "f64")
    a.use_lb_form(omega1)
    b = acs.AllenCahn(phi0.shape, eps, dt, h, bc, "f64")
    a.set_state(phi0)
    b.set_state(phi0)
    a.step(20)
    b.step(20)
    x, y = a.numpy(), b.numpy()
    assert np.abs(x - y).max() <= 1e-13


@pytest.mark.parametrize("vec", [False, True], ids=["scalar", "vector"])
def test_lb_fp32_close_to_fd(acs, vec):
    phi0, eps, dt, h = _problem(3, 0, seed=5, vec=vec)
    p32 = phi0.astype(np.float32)
    a = acs.AllenCahn(phi0.shape, eps, dt, h, 0, "f32")
    a.use_lb_form()
    b = acs.AllenCahn(phi0.shape, eps, dt, h, 0, "f32")
    a.set_state(p32)
    b.set_state(p32)
    a.step(30)
    b.step(30)
    x, y = a.numpy(), b.numpy()
    assert np.abs(x.astype(np.float64) - y).max() <= 2e-5
    assert np.abs(x).max() <= 1.0


def test_lb_long_run_graph_and_energy(acs):
    """Many steps (recorded into a graph) keep the maximum principle and decrease E_h."""
    phi0, eps, dt, h = _problem(2, 2, seed=7)
    s = acs.AllenCahn(phi0.shape, eps, dt, h, 2, "f64")
    s.use_lb_form()
    s.set_state(phi0)
    e0 = s.energy()
    s.step(200)
    ref = oracle.run_fd(phi0, eps, dt, h, 2, 200)
    got = s.numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert s.maxnorm() <= 1.0 and s.energy() < e0
