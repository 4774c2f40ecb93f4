"""GPU parity at the extremes of the launch plans: thousands of tiny batched instances
(more than the per-CTA tensor-map cache covers), a 1D line of four million unknowns, a
3D grid thousands of planes deep on a tiny xy face, and a wide 2D grid whose rows are
not 16-byte multiples (no TMA path).  References: the FP64 oracle, and the
one-thread-per-unknown kernel bit for bit where a tiled kernel runs."""
import numpy as np
import pytest

import oracle
from workloads import BC_DIRICHLET, BC_NEUMANN, BC_PERIODIC, dt_rule, uniform_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


def test_batch_thousands_of_tiny_instances(acs):
    rng = np.random.default_rng(21)
    count = 2500
    n = [int(v) for v in rng.integers(1, 41, size=count)]
    bc = [int(v) for v in rng.integers(0, 3, size=count)]
    eps = [float(v) for v in rng.uniform(0.01, 0.05, size=count)]
    h = [1.0 / (m + 1) if b == BC_DIRICHLET else 1.0 / m for m, b in zip(n, bc)]
    dt = [0.9 * acs.dt_max(2, e, hh)[0] for e, hh in zip(eps, h)]
    b = acs.Batch(n, eps, dt, h, bc, "f32")
    phi0 = [rng.uniform(-1, 1, size=(m, m)).astype(np.float32) for m in n]
    b.set_states(phi0)
    b.step(7)
    got = b.states()
    worst = 0.0
    for k in range(count):
        ref = oracle.run_fd(phi0[k].astype(np.float64), eps[k], dt[k], h[k], bc[k], 7)
        worst = max(worst, float(np.abs(got[k].astype(np.float64) - ref).max()))
    assert worst <= 2e-5
    E, M = b.observe()
    assert np.all(np.isfinite(E)) and np.all(M <= 1.0)


def test_long_1d_line_fp64(acs):
    shape = ((1 << 22) + 3,)
    h, eps = 1.0 / (shape[0] + 1), 2e-6
    dt = dt_rule(1, eps, h)
    phi0 = uniform_field(shape, -1.0, 1.0, 5)
    s = acs.AllenCahn(shape, eps, dt, h, BC_DIRICHLET, "f64")
    s.set_state(phi0)
    s.step(20)
    ref = oracle.run_fd(phi0, eps, dt, h, BC_DIRICHLET, 20)
    assert np.abs(s.numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN, BC_DIRICHLET])
def test_deep_3d_grid_tiled_equals_naive(acs, bc):
    shape = (3001, 4, 8)  # 3001 planes of 4 x 8: many z chunks, one tile per plane
    h, eps = 1.0 / 8, 0.02
    dt = dt_rule(3, eps, h)
    phi0 = uniform_field(shape, -1.0, 1.0, 6)
    a = acs.AllenCahn(shape, eps, dt, h, bc, "f64")
    b = acs.AllenCahn(shape, eps, dt, h, bc, "f64")
    a.set_kernel(acs.ACS_KERNEL_TILED)
    b.set_kernel(acs.ACS_KERNEL_NAIVE)
    a.set_state(phi0)
    b.set_state(phi0)
    a.step(12)
    b.step(12)
    assert np.array_equal(a.numpy(), b.numpy())
    ref = oracle.run_fd(phi0, eps, dt, h, bc, 12)
    assert np.abs(a.numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_wide_2d_rows_not_16_byte_multiples(acs):
    shape = (1001, 4099)  # FP32 rows of 16396 bytes: no TMA tensor map
    h, eps = 1.0 / 4099, 0.002
    dt = dt_rule(2, eps, h)
    phi0 = uniform_field(shape, -1.0, 1.0, 7).astype(np.float32)
    s = acs.AllenCahn(shape, eps, dt, h, BC_NEUMANN, "f32")
    s.set_state(phi0)
    s.step(20)
    got = s.numpy().astype(np.float64)
    ref = oracle.run_fd(phi0.astype(np.float64), eps, dt, h, BC_NEUMANN, 20)
    assert np.abs(got - ref).max() <= 2e-5
    assert np.abs(got).max() <= 1.0
    E = s.energy()
    assert E == pytest.approx(oracle.energy(s.numpy().astype(np.float64), eps, dt, h, BC_NEUMANN), rel=1e-12)
