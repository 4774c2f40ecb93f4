"""GPU parity of the temporally blocked step (K fused steps per pass, ACS_KERNEL_TEMPORAL).

A pass of depth K computes every intermediate level with the single-step arithmetic
(Eq. IE-FD, Remark 1) and re-applies the ghost rule of Eq. (Ddeltax) at each level, so
K steps through it equal K single steps bit for bit.  Checked against the one-thread
kernel for K = 2, 3, 4, every boundary, both precisions, grids smaller than one strip,
partial strips and partial row chunks, step counts that are not multiples of K, and
against the FP64 oracle (max-abs relative 1e-12).
"""
import math

import numpy as np
import pytest

import oracle
from workloads import BC_DIRICHLET, BC_NEUMANN, BC_PERIODIC, cfg2, cfg3, dt_rule, uniform_field

pytestmark = pytest.mark.gpu

BCS = [BC_PERIODIC, BC_NEUMANN, BC_DIRICHLET]
BCN = {0: "P", 1: "HN", 2: "HD"}


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _pair(acs, shape, bc, dtype, seed, depth, chunk=0):
    n = max(shape)
    h, eps = 1.0 / n, 0.02
    dt = dt_rule(len(shape), eps, h)
    phi0 = uniform_field(shape, -1.0, 1.0, seed)
    a = acs.AllenCahn(shape, eps, dt, h, bc, dtype)
    b = acs.AllenCahn(shape, eps, dt, h, bc, dtype)
    a.set_kernel(acs.ACS_KERNEL_TEMPORAL, depth)
    if chunk:
        acs.check(acs.lib().acs_set_variant(a.ctx, 0, chunk))
    b.set_kernel(acs.ACS_KERNEL_NAIVE)
    a.set_state(phi0)
    b.set_state(phi0)
    return a, b, phi0, (eps, dt, h)


# rows a multiple of 16 bytes in both precisions: x sizes multiple of 4
SHAPES = [(1, 4), (3, 8), (7, 4), (33, 64), (130, 256), (61, 124), (257, 260), (40, 512)]


@pytest.mark.parametrize("depth", [2, 3, 4])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("bc", BCS, ids=lambda b: BCN[b])
@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_temporal2d_bitwise_equals_single_steps(acs, shape, bc, dtype, depth):
    a, b, phi0, (eps, dt, h) = _pair(acs, shape, bc, dtype, 300 + bc + depth, depth)
    assert a.get_kernel() == (acs.ACS_KERNEL_TEMPORAL, depth)
    a.step(13)   # passes of depth K plus a remainder
    b.step(13)
    assert np.array_equal(a.numpy(), b.numpy())
    if dtype == "f64":
        assert relerr(a.numpy(), oracle.run_fd(phi0, eps, dt, h, bc, 13)) <= 1e-12


@pytest.mark.parametrize("chunk", [1, 2, 5])
@pytest.mark.parametrize("bc", BCS, ids=lambda b: BCN[b])
def test_temporal2d_row_chunks(acs, bc, chunk):
    """Explicit row chunks (16, 32, 80 rows per warp) that leave a partial last chunk."""
    a, b, _, _ = _pair(acs, (203, 376), bc, "f32", 400 + bc, 4, chunk)
    a.step(24)
    b.step(24)
    assert np.array_equal(a.numpy(), b.numpy())


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_temporal2d_cfg3_full_grid(acs, dtype):
    """The 4096^2 Dirichlet star grid, 40 steps at depth 4, equals the TMA-streamed
    single-step kernel bit for bit."""
    w = cfg3(dtype)
    nd = np.float32 if dtype == "f32" else np.float64
    phi0 = w.phi0().astype(nd)
    a = acs.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, dtype)
    b = acs.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, dtype)
    a.set_kernel(acs.ACS_KERNEL_TEMPORAL, 4)
    b.set_kernel(acs.ACS_KERNEL_TILED)
    a.set_state(phi0)
    b.set_state(phi0)
    a.step(40)
    b.step(40)
    assert np.array_equal(a.numpy(), b.numpy())


@pytest.mark.parametrize("bc", BCS, ids=lambda b: BCN[b])
def test_temporal2d_fex_scheme(acs, bc):
    """The FEX-FD scheme of Remark 2 (no cubic) through depth-4 passes."""
    a, b, phi0, (eps, dt, h) = _pair(acs, (50, 132), bc, "f64", 500 + bc, 4)
    a.set_scheme(acs.ACS_SCHEME_FEX_FD)
    b.set_scheme(acs.ACS_SCHEME_FEX_FD)
    a.step(11)
    b.step(11)
    assert np.array_equal(a.numpy(), b.numpy())
    ref = oracle.run_fd(phi0, eps, dt, h, bc, 11, scheme=oracle.SCHEME_FEX_FD)
    assert relerr(a.numpy(), ref) <= 1e-12


def test_temporal2d_logged_run(acs):
    """A logged run (E_h and max-norm every 10 steps) through depth-3 passes gives the
    same log and state as the single-step kernel."""
    a, b, _, _ = _pair(acs, (96, 128), BC_NEUMANN, "f32", 7, 3)
    Ea, Ma = a.run_logged(50, 10)
    Eb, Mb = b.run_logged(50, 10)
    assert np.array_equal(a.numpy(), b.numpy())
    np.testing.assert_allclose(Ea, Eb, rtol=1e-12)
    assert np.array_equal(Ma, Mb)


SHAPES_3D = [(2, 3, 4), (5, 7, 8), (9, 33, 64), (20, 70, 130), (33, 17, 12), (64, 64, 64), (70, 65, 126),
             (7, 130, 62)]


@pytest.mark.parametrize("bc", BCS, ids=lambda b: BCN[b])
@pytest.mark.parametrize("shape", SHAPES_3D, ids=str)
def test_temporal3d_bitwise_equals_single_steps(acs, shape, bc):
    """3D FP32 at depth 2: windows smaller than the grid and larger, partial windows in
    x and y, partial z chunks, an odd step count (passes plus one single step)."""
    a, b, _, _ = _pair(acs, shape, bc, "f32", 600 + bc, 2)
    assert a.get_kernel() == (acs.ACS_KERNEL_TEMPORAL, 2)
    a.step(11)
    b.step(11)
    assert np.array_equal(a.numpy(), b.numpy())


@pytest.mark.parametrize("chunk", [1, 5, 17])
def test_temporal3d_z_chunks(acs, chunk):
    """Explicit z chunks (1, 5, 17 planes per CTA)."""
    a, b, _, _ = _pair(acs, (41, 60, 72), BC_DIRICHLET, "f32", 700 + chunk, 2, chunk)
    a.step(8)
    b.step(8)
    assert np.array_equal(a.numpy(), b.numpy())


def test_temporal3d_cfg2_full_grid(acs):
    """The 512^3 Neumann grid, 10 steps at depth 2, equals the TMA-streamed single-step
    kernel bit for bit; a logged run through it gives the same E_h log."""
    w = cfg2("f32")
    phi0 = w.phi0().astype(np.float32)
    a = acs.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")
    b = acs.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")
    a.set_kernel(acs.ACS_KERNEL_TEMPORAL, 2)
    b.set_kernel(acs.ACS_KERNEL_TILED)
    a.set_state(phi0)
    b.set_state(phi0)
    a.step(10)
    b.step(10)
    assert np.array_equal(a.numpy(), b.numpy())
    a.set_state(phi0)
    b.set_state(phi0)
    Ea, Ma = a.run_logged(20, 10)
    Eb, Mb = b.run_logged(20, 10)
    assert np.array_equal(a.numpy(), b.numpy())
    np.testing.assert_allclose(Ea, Eb, rtol=1e-12)
    assert np.array_equal(Ma, Mb)


def test_temporal_unsupported_shapes(acs):
    """Rows that are not a multiple of 16 bytes (2D) or of odd length (3D), 1D grids, 3D
    FP64 grids and depths beyond the kernels' have no temporally blocked kernel."""
    s = acs.AllenCahn((33, 65), 0.02, 0.01, 1 / 65, BC_PERIODIC, "f32")
    with pytest.raises(acs.AcsError) as e:
        s.set_kernel(acs.ACS_KERNEL_TEMPORAL, 2)
    assert e.value.status == acs.ACS_E_UNSUPPORTED
    s = acs.AllenCahn((64, 64), 0.02, 0.01, 1 / 64, BC_PERIODIC, "f32")
    with pytest.raises(acs.AcsError):
        s.set_kernel(acs.ACS_KERNEL_TEMPORAL, 5)
    s = acs.AllenCahn((256,), 0.02, 0.01, 1 / 256, BC_PERIODIC, "f32")
    with pytest.raises(acs.AcsError):
        s.set_kernel(acs.ACS_KERNEL_TEMPORAL, 2)
    for shape, dtype, depth in (((8, 8, 8), "f64", 2), ((8, 8, 9), "f32", 2), ((8, 8, 8), "f32", 3)):
        s = acs.AllenCahn(shape, 0.02, 0.01, 1 / 8, BC_PERIODIC, dtype)
        with pytest.raises(acs.AcsError) as e:
            s.set_kernel(acs.ACS_KERNEL_TEMPORAL, depth)
        assert e.value.status == acs.ACS_E_UNSUPPORTED


# Beyond Theorem 2's step-size condition but within Theorem 3's: the root runs without the
# clamp -- the series with its run-time range tests, or the Newton root -- and the states
# stay bounded.  (shape, eps, dt, h, dtype, expected root mode, depths)
UNCLAMPED = [
    ((130, 256), math.sqrt(0.248 / 0.01) / 256, 0.01, 1 / 256, "f32", 1, (2, 3, 4)),
    ((130, 256), math.sqrt(0.2497 / 0.002) / 256, 0.002, 1 / 256, "f64", 1, (2, 4)),
    ((130, 256), math.sqrt(0.2 / 0.5) / 256, 0.5, 1 / 256, "f32", 0, (2, 3, 4)),
    ((130, 256), math.sqrt(0.2 / 0.5) / 256, 0.5, 1 / 256, "f64", 0, (3,)),
    ((20, 70, 130), math.sqrt(0.1658 / 0.01) / 130, 0.01, 1 / 130, "f32", 1, (2,)),
    ((20, 70, 130), math.sqrt(0.1 / 0.5) / 130, 0.5, 1 / 130, "f32", 0, (2,)),
]


@pytest.mark.parametrize("bc", BCS, ids=lambda b: BCN[b])
@pytest.mark.parametrize("case", range(len(UNCLAMPED)))
def test_temporal_unclamped_root_modes(acs, case, bc):
    """Temporal passes equal single steps bit for bit when the root runs without Theorem
    2's clamp (acs_get_root confirms the mode; acs_dt_max that dt exceeds the
    maximum-principle bound but not the energy bound); FP64 also matches the oracle."""
    import ctypes
    shape, eps, dt, h, dtype, mode, depths = UNCLAMPED[case]
    dmp, den = ctypes.c_double(), ctypes.c_double()
    assert acs.lib().acs_dt_max(len(shape), eps, h, ctypes.byref(dmp), ctypes.byref(den)) == 0
    assert dmp.value < dt <= den.value
    phi0 = uniform_field(shape, -1.0, 1.0, 700 + case + bc)
    b = acs.AllenCahn(shape, eps, dt, h, bc, dtype)
    m = ctypes.c_int()
    assert acs.lib().acs_get_root(b.ctx, ctypes.byref(m), None) == 0 and m.value == mode
    b.set_kernel(acs.ACS_KERNEL_NAIVE)
    b.set_state(phi0)
    b.step(13)
    ref = b.numpy()
    assert np.isfinite(ref).all()
    if dtype == "f64":
        assert relerr(ref, oracle.run_fd(phi0, eps, dt, h, bc, 13)) <= 1e-12
    for depth in depths:
        a = acs.AllenCahn(shape, eps, dt, h, bc, dtype)
        a.set_kernel(acs.ACS_KERNEL_TEMPORAL, depth)
        a.set_state(phi0)
        a.step(13)
        assert np.array_equal(a.numpy(), ref), depth
        a.close()
    b.close()
