"""Batched lines (acs_lines_*) on the GPU.

Every line of a batch must equal its standalone 1D run bit for bit (same update and
ghost rule, same coefficients) across the warp-register size classes (up to 32, 64,
..., 2048 unknowns), the shared-memory class beyond them, and every boundary; FP64
lines also match the oracle within 1e-12 relative; per-line E_h / max-norm match the
standalone reductions.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SIDES = [1, 2, 3, 5, 31, 32, 33, 63, 64, 65, 127, 129, 255, 257, 511, 513, 1000, 1024, 1025, 2047, 2048,
         2049, 3000]


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


def _lines(acs, sides, seed):
    n, eps, dt, h, bc = [], [], [], [], []
    rng = np.random.default_rng(seed)
    for k, m in enumerate(sides):
        for b in (0, 1, 2):
            hh = 1.0 / (m + 1) if b == 2 else 1.0 / m
            e = float(rng.uniform(0.005, 0.03))
            n.append(m)
            eps.append(e)
            h.append(hh)
            # include time steps large enough for the Newton solve (small lines)
            dt.append(0.9 * acs.dt_max(1, e, hh)[0])
            bc.append(b)
    return n, eps, dt, h, bc


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_lines_equal_standalone(acs, dtype):
    n, eps, dt, h, bc = _lines(acs, SIDES, 3)
    L = acs.Lines(n, eps, dt, h, bc, dtype)
    nd = np.float32 if dtype == "f32" else np.float64
    rng = np.random.default_rng(5)
    phi0 = [rng.uniform(-1, 1, size=m).astype(nd) for m in n]
    L.set_states(phi0)
    assert all(o % (4 if dtype == "f32" else 2) == 0 for o in L.offsets)
    L.step(7)
    L.step(13)
    got = L.states()
    E, M = L.observe()
    for k in range(len(n)):
        s = acs.AllenCahn((n[k],), eps[k], dt[k], h[k], bc[k], dtype)
        s.set_state(phi0[k])
        s.step(20)
        ref = s.numpy()
        assert np.array_equal(got[k], ref), (n[k], bc[k])
        assert E[k] == pytest.approx(s.energy(), rel=1e-12) and M[k] == s.maxnorm()
        assert np.array_equal(L.view(k).cpu().numpy(), got[k])


def test_lines_fp64_vs_oracle(acs):
    n, eps, dt, h, bc = _lines(acs, [17, 300, 1500, 5000], 8)
    L = acs.Lines(n, eps, dt, h, bc, "f64")
    rng = np.random.default_rng(9)
    phi0 = [rng.uniform(-1, 1, size=m) for m in n]
    L.set_states(phi0)
    L.step(40)
    got = L.states()
    for k in range(len(n)):
        ref = oracle.run_fd(phi0[k], eps[k], dt[k], h[k], bc[k], 40)
        assert np.abs(got[k] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_lines_stationary_profile(acs):
    """The 1D stationary interface tanh(x / (sqrt(2) eps)) on (-1, 1), Neumann ends,
    barely moves: a check of the line path against a solution of the equation."""
    import math
    res = []
    for m in (65, 129, 257):
        hh = 2.0 / (m - 1)
        x = -1.0 + hh * np.arange(m)
        e = 0.05
        prof = np.tanh(x / (math.sqrt(2) * e))
        res.append((m, hh, e, prof))
    n = [r[0] for r in res]
    L = acs.Lines(n, [r[2] for r in res], [0.5 * acs.dt_max(1, r[2], r[1])[0] for r in res],
                  [r[1] for r in res], [1] * len(res), "f64")
    L.set_states([r[3] for r in res])
    L.step(200)
    errs = [np.abs(g - r[3]).max() for g, r in zip(L.states(), res)]
    # second-order spatial error: halving h divides the drift by about four
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[2] > 10


def test_lines_full_workload(acs):
    """The benchmark's 4096-line workload (lengths 32..4096, 2000 steps in one call):
    a sample of 128 lines equals its standalone runs bit for bit; every line keeps
    |phi| <= 1 and a non-increasing E_h."""
    from workloads import LINE_STEPS, line_instances
    lines = line_instances()
    L = acs.Lines([i.n for i in lines], [i.eps for i in lines], [i.dt for i in lines], [i.h for i in lines],
                  [i.bc for i in lines], "f32")
    phi0 = [i.phi0().astype(np.float32) for i in lines]
    L.set_states(phi0)
    E0, _ = L.observe()
    L.step(LINE_STEPS)
    E1, M1 = L.observe()
    assert np.all(E1 <= E0) and np.all(M1 <= 1.0)
    got = L.states()
    for k in range(0, len(lines), len(lines) // 128):
        i = lines[k]
        s = acs.AllenCahn((i.n,), i.eps, i.dt, i.h, i.bc, "f32")
        s.set_state(phi0[k])
        s.step(LINE_STEPS)
        assert np.array_equal(got[k], s.numpy()), k
        s.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("mode", ["series", "newton"])
def test_lines_unclamped_root_modes(acs, dtype, mode):
    """Every size class with the root unclamped: dt above Theorem 2's bound but within
    Theorem 3's (lambda = 0.4993 at dt = 0.002, the series with its range tests; lambda =
    0.4 at dt = 0.5, the Newton root).  Bit-identical to the standalone 1D path; FP64
    within 1e-12 of the oracle."""
    import ctypes
    lam, dt = (0.4993, 0.002) if mode == "series" else (0.4, 0.5)
    n, eps, dts, h, bc = [], [], [], [], []
    for m in SIDES:
        for b in (0, 1, 2):
            hh = 1.0 / (m + 1) if b == 2 else 1.0 / m
            n.append(m)
            h.append(hh)
            eps.append(float(np.sqrt(lam / dt)) * hh)
            dts.append(dt)
            bc.append(b)
    want = acs.ACS_ROOT_SERIES if mode == "series" else acs.ACS_ROOT_NEWTON
    for k in range(len(n)):
        dmp, den = acs.dt_max(1, eps[k], h[k])
        assert dmp < dt <= den
    L = acs.Lines(n, eps, dts, h, bc, dtype)
    nd = np.float32 if dtype == "f32" else np.float64
    rng = np.random.default_rng(9)
    phi0 = [rng.uniform(-1, 1, size=m).astype(nd) for m in n]
    L.set_states(phi0)
    L.step(17)
    got = L.states()
    for k in range(len(n)):
        s = acs.AllenCahn((n[k],), eps[k], dts[k], h[k], bc[k], dtype)
        m = ctypes.c_int()
        assert acs.lib().acs_get_root(s.ctx, ctypes.byref(m), None) == 0 and m.value == want
        s.set_state(phi0[k])
        s.step(17)
        ref = s.numpy()
        s.close()
        assert np.isfinite(ref).all() and np.array_equal(got[k], ref), (n[k], bc[k])
        if dtype == "f64" and k % 5 == 0:
            o = oracle.run_fd(phi0[k].astype(np.float64), eps[k], dts[k], h[k], bc[k], 17)
            assert float(np.abs(got[k] - o).max() / max(np.abs(o).max(), 1e-300)) <= 1e-12
