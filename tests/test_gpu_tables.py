"""The GPU's FP64 path reproduces the numbers the paper prints.

Table 2 (1D traveling wave, Neumann, four grid levels) and Table 3 (2D periodic
self-convergence, two diffusion coefficients, four grids against a fine reference run)
are recomputed with the library's own kernels (the single-problem 1D and 2D paths and
the batched lines) and compared with the printed digits, as the oracle's tests do.
"""
import math

import numpy as np
import pytest

from conftest import read_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


def _wave(inv_dx):
    eps = math.tanh(0.9) / (16 * math.sqrt(2))
    se = 3 * eps / math.sqrt(2)
    T = 1 / se
    h = 1.0 / inv_dx
    k = round(math.log2(inv_dx / 64))
    dt = 5 / 64 ** 2 * 2.0 ** (-2 * k)
    N = round(3 / h)
    x = -0.5 + h * np.arange(N + 1)
    phi0 = 0.5 * (1 - np.tanh(x / (2 * math.sqrt(2) * eps)))
    exact = 0.5 * (1 - np.tanh((x - se * T) / (2 * math.sqrt(2) * eps)))
    return eps, dt, h, N, phi0, exact, math.floor(T / dt)


def _errors(phi, exact, nodes):
    e = phi - exact
    return float(np.abs(e).max()), math.sqrt(float((e * e).sum()) / nodes)


@pytest.mark.parametrize("row", read_golden("table2_traveling_wave_1d.txt"), ids=lambda r: f"dx=1/{int(r[0])}")
def test_table2_on_gpu(acs, row):
    inv_dx, emax, el2 = row
    eps, dt, h, N, phi0, exact, steps = _wave(int(inv_dx))
    s = acs.AllenCahn((N + 1,), eps, dt, h, acs.ACS_BC_NEUMANN, "f64")
    s.set_state(phi0)
    s.step(steps)
    gmax, gl2 = _errors(s.numpy(), exact, N + 1)
    assert gmax == pytest.approx(emax, rel=6e-5, abs=0)
    assert gl2 == pytest.approx(el2, rel=6e-5, abs=0)
    assert s.maxnorm() <= 1.0


def test_table2_as_batched_lines(acs):
    """All four grid levels at once as batched lines give the same bits."""
    rows = read_golden("table2_traveling_wave_1d.txt")
    runs = [_wave(int(r[0])) for r in rows]
    # lines advance together, so run every level for its own step count in turn
    for (eps, dt, h, N, phi0, exact, steps), (inv_dx, emax, el2) in zip(runs, rows):
        L = acs.Lines([N + 1], [eps], [dt], [h], [acs.ACS_BC_NEUMANN], "f64")
        L.set_states([phi0])
        L.step(steps)
        gmax, gl2 = _errors(L.states()[0], exact, N + 1)
        assert gmax == pytest.approx(emax, rel=6e-5, abs=0)
        assert gl2 == pytest.approx(el2, rel=6e-5, abs=0)


def _table3_run(acs, eps2, h, dt):
    n = round(2 * math.pi / h)
    x = h * np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    s = acs.AllenCahn((n, n), math.sqrt(eps2), dt, h, acs.ACS_BC_PERIODIC, "f64")
    s.set_state(0.05 * np.sin(X) * np.sin(Y))
    s.step(round(1 / dt))
    return s.numpy(), n


@pytest.mark.parametrize("eps2", [0.01, 0.2])
def test_table3_on_gpu(acs, eps2):
    rows = [r for r in read_golden("table3_periodic_2d.txt") if r[0] == eps2]
    ref_inv, ref_inv_dt = rows[0][1], rows[0][2]
    ref, nref = _table3_run(acs, eps2, math.pi / ref_inv, 1.0 / ref_inv_dt)
    got = []
    for _, _, _, k, emax, el2 in rows:
        h = math.pi / (10 * k)
        phi, n = _table3_run(acs, eps2, h, h * h * 2 / math.pi ** 2)
        r = nref // n
        assert r * n == nref
        gmax, gl2 = _errors(phi, ref[::r, ::r], (n + 1) ** 2)
        assert gmax == pytest.approx(emax, rel=6e-5, abs=0), (k, gmax, emax)
        assert gl2 == pytest.approx(el2, rel=1e-3, abs=0), (k, gl2, el2)
        got.append(gmax)
    ks = [r[3] for r in rows]
    cr = [math.log(got[i] / got[i + 1]) / math.log(ks[i + 1] / ks[i]) for i in range(len(ks) - 1)]
    assert all(1.9 < c < 2.5 for c in cr), cr
