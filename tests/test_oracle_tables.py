"""Pins of the FD-form oracle to the numbers the paper prints (CPU only).

Table 2 (1D traveling wave, Neumann) and Table 3 (2D periodic, self-convergence)
are reproduced to the printed digits of the maximum-norm error, and the l2
errors to the printed digits (Table 2) or to 1e-3 (Table 3, whose fine reference
run the paper does not fully specify).  A dropped term, a wrong sign of the
reaction or diffusion, a wrong ghost rule for Neumann or periodic, or a wrong
lambda would each move these errors by orders of magnitude.
"""
import math

import numpy as np
import pytest

from conftest import read_golden


def _traveling_wave(orc, inv_dx):
    eps = math.tanh(0.9) / (16 * math.sqrt(2))
    se = 3 * eps / math.sqrt(2)
    T = 1 / se
    h = 1.0 / inv_dx
    k = round(math.log2(inv_dx / 64))
    dt = 5 / 64 ** 2 * 2.0 ** (-2 * k)
    N = round(3 / h)
    x = -0.5 + h * np.arange(N + 1)
    phi0 = 0.5 * (1 - np.tanh(x / (2 * math.sqrt(2) * eps)))
    steps = math.floor(T / dt)
    phi = orc.run_fd(phi0, eps, dt, h, orc.BC_NEUMANN, steps)
    exact = 0.5 * (1 - np.tanh((x - se * T) / (2 * math.sqrt(2) * eps)))
    e = phi - exact
    return float(np.abs(e).max()), math.sqrt(float((e * e).sum()) / (N + 1)), phi


@pytest.mark.parametrize("row", read_golden("table2_traveling_wave_1d.txt")[:3],
                         ids=lambda r: f"dx=1/{int(r[0])}")
def test_table2(orc, row):
    inv_dx, emax, el2 = row
    gmax, gl2, phi = _traveling_wave(orc, int(inv_dx))
    assert gmax == pytest.approx(emax, rel=6e-5, abs=0)
    assert gl2 == pytest.approx(el2, rel=6e-5, abs=0)
    assert np.abs(phi).max() <= 1.0


@pytest.mark.slow
def test_table2_finest(orc):
    inv_dx, emax, el2 = read_golden("table2_traveling_wave_1d.txt")[3]
    gmax, gl2, _ = _traveling_wave(orc, int(inv_dx))
    assert gmax == pytest.approx(emax, rel=6e-5, abs=0)
    assert gl2 == pytest.approx(el2, rel=6e-5, abs=0)


def _table3_run(orc, eps2, h, dt):
    n = round(2 * math.pi / h)
    x = h * np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    u0 = 0.05 * np.sin(X) * np.sin(Y)
    return orc.run_fd(u0, math.sqrt(eps2), dt, h, orc.BC_PERIODIC, round(1 / dt)), n


@pytest.mark.slow
@pytest.mark.parametrize("eps2", [0.01, 0.2])
def test_table3(orc, eps2):
    rows = [r for r in read_golden("table3_periodic_2d.txt") if r[0] == eps2]
    ref_inv, ref_inv_dt = rows[0][1], rows[0][2]
    ref, nref = _table3_run(orc, eps2, math.pi / ref_inv, 1.0 / ref_inv_dt)
    got = []
    for _, _, _, k, emax, el2 in rows:
        h = math.pi / (10 * k)
        dt = h * h * 2 / math.pi ** 2
        phi, n = _table3_run(orc, eps2, h, dt)
        r = nref // n
        assert r * n == nref
        e = phi - ref[::r, ::r]
        gmax = float(np.abs(e).max())
        gl2 = math.sqrt(float((e * e).sum()) / (n + 1) ** 2)
        assert gmax == pytest.approx(emax, rel=6e-5, abs=0), (k, gmax, emax)
        assert gl2 == pytest.approx(el2, rel=1e-3, abs=0), (k, gl2, el2)
        got.append(gmax)
    # second-order convergence in space (the CR column)
    ks = [r[3] for r in rows]
    cr = [math.log(got[i] / got[i + 1]) / math.log(ks[i + 1] / ks[i]) for i in range(len(ks) - 1)]
    assert all(1.9 < c < 2.5 for c in cr), cr


def test_lambda_values(orc):
    """The printed lattice numbers pin lambda = eps^2 dt / dx^2 (Sec. IV.A.1)."""
    h = 1 / 64
    for m, l1, l2 in read_golden("lambda_values.txt"):
        eps = m * math.tanh(0.9) * h / math.sqrt(2)
        assert round(orc.lam(eps, 5 * h * h, h), 4) == pytest.approx(l1, abs=1e-12)
        assert round(orc.lam(eps, 0.2, h), 4) == pytest.approx(l2, abs=1e-12)
