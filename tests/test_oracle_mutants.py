"""Planted mistakes in the oracle must fail its pins (CPU only).

Each case copies ``oracle/acs_oracle.c``, plants one plausible mistake (a
dropped term, a flipped sign, a wrong ghost rule, a wrong coefficient), builds
it into a temporary library and checks that at least one independent pin --
the dense vector form of Eq. (IE-FD-vector-form) or Table 2's first row --
rejects it.  The mutants live only in a temporary directory.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
import oracle.dense as dense
from conftest import read_golden

SRC = os.path.join(os.path.dirname(oracle.__file__), "acs_oracle.c")

MUTANTS = {
    "reaction_sign": ("const double xi = p + lam * lap - a * f;",
                      "const double xi = p + lam * lap + a * f;"),
    "drop_center_term": ("orc_nbr(phi, g, c, idx, k, -1, bc) - 2.0 * phi[idx];",
                         "orc_nbr(phi, g, c, idx, k, -1, bc) - 1.0 * phi[idx];"),
    "neumann_ghost_zero": ("if (bc == ORC_BC_NEUMANN) return phi[idx];",
                           "if (bc == ORC_BC_NEUMANN) return 0.0;"),
    "periodic_wrap_off_by_one": ("int64_t jw = (j < 0) ? j + g->n[k] : j - g->n[k];",
                                 "int64_t jw = (j < 0) ? j + g->n[k] - 1 : j - g->n[k];"),
    "implicit_half_dt": ("const double a = 0.5 * dt;\n    const double b = 1.0 - a;",
                         "const double a = dt;\n    const double b = 1.0 - a;"),
}


def _build_mutant(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", str(path),
                    "-o", str(lib), "-lm"], check=True, capture_output=True)
    L = ctypes.CDLL(str(lib))
    dp = ctypes.POINTER(ctypes.c_double)
    L.acs_oracle_step_fd.restype = ctypes.c_int
    L.acs_oracle_step_fd.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int]
    return L


def _step(L, phi, eps, dt, h, bc):
    p = np.ascontiguousarray(phi, dtype=np.float64)
    out = np.empty_like(p)
    n = (ctypes.c_int64 * 3)(*(list(p.shape) + [1] * (3 - p.ndim)))
    dp = ctypes.POINTER(ctypes.c_double)
    L.acs_oracle_step_fd(p.ndim, n, bc, eps * eps * dt / (h * h), dt, p.ctypes.data_as(dp),
                         out.ctypes.data_as(dp), 0)
    return out


def _pins_pass(L):
    rng = np.random.default_rng(1)
    for bc in (0, 1, 2):
        phi = rng.uniform(-1, 1, (5, 4))
        h, eps, dt = 0.1, 0.05, 0.5
        if not np.allclose(_step(L, phi, eps, dt, h, bc), dense.step(phi, eps, dt, h, bc),
                           rtol=0, atol=2e-14):
            return False
    # Table 2, first row
    inv_dx, emax, _ = read_golden("table2_traveling_wave_1d.txt")[0]
    eps = math.tanh(0.9) / (16 * math.sqrt(2))
    se = 3 * eps / math.sqrt(2)
    h = 1 / inv_dx
    dt = 5 * h * h
    x = -0.5 + h * np.arange(round(3 / h) + 1)
    phi = 0.5 * (1 - np.tanh(x / (2 * math.sqrt(2) * eps)))
    for _ in range(math.floor(1 / se / dt)):
        phi = _step(L, phi, eps, dt, h, 1)
    exact = 0.5 * (1 - np.tanh((x - 1 / se * se) / (2 * math.sqrt(2) * eps)))
    return abs(float(np.abs(phi - exact).max()) - emax) <= 6e-5 * emax


def test_unmutated_copy_passes(tmp_path):
    src = open(SRC).read()
    path = tmp_path / "same.c"
    path.write_text(src)
    lib = tmp_path / "libsame.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", str(path),
                    "-o", str(lib), "-lm"], check=True, capture_output=True)
    L = ctypes.CDLL(str(lib))
    dp = ctypes.POINTER(ctypes.c_double)
    L.acs_oracle_step_fd.restype = ctypes.c_int
    L.acs_oracle_step_fd.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int]
    assert _pins_pass(L)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    assert not _pins_pass(_build_mutant(tmp_path, name))
