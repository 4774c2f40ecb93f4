"""FP64 CPU oracle for the RLB-MIE-FD Allen-Cahn time step (arXiv:2312.07010).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  It shares
no code with the CUDA path (``paper_2312_07010_gb300``) and imports nothing
from it; the product path never calls into it.

``acs_oracle.c`` holds the arithmetic (finite-difference form, collide-and-stream
form, energy, maximum norm, adjoint step); this module only marshals numpy
arrays.  ``dense`` holds the matrix (vector) form built from the paper's
D_{Delta x} matrices, for tiny grids.

Parity status of each function is recorded in the module docstrings of the
tests that pin it: every function here has at least one pin that does not go
through the oracle itself.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

_lib = None

BC_PERIODIC, BC_NEUMANN, BC_DIRICHLET = 0, 1, 2
SCHEME_RLB_MIE_FD, SCHEME_FEX_FD = 0, 1

_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.acs_oracle_cubic_root.restype = ctypes.c_double
        L.acs_oracle_cubic_root.argtypes = [ctypes.c_double, ctypes.c_double]
        L.acs_oracle_cubic_root_array.restype = None
        L.acs_oracle_cubic_root_array.argtypes = [ctypes.c_double, _dp, _dp, ctypes.c_int64]
        L.acs_oracle_step_fd.restype = ctypes.c_int
        L.acs_oracle_step_fd.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, _dp, _dp, ctypes.c_int]
        L.acs_oracle_run_fd.restype = ctypes.c_int
        L.acs_oracle_run_fd.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int64, _dp, _dp, ctypes.c_int]
        L.acs_oracle_step_lb.restype = ctypes.c_int
        L.acs_oracle_step_lb.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.acs_oracle_energy.restype = ctypes.c_double
        L.acs_oracle_energy.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, _dp]
        L.acs_oracle_maxnorm.restype = ctypes.c_double
        L.acs_oracle_maxnorm.argtypes = [ctypes.c_int, _i64p, _dp]
        L.acs_oracle_adjoint_step.restype = ctypes.c_double
        L.acs_oracle_adjoint_step.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
        L.acs_oracle_lambda.restype = ctypes.c_double
        L.acs_oracle_lambda.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.acs_oracle_numthreads.restype = ctypes.c_int
        L.acs_oracle_set_threads.restype = None
        L.acs_oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _dims_n(shape: Sequence[int]) -> Tuple[int, ctypes.Array]:
    d = len(shape)
    if d < 1 or d > 3:
        raise ValueError("dims must be 1, 2 or 3")
    arr = (ctypes.c_int64 * 3)(*(list(int(s) for s in shape) + [1] * (3 - d)))
    return d, arr


def numthreads() -> int:
    return int(lib().acs_oracle_numthreads())


def set_threads(t: int) -> None:
    lib().acs_oracle_set_threads(int(t))


def lam(eps: float, dt: float, h: float) -> float:
    """lambda = eps^2 dt / h^2 (Eq. IE-FD-vector-form: eps^2 = lambda dx^2 / dt)."""
    return float(lib().acs_oracle_lambda(eps, dt, h))


def cubic_root(dt: float, xi):
    """Unique real root of theta + (dt/2)(theta^3 - theta) = xi (Remark 1), elementwise."""
    x = _f64(np.atleast_1d(xi))
    out = np.empty_like(x)
    lib().acs_oracle_cubic_root_array(dt, _ptr(x), _ptr(out), x.size)
    return out.reshape(np.shape(xi)) if np.ndim(xi) else float(out[0])


def step_fd(phi: np.ndarray, eps: float, dt: float, h: float, bc: int,
            scheme: int = SCHEME_RLB_MIE_FD) -> np.ndarray:
    """One step of Eq. (IE-FD) (or the FEX-FD scheme of Remark 2 with scheme=1)."""
    p = _f64(phi)
    d, n = _dims_n(p.shape)
    out = np.empty_like(p)
    rc = lib().acs_oracle_step_fd(d, n, bc, lam(eps, dt, h), dt, _ptr(p), _ptr(out), scheme)
    if rc:
        raise ValueError(f"oracle step_fd failed ({rc})")
    return out


def run_fd(phi: np.ndarray, eps: float, dt: float, h: float, bc: int, steps: int,
           scheme: int = SCHEME_RLB_MIE_FD) -> np.ndarray:
    """``steps`` applications of step_fd (a fresh array is returned)."""
    p = _f64(phi).copy()
    d, n = _dims_n(p.shape)
    tmp = np.empty_like(p)
    rc = lib().acs_oracle_run_fd(d, n, bc, lam(eps, dt, h), dt, int(steps), _ptr(p), _ptr(tmp),
                                 scheme)
    if rc:
        raise ValueError(f"oracle run_fd failed ({rc})")
    return p


def step_lb(phi: np.ndarray, eps: float, dt: float, h: float, bc: int,
            omega1: Optional[float] = None) -> np.ndarray:
    """One collide-and-stream step of the regularized LB form (Eqs. fieq-Fi, fneq, RLB, pine)."""
    p = _f64(phi)
    d, n = _dims_n(p.shape)
    w1 = {1: 1 / 3, 2: 1 / 5, 3: 1 / 6}[d] if omega1 is None else omega1
    out = np.empty_like(p)
    rc = lib().acs_oracle_step_lb(d, n, bc, eps, dt, h, w1, _ptr(p), _ptr(out))
    if rc:
        raise ValueError(f"oracle step_lb failed ({rc})")
    return out


def energy(phi: np.ndarray, eps: float, dt: float, h: float, bc: int) -> float:
    """Discrete free energy of Theorem 3, Eq. (proof2-eq0)."""
    p = _f64(phi)
    d, n = _dims_n(p.shape)
    return float(lib().acs_oracle_energy(d, n, bc, lam(eps, dt, h), dt, h, _ptr(p)))


def maxnorm(phi: np.ndarray) -> float:
    p = _f64(phi)
    d, n = _dims_n(p.shape)
    return float(lib().acs_oracle_maxnorm(d, n, _ptr(p)))


def phase_volume(phi: np.ndarray, h: float) -> float:
    """Volume of the phase phi > 0 measured as h^d sum (1 + phi)/2 (the radius of Sec. IV.B.2's
    shrinking circle / sphere follows from it); math.fsum makes the sum exact before rounding."""
    p = _f64(phi)
    return float(h ** p.ndim * math.fsum(((1.0 + p) / 2.0).ravel()))


def adjoint_step(phi_n: np.ndarray, phi_np1: np.ndarray, adj_np1: np.ndarray, eps: float,
                 dt: float, h: float, bc: int) -> Tuple[np.ndarray, float]:
    """(dL/dphi^n, this step's dL/d(eps^2)) from dL/dphi^{n+1} for one step of Eq. (IE-FD)."""
    a = _f64(phi_n)
    b = _f64(phi_np1)
    g = _f64(adj_np1)
    d, n = _dims_n(a.shape)
    out = np.empty_like(a)
    mu = np.empty_like(a)
    ge = lib().acs_oracle_adjoint_step(d, n, bc, lam(eps, dt, h), dt, h, _ptr(a), _ptr(b),
                                       _ptr(g), _ptr(out), _ptr(mu))
    return out, float(ge)


def grad(phi0: np.ndarray, eps: float, dt: float, h: float, bc: int, steps: int,
         dL_dphiT: np.ndarray, checkpoint_every: int = 0) -> Tuple[np.ndarray, float]:
    """(dL/dphi0, dL/d(eps^2)) of a terminal loss after ``steps`` steps.

    Forward states are kept every ``checkpoint_every`` steps (all of them when 0)
    and each segment is recomputed before its backward sweep.
    """
    C = steps if checkpoint_every <= 0 else int(checkpoint_every)
    C = max(1, C)
    ckpt = {}
    cur = _f64(phi0).copy()
    for s0 in range(0, steps, C):
        ckpt[s0] = cur
        cur = run_fd(cur, eps, dt, h, bc, min(C, steps - s0))
    adj = _f64(dL_dphiT).copy()
    ge_total = 0.0
    seg_starts = sorted(ckpt)
    for s0 in reversed(seg_starts):
        s1 = min(s0 + C, steps)
        states = [ckpt[s0]]
        for _ in range(s1 - s0):
            states.append(step_fd(states[-1], eps, dt, h, bc))
        for k in range(s1 - s0 - 1, -1, -1):
            adj, ge = adjoint_step(states[k], states[k + 1], adj, eps, dt, h, bc)
            ge_total += ge
    return adj, ge_total
