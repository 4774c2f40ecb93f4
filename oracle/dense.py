"""Matrix (vector) form of the RLB-MIE-FD step for tiny grids (test infrastructure).

Eq. (IE-FD-vector-form):
    (Phi^{n+1} - Phi^n)/dt + ((Phi^{n+1})^.3 + (Phi^n)^.3)/2 - (Phi^{n+1} + Phi^n)/2
        = eps^2 Lambda_{dx} Phi^n,
with Lambda_{dx} the Kronecker sum of the one-dimensional matrices D_{dx} of
Eq. (Ddeltax), written out entry by entry here as the paper prints them (the
Neumann matrix with -1 in its two corner diagonal entries, the Dirichlet matrix
with -2 everywhere on the diagonal, the periodic matrix with the two wrap-around
ones).  Phi is ordered with the last index fastest, so for d = 3
Lambda = D (x) I (x) I + I (x) D (x) I + I (x) I (x) D (the paper's d = 3 line
repeats the I (x) I (x) D term; the Kronecker sum is meant).

The cubic of each node is solved with ``numpy.roots`` (the real root), a
library routine independent of the C oracle's Newton iteration.
Nothing here is shared with, or called by, the CUDA path.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

BC_PERIODIC, BC_NEUMANN, BC_DIRICHLET = 0, 1, 2


def D_matrix(m: int, h: float, bc: int) -> np.ndarray:
    """The m x m matrix D_{dx} of Eq. (Ddeltax) for one axis with m unknowns."""
    D = np.zeros((m, m))
    for i in range(m):
        D[i, i] = -2.0
        if i > 0:
            D[i, i - 1] = 1.0
        if i < m - 1:
            D[i, i + 1] = 1.0
    if bc == BC_NEUMANN:
        D[0, 0] += 1.0
        D[m - 1, m - 1] += 1.0
    elif bc == BC_PERIODIC:
        D[0, m - 1] += 1.0
        D[m - 1, 0] += 1.0
    elif bc != BC_DIRICHLET:
        raise ValueError(bc)
    return D / (h * h)


def Lambda_matrix(shape: Sequence[int], h: float, bc: int) -> np.ndarray:
    """Kronecker sum of the per-axis D matrices (C order: last axis fastest)."""
    shape = [int(s) for s in shape]
    total = int(np.prod(shape))
    L = np.zeros((total, total))
    for k in range(len(shape)):
        mats = [np.eye(s) for s in shape]
        mats[k] = D_matrix(shape[k], h, bc)
        term = mats[0]
        for m in mats[1:]:
            term = np.kron(term, m)
        L += term
    return L


def real_root(a3: float, a1: float, c0: float) -> float:
    """The real root of a3 t^3 + a1 t - c0 with a3 >= 0, a1 > 0 (unique: the derivative is > 0)."""
    if a3 == 0.0:
        return c0 / a1
    r = np.roots([a3, 0.0, a1, -c0])
    real = r[np.argmin(np.abs(r.imag))].real
    return float(real)


def step(phi: np.ndarray, eps: float, dt: float, h: float, bc: int) -> np.ndarray:
    """One step of Eq. (IE-FD-vector-form): solve per node
    Phi' + dt/2 (Phi'^3 - Phi') = Phi - dt/2 (Phi^3 - Phi) + dt eps^2 Lambda Phi."""
    shape = phi.shape
    P = np.asarray(phi, dtype=np.float64).reshape(-1)
    L = Lambda_matrix(shape, h, bc)
    rhs = P - 0.5 * dt * (P ** 3 - P) + dt * eps * eps * (L @ P)
    out = np.array([real_root(0.5 * dt, 1.0 - 0.5 * dt, r) for r in rhs])
    return out.reshape(shape)


def energy(phi: np.ndarray, eps: float, dt: float, h: float, bc: int) -> float:
    """Eq. (proof2-eq0) with the explicit matrix: dx^d [1/4 sum (phi^2-1)^2 - lambda/(2 dt) Phi^T Lambda Phi],
    Lambda = dx^2 Lambda_{dx}, lambda = eps^2 dt / dx^2."""
    P = np.asarray(phi, dtype=np.float64).reshape(-1)
    d = phi.ndim
    lam = eps * eps * dt / (h * h)
    Lam = (h * h) * Lambda_matrix(phi.shape, h, bc)
    return float(h ** d * (0.25 * np.sum((P * P - 1.0) ** 2) - lam / (2.0 * dt) * (P @ Lam @ P)))


def jacobian(phi_n: np.ndarray, phi_np1: np.ndarray, eps: float, dt: float, h: float,
             bc: int) -> np.ndarray:
    """d Phi^{n+1} / d Phi^n by implicit differentiation of the vector form:
    diag(1 + dt/2 (3 Phi'^2 - 1)) dPhi' = (diag(1 - dt/2 (3 Phi^2 - 1)) + dt eps^2 Lambda) dPhi."""
    P = np.asarray(phi_n, dtype=np.float64).reshape(-1)
    Q = np.asarray(phi_np1, dtype=np.float64).reshape(-1)
    L = Lambda_matrix(phi_n.shape, h, bc)
    right = np.diag(1.0 - 0.5 * dt * (3 * P * P - 1.0)) + dt * eps * eps * L
    left = 1.0 + 0.5 * dt * (3 * Q * Q - 1.0)
    return right / left[:, None]


def d_step_d_eps2(phi_n: np.ndarray, phi_np1: np.ndarray, dt: float, h: float, bc: int) -> np.ndarray:
    """d Phi^{n+1} / d(eps^2) with dt, dx fixed: dt Lambda Phi^n / (1 + dt/2 (3 Phi'^2 - 1))."""
    P = np.asarray(phi_n, dtype=np.float64).reshape(-1)
    Q = np.asarray(phi_np1, dtype=np.float64).reshape(-1)
    L = Lambda_matrix(phi_n.shape, h, bc)
    return (dt * (L @ P)) / (1.0 + 0.5 * dt * (3 * Q * Q - 1.0))
