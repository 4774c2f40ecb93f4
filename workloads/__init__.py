"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the time step itself: it only draws initial
fields and lists the workload parameters (grid, boundary, interfacial parameter,
step size, step count).  Both the CPU oracle and the CUDA path consume what it
returns; neither is imported here.

Workloads follow the paper's problem statement (Sec. I, Eq. ACE: phi_t =
eps^2 lap(phi) - f(phi) on a hypercube with periodic, homogeneous Neumann or
homogeneous Dirichlet boundaries) at the sizes of the five benchmark cases:

  * ``cfg1_2d_periodic_128``  2D, 128^2, periodic, h = 1/128, eps = 0.02,
    phi0 ~ U[-0.9, 0.9] (seed 0), FP64, 1000 steps, E_h and max-norm every 10.
  * ``cfg2_3d_neumann_512``   3D, 512^3, Neumann, h = 1/512, eps = 0.01,
    phi0 ~ U[-1, 1] (seed 1), FP32 (and FP64), 200 steps.
  * ``cfg3_2d_dirichlet_4096`` 2D, 4096^2, Dirichlet, h = 2/4097, eps = 0.005,
    star-shaped interface, FP32 and FP64, 2000 steps, energy every 50.
  * ``cfg4_batched_256``      256 independent 2D instances (seed 2).
  * ``cfg5_adjoint_1024``     2D, 1024^2, periodic, h = 1/1024, eps = 0.01,
    phi0 ~ U[-0.5, 0.5] (seed 3), 500 steps, checkpoints every 50.

Step-size rule (the paper gives none for these cases): 90 % of the tighter of
the maximum-principle bound dt <= 1 - 2 d lambda (Theorem 2, Eq.
maximum-condition) and the relaxation requirement s > 1, i.e. lambda < omega1,
with lambda = eps^2 dt / h^2 and the paper's weights omega1 = 1/3, 1/5, 1/6 for
d = 1, 2, 3 (Sec. IV, first paragraph).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

BC_PERIODIC = 0
BC_NEUMANN = 1
BC_DIRICHLET = 2
BC_NAMES = {BC_PERIODIC: "periodic", BC_NEUMANN: "neumann", BC_DIRICHLET: "dirichlet"}

# Lattice weights used in the paper's experiments (Sec. IV): omega1 per dimension.
PAPER_OMEGA1 = {1: 1.0 / 3.0, 2: 1.0 / 5.0, 3: 1.0 / 6.0}


def dt_rule(dims: int, eps: float, h: float, safety: float = 0.9,
            omega1: Optional[float] = None) -> float:
    """Step size: ``safety`` times the tighter of the maximum-principle bound and s > 1.

    Theorem 2: dt <= 1 - 2 d lambda with lambda = eps^2 dt / h^2, i.e.
    dt <= 1 / (1 + 2 d eps^2 / h^2); and s = omega1 / lambda > 1, i.e.
    dt < omega1 h^2 / eps^2.
    """
    w1 = PAPER_OMEGA1[dims] if omega1 is None else omega1
    r = eps * eps / (h * h)
    return safety * min(1.0 / (1.0 + 2.0 * dims * r), w1 / r)


def uniform_field(shape: Tuple[int, ...], lo: float, hi: float, seed: int) -> np.ndarray:
    """i.i.d. uniform initial field, float64, C order (last index fastest)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=tuple(int(s) for s in shape))


def node_coords(n: int, h: float, x0: float) -> np.ndarray:
    """Node positions x_i = x0 + i h, i = 0..n-1."""
    return x0 + h * np.arange(n, dtype=np.float64)


def star_field(n: int, h: float, eps: float) -> np.ndarray:
    """Star-shaped interface on [-1, 1]^2 with Dirichlet nodes x_i = -1 + (i+1) h.

    phi0 = tanh((0.5 + 0.1 cos(6 theta) - r) / (sqrt(2) eps)); axis 1 (fastest) is x,
    axis 0 is y.
    """
    c = node_coords(n, h, -1.0 + h)
    y, x = np.meshgrid(c, c, indexing="ij")
    r = np.sqrt(x * x + y * y)
    th = np.arctan2(y, x)
    return np.tanh((0.5 + 0.1 * np.cos(6.0 * th) - r) / (math.sqrt(2.0) * eps))


def tanh_disc(n: int, h: float, eps: float, radius: float = 0.3,
              center: Tuple[float, float] = (0.5, 0.5)) -> np.ndarray:
    """Disc target tanh((R - |x - c|) / (sqrt(2) eps)) on the periodic nodes x_i = i h."""
    c = node_coords(n, h, 0.0)
    y, x = np.meshgrid(c, c, indexing="ij")
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2)
    return np.tanh((radius - r) / (math.sqrt(2.0) * eps))


@dataclass
class Workload:
    """One stepping problem: grid, boundary, parameters and how phi0 is drawn."""
    name: str
    dims: int
    n: Tuple[int, ...]
    h: float
    eps: float
    dt: float
    bc: int
    steps: int
    dtype: str                      # "f32" or "f64"
    init: str = "uniform"           # "uniform", "star", "tanh_disc"
    lo: float = -1.0
    hi: float = 1.0
    seed: int = 0
    log_every: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def numel(self) -> int:
        return int(np.prod(self.n))

    def phi0(self) -> np.ndarray:
        """float64 initial field (cast to float32 by FP32 users)."""
        if self.init == "uniform":
            return uniform_field(self.n, self.lo, self.hi, self.seed)
        if self.init == "star":
            return star_field(self.n[0], self.h, self.eps)
        if self.init == "tanh_disc":
            return tanh_disc(self.n[0], self.h, self.eps)
        raise ValueError(self.init)

    def scaled(self, n: int, steps: Optional[int] = None) -> "Workload":
        """Same recipe on a smaller grid n^d (h scaled so the domain is kept)."""
        L = self.h * (self.n[0] + (1 if self.bc == BC_DIRICHLET else 0))
        hn = L / (n + (1 if self.bc == BC_DIRICHLET else 0))
        w = Workload(self.name + f"_n{n}", self.dims, (n,) * self.dims, hn, self.eps,
                     dt_rule(self.dims, self.eps, hn), self.bc,
                     self.steps if steps is None else steps, self.dtype, self.init,
                     self.lo, self.hi, self.seed, self.log_every, dict(self.extra))
        return w


def cfg1() -> Workload:
    h = 1.0 / 128
    return Workload("cfg1_2d_periodic_128", 2, (128, 128), h, 0.02, dt_rule(2, 0.02, h),
                    BC_PERIODIC, 1000, "f64", "uniform", -0.9, 0.9, 0, 10)


def cfg2(dtype: str = "f32") -> Workload:
    h = 1.0 / 512
    return Workload("cfg2_3d_neumann_512", 3, (512, 512, 512), h, 0.01, dt_rule(3, 0.01, h),
                    BC_NEUMANN, 200, dtype, "uniform", -1.0, 1.0, 1, 50)


def cfg3(dtype: str = "f32") -> Workload:
    h = 2.0 / 4097
    return Workload("cfg3_2d_dirichlet_4096", 2, (4096, 4096), h, 0.005, dt_rule(2, 0.005, h),
                    BC_DIRICHLET, 2000, dtype, "star", seed=0, log_every=50)


def cfg5() -> Workload:
    h = 1.0 / 1024
    return Workload("cfg5_adjoint_1024", 2, (1024, 1024), h, 0.01, dt_rule(2, 0.01, h),
                    BC_PERIODIC, 500, "f32", "uniform", -0.5, 0.5, 3, 0,
                    {"checkpoint_every": 50, "target": "tanh_disc", "radius": 0.3})


def adjoint_target(w: Workload) -> np.ndarray:
    return tanh_disc(w.n[0], w.h, w.eps, w.extra.get("radius", 0.3))


@dataclass
class BatchInstance:
    n: int
    h: float
    eps: float
    dt: float
    bc: int
    seed: int

    def phi0(self) -> np.ndarray:
        return uniform_field((self.n, self.n), -1.0, 1.0, self.seed)


def batched_instances(count: int = 256, seed: int = 2, n_lo: int = 64, n_hi: int = 1024,
                      steps: int = 500) -> List[BatchInstance]:
    """Instances of the batched workload: side log-uniform in [n_lo, n_hi],
    eps ~ U[0.005, 0.03], boundary uniform over {periodic, Neumann, Dirichlet}.

    Unit square: h = 1/n (periodic, Neumann) or 1/(n+1) (Dirichlet interior nodes).
    Each instance's phi0 ~ U[-1, 1] is drawn from its own seed (seed*100003 + index).
    """
    rng = np.random.default_rng(seed)
    sides = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))
    sides = np.clip(np.rint(sides).astype(np.int64), n_lo, n_hi)
    epss = rng.uniform(0.005, 0.03, size=count)
    bcs = rng.integers(0, 3, size=count)
    out = []
    for i in range(count):
        n = int(sides[i])
        bc = int(bcs[i])
        h = 1.0 / (n + 1) if bc == BC_DIRICHLET else 1.0 / n
        eps = float(epss[i])
        out.append(BatchInstance(n, h, eps, dt_rule(2, eps, h), bc, seed * 100003 + i))
    return out


BATCH_STEPS = 500


@dataclass
class LineInstance:
    n: int
    h: float
    eps: float
    dt: float
    bc: int
    seed: int

    def phi0(self) -> np.ndarray:
        return uniform_field((self.n,), -1.0, 1.0, self.seed)


def line_instances(count: int = 4096, seed: int = 4, n_lo: int = 32, n_hi: int = 4096) -> List[LineInstance]:
    """Lines of the batched 1D workload: length log-uniform in [n_lo, n_hi], eps ~
    U[0.005, 0.03], boundary uniform over {periodic, Neumann, Dirichlet} on the unit
    interval (h = 1/n, or 1/(n+1) for Dirichlet interior nodes); phi0 ~ U[-1, 1] from
    the line's own seed (seed*100003 + index); dt by dt_rule for d = 1."""
    rng = np.random.default_rng(seed)
    sides = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))
    sides = np.clip(np.rint(sides).astype(np.int64), n_lo, n_hi)
    epss = rng.uniform(0.005, 0.03, size=count)
    bcs = rng.integers(0, 3, size=count)
    out = []
    for i in range(count):
        n = int(sides[i])
        bc = int(bcs[i])
        h = 1.0 / (n + 1) if bc == BC_DIRICHLET else 1.0 / n
        eps = float(epss[i])
        out.append(LineInstance(n, h, eps, dt_rule(1, eps, h), bc, seed * 100003 + i))
    return out


LINE_STEPS = 2000
