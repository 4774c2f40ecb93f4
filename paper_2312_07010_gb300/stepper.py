"""Python front end of libacs: device memory and streams from PyTorch, compute in CUDA.

``AllenCahn`` wraps one ``acs_ctx`` (include/acs.h): it allocates the state and the
work buffer as torch tensors on the GPU, binds them with the current CUDA stream,
and forwards every call to the C ABI.  ``AllenCahnFunction`` is the
``torch.autograd.Function`` whose backward is the library's hand-written adjoint.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from ._lib import (ACS_F32, ACS_F64, ACS_KERNEL_AUTO, ACS_KERNEL_LB, AcsError, check, lib)

_DT = {"f32": (ACS_F32, torch.float32, np.float32), "f64": (ACS_F64, torch.float64, np.float64)}


def dt_max(dims: int, eps: float, h: float) -> Tuple[float, float]:
    """(dt bound of Theorem 2, dt bound of Theorem 3) -- acs_dt_max."""
    a = ctypes.c_double()
    b = ctypes.c_double()
    check(lib().acs_dt_max(dims, eps, h, ctypes.byref(a), ctypes.byref(b)), "acs_dt_max")
    return a.value, b.value


class AllenCahn:
    """One Allen-Cahn problem on an n[0] x ... x n[d-1] grid (last axis fastest).

    shape  grid shape (d = len(shape) in 1..3); eps, dt, h, bc as in acs_create;
    dtype  "f32" or "f64".
    """

    def __init__(self, shape: Sequence[int], eps: float, dt: float, h: float, bc: int,
                 dtype: str = "f32", device: Optional[torch.device] = None,
                 stream: Optional[torch.cuda.Stream] = None):
        self.L = lib()
        self.shape = tuple(int(s) for s in shape)
        self.dims = len(self.shape)
        self.eps, self.dt, self.h, self.bc = float(eps), float(dt), float(h), int(bc)
        self.dtype_name = dtype
        code, self.tdtype, self.ndtype = _DT[dtype]
        n = (ctypes.c_int64 * 3)(*(list(self.shape) + [1] * (3 - self.dims)))
        ctx = ctypes.c_void_p()
        rc = self.L.acs_create(self.dims, n, self.eps, self.dt, self.h, self.bc, code, ctypes.byref(ctx))
        self.create_status = check(rc, "acs_create")
        self.ctx = ctx
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        self.phi = torch.empty(self.shape, dtype=self.tdtype, device=self.device)
        wb = int(self.L.acs_work_bytes(self.ctx))
        self.work = torch.empty(wb, dtype=torch.uint8, device=self.device)
        check(self.L.acs_bind(self.ctx, ctypes.c_void_p(self.phi.data_ptr()),
                              ctypes.c_void_p(self.work.data_ptr()), wb,
                              ctypes.c_void_p(self.stream.cuda_stream)), "acs_bind")
        self._grad_buf = None

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.L.acs_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def numel(self) -> int:
        return int(np.prod(self.shape))

    # ------------------------------------------------------------------ state
    def set_state(self, phi0) -> None:
        """Initial state from a CUDA tensor or a host array (numpy / CPU tensor)."""
        if isinstance(phi0, torch.Tensor) and phi0.is_cuda:
            t = phi0.to(self.tdtype).contiguous()
            if tuple(t.shape) != self.shape:
                raise ValueError(f"shape {tuple(t.shape)} != {self.shape}")
            check(self.L.acs_set_state(self.ctx, ctypes.c_void_p(t.data_ptr())), "acs_set_state")
            if t.data_ptr() != self.phi.data_ptr():
                self._keep = t  # alive until the stream has copied it
            return
        a = np.ascontiguousarray(np.asarray(phi0, dtype=self.ndtype))
        if a.shape != self.shape:
            raise ValueError(f"shape {a.shape} != {self.shape}")
        check(self.L.acs_set_state_host(self.ctx, ctypes.c_void_p(a.ctypes.data)), "acs_set_state_host")
        self.sync()

    def set_state_host(self, host: torch.Tensor) -> None:
        """acs_set_state_host from a (preferably pinned) CPU tensor; asynchronous for pinned memory."""
        check(self.L.acs_set_state_host(self.ctx, ctypes.c_void_p(host.data_ptr())), "acs_set_state_host")

    def get_state_host(self, out: torch.Tensor) -> None:
        """acs_get_state_host into a CPU tensor of the state's shape and dtype (synchronizes)."""
        check(self.L.acs_get_state_host(self.ctx, ctypes.c_void_p(out.data_ptr())), "acs_get_state_host")

    def state(self) -> torch.Tensor:
        """The bound state tensor (valid after the stream has reached this point)."""
        return self.phi

    def numpy(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=self.ndtype)
        check(self.L.acs_get_state_host(self.ctx, ctypes.c_void_p(out.ctypes.data)), "acs_get_state_host")
        return out

    # ------------------------------------------------------------------ stepping
    def set_kernel(self, kernel: int, depth: int = 1) -> None:
        check(self.L.acs_set_kernel(self.ctx, int(kernel), int(depth)), "acs_set_kernel")

    def get_kernel(self) -> Tuple[int, int]:
        k = ctypes.c_int()
        d = ctypes.c_int()
        check(self.L.acs_get_kernel(self.ctx, ctypes.byref(k), ctypes.byref(d)), "acs_get_kernel")
        return k.value, d.value

    def use_lb_form(self, omega1: float = 0.0) -> None:
        """Step with the collide-and-stream population form (acs_lb_bind + ACS_KERNEL_LB):
        allocates the (2d+1) population arrays; omega1 = 0 takes the paper's weight."""
        nb = int(self.L.acs_lb_bytes(self.ctx))
        self._pop = torch.empty(nb, dtype=torch.uint8, device=self.device)
        check(self.L.acs_lb_bind(self.ctx, ctypes.c_void_p(self._pop.data_ptr()), nb, float(omega1)), "acs_lb_bind")
        self.set_kernel(ACS_KERNEL_LB)

    def set_scheme(self, scheme: int) -> None:
        check(self.L.acs_set_scheme(self.ctx, int(scheme)), "acs_set_scheme")

    def step(self, n: int = 1) -> None:
        check(self.L.acs_step(self.ctx, int(n)), "acs_step")

    @property
    def steps_done(self) -> int:
        return int(self.L.acs_steps_done(self.ctx))

    def sync(self) -> None:
        check(self.L.acs_sync(self.ctx), "acs_sync")

    # ------------------------------------------------------------------ reductions
    def energy(self, allow_nonfinite: bool = False) -> float:
        v = ctypes.c_double()
        rc = self.L.acs_energy(self.ctx, ctypes.byref(v))
        if not (allow_nonfinite and rc == -5):
            check(rc, "acs_energy")
        return v.value

    def maxnorm(self, allow_nonfinite: bool = False) -> float:
        v = ctypes.c_double()
        rc = self.L.acs_maxnorm(self.ctx, ctypes.byref(v))
        if not (allow_nonfinite and rc == -5):
            check(rc, "acs_maxnorm")
        return v.value

    def phase_volume(self) -> float:
        """h^d sum (1 + phi) / 2: the volume of the phase phi > 0 (acs_phase_volume)."""
        v = ctypes.c_double()
        check(self.L.acs_phase_volume(self.ctx, ctypes.byref(v)), "acs_phase_volume")
        return v.value

    def observe_async(self, out2: torch.Tensor) -> None:
        """{E_h, max|phi|} into a 2-element float64 CUDA tensor, no synchronization."""
        check(self.L.acs_observe_async(self.ctx, ctypes.c_void_p(out2.data_ptr())), "acs_observe_async")

    def run_logged(self, n_steps: int, every: int) -> Tuple[np.ndarray, np.ndarray]:
        m = n_steps // every + 1
        e = np.empty(m)
        x = np.empty(m)
        dp = ctypes.POINTER(ctypes.c_double)
        check(self.L.acs_run_logged(self.ctx, int(n_steps), int(every), e.ctypes.data_as(dp),
                                    x.ctypes.data_as(dp)), "acs_run_logged")
        return e, x

    # ------------------------------------------------------------------ adjoint
    def record_for_grad(self, max_steps: int, every: int) -> None:
        """Enable checkpoint recording from the current state (acs_grad_bind)."""
        nb = int(self.L.acs_grad_work_bytes(self.ctx, int(max_steps), int(every)))
        self._grad_buf = torch.empty(nb, dtype=torch.uint8, device=self.device)
        check(self.L.acs_grad_bind(self.ctx, ctypes.c_void_p(self._grad_buf.data_ptr()), nb, int(max_steps),
                                   int(every)), "acs_grad_bind")

    def grad(self, dL_dphiT: torch.Tensor) -> Tuple[torch.Tensor, float]:
        """(dL/dphi0, dL/d(eps^2)) for the recorded steps, given dL/dphi_T."""
        g = dL_dphiT.to(self.tdtype).contiguous()
        out = torch.empty_like(g)
        ge = ctypes.c_double()
        check(self.L.acs_grad(self.ctx, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                              ctypes.byref(ge)), "acs_grad")
        return out, ge.value


class AllenCahnFunction(torch.autograd.Function):
    """phi_T = S^steps(phi0; eps^2): differentiable in phi0 and eps^2 (dt, h fixed).

    forward(phi0, eps2, steps, dt, h, bc, checkpoint_every) runs the CUDA stepper
    with checkpoint recording; backward runs the hand-written adjoint (acs_grad).
    checkpoint_every = 1 stores every state (steps + 1 of them) and the backward pass
    recomputes nothing; larger values trade memory for one recomputed forward.
    """

    @staticmethod
    def forward(ctx, phi0: torch.Tensor, eps2: torch.Tensor, steps: int, dt: float, h: float, bc: int,
                checkpoint_every: int = 50):
        dtype = "f64" if phi0.dtype == torch.float64 else "f32"
        solver = AllenCahn(tuple(phi0.shape), math.sqrt(float(eps2)), dt, h, bc, dtype, device=phi0.device)
        solver.set_state(phi0.detach())
        solver.record_for_grad(max(1, int(steps)), int(checkpoint_every))
        solver.step(int(steps))
        ctx.solver = solver
        ctx.eps2_dtype = eps2.dtype
        return solver.phi.clone()

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        solver = ctx.solver
        g0, ge = solver.grad(grad_out.contiguous())
        geps = torch.tensor(ge, dtype=ctx.eps2_dtype, device=grad_out.device)
        ctx.solver = None
        solver.close()
        return g0, geps, None, None, None, None, None


def allen_cahn(phi0: torch.Tensor, eps2: torch.Tensor, steps: int, dt: float, h: float, bc: int,
               checkpoint_every: int = 50) -> torch.Tensor:
    return AllenCahnFunction.apply(phi0, eps2, steps, dt, h, bc, checkpoint_every)
