"""Pipelined host-to-host runs (``acs_pipe_*`` in include/acs.h).

``Pipeline`` runs a stream of independent jobs -- host phi^0 in, ``steps`` steps with
E_h / max|phi| logged every ``every`` steps, host phi^N out -- on ``slots`` (2 to 4)
device states taken in turn, so each job's copies overlap its neighbours' compute.  Results equal
``AllenCahn.set_state_host`` + ``run_logged`` + ``get_state_host`` bit for bit.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import numpy as np
import torch

from ._lib import check, lib
from .stepper import _DT


class Pipeline:
    """shape, eps, dt, h, bc, dtype as for ``AllenCahn``; ``stream`` runs the steps."""

    def __init__(self, shape: Sequence[int], eps: float, dt: float, h: float, bc: int,
                 dtype: str = "f32", slots: int = 3, device: Optional[torch.device] = None,
                 stream: Optional[torch.cuda.Stream] = None):
        self.L = lib()
        self.shape = tuple(int(s) for s in shape)
        self.dims = len(self.shape)
        code, self.tdtype, self.ndtype = _DT[dtype]
        n = (ctypes.c_int64 * 3)(*(list(self.shape) + [1] * (3 - self.dims)))
        p = ctypes.c_void_p()
        self.create_status = check(self.L.acs_pipe_create(self.dims, n, float(eps), float(dt), float(h), int(bc),
                                                          code, int(slots), ctypes.byref(p)), "acs_pipe_create")
        self.slots = int(slots)
        self.p = p
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        nb = int(self.L.acs_pipe_bytes(self.p))
        self.buf = torch.empty(nb, dtype=torch.uint8, device=self.device)
        check(self.L.acs_pipe_bind(self.p, ctypes.c_void_p(self.buf.data_ptr()), nb,
                                   ctypes.c_void_p(self.stream.cuda_stream)), "acs_pipe_bind")
        self._held: List[object] = []

    def context(self, slot: int) -> ctypes.c_void_p:
        """The acs_ctx of a slot (for acs_set_kernel / acs_set_scheme on every slot)."""
        return ctypes.c_void_p(self.L.acs_pipe_context(self.p, int(slot)))

    def host_buffer(self) -> torch.Tensor:
        """A page-locked CPU tensor of the state's shape and dtype."""
        return torch.empty(self.shape, dtype=self.tdtype).pin_memory()

    def log_buffer(self, steps: int, every: int) -> torch.Tensor:
        """A page-locked (steps // every + 1, 2) float64 tensor for {E_h, max|phi|}."""
        return torch.empty((steps // every + 1, 2), dtype=torch.float64).pin_memory()

    def submit(self, h_in: torch.Tensor, h_out: torch.Tensor, steps: int, every: int = 0,
               log: Optional[torch.Tensor] = None) -> None:
        """Enqueue one job (returns at once); the buffers are held until ``wait``."""
        for t in (h_in, h_out):
            if t.device.type != "cpu" or t.dtype != self.tdtype or tuple(t.shape) != self.shape \
                    or not t.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU tensors of the state's shape and dtype")
        lp = None
        if every > 0:
            if log is None or log.dtype != torch.float64 or log.numel() < 2 * (steps // every + 1) \
                    or log.device.type != "cpu" or not log.is_contiguous():
                raise ValueError("every > 0 needs a contiguous float64 CPU log of 2 (steps // every + 1) values")
            lp = ctypes.cast(ctypes.c_void_p(log.data_ptr()), ctypes.POINTER(ctypes.c_double))
        check(self.L.acs_pipe_submit(self.p, ctypes.c_void_p(h_in.data_ptr()), ctypes.c_void_p(h_out.data_ptr()),
                                     int(steps), int(every), lp), "acs_pipe_submit")
        self._held.append((h_in, h_out, log))

    def wait(self) -> None:
        """Wait for every submitted job (raises on a kernel timeout or a non-finite log)."""
        rc = self.L.acs_pipe_wait(self.p)
        self._held.clear()
        check(rc, "acs_pipe_wait")

    def close(self):
        if getattr(self, "p", None) is not None and self.p.value:
            self.L.acs_pipe_destroy(self.p)
            self.p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
