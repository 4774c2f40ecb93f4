"""Batched lines (acs_lines_*): many independent 1D problems advanced together.

``Lines`` packs the lines' states into one device buffer (torch) and forwards to the
C ABI; line i is ``phi[offsets[i] : offsets[i] + n_i]``.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence, Tuple

import numpy as np
import torch

from ._lib import ACS_F32, ACS_F64, check, lib


class Lines:
    def __init__(self, n: Sequence[int], eps: Sequence[float], dt: Sequence[float], h: Sequence[float],
                 bc: Sequence[int], dtype: str = "f32", stream=None):
        self.L = lib()
        self.count = len(n)
        self.n = [int(v) for v in n]
        code = ACS_F32 if dtype == "f32" else ACS_F64
        self.tdtype = torch.float32 if dtype == "f32" else torch.float64
        self.ndtype = np.float32 if dtype == "f32" else np.float64
        arr = lambda t, v: (t * self.count)(*v)
        h_ = ctypes.c_void_p()
        rc = self.L.acs_lines_create(self.count, arr(ctypes.c_int64, self.n), arr(ctypes.c_double, eps),
                                     arr(ctypes.c_double, dt), arr(ctypes.c_double, h), arr(ctypes.c_int, bc),
                                     code, ctypes.byref(h_))
        self.create_status = check(rc, "acs_lines_create")
        self.h = h_
        self.numel = int(self.L.acs_lines_numel(self.h))
        offs = (ctypes.c_int64 * self.count)()
        check(self.L.acs_lines_offsets(self.h, offs), "acs_lines_offsets")
        self.offsets = [int(v) for v in offs]
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self.phi = torch.zeros(self.numel, dtype=self.tdtype, device="cuda")
        wb = int(self.L.acs_lines_work_bytes(self.h))
        self.work = torch.empty(wb, dtype=torch.uint8, device="cuda")
        check(self.L.acs_lines_bind(self.h, ctypes.c_void_p(self.phi.data_ptr()),
                                    ctypes.c_void_p(self.work.data_ptr()), wb,
                                    ctypes.c_void_p(self.stream.cuda_stream)), "acs_lines_bind")

    def view(self, i: int) -> torch.Tensor:
        o = self.offsets[i]
        return self.phi[o:o + self.n[i]]

    def set_states(self, states: List[np.ndarray]) -> None:
        host = torch.zeros(self.numel, dtype=self.tdtype)
        for i, s in enumerate(states):
            o = self.offsets[i]
            host[o:o + self.n[i]] = torch.from_numpy(np.ascontiguousarray(s, dtype=self.ndtype).reshape(-1))
        self.phi.copy_(host.to("cuda"))
        torch.cuda.synchronize()

    def states(self) -> List[np.ndarray]:
        torch.cuda.synchronize()
        host = self.phi.cpu().numpy()
        return [host[o:o + n].copy() for o, n in zip(self.offsets, self.n)]

    def step(self, n: int) -> None:
        check(self.L.acs_lines_step(self.h, int(n)), "acs_lines_step")

    def observe(self) -> Tuple[np.ndarray, np.ndarray]:
        e = np.empty(self.count)
        m = np.empty(self.count)
        dp = ctypes.POINTER(ctypes.c_double)
        check(self.L.acs_lines_observe(self.h, e.ctypes.data_as(dp), m.ctypes.data_as(dp)), "acs_lines_observe")
        return e, m

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.acs_lines_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
