"""Batched stepping (acs_batch_*): many independent 2D problems in one persistent launch.

``Batch`` packs the instances' states into one device buffer (torch) and forwards to the
C ABI; row y, column x of instance i is ``phi[offsets[i] + y * ld[i] + x]`` with the row
stride ``ld[i]`` (n_i rounded up to 16 bytes) from acs_batch_row_strides.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence, Tuple

import numpy as np
import torch

from ._lib import ACS_F32, ACS_F64, check, lib


class Batch:
    def __init__(self, n: Sequence[int], eps: Sequence[float], dt: Sequence[float], h: Sequence[float],
                 bc: Sequence[int], dtype: str = "f32", stream=None):
        self.L = lib()
        self.count = len(n)
        self.n = [int(v) for v in n]
        code = ACS_F32 if dtype == "f32" else ACS_F64
        self.tdtype = torch.float32 if dtype == "f32" else torch.float64
        self.ndtype = np.float32 if dtype == "f32" else np.float64
        arr = lambda t, v: (t * self.count)(*v)
        b = ctypes.c_void_p()
        rc = self.L.acs_batch_create(self.count, arr(ctypes.c_int64, self.n), arr(ctypes.c_double, eps),
                                     arr(ctypes.c_double, dt), arr(ctypes.c_double, h), arr(ctypes.c_int, bc),
                                     code, ctypes.byref(b))
        self.create_status = check(rc, "acs_batch_create")
        self.b = b
        self.numel = int(self.L.acs_batch_numel(self.b))
        offs = (ctypes.c_int64 * self.count)()
        check(self.L.acs_batch_offsets(self.b, offs), "acs_batch_offsets")
        self.offsets = [int(v) for v in offs]
        lds = (ctypes.c_int64 * self.count)()
        check(self.L.acs_batch_row_strides(self.b, lds), "acs_batch_row_strides")
        self.ld = [int(v) for v in lds]
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self.phi = torch.zeros(self.numel, dtype=self.tdtype, device="cuda")
        wb = int(self.L.acs_batch_work_bytes(self.b))
        self.work = torch.empty(wb, dtype=torch.uint8, device="cuda")
        check(self.L.acs_batch_bind(self.b, ctypes.c_void_p(self.phi.data_ptr()), ctypes.c_void_p(self.work.data_ptr()),
                                    wb, ctypes.c_void_p(self.stream.cuda_stream)), "acs_batch_bind")

    def view(self, i: int) -> torch.Tensor:
        """Instance i as an n_i x n_i strided view of the packed device buffer."""
        o, n, ld = self.offsets[i], self.n[i], self.ld[i]
        return self.phi[o:o + n * ld].view(n, ld)[:, :n]

    def pack(self, states: List[np.ndarray]) -> torch.Tensor:
        """Host (CPU) tensor of the packed layout holding `states` (zero padding)."""
        host = torch.zeros(self.numel, dtype=self.tdtype)
        for i, s in enumerate(states):
            o, n, ld = self.offsets[i], self.n[i], self.ld[i]
            a = torch.from_numpy(np.ascontiguousarray(s, dtype=self.ndtype).reshape(n, n))
            host[o:o + n * ld].view(n, ld)[:, :n] = a
        return host

    def unpack(self, host: np.ndarray) -> List[np.ndarray]:
        """The instances' states (copies) out of a packed host array."""
        return [host[o:o + n * ld].reshape(n, ld)[:, :n].copy()
                for o, n, ld in zip(self.offsets, self.n, self.ld)]

    def set_states(self, states: List[np.ndarray]) -> None:
        self.phi.copy_(self.pack(states).to("cuda"))
        torch.cuda.synchronize()

    def states(self) -> List[np.ndarray]:
        torch.cuda.synchronize()
        return self.unpack(self.phi.cpu().numpy())

    def set_config(self, ctas_per_sm: int, blocks_per_ticket: int, order: int) -> None:
        check(self.L.acs_batch_set_config(self.b, int(ctas_per_sm), int(blocks_per_ticket), int(order)),
              "acs_batch_set_config")

    def get_config(self) -> Tuple[int, int, int]:
        v = [ctypes.c_int() for _ in range(3)]
        check(self.L.acs_batch_get_config(self.b, *[ctypes.byref(x) for x in v]), "acs_batch_get_config")
        return tuple(x.value for x in v)

    def set_temporal(self, depth: int, rows_per_unit: int = 0, order: int = 0) -> None:
        """K = depth steps per pass through HBM (1: single steps); units of at most
        rows_per_unit rows (0: the library's default), in instance order (0) or the
        largest instances first (1)."""
        check(self.L.acs_batch_set_temporal(self.b, int(depth), int(rows_per_unit), int(order)),
              "acs_batch_set_temporal")

    def get_temporal(self) -> Tuple[int, int, int]:
        v = [ctypes.c_int() for _ in range(3)]
        check(self.L.acs_batch_get_temporal(self.b, *[ctypes.byref(x) for x in v]), "acs_batch_get_temporal")
        return tuple(x.value for x in v)

    def autotune(self) -> float:
        """Time the launch configurations on the bound batch (state unchanged); returns
        the winner's microseconds per step."""
        us = ctypes.c_double()
        check(self.L.acs_batch_autotune(self.b, ctypes.byref(us)), "acs_batch_autotune")
        return us.value

    def step(self, n: int) -> None:
        check(self.L.acs_batch_step(self.b, int(n)), "acs_batch_step")

    def observe(self) -> Tuple[np.ndarray, np.ndarray]:
        e = np.empty(self.count)
        m = np.empty(self.count)
        dp = ctypes.POINTER(ctypes.c_double)
        check(self.L.acs_batch_observe(self.b, e.ctypes.data_as(dp), m.ctypes.data_as(dp)), "acs_batch_observe")
        return e, m

    def close(self) -> None:
        if getattr(self, "b", None) is not None and self.b.value:
            self.L.acs_batch_destroy(self.b)
            self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
