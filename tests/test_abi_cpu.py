"""The C-ABI library without a GPU: it loads, exports every symbol include/acs.h
declares, and its host-only logic (argument validation, step-size conditions,
status strings) behaves as documented.  No call here touches a device."""
import ctypes
import math
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "acs.h")


@pytest.fixture(scope="module")
def L():
    from paper_2312_07010_gb300 import build, lib
    build.build()
    return lib()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"ACS_API\s+[\w\s\*]+?\b(acs_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("acs_create", "acs_step", "acs_energy", "acs_maxnorm", "acs_grad", "acs_bind",
              "acs_batch_create", "acs_batch_step"):
        assert s in syms


def test_every_declared_symbol_is_exported(L):
    from paper_2312_07010_gb300 import SIGNATURES
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing
    assert sorted(SIGNATURES) == declared_symbols()


def _create(L, dims, n, eps, dt, h, bc, dtype=0):
    ctx = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    rc = L.acs_create(dims, arr, eps, dt, h, bc, dtype, ctypes.byref(ctx))
    return rc, ctx


def test_create_validates_arguments(L):
    good = (2, (8, 8), 0.02, 0.01, 1 / 8, 0)
    rc, ctx = _create(L, *good)
    assert rc == 0 and ctx.value
    L.acs_destroy(ctx)
    bad = [
        (0, (8,), 0.02, 0.01, 0.1, 0), (4, (8, 8, 8), 0.02, 0.01, 0.1, 0),
        (1, (0,), 0.02, 0.01, 0.1, 0), (2, (8, -1), 0.02, 0.01, 0.1, 0),
        (1, (8,), -0.1, 0.01, 0.1, 0), (1, (8,), 0.02, 0.0, 0.1, 0), (1, (8,), 0.02, 2.0, 0.1, 0),
        (1, (8,), 0.02, 0.01, 0.0, 0), (1, (8,), 0.02, 0.01, 0.1, 3), (1, (8,), math.nan, 0.01, 0.1, 0),
        (1, (8,), 0.02, math.inf, 0.1, 0), (3, (1 << 14, 1 << 14, 1 << 14), 0.02, 0.01, 0.1, 0),
        # (2^24 + 1) * 2^40 wraps to 2^40 in int64: rejected before the product is formed
        (2, ((1 << 24) + 1, 1 << 40), 0.02, 0.01, 0.1, 0), (3, (3, 1 << 62, 1 << 62), 0.02, 0.01, 0.1, 0),
    ]
    for args in bad:
        rc, ctx = _create(L, *args)
        assert rc == -1, args
        assert not ctx.value
    rc, ctx = _create(L, 1, (8,), 0.02, 0.01, 0.1, 0, dtype=7)
    assert rc == -1


def test_noalloc_rejects_overflowing_shapes_on_host(L):
    """acs_observe_noalloc validates the shape before any CUDA call, with the same
    overflow-safe limit as acs_create; the device pointers here are never touched."""
    fake = ctypes.c_void_p(1 << 20)  # aligned, never dereferenced: the call returns first
    for dims, n in ((2, ((1 << 24) + 1, 1 << 40)), (3, (1 << 21, 1 << 21, 1)), (2, (0, 8))):
        arr = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
        assert L.acs_observe_noalloc(dims, arr, 0.1, 0.1, 0, 0, fake, fake, None) == -1


def test_batch_config_validation_on_host(L):
    """acs_batch_set_config checks its ranges before any CUDA call (the batch is not bound)."""
    n = (ctypes.c_int64 * 2)(16, 24)
    d = (ctypes.c_double * 2)
    bc = (ctypes.c_int * 2)(0, 2)
    b = ctypes.c_void_p()
    assert L.acs_batch_create(2, n, d(0.02, 0.02), d(0.01, 0.01), d(1 / 16, 1 / 25), bc, 0, ctypes.byref(b)) >= 0
    for bad in ((-1, 1, 0), (0, 0, 0), (0, 17, 0), (1, 1, 2)):
        assert L.acs_batch_set_config(b, *bad) == -1, bad
    assert L.acs_batch_set_config(b, 2, 4, 1) == 0
    v = [ctypes.c_int() for _ in range(3)]
    assert L.acs_batch_get_config(b, *[ctypes.byref(x) for x in v]) == 0
    assert [x.value for x in v] == [2, 4, 1]
    assert L.acs_batch_autotune(b, None) == -6  # not bound
    L.acs_batch_destroy(b)


def test_batch_temporal_validation_on_host(L):
    """acs_batch_set_temporal checks its ranges and the batch's eligibility (FP32) before
    any CUDA call."""
    n = (ctypes.c_int64 * 2)(16, 24)
    d = (ctypes.c_double * 2)
    bc = (ctypes.c_int * 2)(0, 2)
    v = [ctypes.c_int() for _ in range(3)]
    b = ctypes.c_void_p()
    assert L.acs_batch_create(2, n, d(0.02, 0.02), d(0.01, 0.01), d(1 / 16, 1 / 25), bc, 0, ctypes.byref(b)) >= 0
    for bad in ((0, 0, 0), (5, 0, 0), (2, -1, 0), (2, 8, 0), (4, (1 << 20) + 1, 0), (2, 0, 2), (2, 0, -1)):
        assert L.acs_batch_set_temporal(b, *bad) == -1, bad
    assert L.acs_batch_get_temporal(b, *[ctypes.byref(x) for x in v]) == 0
    assert [x.value for x in v] == [1, 64, 0]
    for depth, rows, order in ((2, 16, 1), (3, 0, 0), (4, 4096, 1), (1, 0, 0)):
        assert L.acs_batch_set_temporal(b, depth, rows, order) == 0
        assert L.acs_batch_get_temporal(b, *[ctypes.byref(x) for x in v]) == 0
        assert [x.value for x in v] == [depth, rows or 64, order]
    L.acs_batch_destroy(b)
    # FP64: the temporally blocked kernel is FP32 only
    assert L.acs_batch_create(2, n, d(0.02, 0.02), d(0.01, 0.01), d(1 / 16, 1 / 25), bc, 1, ctypes.byref(b)) >= 0
    assert L.acs_batch_set_temporal(b, 2, 0, 0) == -7
    assert L.acs_batch_set_temporal(b, 1, 0, 0) == 0
    L.acs_batch_destroy(b)
    # an instance on the Newton root (a time step beyond the series' range, Remark 1)
    assert L.acs_batch_create(2, n, d(0.02, 0.02), d(0.01, 1.9), d(1 / 16, 1 / 25), bc, 0, ctypes.byref(b)) >= 0
    assert L.acs_batch_set_temporal(b, 2, 0, 1) == 0
    L.acs_batch_destroy(b)


def test_create_warns_on_step_conditions(L):
    h = 1 / 64
    eps = 8 * math.tanh(0.9) * h / math.sqrt(2)
    # dt = 5 h^2 satisfies Theorem 2; dt = 1/5 (lambda = 3.28) violates Theorems 2 and 3
    rc, ctx = _create(L, 1, (193,), eps, 5 * h * h, h, 1)
    assert rc == 0
    L.acs_destroy(ctx)
    rc, ctx = _create(L, 1, (193,), eps, 0.2, h, 1)
    assert rc == 2
    L.acs_destroy(ctx)
    # between the two bounds: only the maximum principle warning
    dmp = ctypes.c_double()
    den = ctypes.c_double()
    assert L.acs_dt_max(1, 0.1, 0.1, ctypes.byref(dmp), ctypes.byref(den)) == 0
    rc, ctx = _create(L, 1, (16,), 0.1, 0.5 * (dmp.value + den.value), 0.1, 0)
    assert rc == 1
    L.acs_destroy(ctx)


def test_dt_max_matches_the_theorems(L):
    for d in (1, 2, 3):
        for eps, h in ((0.02, 1 / 128), (0.01, 1 / 512), (0.3, 0.1)):
            a = ctypes.c_double()
            b = ctypes.c_double()
            assert L.acs_dt_max(d, eps, h, ctypes.byref(a), ctypes.byref(b)) == 0
            lam = eps * eps * a.value / (h * h)
            assert a.value == pytest.approx(1 - 2 * d * lam, rel=1e-14)        # Theorem 2 at equality
            lam = eps * eps * b.value / (h * h)
            assert b.value == pytest.approx(4 * (1 - 2 * d * lam), rel=1e-14)  # Theorem 3 at equality
    assert L.acs_dt_max(0, 0.1, 0.1, None, None) == -1


def test_strerror_and_version(L):
    for s in (0, 1, 2, -1, -2, -3, -4, -5, -6, -7, 99):
        assert isinstance(L.acs_strerror(s), bytes) and L.acs_strerror(s)
    assert re.match(rb"^\d+\.\d+\.\d+$", L.acs_version())


def test_unbound_context_rejects_device_calls(L):
    rc, ctx = _create(L, 2, (8, 8), 0.02, 0.01, 1 / 8, 0)
    assert rc == 0
    assert L.acs_step(ctx, 1) == -6
    v = ctypes.c_double()
    assert L.acs_energy(ctx, ctypes.byref(v)) == -6
    assert L.acs_step(ctx, -1) == -1
    assert L.acs_work_bytes(ctx) >= 8 * 8 * 4
    assert L.acs_set_kernel(ctx, 9, 1) == -1
    assert L.acs_set_kernel(ctx, 3, 0) == -1
    assert L.acs_set_scheme(ctx, 5) == -1
    L.acs_destroy(ctx)
    L.acs_destroy(None)


def test_lb_form_host_logic(L):
    """Population form: buffer size (2d+1) (n^d + 8192) elements; weight and order checks.
    The pointer is never dereferenced by these calls (no device work)."""
    fake = ctypes.c_void_p(1 << 20)
    for dims, n in ((1, (40,)), (2, (12, 10)), (3, (6, 5, 4))):
        for dtype, es in ((0, 4), (1, 8)):
            rc, ctx = _create(L, dims, n, 0.02, 0.01, 0.1, 1, dtype)
            assert rc == 0
            tot = math.prod(n)
            assert L.acs_lb_bytes(ctx) == (2 * dims + 1) * (tot + 8192) * es
            # selecting the form before binding its buffer is out of order
            assert L.acs_set_kernel(ctx, 4, 1) == -6
            nb = L.acs_lb_bytes(ctx)
            assert L.acs_lb_bind(ctx, fake, nb - 1, 0.0) == -3
            assert L.acs_lb_bind(ctx, fake, nb, 1.0 / (2 * dims) * 1.01) == -1
            assert L.acs_lb_bind(ctx, ctypes.c_void_p((1 << 20) + 4), nb, 0.0) == -1
            assert L.acs_lb_bind(ctx, fake, nb, math.nan) == -1
            assert L.acs_lb_bind(ctx, fake, nb, 0.0) == 0
            assert L.acs_set_kernel(ctx, 4, 1) == 0
            k, d = ctypes.c_int(), ctypes.c_int()
            assert L.acs_get_kernel(ctx, ctypes.byref(k), ctypes.byref(d)) == 0 and k.value == 4
            # the population form exists for the paper's scheme only
            assert L.acs_set_scheme(ctx, 1) == -7
            assert L.acs_set_scheme(ctx, 0) == 0
            L.acs_destroy(ctx)


def test_lines_create_limits(L):
    """Batched lines: per-line validation and the on-chip length limits (host only)."""
    def create(ns, dtype=0):
        k = len(ns)
        h = ctypes.c_void_p()
        rc = L.acs_lines_create(k, (ctypes.c_int64 * k)(*ns), (ctypes.c_double * k)(*([0.02] * k)),
                                (ctypes.c_double * k)(*([0.01] * k)), (ctypes.c_double * k)(*([0.1] * k)),
                                (ctypes.c_int * k)(*([1] * k)), dtype, ctypes.byref(h))
        return rc, h
    rc, h = create([1, 5, 33, 2048, 28672])
    assert rc == 0
    offs = (ctypes.c_int64 * 5)()
    assert L.acs_lines_offsets(h, offs) == 0
    assert list(offs) == [0, 4, 12, 48, 2096]
    assert L.acs_lines_numel(h) == 2096 + 28672
    L.acs_lines_destroy(h)
    assert create([28673])[0] == -1
    rc, h = create([14336], 1)
    assert rc == 0
    L.acs_lines_destroy(h)
    assert create([14337], 1)[0] == -1
    assert create([0])[0] == -1


def test_pipe_host_logic(L):
    """Pipelined runner: validation as acs_create, two states + two work areas, and the
    order checks of submit / bind (host only: nothing is bound, nothing is copied)."""
    def create(dims, n, eps=0.02, dt=0.01, h=0.1, bc=1, dtype=0, slots=2):
        p = ctypes.c_void_p()
        nn = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
        return L.acs_pipe_create(dims, nn, eps, dt, h, bc, dtype, slots, ctypes.byref(p)), p
    for dims, n, dtype, es, slots in ((1, (1000,), 0, 4, 2), (2, (33, 65), 1, 8, 3), (3, (16, 8, 12), 0, 4, 4)):
        rc, p = create(dims, n, dtype=dtype, slots=slots)
        assert rc == 0
        rc2, ctx = _create(L, dims, n, 0.02, 0.01, 0.1, 1, dtype)
        up = lambda x: (x + 255) // 256 * 256
        assert L.acs_pipe_bytes(p) == slots * (up(math.prod(n) * es) + up(L.acs_work_bytes(ctx)))
        L.acs_destroy(ctx)
        cs = [L.acs_pipe_context(p, k) for k in range(slots)]
        assert all(cs) and len(set(cs)) == slots
        assert L.acs_pipe_context(p, slots) is None and L.acs_pipe_context(p, -1) is None
        one = ctypes.c_void_p(1 << 20)
        log = (ctypes.c_double * 64)()
        assert L.acs_pipe_submit(p, one, one, 10, 0, None) == -6      # not bound
        assert L.acs_pipe_submit(p, one, one, -1, 0, None) == -1
        assert L.acs_pipe_submit(p, one, one, 10, -1, None) == -1
        assert L.acs_pipe_submit(p, one, one, 10, 5, None) == -1      # logging needs a log
        assert L.acs_pipe_submit(p, one, one, 10 ** 6, 1, log) == -1  # more than 4096 entries
        assert L.acs_pipe_submit(p, None, one, 10, 0, None) == -1
        assert L.acs_pipe_wait(p) == 0                                # nothing submitted
        assert L.acs_pipe_bind(p, ctypes.c_void_p((1 << 20) + 16), L.acs_pipe_bytes(p), None) == -1
        assert L.acs_pipe_bind(p, one, L.acs_pipe_bytes(p) - 1, None) == -3
        L.acs_pipe_destroy(p)
    assert create(3, (8, 8, 8), dt=2.5)[0] == -1
    assert create(4, (8, 8, 8))[0] == -1
    assert create(3, (8, 8, 8), slots=1)[0] == -1
    assert create(3, (8, 8, 8), slots=5)[0] == -1
    rc, p = create(2, (32, 32), eps=0.5, dt=0.5, h=1 / 32)
    rc2, ctx = _create(L, 2, (32, 32), 0.5, 0.5, 1 / 32, 1)
    assert rc > 0 and rc == rc2  # the step conditions fail: acs_create's warning
    L.acs_destroy(ctx)
    L.acs_pipe_destroy(p)
    L.acs_pipe_destroy(None)


def _root(L, dims, n, eps, dt, h, bc, dtype):
    rc, ctx = _create(L, dims, n, eps, dt, h, bc, dtype)
    assert rc >= 0
    mode, split = ctypes.c_int(), ctypes.c_int()
    assert L.acs_get_root(ctx, ctypes.byref(mode), ctypes.byref(split)) == 0
    L.acs_destroy(ctx)
    return mode.value, split.value


def test_fp64_series_split_decisions(L):
    """The stated FP64 workloads take the series with its FP32 tail (512^3 Neumann, 4096^2
    Dirichlet), the 128^2 periodic one the Newton root; FP32 contexts never split."""
    assert L.acs_get_root(None, None, None) == -1
    assert _root(L, 3, (512, 512, 512), 0.01, 0.005685895945577131, 1 / 512, 1, 1) == (1, 1)
    assert _root(L, 2, (4096, 4096), 0.005, 0.0017157758860686684, 2 / 4097, 2, 1) == (1, 1)
    assert _root(L, 2, (128, 128), 0.02, 0.0274658203125, 1 / 128, 0, 1) == (0, 0)
    assert _root(L, 3, (512, 512, 512), 0.01, 0.005685895945577131, 1 / 512, 1, 0) == (1, 0)
    # FEX-FD has no cubic
    rc, ctx = _create(L, 2, (64, 64), 0.02, 0.001, 1 / 64, 0, 1)
    assert L.acs_set_scheme(ctx, 1) == 0
    mode = ctypes.c_int()
    assert L.acs_get_root(ctx, ctypes.byref(mode), None) == 0 and mode.value == 2
    L.acs_destroy(ctx)


def _tail_error(dt, xs):
    """Largest |xi x2^6 (T32 - T)| over xs: T = sum_{k>=6} q_k x2^(k-6) evaluated exactly
    (mpmath) from the FP64 coefficients and the FP64 x2 = xi^2, T32 as the FP64 kernels
    form it -- x2 truncated to FP32 on the integer units, FP32 coefficients, FP32 Horner
    (emulated: each fma exact in FP64, then rounded to FP32)."""
    import numpy as np
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    C = [1, 1, 3, 12, 55, 273, 1428, 7752, 43263]
    a = 0.5 * dt
    b = 1.0 - a
    q = [C[k] * (-a) ** k / b ** (3 * k + 1) for k in range(9)]  # q[0] is not used here
    qf = [np.float32(q[k]) for k in (6, 7, 8)]
    worst = 0.0
    for xi in xs:
        x2 = float(np.float64(xi) * np.float64(xi))
        u = np.array([x2]).view(np.uint64)[0]
        hi, lo = int(u >> np.uint64(32)), int(u & np.uint64(0xFFFFFFFF))
        e = (hi >> 20) - 896
        m = (((hi << 3) & 0xFFFFFFFF) | (lo >> 29)) & 0x7FFFFF
        x2f = 0.0 if e <= 0 else float(np.array([(e << 23) | m], dtype=np.uint32).view(np.float32)[0])
        t = qf[2]
        for k in (7, 6):
            t = np.float32(float(t) * x2f + float(qf[k - 6]))  # fma: exact product, one FP64 rounding
        T = sum(mpmath.mpf(q[k]) * mpmath.mpf(x2) ** (k - 6) for k in (6, 7, 8))
        err = abs(mpmath.mpf(xi) * mpmath.mpf(x2) ** 6 * (mpmath.mpf(float(t)) - T))
        worst = max(worst, float(err))
    return worst


def test_fp64_series_split_error_bound(L):
    """Wherever the library enables the FP32 tail, its effect on theta stays below 2^-58 for
    |xi| <= 1 (the clamped range under Theorem 2), the bound the split is admitted by:
    at the stated workloads' time steps and at the largest time step that still splits."""
    import numpy as np
    xs = list(np.linspace(-1.0, 1.0, 801)) + [1.0, -1.0, 0.999999, 2.0 ** -30]
    for dt in (0.005685895945577131, 0.0017157758860686684):
        assert _tail_error(dt, xs) <= 2.0 ** -58
    # the largest dt (series, Theorem 2 holding: 2D with a fine grid) whose context splits
    lo, hi = 0.001, 0.05
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if _root(L, 2, (64, 64), 0.001, mid, 1 / 64, 1, 1)[1]:
            lo = mid
        else:
            hi = mid
    assert _root(L, 2, (64, 64), 0.001, lo, 1 / 64, 1, 1) == (1, 1)
    assert _tail_error(lo, xs) <= 2.0 ** -58
