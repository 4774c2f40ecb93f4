"""GPU: the pipelined host-to-host runner (acs_pipe_*) against one context and the oracle.

Each job of a pipeline must give, bit for bit, what acs_set_state_host + acs_run_logged +
acs_get_state_host give on a single context (same kernels, same graphs), whatever the
neighbouring jobs are; FP64 jobs also match the oracle to 1e-12 (relative max-abs).
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import BC_DIRICHLET, BC_NEUMANN, BC_PERIODIC, dt_rule, uniform_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


def _single(acs, shape, eps, dt, h, bc, dtype, phi0, steps, every):
    s = acs.AllenCahn(shape, eps, dt, h, bc, dtype)
    s.set_state(phi0)
    E, M = s.run_logged(steps, every) if every else (None, None)
    if not every:
        s.step(steps)
    return s.numpy(), E, M


@pytest.mark.parametrize("slots", [2, 3, 4])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shape,bc", [((4099,), BC_NEUMANN), ((130, 257), BC_PERIODIC), ((33, 17, 24), BC_DIRICHLET),
                                      ((64, 64, 64), BC_NEUMANN)], ids=str)
def test_jobs_equal_single_context_runs(acs, shape, bc, dtype, slots):
    d = len(shape)
    h, eps = 1.0 / max(shape), 0.02
    dt = dt_rule(d, eps, h)
    nd = np.float32 if dtype == "f32" else np.float64
    steps, every = 37, 10
    jobs = [uniform_field(shape, -1.0, 1.0, 100 + j).astype(nd) for j in range(5)]
    pipe = acs.Pipeline(shape, eps, dt, h, bc, dtype, slots=slots)
    ins = [torch.from_numpy(j).pin_memory() for j in jobs]
    outs = [pipe.host_buffer() for _ in jobs]
    logs = [pipe.log_buffer(steps, every) for _ in jobs]
    for i in range(len(jobs)):
        pipe.submit(ins[i], outs[i], steps, every, logs[i])
    pipe.wait()
    for i, j in enumerate(jobs):
        ref, E, M = _single(acs, shape, eps, dt, h, bc, dtype, j, steps, every)
        assert np.array_equal(outs[i].numpy(), ref)
        assert np.array_equal(logs[i].numpy()[:, 0], E)
        assert np.array_equal(logs[i].numpy()[:, 1], M)
        if dtype == "f64" and i < 2:
            orc = oracle.run_fd(j, eps, dt, h, bc, steps)
            assert float(np.abs(outs[i].numpy() - orc).max() / np.abs(orc).max()) <= 1e-12


def test_unlogged_jobs_reused_buffers_and_rebind(acs):
    """every = 0 (no log), one output buffer reused by consecutive waits, an odd number
    of jobs per wait, and the same pipeline bound again."""
    shape, bc = (96, 80), BC_NEUMANN
    h, eps = 1 / 96, 0.02
    dt = dt_rule(2, eps, h)
    pipe = acs.Pipeline(shape, eps, dt, h, bc, "f32", slots=2)
    out = pipe.host_buffer()
    for rnd in range(3):
        phi0 = uniform_field(shape, -1.0, 1.0, 7 + rnd).astype(np.float32)
        src = torch.from_numpy(phi0).pin_memory()
        for _ in range(3):
            pipe.submit(src, out, 25)
        pipe.wait()
        ref, _, _ = _single(acs, shape, eps, dt, h, bc, "f32", phi0, 25, 0)
        assert np.array_equal(out.numpy(), ref)


def test_pageable_buffers_still_correct(acs):
    shape, bc = (40, 40, 40), BC_PERIODIC
    h, eps = 1 / 40, 0.02
    dt = dt_rule(3, eps, h)
    pipe = acs.Pipeline(shape, eps, dt, h, bc, "f64")
    phi0 = uniform_field(shape, -0.9, 0.9, 3)
    src = torch.from_numpy(phi0.copy())
    out = torch.empty(shape, dtype=torch.float64)
    log = torch.empty((5, 2), dtype=torch.float64)
    pipe.submit(src, out, 40, 10, log)
    pipe.wait()
    ref, E, M = _single(acs, shape, eps, dt, h, bc, "f64", phi0, 40, 10)
    assert np.array_equal(out.numpy(), ref)
    assert np.array_equal(log.numpy()[:, 0], E)


def test_nonfinite_log_reported(acs):
    """A state holding NaN logs a NaN energy: wait raises ACS_E_NONFINITE, outputs written."""
    shape = (16, 16)
    pipe = acs.Pipeline(shape, 0.02, 0.01, 1 / 16, BC_NEUMANN, "f32")
    phi0 = np.zeros(shape, np.float32)
    phi0[3, 4] = np.nan
    src = torch.from_numpy(phi0).pin_memory()
    out = pipe.host_buffer()
    log = pipe.log_buffer(4, 2)
    pipe.submit(src, out, 4, 2, log)
    with pytest.raises(acs.AcsError) as e:
        pipe.wait()
    assert e.value.status == -5
    assert np.isnan(log.numpy()[0, 0])
