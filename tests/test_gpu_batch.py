"""Batched stepping (acs_batch_*) on the GPU.

Every instance of a batched launch must equal its standalone run bit for bit (same
kernel arithmetic, same coefficients); FP64 instances also match the oracle within
1e-12 relative; per-instance E_h / max-norm match the standalone reductions; and the
bounded grid barrier turns an injected missing arrival into ACS_E_TIMEOUT.
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import batched_instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


def _instances(count, seed, n_lo, n_hi):
    return batched_instances(count=count, seed=seed, n_lo=n_lo, n_hi=n_hi)


@pytest.mark.parametrize("steps", [1, 2, 37])
def test_batch_equals_standalone_fp32(acs, steps):
    inst = _instances(24, 5, 8, 300)
    b = acs.Batch([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
                  [i.bc for i in inst], "f32")
    phi0 = [i.phi0().astype(np.float32) for i in inst]
    b.set_states(phi0)
    b.step(steps)
    got = b.states()
    E, M = b.observe()
    for k, i in enumerate(inst):
        s = acs.AllenCahn((i.n, i.n), i.eps, i.dt, i.h, i.bc, "f32")
        s.set_state(phi0[k])
        s.step(steps)
        assert np.array_equal(got[k], s.numpy()), k
        # states are bit-identical; the reductions may sum in another order
        assert E[k] == pytest.approx(s.energy(), rel=1e-12) and M[k] == s.maxnorm()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_ragged_small_sides(acs, dtype):
    """Sides that end mid-vector, are smaller than one vector, or straddle a block
    edge, under every boundary: each instance equals its standalone run bit for bit."""
    sides = [1, 2, 3, 5, 7, 8, 9, 63, 65, 127, 129, 131, 132, 133]
    n, eps, dt, h, bc = [], [], [], [], []
    for k, m in enumerate(sides):
        for b in (0, 1, 2):
            hh = 1.0 / (m + 1) if b == 2 else 1.0 / m
            e = 0.02 + 0.001 * k
            n.append(m)
            eps.append(e)
            h.append(hh)
            dt.append(acs.dt_max(2, e, hh)[0] * 0.9)
            bc.append(b)
    bt = acs.Batch(n, eps, dt, h, bc, dtype)
    nd = np.float32 if dtype == "f32" else np.float64
    rng = np.random.default_rng(11)
    phi0 = [rng.uniform(-1, 1, size=(m, m)).astype(nd) for m in n]
    bt.set_states(phi0)
    vx = 4 if dtype == "f32" else 2
    assert bt.ld == [(m + vx - 1) // vx * vx for m in n]
    assert all(o % vx == 0 for o in bt.offsets)
    bt.step(5)
    got = bt.states()
    for k in range(len(n)):
        s = acs.AllenCahn((n[k], n[k]), eps[k], dt[k], h[k], bc[k], dtype)
        s.set_state(phi0[k])
        s.step(5)
        assert np.array_equal(got[k], s.numpy()), (n[k], bc[k])
        # the strided device view holds the same state
        assert np.array_equal(bt.view(k).cpu().numpy(), got[k])


def test_batch_fp64_vs_oracle(acs):
    inst = _instances(6, 9, 16, 200)
    b = acs.Batch([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
                  [i.bc for i in inst], "f64")
    phi0 = [i.phi0() for i in inst]
    b.set_states(phi0)
    b.step(20)
    got = b.states()
    for k, i in enumerate(inst):
        ref = oracle.run_fd(phi0[k], i.eps, i.dt, i.h, i.bc, 20)
        assert np.abs(got[k] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_batch_calls_compose(acs):
    inst = _instances(10, 3, 30, 260)
    args = ([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
            [i.bc for i in inst], "f32")
    a = acs.Batch(*args)
    b = acs.Batch(*args)
    phi0 = [i.phi0().astype(np.float32) for i in inst]
    a.set_states(phi0)
    b.set_states(phi0)
    a.step(12)
    for _ in range(4):
        b.step(3)
    for x, y in zip(a.states(), b.states()):
        assert np.array_equal(x, y)


def test_batch_barrier_timeout_is_reported(acs):
    """A missing arrival at the grid barrier (injected on the host side, no GPU fault)
    ends the launch after the bounded wait and is reported as ACS_E_TIMEOUT."""
    inst = _instances(8, 4, 64, 200)
    b = acs.Batch([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
                  [i.bc for i in inst], "f32")
    b.set_states([i.phi0().astype(np.float32) for i in inst])
    L = acs.lib()
    assert L.acs_batch_inject_fault(b.b, 1) == 0
    b.step(4)
    with pytest.raises(acs.AcsError) as e:
        b.observe()
    assert e.value.status == -4
    assert L.acs_batch_inject_fault(b.b, 0) == 0
    b.set_states([i.phi0().astype(np.float32) for i in inst])
    b.step(4)
    E, M = b.observe()
    assert np.isfinite(E).all() and (M <= 1.0).all()


def test_batch_full_workload(acs):
    """The benchmark's 256-instance workload (sides 64..1024, 500 steps in one call):
    every instance equals its standalone run bit for bit, keeps |phi| <= 1, and its
    E_h does not increase."""
    from workloads import BATCH_STEPS
    inst = batched_instances()
    b = acs.Batch([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
                  [i.bc for i in inst], "f32")
    phi0 = [i.phi0().astype(np.float32) for i in inst]
    b.set_states(phi0)
    E0, _ = b.observe()
    b.step(BATCH_STEPS)
    E1, M1 = b.observe()
    got = b.states()
    assert np.all(E1 <= E0) and np.all(M1 <= 1.0)
    for k, i in enumerate(inst):
        s = acs.AllenCahn((i.n, i.n), i.eps, i.dt, i.h, i.bc, "f32")
        s.set_state(phi0[k])
        s.step(BATCH_STEPS)
        assert np.array_equal(got[k], s.numpy()), k
        s.close()


def _standalone(acs, inst, phi0, steps):
    out = []
    for k, i in enumerate(inst):
        s = acs.AllenCahn((i.n, i.n), i.eps, i.dt, i.h, i.bc, "f32")
        s.set_state(phi0[k])
        s.step(steps)
        out.append(s.numpy())
        s.close()
    return out


@pytest.mark.parametrize("cfg", [(1, 1, 0), (2, 4, 1), (3, 2, 1), (0, 16, 0), (1, 3, 1)], ids=str)
def test_batch_launch_configs_bitwise(acs, cfg):
    """Every launch configuration (CTAs per SM, blocks per ticket, block order) gives the
    standalone runs' bits."""
    inst = _instances(30, 9, 8, 400)
    b = acs.Batch([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
                  [i.bc for i in inst], "f32")
    b.set_config(*cfg)
    c, ch, order = b.get_config()
    assert (ch, order) == cfg[1:] and c >= 1
    phi0 = [i.phi0().astype(np.float32) for i in inst]
    b.set_states(phi0)
    b.step(9)
    got = b.states()
    for k, ref in enumerate(_standalone(acs, inst, phi0, 9)):
        assert np.array_equal(got[k], ref), k
    b.close()


def test_batch_autotune_keeps_state_bits_and_cache(acs, tmp_path, monkeypatch):
    """acs_batch_autotune reads the state only, its choice keeps the standalone bits, and
    a second batch of the same workload class takes the cached choice at bind."""
    monkeypatch.setenv("ACS_TUNE_CACHE", str(tmp_path / "tune.txt"))
    inst = _instances(40, 77, 16, 320)
    args = ([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
            [i.bc for i in inst], "f32")
    b = acs.Batch(*args)
    phi0 = [i.phi0().astype(np.float32) for i in inst]
    b.set_states(phi0)
    us = b.autotune()
    assert us > 0
    for k, st in enumerate(b.states()):
        assert np.array_equal(st, phi0[k]), k
    cfg = b.get_config()
    assert "batch/" in (tmp_path / "tune.txt").read_text()
    b.step(12)
    got = b.states()
    for k, ref in enumerate(_standalone(acs, inst, phi0, 12)):
        assert np.array_equal(got[k], ref), k
    b.close()
    b2 = acs.Batch(*args)
    assert b2.get_config() == cfg
    b2.close()
