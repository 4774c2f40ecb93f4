"""Temporal blocking of the batched form (acs_batch_set_temporal) on the GPU.

A pass of depth K gives every instance the bits of K single steps, so each batched
run with temporal blocking must equal the single-step batched run (and the standalone
runs) bit for bit, for every depth, unit height and block order, with step counts
that are and are not multiples of K (the remainder runs as single steps) and pass
counts of both parities (the state ends in either buffer).  The per-instance waits
that replace the grid barrier turn an injected missing completion into
ACS_E_TIMEOUT.
"""
import numpy as np
import pytest

import oracle
from workloads import batched_instances, dt_rule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acs():
    import paper_2312_07010_gb300 as P
    P.build.build()
    P.lib()
    return P


def _ragged_batch():
    """Sides below one vector, mid-vector, around one strip (120 written columns of a
    128-column window) and several strips, under every boundary."""
    sides = [1, 2, 3, 5, 17, 64, 119, 120, 121, 129, 241, 250, 333, 517]
    n, eps, dt, h, bc = [], [], [], [], []
    for k, m in enumerate(sides):
        for b in (0, 1, 2):
            hh = 1.0 / (m + 1) if b == 2 else 1.0 / m
            e = 0.005 + 0.002 * ((3 * k + b) % 12)
            n.append(m)
            eps.append(e)
            dt.append(dt_rule(2, e, hh))
            h.append(hh)
            bc.append(b)
    rng = np.random.default_rng(11)
    phi0 = [rng.uniform(-1, 1, (m, m)).astype(np.float32) for m in n]
    return (n, eps, dt, h, bc), phi0


def _run(acs, args, phi0, steps, depth=1, rows=0, order=0):
    b = acs.Batch(*args, "f32")
    b.set_config(0, 1, order)
    b.set_temporal(depth, rows, order)
    assert b.get_temporal()[0] == depth
    b.set_states(phi0)
    b.step(steps)
    out = b.states()
    E, M = b.observe()
    b.close()
    return out, E, M


@pytest.fixture(scope="module")
def ragged():
    return _ragged_batch()


@pytest.mark.parametrize("steps", [8, 13])
@pytest.mark.parametrize("depth,rows,order", [(2, 16, 0), (2, 64, 1), (3, 32, 0), (3, 0, 1), (4, 16, 1),
                                              (4, 64, 0), (4, 128, 1)], ids=str)
def test_temporal_batch_bitwise(acs, ragged, depth, rows, order, steps):
    args, phi0 = ragged
    ref, E0, M0 = _run(acs, args, phi0, steps)
    got, E1, M1 = _run(acs, args, phi0, steps, depth, rows, order)
    for k in range(len(ref)):
        assert np.array_equal(got[k], ref[k]), (k, args[0][k], args[4][k])
    assert np.array_equal(E0, E1) and np.array_equal(M0, M1)


def test_temporal_batch_equals_standalone(acs, ragged):
    """Against the single-problem path (a different kernel), 4 passes of depth 3 + 1."""
    args, phi0 = ragged
    got, _, _ = _run(acs, args, phi0, 13, 3, 32, 1)
    n, eps, dt, h, bc = args
    for k in range(len(n)):
        s = acs.AllenCahn((n[k], n[k]), eps[k], dt[k], h[k], bc[k], "f32")
        s.set_state(phi0[k])
        s.step(13)
        assert np.array_equal(got[k], s.numpy()), k
        s.close()


def test_temporal_batch_calls_compose(acs, ragged):
    """Calls that end mid-block compose: 3 + 5 + 4 steps equal 12 single steps."""
    args, phi0 = ragged
    ref, _, _ = _run(acs, args, phi0, 12)
    b = acs.Batch(*args, "f32")
    b.set_temporal(4, 32)
    b.set_states(phi0)
    for k in (3, 5, 4):
        b.step(k)
    for x, y in zip(ref, b.states()):
        assert np.array_equal(x, y)
    b.close()


def test_temporal_batch_full_workload_vs_single_and_oracle(acs):
    """The 256-instance workload (sides 64..1024, all three boundaries), 40 steps at depth
    4: bit-identical to the single-step batched kernel; a sample of instances within
    2e-5 of the FP64 oracle; |phi| <= 1 and E_h not increased."""
    inst = batched_instances()
    args = ([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
            [i.bc for i in inst])
    phi0 = [i.phi0().astype(np.float32) for i in inst]
    steps = 40
    ref, _, _ = _run(acs, args, phi0, steps)
    b = acs.Batch(*args, "f32")
    b.set_temporal(4, 64)
    b.set_states(phi0)
    E0, _ = b.observe()
    b.step(steps)
    E1, M1 = b.observe()
    got = b.states()
    b.close()
    assert np.all(E1 <= E0) and np.all(M1 <= 1.0)
    for k in range(len(inst)):
        assert np.array_equal(got[k], ref[k]), k
    small = sorted(range(len(inst)), key=lambda k: inst[k].n)[:6]
    for k in small:
        i = inst[k]
        o = oracle.run_fd(phi0[k].astype(np.float64), i.eps, i.dt, i.h, i.bc, steps)
        assert np.max(np.abs(got[k] - o)) <= 2e-5, k


def test_temporal_batch_timeout_is_reported(acs):
    """An uncounted unit completion (injected on the host side, no GPU fault) leaves the
    next pass of its instance waiting; the bounded wait ends the launch and the next
    observe reports ACS_E_TIMEOUT.  Disarmed, the batch steps normally again."""
    inst = batched_instances(count=8, seed=4, n_lo=64, n_hi=200)
    args = ([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
            [i.bc for i in inst])
    phi0 = [i.phi0().astype(np.float32) for i in inst]
    b = acs.Batch(*args, "f32")
    b.set_temporal(2, 32)
    b.set_states(phi0)
    L = acs.lib()
    assert L.acs_batch_inject_fault(b.b, 1) == 0
    b.step(8)
    with pytest.raises(acs.AcsError) as e:
        b.observe()
    assert e.value.status == -4
    assert L.acs_batch_inject_fault(b.b, 0) == 0
    b.set_states(phi0)
    b.step(8)
    got = b.states()
    b.close()
    ref, _, _ = _run(acs, args, phi0, 8)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)


def test_temporal_batch_unsupported_and_autotune(acs, tmp_path, monkeypatch):
    """FP64 batches refuse depth >= 2; the autotuner's choice (single-step or temporal)
    keeps the single-step bits, leaves the state unchanged, and is taken from the cache
    by a second batch of the same class."""
    inst = batched_instances(count=40, seed=77, n_lo=16, n_hi=700)
    args = ([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
            [i.bc for i in inst])
    b64 = acs.Batch(*args, "f64")
    with pytest.raises(acs.AcsError) as e:
        b64.set_temporal(2)
    assert e.value.status == -7
    b64.close()
    monkeypatch.setenv("ACS_TUNE_CACHE", str(tmp_path / "tune.txt"))
    phi0 = [i.phi0().astype(np.float32) for i in inst]
    ref, _, _ = _run(acs, args, phi0, 21)
    b = acs.Batch(*args, "f32")
    b.set_states(phi0)
    assert b.autotune() > 0
    for k, st in enumerate(b.states()):
        assert np.array_equal(st, phi0[k]), k
    cfg, tcfg = b.get_config(), b.get_temporal()
    b.step(21)
    for k, st in enumerate(b.states()):
        assert np.array_equal(st, ref[k]), k
    b.close()
    b2 = acs.Batch(*args, "f32")
    assert b2.get_config() == cfg and b2.get_temporal() == tcfg
    b2.close()


def test_temporal_batch_all_root_modes(acs):
    """Instances in every root mode the per-unit dispatch selects: the series under
    Theorem 2's clamp, the series with its run-time range tests (time step above the
    maximum-principle bound, so no clamp), and the Newton root with and without the clamp.
    Every depth gives the single-step kernel's bits (NaN-aware, since states beyond the
    theorems' conditions may grow) and the standalone runs' bits."""
    import ctypes
    cases = [(256, 0.03, 0.006, 1 / 256, 1),        # series, no clamp (dt > 1 / (1 + 4 eps^2 / h^2))
             (200, 0.03, 0.008, 1 / 200, 0),        # series, no clamp
             (64, 0.02, 0.5, 1 / 64, 2),            # Newton, no clamp
             (100, 0.02, 0.3, 1 / 101, 2),          # Newton, no clamp
             (77, 0.01, 0.05, 1 / 77, 1),           # Newton under the clamp
             (300, 0.03, dt_rule(2, 0.03, 1 / 300), 1 / 300, 0)]  # series under the clamp
    L = acs.lib()
    modes = []
    for n, eps, dt, h, bc in cases:
        c = ctypes.c_void_p()
        nn = (ctypes.c_int64 * 3)(n, n, 1)
        assert L.acs_create(2, nn, eps, dt, h, bc, 0, ctypes.byref(c)) >= 0
        m = ctypes.c_int()
        assert L.acs_get_root(c, ctypes.byref(m), None) == 0
        modes.append(m.value)
        L.acs_destroy(c)
    assert modes == [acs.ACS_ROOT_SERIES, acs.ACS_ROOT_SERIES, acs.ACS_ROOT_NEWTON, acs.ACS_ROOT_NEWTON,
                     acs.ACS_ROOT_NEWTON, acs.ACS_ROOT_SERIES]
    args = tuple(list(x) for x in zip(*cases))
    rng = np.random.default_rng(21)
    phi0 = [rng.uniform(-1, 1, (n, n)).astype(np.float32) for n in args[0]]
    for steps in (8, 13):
        ref, _, _ = _run_nan(acs, args, phi0, steps)
        for depth in (2, 3, 4):
            got, _, _ = _run_nan(acs, args, phi0, steps, depth, 32, depth % 2)
            for k in range(len(cases)):
                assert np.array_equal(got[k], ref[k], equal_nan=True), (steps, depth, k)
    for k, (n, eps, dt, h, bc) in enumerate(cases):
        s = acs.AllenCahn((n, n), eps, dt, h, bc, "f32")
        s.set_state(phi0[k])
        s.step(13)
        assert np.array_equal(got[k], s.numpy(), equal_nan=True), k
        s.close()


def _run_nan(acs, args, phi0, steps, depth=1, rows=0, order=0):
    """_run without the reductions (states beyond the theorems' conditions may not stay
    finite, which acs_batch_observe reports as an error)."""
    b = acs.Batch(*args, "f32")
    b.set_temporal(depth, rows, order)
    b.set_states(phi0)
    b.step(steps)
    out = b.states()
    b.close()
    return out, None, None
