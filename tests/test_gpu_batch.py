"""GPU tests of the batched persistent form (nmf_batch_*), through the C ABI.

* parity: every problem of a batch of uneven (n, m, k), after sweeps of the
  compensated pass, agrees with the FP64 oracle to the compensated pass's
  bar (1e-9 per sweep from an oracle-warmed state), and after the FP32 pass
  to its bar (max(2e-4, 4e-7 cond) of the half-sweep's Gram);
* the device-driven mixed schedule brings every problem to its relative-KKT
  target, and the converged objective matches the FP64 one-problem form;
* a problem's iterates are bitwise the same alone and in a mix of other
  problems (its partition and reduction order depend only on itself);
* the autotuner returns one of its candidates, and the batch still agrees
  with the oracle afterwards.
"""
import numpy as np
import pytest

import oracle
import synth
from _parity import colmax_rel, objective_ratios

pytestmark = pytest.mark.gpu


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import StreamingNMFBatch, StreamingNMF, build
    build.build()
    return StreamingNMFBatch, StreamingNMF


def _rel_y(a, b):
    """Largest relative error of one column of Y (k x m)."""
    return colmax_rel(a, b, axis=0)


def _rel_x(a, b):
    """Largest relative error of one row of X (n x k)."""
    return colmax_rel(a, b, axis=1)


def _state(n, m, k, seed, warm_sweeps=15, near_truth=False):
    M, X0, Y0 = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=seed)
    X, Y = synth.near_truth_factors(X0, Y0, 0.1, seed=seed) if near_truth else synth.init_factors(n, m, k, seed=seed)
    if warm_sweeps:
        X, Y, _, _, _, _, st = oracle.anls(M, X, Y, max_sweeps=warm_sweeps)
        assert st == oracle.OK
    return M, np.ascontiguousarray(X), np.ascontiguousarray(Y)


# uneven shapes: several (k, cluster size) classes, ragged tiles and row blocks
SHAPES = [(700, 150, 4), (333, 97, 2), (1200, 64, 8), (2100, 40, 3), (450, 210, 6), (3500, 33, 4)]


def _batch(B, states, **kw):
    b = B([(M.shape[0], X.shape[1], M.shape[1]) for M, X, Y in states], kkt_target=kw.pop("kkt_target", 0.0),
          **kw)
    for j, (M, X, Y) in enumerate(states):
        b.append_columns(j, np.asfortranarray(M.astype(np.float32)))
        b.set_factors(j, X, Y)
    return b


@pytest.mark.parametrize("mode", [2, 0])
def test_batch_one_sweep_parity(mode):
    """Per column of Y and row of X.  mode 2 (compensated): 1e-7.  mode 0
    (FP32 contraction, ~1e-7 relative on B and P): the error of each
    half-sweep is amplified by the condition number of its Gram (G = X^T X
    for Y, H = Y Y^T for X), so the bar is min(1e-2, max(2e-3, 4e-7 cond)).
    Both: the per-column objective check of tests/_parity.py."""
    B, _ = _lib()
    # states near the generating factors: the Grams are conditioned as on the
    # data the pass is used for, so that the per-row value bar means something
    states = [_state(n, m, k, seed=31 * n + k, near_truth=True) for n, m, k in SHAPES]
    ref = [oracle.sweep(M, X, Y) for M, X, Y in states]
    with _batch(B, states) as b:
        b.set_pass_mode(mode)
        stats, nrun = b.sweep(1)
        assert nrun == 1
        for j, (Xo, Yo, _, _, st) in enumerate(ref):
            assert st == oracle.OK
            X0 = states[j][1]
            if mode == 2:
                bar_y = bar_x = 1e-7
            else:
                bar_y = min(1e-2, max(2e-3, 4e-7 * np.linalg.cond(X0.T @ X0)))
                bar_x = min(1e-2, max(2e-3, 4e-7 * np.linalg.cond(Yo @ Yo.T)))
            Xg, Yg, _, _ = b.get_factors(j)
            assert stats[j]["sweeps"] == 1
            assert _rel_y(Yg, Yo) <= bar_y, (j, _rel_y(Yg, Yo), bar_y)
            assert _rel_x(Xg, Xo) <= bar_x, (j, _rel_x(Xg, Xo), bar_x)
            ry, rx, _ = objective_ratios(states[j][0], X0, Xg, Yg, "df" if mode == 2 else "f32")
            assert ry <= 1.0 and rx <= 1.0, (j, ry, rx)


def test_batch_three_sweeps_compensated():
    B, _ = _lib()
    states = [_state(n, m, k, seed=7 * n + m) for n, m, k in SHAPES[:4]]
    ref = []
    for M, X, Y in states:
        Xo, Yo = X, Y
        for _ in range(3):
            Xo, Yo, _, _, st = oracle.sweep(M, Xo, Yo)
        ref.append((Xo, Yo))
    with _batch(B, states) as b:
        b.set_pass_mode(2)
        stats, nrun = b.sweep(3)
        assert nrun == 3
        for j, (Xo, Yo) in enumerate(ref):
            Xg, Yg, _, _ = b.get_factors(j)
            assert stats[j]["fp64_sweeps"] == 3
            assert _rel_y(Yg, Yo) <= 3e-9
            assert _rel_x(Xg, Xo) <= 3e-9


def test_batch_alone_equals_mixed():
    """Bitwise: a problem's results do not depend on its batch mates."""
    B, _ = _lib()
    states = [_state(n, m, k, seed=11 * n + 3 * k) for n, m, k in SHAPES]
    j0 = 0
    with _batch(B, states) as b:
        b.set_pass_mode(2)
        b.set_schedule(32, 8)
        b.sweep(4)
        Xm, Ym, xmm, ymm = b.get_factors(j0)
    with _batch(B, [states[j0]]) as b1:
        b1.set_pass_mode(2)
        b1.set_schedule(32, 8)
        b1.sweep(4)
        Xa, Ya, xma, yma = b1.get_factors(0)
    assert np.array_equal(Xm, Xa) and np.array_equal(Ym, Ya)
    assert np.array_equal(xmm, xma) and np.array_equal(ymm, yma)


def test_batch_mixed_schedule_reaches_target():
    """Device-driven schedule: FP32 passes, then compensated passes, until
    each problem's own relative KKT target; the objective matches the FP64
    one-problem form run to the same target."""
    B, S = _lib()
    # Sec. 5.4 uniform recipe; the oracle reaches 1e-8 from these starts in
    # 1548, 416, 511 and 497 sweeps (some seeds need far more than 20000)
    cases = [(200, 50, 3, 100), (240, 60, 2, 101), (160, 40, 2, 7), (220, 55, 3, 3)]
    states = []
    for n, m, k, seed in cases:
        M, _, _ = synth.paper_uniform(n, m, k, seed=seed)
        X, Y = synth.init_factors(n, m, k, seed=seed)
        states.append((M.astype(np.float32).astype(np.float64), X, Y))
    with _batch(B, states, kkt_target=1e-8, max_sweeps=20000) as b:
        stats, nrun = b.sweep(0)
        for j, (M, X, Y) in enumerate(states):
            st = stats[j]
            assert st["converged"] == 1, (j, st)
            assert 0 < st["kkt_rel"] <= 1e-8
            assert st["fp64_sweeps"] >= 1      # the schedule moved to the compensated pass
            assert st["fp64_sweeps"] < st["sweeps"]
            n, k = X.shape
            h = S(n, k, M.shape[1], prec=0, kkt_target=1e-8, max_sweeps=20000)
            h.append_columns(np.asfortranarray(M))
            h.set_factors(X, Y)
            s64 = h.sweep(0)
            h.close()
            assert s64["converged"] == 1
            assert abs(st["f"] - s64["f"]) <= 1e-6 * abs(s64["f"])


def test_batch_autotune_then_parity():
    B, _ = _lib()
    states = [_state(n, m, k, seed=5 * n + 2 * m) for n, m, k in SHAPES[:3]]
    with _batch(B, states) as b:
        t = b.autotune(trial_sweeps=2)
        assert t["cols_per_item"] in (16, 32, 64, 128, 256)
        assert t["stage_cap"] in (2, 8)
        assert t["ms_per_sweep"] > 0
        # continue from the tuned state with the compensated pass: one sweep
        # against the oracle from the same state
        X0 = [b.get_factors(j)[:2] for j in range(len(states))]
        b.set_pass_mode(2)
        b.sweep(1)
        for j, (M, _, _) in enumerate(states):
            Xo, Yo, _, _, st = oracle.sweep(M, X0[j][0], X0[j][1])
            Xg, Yg, _, _ = b.get_factors(j)
            assert _rel_y(Yg, Yo) <= 1e-9
            assert _rel_x(Xg, Xo) <= 1e-9
        assert b.launches > 0


def test_batch_rejects_bad_input():
    B, _ = _lib()
    from paper_2101_08431_gb300 import NMFError
    with pytest.raises(NMFError):
        B([(100, 9, 20)])          # rank 9 is not supported
    M, X, Y = _state(300, 40, 3, seed=1, warm_sweeps=0)
    with B([(300, 3, 40), (300, 3, 40)]) as b:
        b.append_columns(0, np.asfortranarray(M.astype(np.float32)))
        b.set_factors(0, X, Y)
        with pytest.raises(NMFError):   # problem 1 has no factors
            b.sweep(1)
        with pytest.raises(NMFError):
            b.set_pass_mode(1)          # the FP64-accumulated pass is not a batch mode


def test_bounded_wait_reports_timeout():
    """The dependency wait of the batched form gives up after its poll limit
    on a counter nothing increments, and reports NMF_ETIMEOUT through the
    control block; the context stays usable."""
    _lib()
    import time
    import torch
    from paper_2101_08431_gb300 import _native
    L = _native.load()
    t0 = time.time()
    assert L.nmf_selftest_bounded_wait(20000, None) == _native.NMF_ETIMEOUT
    assert time.time() - t0 < 30.0
    assert L.nmf_selftest_bounded_wait(0, None) == _native.NMF_EINVAL
    x = torch.ones(16, device="cuda")
    assert float(x.sum().item()) == 16.0        # the device still answers
