"""GPU parity of the rank-16 tensor-core M pass (split-BF16 tcgen05
contractions, FP32 column solves, FP64 row solves), through the C ABI.

The FP32-class pass of the mixed form at k = 16 runs B = X^T M and P = M Y^T
as (M_hi + M_lo)(V_hi + V_lo) BF16 products with FP32 accumulation.  Each of
hi, lo carries 8 significant bits, so the pair represents a value to within
2^-16 of its magnitude; a product of two split values is then within
2 * 2^-16 = 2^-15 (tests/test_split_bf16_bound.py pins both), and an FP32 sum
of L terms adds at most 2 (L - 1) 2^-24 of the sum of magnitudes.  So the
right-hand side the GPU solves differs from the FP64 one by at most
u * sum_r |x_r| |m_r| per component, u = 2^-15 + 2 (L - 1) 2^-24.

Each half-sweep is judged per column (Y) and per row (X) against the
oracle's solve of the same subproblem (eq. "qp", Sec. 2): Y against the
oracle's column solve with the input X, X against its row solve with the
GPU's new Y (so the X check measures the row pass alone):
* the subproblem objective: phi(v) - phi(v*) must stay within the first-order
  bound sum_a w_a |v_a - v*_a|, w = u sum|.||.| + kappa |G| (|v| + |v*|) +
  tol, kappa = 2^-18 for the FP32 column solve's rounding of G and of the
  solution (2^-40 for the FP64 row solve), tol the Lawson-Hanson entering
  tolerance (tests/_parity.py derives it); a zero column exceeds it ~1e4
  times and a 10% error ~1e3 times;
* values: the largest per-column (per-row) relative error, at most
  min(1e-2, max(5e-4, 3e-5 cond)) of the half-sweep's Gram -- capped at 1e-2;
* passive sets differ only where the positive value is below that bar times
  the column's (row's) largest value.
States are reached by oracle sweeps from a start near the generating factors,
where the Grams are conditioned as on the data this pass is used for.

Shapes cover a single CTA per column range (C = 1), clusters of 2, 4 and 16
CTAs (rows split), CTAs that own no rows, a ragged last tile of columns and
several tiles per cluster.
"""
import numpy as np
import pytest

import oracle
import synth
from _parity import colmax_rel, masks_differ_only_at_small_values, objective_ratios

pytestmark = pytest.mark.gpu


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import StreamingNMF, build
    build.build()
    return StreamingNMF


VALUE_CAP = 1e-2


def _warm_state(n, m, seed, sweeps, near_truth=True):
    M, X0, Y0 = synth.pdf_like(n, m, 16, noise=1e-3, relative=True, seed=seed)
    M32 = np.asfortranarray(M.astype(np.float32))
    M64 = M32.astype(np.float64)
    if near_truth:
        X, Y = synth.near_truth_factors(X0, Y0, 0.1, seed=seed)
    else:
        X, Y = synth.init_factors(n, m, 16, seed=seed)
    if sweeps:
        X, Y, _, _, _, _, st = oracle.anls(M64, X, Y, max_sweeps=sweeps)
        assert st == oracle.OK
    return M32, M64, np.ascontiguousarray(X), np.ascontiguousarray(Y)


def _check_sweep(M64, X, Xg, Yg, xmg=None, ymg=None, J=None, I=None):
    """Y half against the oracle's column solves with the input X; X half
    against its row solves with the GPU's Y.  J, I: sampled columns / rows."""
    ry, rx, (Yref, ymo, Xref, xmo) = objective_ratios(M64, X, Xg, Yg, "tc16", J=J, I=I)
    halves = (("Y", X.T @ X, Yg if J is None else Yg[:, J], Yref, ymg if (ymg is None or J is None) else ymg[J],
               ymo, ry),
              ("X", Yg @ Yg.T, (Xg if I is None else Xg[I, :]).T, Xref.T,
               xmg if (xmg is None or I is None) else xmg[I], xmo, rx))
    for label, G, V, Vref, mask, mask_ref, ratio in halves:
        cond = np.linalg.cond(G)
        bar = min(VALUE_CAP, max(5e-4, 3e-5 * cond))
        err = colmax_rel(V, Vref, axis=0)
        ok_m, nd, worst = (True, 0, 0.0) if mask is None else \
            masks_differ_only_at_small_values(V, Vref, mask, mask_ref, bar)
        print("  %s: objective excess / bound max %.2e; per-column rel err %.2e (bar %.1e, cond %.1e); "
              "mask differences %d (largest value there %.2e)" % (label, ratio, err, bar, cond, nd, worst))
        assert ratio <= 1.0, (label, ratio)
        assert err <= bar, (label, err, bar)
        assert ok_m, (label, worst, bar)


# (n, m, seed): C = 1 (200 rows); C = 2 (700, 1000); C = 4 (2048); C = 16 with
# empty CTAs (4100); ragged last tiles (m = 50, 150, 290 not multiples of 16)
SHAPES = [(200, 50, 1), (700, 150, 2), (1000, 64, 3), (2048, 300, 4), (4100, 290, 8)]


@pytest.mark.parametrize("n,m,seed", SHAPES)
def test_tc16_one_sweep_parity(n, m, seed):
    S = _lib()
    M32, M64, X, Y = _warm_state(n, m, seed, sweeps=12)
    h = S(n, 16, m, prec=1, kkt_target=0.0)
    h.append_columns(M32)
    h.set_factors(X, Y)
    h.set_pass_mode(0)
    h.sweep(1)
    Xg, Yg, xmg, ymg = h.get_factors()
    h.close()
    print("tc16 n=%d m=%d" % (n, m))
    _check_sweep(M64, X, Xg, Yg, xmg, ymg)


def test_tc16_cold_start_sweeps_decrease_objective():
    """From the U[0,1] start, tensor-core sweeps decrease the objective the
    oracle computes for each iterate (Sec. 2: every ANLS half-step is a
    minimisation, up to the pass's rounding)."""
    S = _lib()
    n, m = 1000, 96
    M32, M64, X, Y = _warm_state(n, m, 9, sweeps=0, near_truth=False)
    h = S(n, 16, m, prec=1, kkt_target=0.0)
    h.append_columns(M32)
    h.set_factors(X, Y)
    h.set_pass_mode(0)
    f_prev = oracle.objective(M64, X, Y)
    for _ in range(6):
        h.sweep(1)
        Xg, Yg, _, _ = h.get_factors()
        f = oracle.objective(M64, Xg, Yg)
        assert f <= f_prev * (1 + 1e-5), (f, f_prev)
        f_prev = f
    h.close()


def test_tc16_well_conditioned_tight_bar():
    """Components with nearly disjoint supports: cond(G) is small, so the value
    bar is the pass's own error, 5e-4 (split-BF16 products are good to ~1e-5)."""
    S = _lib()
    n, m, k = 3000, 500, 16
    g = np.random.default_rng(41)
    r = np.arange(n, dtype=np.float64)
    X0 = np.stack([np.exp(-0.5 * ((r - (c + 0.5) * n / k) / (n / (8.0 * k))) ** 2) for c in range(k)], axis=1)
    Y0 = g.uniform(0.1, 1.0, size=(k, m))
    M = X0 @ Y0
    M += g.normal(0.0, 1e-3 * np.sqrt(np.mean(M ** 2)), size=M.shape)
    M32 = np.asfortranarray(M.astype(np.float32))
    M64 = M32.astype(np.float64)
    X, Y = synth.near_truth_factors(X0, Y0, 0.1, seed=41)
    X, Y, _, _, _, _, st = oracle.anls(M64, X, Y, max_sweeps=8)
    assert st == oracle.OK
    X, Y = np.ascontiguousarray(X), np.ascontiguousarray(Y)
    h = S(n, k, m, prec=1, kkt_target=0.0)
    h.append_columns(M32)
    h.set_factors(X, Y)
    h.set_pass_mode(0)
    h.sweep(1)
    Xg, Yg, xmg, ymg = h.get_factors()
    h.close()
    print("well-conditioned: cond G %.1f" % np.linalg.cond(X.T @ X))
    _check_sweep(M64, X, Xg, Yg, xmg, ymg)


def test_tc16_full_size_sampled():
    """The 8192 x 16384 x 16 workload (512 MB of FP32 M) in the launch
    configuration the benchmark times: one tensor-core sweep from the U[0,1]
    start, checked on 512 sampled columns (the oracle's column solve with the
    input X) and 1024 sampled rows (the oracle's row solve with the sweep's
    own new Y, so that every sampled row is an exact one-row problem)."""
    S = _lib()
    n, m, k = 8192, 16384, 16
    M, _, _ = synth.pdf_like(n, m, k, noise=1e-4, relative=True, seed=3)
    M32 = np.asfortranarray(M.astype(np.float32))
    del M
    X, Y = synth.init_factors(n, m, k, seed=3)
    h = S(n, k, m, prec=1, kkt_target=0.0)
    h.append_columns(M32)
    h.set_factors(X, Y)
    h.set_pass_mode(0)
    h.sweep(1)
    Xg, Yg, _, _ = h.get_factors()
    kk = h.objective_kkt()
    h.close()
    g = np.random.default_rng(5)
    J = np.sort(g.choice(m, size=512, replace=False))
    I = np.sort(g.choice(n, size=1024, replace=False))
    print("full size, sampled columns and rows")
    _check_sweep(M32, X, Xg, Yg, J=J, I=I)
    f_or = oracle.objective(M32.astype(np.float64), Xg, Yg)
    print("  f %.6e vs oracle %.6e" % (kk["f"], f_or))
    assert abs(kk["f"] - f_or) <= 1e-3 * abs(f_or)


def test_tc16_ring_eviction_window():
    """Streaming append past the ring capacity: the resident window wraps
    around the ring's end (head != 0), so the converters and the column solves
    address physical columns through the ring; one sweep on the window against
    the oracle's sweep of the same window."""
    S = _lib()
    n, k, mcap = 1000, 16, 64
    M, X0, Y0 = synth.pdf_like(n, 80, k, noise=1e-3, relative=True, seed=8)
    M32 = np.asfortranarray(M.astype(np.float32))
    W64 = M32[:, 16:80].astype(np.float64)          # the newest 64 columns
    X, Y = synth.near_truth_factors(X0, Y0[:, 16:80], 0.1, seed=8)
    X, Y, _, _, _, _, st = oracle.anls(W64, X, Y, max_sweeps=10)
    assert st == oracle.OK
    X, Y = np.ascontiguousarray(X), np.ascontiguousarray(Y)
    h = S(n, k, mcap, prec=1, kkt_target=0.0)
    h.append_columns(np.asfortranarray(M32[:, :40]))
    h.append_columns(np.asfortranarray(M32[:, 40:80]))   # evicts the 16 oldest; the window wraps
    assert h.m == mcap
    h.set_factors(X, Y)
    h.set_pass_mode(0)
    h.sweep(1)
    Xg, Yg, xmg, ymg = h.get_factors()
    h.close()
    print("ring window")
    _check_sweep(W64, X, Xg, Yg, xmg, ymg)


def test_tc16_graph_replay_matches_plain_launches():
    """Sweeps in chunks of 32 are captured into a CUDA graph the second time
    their signature is seen and replayed after that; the tensor-core pass's
    cluster launches must give bitwise the same iterates replayed as launched
    one sweep at a time (every partition and reduction order is fixed)."""
    S = _lib()
    n, m = 700, 150
    M32, M64, X, Y = _warm_state(n, m, 2, sweeps=4)
    out = []
    for chunked in (True, False):
        h = S(n, 16, m, prec=1, kkt_target=0.0)
        h.append_columns(M32)
        h.set_factors(X, Y)
        h.set_pass_mode(0)
        if chunked:
            h.sweep(96)          # chunk 1 plain, chunk 2 captured, chunk 3 replayed
        else:
            for _ in range(96):
                h.sweep(1)
        out.append(h.get_factors())
        h.close()
    (Xa, Ya, xa, ya), (Xb, Yb, xb, yb) = out
    assert np.array_equal(Xa, Xb) and np.array_equal(Ya, Yb)
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)


def test_tc16_bounded_wait_reports_timeout():
    """The rank-16 pass's wait gives up after its wall-time limit on an
    mbarrier nothing arrives on, raises its abort flag and returns
    NMF_ETIMEOUT; the context stays usable."""
    _lib()
    import time
    import torch
    from paper_2101_08431_gb300 import _native
    L = _native.load()
    t0 = time.time()
    assert L.nmf_selftest_tc16_wait(200, None) == _native.NMF_ETIMEOUT
    dt = time.time() - t0
    assert 0.15 < dt < 30.0, dt
    x = torch.ones(16, device="cuda")
    assert float(x.sum().item()) == 16.0        # the device still answers


# ---------------------------------------------------------------------------
# Refinement at rank 16 beyond the rows of the cluster-fused FP64-class kernels
# (n > ~3840): compensated reference sweeps and incremental sweeps
# ---------------------------------------------------------------------------
REF_N, REF_M, REF_SEED = 4100, 290, 8


def _refined_state(sweeps):
    """A state of the refinement phase: oracle sweeps from near the generating
    factors (FP64 throughout)."""
    return _warm_state(REF_N, REF_M, REF_SEED, sweeps=sweeps)


def test_tc16_reference_sweep_matches_the_oracle():
    """Pass mode 2 at n = 4100, k = 16: the compensated reference sweep
    (double-float B = X^T M and P = M Y^T, FP64 column and row solves)
    against one oracle sweep: per column / row within 1e-7 (the compensated
    pass's bar) and the subproblem objective within its first-order bound
    with the compensated contraction unit."""
    S = _lib()
    M32, M64, X, Y = _refined_state(40)
    h = S(REF_N, 16, REF_M, prec=1, kkt_target=0.0)
    h.append_columns(M32)
    h.set_factors(X, Y)
    h.set_pass_mode(2)
    h.sweep(1)
    Xg, Yg, xmg, ymg = h.get_factors()
    h.close()
    Xo, Yo, _, _, _ = oracle.sweep(M64, X, Y)
    ey, ex = colmax_rel(Yg, Yo, axis=0), colmax_rel(Xg, Xo, axis=1)
    ry, rx, _ = objective_ratios(M64, X, Xg, Yg, "df")
    print("reference sweep n=%d m=%d: per-column %.2e per-row %.2e; objective ratios %.2e %.2e" %
          (REF_N, REF_M, ey, ex, ry, rx))
    assert ey <= 1e-7 and ex <= 1e-7
    assert ry <= 1.0 and rx <= 1.0


def test_tc16_incremental_chunk_matches_the_oracle():
    """Pass mode 3 at n = 4100, k = 16: a chunk of one recording reference
    sweep and 31 incremental sweeps (tensor-core change terms on the FP64
    references) against 32 oracle sweeps from the same refined state: per
    column / row within 1e-7."""
    S = _lib()
    M32, M64, X, Y = _refined_state(40)
    h = S(REF_N, 16, REF_M, prec=1, kkt_target=0.0)
    h.append_columns(M32)
    h.set_factors(X, Y)
    h.set_pass_mode(3)
    h.sweep(32)
    Xg, Yg, _, _ = h.get_factors()
    h.close()
    Xo, Yo, _, _, _, _, _ = oracle.anls(M64, X, Y, max_sweeps=32)
    ey, ex = colmax_rel(Yg, Yo, axis=0), colmax_rel(Xg, Xo, axis=1)
    print("32 sweeps (1 reference + 31 incremental): per-column %.2e per-row %.2e" % (ey, ex))
    assert ey <= 1e-7 and ex <= 1e-7


def test_tc16_mixed_run_reaches_the_target_the_oracle_certifies():
    """The mixed schedule at n = 4100, k = 16 (tensor-core passes, then the
    reference / incremental refinement) to relative KKT 1e-8 from a state
    near the generating factors: the oracle's KKT of the returned iterate is
    within the target.  (The run's own f is measured through the change
    terms' 2^-15 rounding, which the cancellation in the Gram form of f
    amplifies; it is checked loosely.)"""
    S = _lib()
    M32, M64, X, Y = _refined_state(0)
    h = S(REF_N, 16, REF_M, prec=1, kkt_target=1e-8, max_sweeps=40000)
    h.append_columns(M32)
    h.set_factors(X, Y)
    st = h.sweep(0)
    Xg, Yg, _, _ = h.get_factors()
    h.close()
    kk = oracle.kkt(M64, Xg, Yg)
    print("mixed run: %d sweeps (%d refinement), f %.12e (oracle %.12e), rel KKT %.3e (oracle %.3e)" %
          (st["sweeps"], st["fp64_sweeps"], st["f"], kk["f"], st["kkt_rel"], kk["rel"]))
    assert st["converged"] == 1 and st["fp64_sweeps"] > 0
    assert kk["rel"] <= 1.05e-8
    assert st["f"] == pytest.approx(kk["f"], rel=1e-3)
