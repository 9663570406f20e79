"""GPU parity of the ANLS sweep against the CPU oracle, through the C ABI.

Every comparison is per column of Y and per row of X (the largest relative
error of one column / row, columns below 1e-3 of the largest measured
against 1e-3 of it), so a few wrong small columns cannot hide in a norm of
the whole factor.  Bars (the rounding of each pass's contraction, ~1e-16
FP64, ~1e-13 double-float, ~1e-7 FP32 relative, amplified by the condition
number of the half-sweep's Gram and, per column, by the cancellation in its
right-hand side, with margin):
* FP64 form and FP64-accumulated passes: one sweep from the same state
  agrees with the oracle to 1e-9 per column and row, and the passive sets
  agree except on degenerate entries;
* compensated FP32 (double-float) refinement passes of the mixed form: 1e-7;
* FP32 passes: 2e-3 after one sweep;
* per column and row, the subproblem's objective (eq. "qp") of the GPU's
  solution is within the first-order bound of its pass's rounding of the
  optimum the oracle finds for the same subproblem (tests/_parity.py);
* statistics of the iterate (f, KKT) agree with the oracle's direct
  computation from the residual.
Each case starts from a state reached by oracle sweeps, so that the
comparison measures one sweep, not the amplification of rounding along a
trajectory from a random start.
"""
import numpy as np
import pytest

import oracle
import synth
from _parity import colmax_rel, objective_ratios

pytestmark = pytest.mark.gpu

PREC_FP64, PREC_MIXED = 0, 1


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import StreamingNMF, build
    build.build()
    return StreamingNMF


def _rel_y(a, b):
    """Largest relative error of one column of Y (k x m)."""
    return colmax_rel(a, b, axis=0)


def _rel_x(a, b):
    """Largest relative error of one row of X (n x k)."""
    return colmax_rel(a, b, axis=1)


def _objective(M, X, Xg, Yg, kind):
    """Per column and row: the subproblem objective within its first-order
    bound of the pass's rounding (both halves)."""
    ry, rx, _ = objective_ratios(M, X, Xg, Yg, kind)
    assert ry <= 1.0 and rx <= 1.0, (kind, ry, rx)


def _state(n, m, k, seed, warm_sweeps=15, noise=1e-3, near_truth=False):
    M, X0, Y0 = synth.pdf_like(n, m, k, noise=noise, relative=True, seed=seed)
    X, Y = synth.near_truth_factors(X0, Y0, 0.1, seed=seed) if near_truth else synth.init_factors(n, m, k, seed=seed)
    if warm_sweeps:
        X, Y, _, _, _, _, st = oracle.anls(M, X, Y, max_sweeps=warm_sweeps)
        assert st == oracle.OK
    return M, np.ascontiguousarray(X), np.ascontiguousarray(Y)


def _handle(StreamingNMF, M, X, Y, prec, mode=None, **kw):
    n, m = M.shape
    h = StreamingNMF(n, X.shape[1], kw.pop("m_capacity", m), prec=prec, kkt_target=0.0, **kw)
    cols = M.astype(np.float32) if prec == PREC_MIXED else M
    h.append_columns(np.asfortranarray(cols))
    h.set_factors(X, Y)
    if mode is not None:
        h.set_pass_mode(mode)
    return h


def _masks_agree(vals_gpu, mask_gpu, vals_ref, rel_tol):
    """Passive sets equal except where the component is ~0 on one side."""
    k = vals_ref.shape[0]
    bits = ((mask_gpu[None, :] >> np.arange(k)[:, None]) & 1).astype(bool)
    ref_pos = vals_ref > 0
    scale = np.abs(vals_ref).max(axis=0, keepdims=True) + 1e-300
    degenerate = (np.abs(vals_ref) <= rel_tol * scale) | (np.abs(vals_gpu) <= rel_tol * scale)
    return np.all((bits == ref_pos) | degenerate)


CASES = [  # (n, m, k) -- several tiles, ragged tails, rows not a multiple of 32
    (1000, 300, 4), (777, 123, 3), (1500, 257, 8), (333, 64, 1), (2100, 190, 5),
    (450, 97, 2), (640, 130, 6), (900, 77, 7), (800, 100, 16),
]


@pytest.mark.parametrize("n,m,k", CASES)
def test_fp64_one_sweep_parity(n, m, k):
    S = _lib()
    M, X, Y = _state(n, m, k, seed=n + m + k)
    Xo, Yo, xmo, ymo, st = oracle.sweep(M, X, Y)
    assert st == oracle.OK
    with _handle(S, M, X, Y, PREC_FP64) as h:
        h.sweep(1)
        Xg, Yg, xmg, ymg = h.get_factors()
    assert _rel_y(Yg, Yo) <= 1e-9
    assert _rel_x(Xg, Xo) <= 1e-9
    _objective(M, X, Xg, Yg, "fp64")
    assert _masks_agree(Yg, ymg, Yo, 1e-9)
    assert _masks_agree(Xg.T, xmg, Xo.T, 1e-9)


@pytest.mark.parametrize("n,m,k", CASES[:4])
def test_refinement_pass_one_sweep_parity(n, m, k):
    """FP32-stored M with FP64 accumulation solves the same problem exactly
    (M holds FP32-representable values)."""
    S = _lib()
    M, X, Y = _state(n, m, k, seed=2 * n + k)
    Xo, Yo, _, _, _ = oracle.sweep(M, X, Y)
    with _handle(S, M, X, Y, PREC_MIXED, mode=1) as h:
        h.sweep(1)
        Xg, Yg, xmg, ymg = h.get_factors()
    assert _rel_y(Yg, Yo) <= 1e-9
    assert _rel_x(Xg, Xo) <= 1e-9
    _objective(M, X, Xg, Yg, "fp64")


@pytest.mark.parametrize("n,m,k", CASES)
def test_compensated_pass_one_sweep_parity(n, m, k):
    """The compensated FP32 (double-float) contraction of the mixed form's
    refinement sweeps carries ~44-46 significant bits (B and P to ~1e-13
    relative); one sweep agrees with the FP64 oracle to 1e-7 per column and
    row (1e-13 amplified by cond(H) <= ~1e4 at k = 8 and by the cancellation
    in a small column's right-hand side)."""
    S = _lib()
    M, X, Y = _state(n, m, k, seed=5 * n + k)
    Xo, Yo, _, _, _ = oracle.sweep(M, X, Y)
    with _handle(S, M, X, Y, PREC_MIXED, mode=2) as h:
        h.sweep(1)
        Xg, Yg, xmg, ymg = h.get_factors()
    assert _rel_y(Yg, Yo) <= 1e-7
    assert _rel_x(Xg, Xo) <= 1e-7
    _objective(M, X, Xg, Yg, "df")
    assert _masks_agree(Yg, ymg, Yo, 1e-9)


@pytest.mark.parametrize("n,m,k", CASES[:4])
def test_fp32_pass_one_sweep(n, m, k):
    S = _lib()
    M, X, Y = _state(n, m, k, seed=3 * n + k, warm_sweeps=40)
    Xo, Yo, _, _, _ = oracle.sweep(M, X, Y)
    with _handle(S, M, X, Y, PREC_MIXED, mode=0) as h:
        h.sweep(1)
        Xg, Yg, xmg, ymg = h.get_factors()
    assert _rel_y(Yg, Yo) <= 2e-3
    assert _rel_x(Xg, Xo) <= 2e-3
    _objective(M, X, Xg, Yg, "f32")
    assert _masks_agree(Yg, ymg, Yo, 1e-3)


@pytest.mark.parametrize("n,m,k", CASES[:4] + [(800, 100, 16)])
def test_incremental_chunk_tracks_the_oracle(n, m, k):
    """Pass mode 3: one chunk of 32 sweeps, a compensated sweep that records
    the reference contractions and 31 incremental sweeps (FP32 contraction
    of the change of X and Y since the references).  It tracks 32 oracle
    sweeps, and 32 compensated sweeps, to 1e-7 per column and row, from a
    state of the refinement phase (near the generating factors, after oracle
    sweeps): there the change of X and Y over a chunk is small, so the FP32
    contraction of the change is FP64-accurate."""
    S = _lib()
    M, X, Y = _state(n, m, k, seed=11 * n + k, warm_sweeps=100, near_truth=True)
    Xo, Yo, _, _, _, _, st = oracle.anls(M, X, Y, max_sweeps=32)
    assert st == oracle.OK
    out = {}
    for mode in (3, 2):
        with _handle(S, M, X, Y, PREC_MIXED, mode=mode) as h:
            stt = h.sweep(32)
            assert stt["sweeps"] == 32 and stt["fp64_sweeps"] == 32
            out[mode] = h.get_factors()
    (Xi, Yi, _, ymi), (Xd, Yd, _, _) = out[3], out[2]
    assert _rel_y(Yi, Yo) <= 1e-7 and _rel_x(Xi, Xo) <= 1e-7, (_rel_y(Yi, Yo), _rel_x(Xi, Xo))
    assert _rel_y(Yi, Yd) <= 1e-7 and _rel_x(Xi, Xd) <= 1e-7
    assert _masks_agree(Yi, ymi, Yo, 1e-9)


def test_chain_warm_start_takes_the_oracle_chain_steps():
    """Sec. 2's chain, the paper's own warm start: column j starts from column
    j - 1's new solution, one column after another.  On the oracle's chain
    state (PDF-like 400 x 200 x 4 after 100 sweeps) one GPU sweep with
    NMF_WARM_CHAIN gives the oracle's sweep (unique solutions, 1e-9 per
    column and row), and its column solves take the entering steps of the
    oracle's warm-started chain -- a small fraction of the cold solver's,
    which the cold GPU sweep matches."""
    S = _lib()
    from paper_2101_08431_gb300 import NMF_WARM_CHAIN, NMF_WARM_COLD
    n, m, k = 400, 200, 4
    M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=1)
    X, Y = synth.init_factors(n, m, k, seed=1)
    X, Y, _, _, _, _, st = oracle.anls(M, X, Y, max_sweeps=100)
    X, Y = np.ascontiguousarray(X), np.ascontiguousarray(Y)
    G, B = X.T @ X, X.T @ M
    cold = chain = 0
    prev = Y[:, 0]                       # column 0 starts from its previous-sweep solution
    for j in range(m):
        _, _, oc, _ = oracle.nnls(G, B[:, j])
        yw, _, ow, _, _ = oracle.nnls_warm(G, B[:, j], prev)
        cold += oc
        chain += ow
        prev = yw
    Xo, Yo, _, _, _ = oracle.sweep(M, X, Y)
    steps = {}
    for ws in (NMF_WARM_CHAIN, NMF_WARM_COLD):
        with _handle(S, M, X, Y, PREC_FP64, warm_start=ws) as h:
            stt = h.sweep(1)
            Xg, Yg, _, _ = h.get_factors()
        steps[ws] = stt["entering_steps"]
        assert _rel_y(Yg, Yo) <= 1e-9 and _rel_x(Xg, Xo) <= 1e-9
    print("entering steps: GPU chain %d, oracle chain %d; GPU cold %d, oracle cold %d"
          % (steps[NMF_WARM_CHAIN], chain, steps[NMF_WARM_COLD], cold))
    assert abs(steps[NMF_WARM_CHAIN] - chain) <= 2
    assert abs(steps[NMF_WARM_COLD] - cold) <= 2
    assert steps[NMF_WARM_CHAIN] <= 0.25 * steps[NMF_WARM_COLD]


def test_ten_fp64_sweeps_track_the_oracle():
    S = _lib()
    M, X, Y = _state(1200, 400, 4, seed=7, warm_sweeps=30)
    Xo, Yo, _, _, _, _, _ = oracle.anls(M, X, Y, max_sweeps=10)
    with _handle(S, M, X, Y, PREC_FP64) as h:
        h.sweep(10)
        Xg, Yg, _, _ = h.get_factors()
    assert _rel_y(Yg, Yo) <= 1e-9 and _rel_x(Xg, Xo) <= 1e-9


@pytest.mark.parametrize("prec,mode", [(PREC_FP64, None), (PREC_MIXED, 1)])
def test_iterate_statistics_match_oracle(prec, mode):
    """f and the KKT error of iterate t, measured during sweep t from the
    Grams, equal the oracle's residual-based values at that iterate."""
    S = _lib()
    M, X, Y = _state(800, 200, 4, seed=11, warm_sweeps=25)
    ref = oracle.kkt(M, X, Y)
    with _handle(S, M, X, Y, prec, mode=mode) as h:
        st = h.sweep(1)
        assert st["measured_iter"] == 0
        assert st["f"] == pytest.approx(ref["f"], rel=1e-9)
        assert st["kkt_abs"] == pytest.approx(ref["E_abs"], rel=1e-6, abs=1e-12 * ref["s_g"])
        assert st["kkt_rel"] == pytest.approx(ref["rel"], rel=1e-6, abs=1e-14)
        # the explicit objective / KKT pass at the new iterate
        Xg, Yg, _, _ = h.get_factors()
        ref2 = oracle.kkt(M, Xg, Yg)
        ok = h.objective_kkt()
        assert ok["f"] == pytest.approx(ref2["f"], rel=1e-9)
        assert ok["kkt_abs"] == pytest.approx(ref2["E_abs"], rel=1e-6, abs=1e-12 * ref2["s_g"])


@pytest.mark.parametrize("case", ["uniform", "pdf"])
def test_run_to_target_matches_oracle_fp64(case):
    """Runs to relative KKT 1e-8 (small-residual PDF-like data converge very
    slowly under ANLS, so the PDF case starts from a near-converged oracle
    state).  The GPU stops at an iterate the oracle certifies, after about as
    many sweeps as the oracle, at the same objective and passive sets."""
    S = _lib()
    if case == "uniform":            # the Sec. 5.4 recipe, from the U[0,1] start
        n, m, k = 200, 50, 3
        M, _, _ = synth.paper_uniform(n, m, k, sigma=0.1, seed=0)
        X, Y = synth.init_factors(n, m, k, seed=0)
    else:
        n, m, k = 400, 100, 4
        M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=2)
        X, Y = synth.init_factors(n, m, k, seed=0)
        X, Y, _, _, _, _, _ = oracle.anls(M, X, Y, max_sweeps=3000)
    Xo, Yo, xmo, ymo, sw, tr, st = oracle.anls(M, X, Y, max_sweeps=20000, kkt_target=1e-8, want_trace=True)
    assert st == oracle.OK and tr[-1, 2] <= 1e-8
    h = S(n, k, m, prec=PREC_FP64, kkt_target=1e-8, max_sweeps=20000)
    h.append_columns(np.asfortranarray(M))
    h.set_factors(X, Y)
    stt = h.sweep(0)
    Xg, Yg, xmg, ymg = h.get_factors()
    h.close()
    assert stt["converged"] == 1 and stt["kkt_rel"] <= 1e-8
    assert oracle.kkt(M, Xg, Yg)["rel"] <= 1.01e-8
    assert abs(stt["sweeps"] - sw) <= max(3, 0.02 * sw)
    assert oracle.objective(M, Xg, Yg) == pytest.approx(tr[-1, 0], rel=1e-8)
    np.testing.assert_array_equal(ymg, ymo)
    np.testing.assert_allclose(Xg @ Yg, Xo @ Yo, rtol=0, atol=1e-6 * np.abs(M).max())


def test_absolute_kkt_stop_matches_the_oracle_trace():
    """kkt_abs_target: the paper's own stopping rule, absolute E <= 1e-6
    (Sec. 5.1), on its Sec. 5.4 synthetic recipe at (2000, 50, 3).  The FP64
    form stops at the first iterate of the oracle's trajectory whose E is
    below the target, and the oracle certifies the returned iterate."""
    S = _lib()
    n, m, k = 2000, 50, 3
    M, _, _ = synth.paper_uniform(n, m, k, sigma=0.1, seed=0)
    X, Y = synth.init_factors(n, m, k, seed=0)
    _, _, _, _, _, tr, st = oracle.anls(M, X, Y, max_sweeps=2700, want_trace=True)
    hit = int(np.nonzero(tr[:, 1] <= 1e-6)[0][0])
    h = S(n, k, m, prec=PREC_FP64, kkt_target=0.0, kkt_abs_target=1e-6, max_sweeps=20000)
    h.append_columns(np.asfortranarray(M))
    h.set_factors(X, Y)
    stt = h.sweep(0)
    Xg, Yg, _, _ = h.get_factors()
    h.close()
    assert stt["converged"] == 1 and stt["kkt_abs"] <= 1e-6
    assert abs(stt["sweeps"] - (hit + 1)) <= 2, (stt["sweeps"], hit)
    assert oracle.kkt(M, Xg, Yg)["E_abs"] <= 1.001e-6


def test_mixed_run_to_target_beats_fp32_floor():
    S = _lib()
    n, m, k = 600, 300, 4
    M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=4)
    X, Y = synth.init_factors(n, m, k, seed=4)
    h = S(n, k, m, prec=PREC_MIXED, kkt_target=1e-8, max_sweeps=20000)
    h.append_columns(np.asfortranarray(M.astype(np.float32)))
    h.set_factors(X, Y)
    stt = h.sweep(0)
    Xg, Yg, _, _ = h.get_factors()
    h.close()
    assert stt["converged"] == 1 and stt["fp64_sweeps"] >= 1
    assert oracle.kkt(M, Xg, Yg)["rel"] <= 1.05e-8


def test_incremental_run_to_target_matches_compensated_run():
    """From the same start, the automatic schedule (FP32 sweeps, then chunks of
    a reference-recording compensated sweep and incremental sweeps) and the
    compensated pass alone reach relative KKT 1e-8 at iterates the oracle
    certifies.  (Their objectives agree to 1e-6: two points of the same
    valley that both meet the KKT target, on different trajectories.)"""
    S = _lib()
    n, m, k = 700, 260, 4
    M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=6)
    X, Y = synth.init_factors(n, m, k, seed=6)
    res = {}
    for mode in (-1, 2):
        h = S(n, k, m, prec=PREC_MIXED, kkt_target=1e-8, max_sweeps=40000)
        h.append_columns(np.asfortranarray(M.astype(np.float32)))
        h.set_factors(X, Y)
        h.set_pass_mode(mode)
        stt = h.sweep(0)
        Xg, Yg, _, _ = h.get_factors()
        h.close()
        assert stt["converged"] == 1
        assert oracle.kkt(M, Xg, Yg)["rel"] <= 1.05e-8
        res[mode] = oracle.objective(M, Xg, Yg)
    print("objectives: automatic %.12e, compensated %.12e" % (res[-1], res[2]))
    assert res[-1] == pytest.approx(res[2], rel=1e-6)


def test_edge_cases():
    S = _lib()
    rs = np.random.default_rng(0)
    # single column, tiny n, k = 1
    for n, m, k in ((5, 1, 1), (33, 1, 2), (7, 3, 3)):
        M = rs.uniform(0, 1, size=(n, m)).astype(np.float32).astype(np.float64)
        X = rs.uniform(0, 1, size=(n, k))
        Y = rs.uniform(0, 1, size=(k, m))
        Xo, Yo, _, _, _ = oracle.sweep(M, X, Y)
        with _handle(S, M, X, Y, PREC_FP64) as h:
            h.sweep(1)
            Xg, Yg, _, _ = h.get_factors()
        assert _rel_y(Yg, Yo) <= 1e-10 and _rel_x(Xg, Xo) <= 1e-10
    # an all-zero column of M gives y = 0
    M, X, Y = _state(300, 40, 3, seed=5)
    M[:, 7] = 0.0
    Xo, Yo, _, _, _ = oracle.sweep(M, X, Y)
    with _handle(S, M, X, Y, PREC_FP64) as h:
        h.sweep(1)
        Xg, Yg, _, ymg = h.get_factors()
    assert np.all(Yg[:, 7] == 0) and ymg[7] == 0
    assert _rel_y(Yg, Yo) <= 1e-10


def test_ring_buffer_append_and_evict():
    """Columns appended past the capacity evict the oldest; the sweep works on
    the resident window exactly as the oracle does on that window."""
    S = _lib()
    n, k, cap = 500, 3, 120
    M, X, Y = _state(n, 200, k, seed=9, warm_sweeps=20)
    h = S(n, k, cap, prec=PREC_FP64, kkt_target=0.0)
    h.append_columns(np.asfortranarray(M[:, :100]))
    h.set_factors(X, Y[:, :100])
    h.sweep(2)
    h.append_columns(np.asfortranarray(M[:, 100:200]))     # evicts 80 columns
    assert h.m == cap
    Xg, Yg, _, _ = h.get_factors()
    # the new columns were seeded with the newest resident column's y
    np.testing.assert_array_equal(Yg[:, 20:], np.repeat(Yg[:, 19:20], 100, axis=1))
    Xo, Yo, _, _, _ = oracle.sweep(M[:, 80:200], Xg, Yg)
    h.sweep(1)
    Xg2, Yg2, _, _ = h.get_factors()
    h.close()
    assert _rel_y(Yg2, Yo) <= 1e-10 and _rel_x(Xg2, Xo) <= 1e-10


def test_nonfinite_input_is_reported():
    S = _lib()
    h = S(64, 2, 8, prec=PREC_FP64)
    cols = np.ones((64, 2))
    cols[3, 1] = np.nan
    from paper_2101_08431_gb300 import NMFError
    with pytest.raises(NMFError) as e:
        h.append_columns(np.asfortranarray(cols))
    assert e.value.status == 7
    h.close()


def test_measured_fma_peaks_are_plausible():
    """nmf_measure_fma_peaks (the denominators of the ALU rooflines): FP64 and
    FP32 FMA throughput of the device, positive and within an order of
    magnitude of a Blackwell part's nominal rates (FP64 ~1.2 TFLOP/s on
    GB300, FP32 SIMT ~80 TFLOP/s at the maximum clock)."""
    _lib()
    from paper_2101_08431_gb300 import measure_fma_peaks
    pk = measure_fma_peaks()
    assert 0.1 < pk["fp64_tflops"] < 100.0, pk
    assert 8.0 < pk["fp32_tflops"] < 400.0, pk
    assert pk["fp32_tflops"] > pk["fp64_tflops"], pk
