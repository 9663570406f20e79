"""Parity at the benchmarked sizes, in the launch configurations bench.py times.

* the benchmark workload (PDF-like n=3000, m=2000, k=4, the bench's data and
  handle configuration): one sweep of each pass from an oracle-warmed state
  against the oracle's sweep, every entry compared;
* the batched workload (256 problems of uneven n, m, k; 2.5 GB of FP32 M):
  one compensated-pass sweep of the whole batch, checked against the oracle
  on a sample of problems (every entry of each sampled problem).
"""
import numpy as np
import pytest

import bench
import oracle
import synth
from _parity import colmax_rel, objective_ratios

pytestmark = pytest.mark.gpu


def _rel_y(a, b):
    """Largest relative error of one column of Y (k x m)."""
    return colmax_rel(a, b, axis=0)


def _rel_x(a, b):
    """Largest relative error of one row of X (n x k)."""
    return colmax_rel(a, b, axis=1)


def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def bench_state():
    _need_gpu()
    M32, M64, X0, Y0 = bench.make_data(0)
    X, Y, _, _, _, _, st = oracle.anls(M64, X0, Y0, max_sweeps=10)
    assert st == oracle.OK
    Xo, Yo, xmo, ymo, st = oracle.sweep(M64, X, Y)
    assert st == oracle.OK
    return M32, M64, np.ascontiguousarray(X), np.ascontiguousarray(Y), Xo, Yo


@pytest.mark.parametrize("prec,mode,bar,kind", [(0, None, 1e-9, "fp64"), (1, 2, 1e-7, "df"), (1, 1, 1e-9, "fp64"),
                                                (1, 0, 2e-3, "f32")])
def test_benchmark_workload_one_sweep(bench_state, prec, mode, bar, kind):
    """The 3000 x 2000 x 4 workload in each pass, per column of Y and row of
    X (bars of tests/test_gpu_sweep.py), with the per-column objective check."""
    from paper_2101_08431_gb300 import StreamingNMF
    M32, M64, X, Y, Xo, Yo = bench_state
    h = StreamingNMF(bench.N_ROWS, bench.RANK_K, bench.M_COLS, prec=prec, kkt_target=0.0)
    h.append_columns(M64 if prec == 0 else M32)
    h.set_factors(X, Y)
    if mode is not None:
        h.set_pass_mode(mode)
    h.sweep(1)
    Xg, Yg, _, _ = h.get_factors()
    h.close()
    assert _rel_y(Yg, Yo) <= bar, _rel_y(Yg, Yo)
    assert _rel_x(Xg, Xo) <= bar, _rel_x(Xg, Xo)
    ry, rx, _ = objective_ratios(M64, X, Xg, Yg, kind)
    assert ry <= 1.0 and rx <= 1.0, (ry, rx)


def test_batched_workload_sampled():
    _need_gpu()
    from paper_2101_08431_gb300 import StreamingNMFBatch
    shapes = synth.batch_problem_shapes(bench.BATCH_NPROB)
    b = StreamingNMFBatch([(n, k, m) for n, m, k, _ in shapes], kkt_target=0.0)
    data = {}
    sample = [0, 17, 64, 101, 150, 199, 230, 255]
    for j, (n, m, k, seed) in enumerate(shapes):
        M, _, _ = synth.pdf_like(n, m, k, noise=bench.NOISE, relative=True, seed=seed)
        X, Y = synth.init_factors(n, m, k, seed=seed)
        b.append_columns(j, np.asfortranarray(M, dtype=np.float32))
        b.set_factors(j, X, Y)
        if j in sample:
            data[j] = (M, X, Y)
    b.set_pass_mode(2)
    stats, nrun = b.sweep(1)
    assert nrun == 1
    for j in sample:
        M, X, Y = data[j]
        Xo, Yo, _, _, st = oracle.sweep(M, X, Y)
        assert st == oracle.OK
        Xg, Yg, _, _ = b.get_factors(j)
        assert stats[j]["sweeps"] == 1
        # one sweep from the U[0,1] start: the compensated pass's 1e-9, scaled
        # by the conditioning of the half-sweep's Gram where it is poor
        bar_y = max(1e-9, 1e-13 * np.linalg.cond(X.T @ X))
        bar_x = max(1e-9, 1e-13 * np.linalg.cond(Yo @ Yo.T))
        assert _rel_y(Yg, Yo) <= bar_y, (j, shapes[j], _rel_y(Yg, Yo))
        assert _rel_x(Xg, Xo) <= bar_x, (j, shapes[j], _rel_x(Xg, Xo))
    b.close()
