"""GPU tests of the streaming server (nmf_server_*), through the C ABI.

* every completed chunk leaves its stream at an iterate the oracle certifies
  on the resident window (relative KKT <= the target), including after the
  ring has evicted old columns;
* a stream's results are bitwise the same served alone and served while
  other streams' chunks arrive and run in the same rounds;
* admission follows the HBM budget: a stream that does not fit waits until
  another one closes;
* streams with chunks in flight share rounds (continuous batching).
"""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _srv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import StreamingServer, build
    build.build()
    return StreamingServer


def _stream_data(n, m, k, seed):
    M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=seed)
    return np.asfortranarray(M.astype(np.float32))


def _wait(srv, tickets, timeout=120.0):
    """Results of the given tickets (dict ticket -> result)."""
    want, got, t0 = set(tickets), {}, time.time()
    while want - set(got):
        for r in srv.poll(wait_ms=200):
            got[r["ticket"]] = r
        assert time.time() - t0 < timeout, "chunks did not complete"
    return got


def test_chunks_certified_by_oracle_with_eviction():
    S = _srv()
    n, k, mcap = 300, 3, 120
    M = _stream_data(n, 300, k, seed=21)
    sizes = [60, 7, 13, 1, 25, 40, 64, 30]
    with S(kkt_target=1e-6, max_sweeps_per_chunk=5000) as srv:
        sid = srv.open_stream(n, k, mcap, seed=5)
        c0 = 0
        for c in sizes:
            t = srv.submit(sid, M[:, c0:c0 + c])
            c0 += c
            r = _wait(srv, [t])[t]
            assert r["converged"] == 1 and r["kkt_rel"] <= 1e-6
            X, Y, xm, ym = srv.get_factors(sid)
            m = min(c0, mcap)
            assert r["m"] == m and Y.shape == (k, m)
            window = M[:, c0 - m:c0].astype(np.float64)
            assert oracle.kkt(window, X, Y)["rel"] <= 1.05e-6
        st = srv.stats()
        assert st["chunks_done"] == len(sizes) and st["columns_done"] == sum(sizes)


def _serve_A(S, others):
    """Stream A's chunks one at a time (each after the previous completes);
    `others` streams receive all their chunks at once.  Returns A's X, Y
    after every chunk."""
    n, k, mcap = 256, 4, 100
    MA = _stream_data(n, 160, k, seed=3)
    sizes = [40, 16, 30, 5, 64]
    out = []
    with S(kkt_target=1e-6, max_sweeps_per_chunk=4000, sweeps_per_round=8) as srv:
        a = srv.open_stream(n, k, mcap, seed=11)
        for i in range(others):
            ni, ki = 200 + 37 * i, 2 + i % 4
            Mo = _stream_data(ni, 200, ki, seed=50 + i)
            sid = srv.open_stream(ni, ki, 150, seed=70 + i)
            for c0 in range(0, 200, 25):
                srv.submit(sid, Mo[:, c0:c0 + 25])
        c0 = 0
        for c in sizes:
            t = srv.submit(a, MA[:, c0:c0 + c])
            c0 += c
            _wait(srv, [t])
            X, Y, _, _ = srv.get_factors(a)
            out.append((X, Y))
        st = srv.stats()
    return out, st


def test_stream_alone_equals_in_mix():
    S = _srv()
    alone, _ = _serve_A(S, 0)
    mixed, st = _serve_A(S, 4)
    assert st["max_streams_in_round"] >= 2          # the mix really shared rounds
    for (Xa, Ya), (Xm, Ym) in zip(alone, mixed):
        assert np.array_equal(Xa, Xm) and np.array_equal(Ya, Ym)


def test_admission_by_footprint():
    S = _srv()
    n, k, mcap = 400, 3, 200
    M = _stream_data(n, 80, k, seed=9)
    with S() as probe:     # footprint of one stream of this shape
        sid = probe.open_stream(n, k, mcap)
        t = probe.submit(sid, M[:, :40])
        _wait(probe, [t])
        one = probe.stats()["hbm_in_use_bytes"]
    assert one > 0
    with S(hbm_budget_bytes=int(2.5 * one), kkt_target=1e-5) as srv:
        ids = [srv.open_stream(n, k, mcap, seed=i) for i in range(3)]
        tk = [srv.submit(i, M[:, :40]) for i in ids]
        got = _wait(srv, tk[:2])
        st = srv.stats()
        assert st["streams_admitted"] == 2 and st["streams_queued"] == 1
        assert not any(r["stream"] == ids[2] for r in got.values())
        srv.close_stream(ids[0])        # frees its memory: the third stream is admitted
        r3 = _wait(srv, [tk[2]])[tk[2]]
        assert r3["stream"] == ids[2] and r3["converged"] == 1
        st = srv.stats()
        assert st["streams_admitted"] == 2 and st["streams_queued"] == 0
        assert st["hbm_in_use_bytes"] <= st["hbm_budget_bytes"]


def test_continuous_batching_overlaps_streams():
    S = _srv()
    with S(kkt_target=1e-5, max_sweeps_per_chunk=50000) as srv:
        tickets = []
        for i in range(6):
            n, k = 256 + 64 * i, 2 + i % 5
            M = _stream_data(n, 96, k, seed=100 + i)
            sid = srv.open_stream(n, k, 96, seed=i)
            for c0 in range(0, 96, 32):
                tickets.append(srv.submit(sid, M[:, c0:c0 + 32]))
        got = _wait(srv, tickets)
        assert all(r["converged"] == 1 for r in got.values())
        assert all(r["t_done_s"] >= r["t_submit_s"] for r in got.values())
        st = srv.stats()
        assert st["max_streams_in_round"] >= 4
        assert st["stream_rounds"] > st["rounds"]
