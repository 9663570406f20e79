"""Column-sharded sweeps through the C ABI (the multi-GPU data path): two
ranks, each a process with its own handle holding half of the time columns,
exchange P = M Y^T and H = Y Y^T once per sweep with a gloo all-reduce on the
host, and must reproduce the oracle's sweeps of the whole problem (Alg.
"anls", Sec. 2: the Y half is per column, the X half needs only P and H).
Both ranks share the one GPU here; their kernels never wait on each other
(the exchange is on the host), so nothing on the device depends on the two
processes running at the same time."""
import os

import numpy as np
import pytest

import oracle
import synth
from _parity import colmax_rel

pytestmark = pytest.mark.gpu

N, M_COLS, K, SWEEPS = 900, 260, 4, 3


def _rank_main(rank, world, port, outdir, prec, mode):
    import torch
    import torch.distributed as dist
    from paper_2101_08431_gb300 import StreamingNMF, build
    build.build()
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    M, X, Y = _problem()
    lo, hi = rank * M_COLS // world, (rank + 1) * M_COLS // world
    cols = M[:, lo:hi].astype(np.float32) if prec == 1 else M[:, lo:hi]
    h = StreamingNMF(N, K, hi - lo, prec=prec, kkt_target=0.0)
    h.append_columns(np.asfortranarray(cols))
    h.set_factors(X, Y[:, lo:hi])
    if mode is not None:
        h.set_pass_mode(mode)
    stats = []
    for _ in range(SWEEPS):
        sb, mb = h.shard_y_half()
        ts, tm = torch.from_numpy(sb), torch.from_numpy(mb)
        dist.all_reduce(ts, op=dist.ReduceOp.SUM)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        stats.append(h.shard_x_half(ts.numpy(), tm.numpy()))
    Xg, Yg, xm, ym = h.get_factors()
    h.close()
    np.savez(os.path.join(outdir, "rank%d.npz" % rank), X=Xg, Y=Yg, xm=xm, ym=ym,
             f=np.array([s["f"] for s in stats]), rel=np.array([s["kkt_rel"] for s in stats]))
    dist.barrier()
    dist.destroy_process_group()


def _problem():
    M, _, _ = synth.pdf_like(N, M_COLS, K, noise=1e-3, relative=True, seed=77)
    X, Y = synth.init_factors(N, M_COLS, K, seed=77)
    X, Y, _, _, _, _, st = oracle.anls(M, X, Y, max_sweeps=20)
    assert st == oracle.OK
    return M, np.ascontiguousarray(X), np.ascontiguousarray(Y)


@pytest.mark.parametrize("prec,mode,bar", [(0, None, 1e-9), (1, 2, 1e-7)])
def test_two_rank_column_sharded_sweeps_match_the_oracle(tmp_path, prec, mode, bar):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.spawn(_rank_main, args=(2, port, str(tmp_path), prec, mode), nprocs=2, join=True)
    r = [np.load(os.path.join(str(tmp_path), "rank%d.npz" % i)) for i in range(2)]
    # every rank holds the same X, bit for bit
    assert np.array_equal(r[0]["X"], r[1]["X"]) and np.array_equal(r[0]["xm"], r[1]["xm"])
    M, X, Y = _problem()
    Xo, Yo, xmo, ymo, _, _, st = oracle.anls(M, X, Y, max_sweeps=SWEEPS)
    Yg = np.concatenate([r[0]["Y"], r[1]["Y"]], axis=1)
    assert colmax_rel(Yg, Yo, axis=0) <= bar and colmax_rel(r[0]["X"], Xo, axis=1) <= bar
    # statistics of the whole problem: iterate 0 is unmeasured, iterates 1, 2
    # equal the oracle's residual-based values
    assert r[0]["rel"][0] == -1.0
    Xs, Ys = X, Y
    for t in range(1, SWEEPS):
        Xs, Ys, _, _, _ = oracle.sweep(M, Xs, Ys)
        ref = oracle.kkt(M, Xs, Ys)
        for i in range(2):
            assert r[i]["f"][t] == pytest.approx(ref["f"], rel=1e-8)
            assert r[i]["rel"][t] == pytest.approx(ref["rel"], rel=1e-5)
