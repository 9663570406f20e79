"""Host-side multi-rank logic on CPU (gloo, world size 2).

1. Column sharding of one sweep: each rank owns a contiguous block of time
   columns, solves its Y columns (Y-update needs only X), forms the partial
   P_g = M_g Y_g^T and H_g = Y_g Y_g^T, and one all-reduce (sum) gives every
   rank the full P and H for the X-update.  The result equals the
   single-process oracle sweep.
2. The benchmark's multi-GPU reduction: the step time is the MAX over ranks
   and the whole-job value counts every rank's units.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, M, X, Y, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, m = M.shape
    k = X.shape[1]
    c0, c1 = rank * m // world, (rank + 1) * m // world
    G = X.T @ X
    Yl = np.zeros((k, c1 - c0))
    for j in range(c0, c1):
        Yl[:, j - c0] = oracle.nnls(G, X.T @ M[:, j])[0]
    P = torch.from_numpy(M[:, c0:c1] @ Yl.T)
    H = torch.from_numpy(Yl @ Yl.T)
    dist.all_reduce(P)
    dist.all_reduce(H)
    Xn = np.zeros_like(X)
    for i in range(n):
        Xn[i] = oracle.nnls(H.numpy(), P.numpy()[i])[0]
    # the benchmark's reduction of the per-rank step time
    t = torch.tensor([float(10 + rank)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    width = (m + world - 1) // world             # gloo gathers equal sizes: pad
    pad = np.zeros((k, width))
    pad[:, : c1 - c0] = Yl
    Yg = [torch.zeros(k, width, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(Yg, torch.from_numpy(pad))
    if rank == 0:
        parts = [Yg[r].numpy()[:, : (r + 1) * m // world - r * m // world] for r in range(world)]
        q.put((Xn, np.concatenate(parts, axis=1), float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_column_sharded_sweep_equals_single_process():
    import oracle
    import synth
    n, m, k = 120, 37, 3
    M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, seed=1)
    X, Y = synth.init_factors(n, m, k, seed=1)
    X, Y, _, _, _, _, _ = oracle.anls(M, X, Y, max_sweeps=10)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, M, X, Y, q)) for r in range(2)]
    for p in procs:
        p.start()
    Xn, Yn, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    Xo, Yo, _, _, _ = oracle.sweep(M, X, Y)
    np.testing.assert_allclose(Yn, Yo, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Xn, Xo, rtol=1e-9, atol=1e-12)
    assert tmax == 11.0
