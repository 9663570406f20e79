"""nmf_sweep_noalloc: the sweep for callers that cannot allocate device memory.

Some callers must not allocate where they run the sweep: a latency-critical
loop that cannot block on cudaMalloc, a plug-in whose host framework has
reserved all device memory, code that may allocate only at start-up.  For
them the library offers one entry point whose working memory is a fixed
__device__ array inside the library.  This test drives it through the C ABI,
two calls in a row, and checks each result against the handle-based entry
point running the same FP64-accumulated M pass, within the 1e-10 relative
bar of the other FP64 parity tests.  It is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_noalloc_sweep_matches_handle_sweep_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import NMF_PREC_MIXED, StreamingNMF, _native, build
    build.build()
    L = _native.load()
    n, m, k = 1000, 300, 4
    ldm = (n + 31) // 32 * 32
    M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=21)
    X, Y = synth.init_factors(n, m, k, seed=21)
    X, Y, _, _, _, _, _ = oracle.anls(M, X, Y, max_sweeps=15)
    M32 = np.asfortranarray(M.astype(np.float32))

    # the handle-based entry point, FP64-accumulated pass, two sweeps
    with StreamingNMF(n, k, m, prec=NMF_PREC_MIXED, kkt_target=0.0) as h:
        h.append_columns(M32)
        h.set_factors(X, Y)
        h.set_pass_mode(1)
        h.sweep(1)
        X1, Y1, _, _ = h.get_factors()
        h.sweep(1)
        X2, Y2, _, _ = h.get_factors()

    # the allocation-free entry point on caller-owned device buffers
    dev = torch.device("cuda", 0)
    Md = torch.zeros((m, ldm), dtype=torch.float32, device=dev)      # column-major n x m, ld = ldm
    Md[:, :n] = torch.from_numpy(np.ascontiguousarray(M32.T))
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)            # n x k row-major
    Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).to(dev)          # k x m column-major
    st = torch.zeros(16, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    results = []
    for _ in range(2):
        s = L.nmf_sweep_noalloc(C.c_void_p(Md.data_ptr()), n, m, ldm, k, C.c_void_p(Xd.data_ptr()),
                                C.c_void_p(Yd.data_ptr()), C.c_void_p(st.data_ptr()), C.c_void_p(stream))
        assert s == _native.NMF_OK
        torch.cuda.synchronize(dev)
        results.append((Xd.cpu().numpy().copy(), Yd.cpu().numpy().T.copy(), st.cpu().numpy().copy()))
    (Xa, Ya, sa), (Xb, Yb, sb) = results
    assert _rel(Xa, X1) <= 1e-10 and _rel(Ya, Y1) <= 1e-10
    assert _rel(Xb, X2) <= 1e-10 and _rel(Yb, Y2) <= 1e-10
    # the record of the incoming iterate of the first call: its objective
    assert sa[1] == pytest.approx(oracle.objective(M, X, Y), rel=1e-9)
    assert sb[1] == pytest.approx(oracle.objective(M, X1, Y1), rel=1e-9)


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import _native, build
    build.build()
    L = _native.load()
    dev = torch.device("cuda", 0)
    buf = torch.zeros(64, dtype=torch.float64, device=dev)
    p = C.c_void_p(buf.data_ptr())
    assert L.nmf_sweep_noalloc(p, 4096, 10, 4096, 4, p, p, None, None) == _native.NMF_ECAPACITY
    assert L.nmf_sweep_noalloc(p, 100, 5000, 128, 4, p, p, None, None) == _native.NMF_ECAPACITY
    assert L.nmf_sweep_noalloc(p, 100, 10, 128, 9, p, p, None, None) == _native.NMF_ECAPACITY
    assert L.nmf_sweep_noalloc(p, 100, 10, 100, 4, p, p, None, None) == _native.NMF_EINVAL
