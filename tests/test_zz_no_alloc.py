"""nmf_sweep_noalloc: the sweep for callers that cannot allocate device memory.

Some callers must not allocate where they run the sweep: a latency-critical
loop that cannot block on cudaMalloc, a plug-in whose host framework has
reserved all device memory, code that may allocate only at start-up.  For
them the library offers one entry point whose working memory is a fixed
__device__ array inside the library.  This test drives it through the C ABI,
a larger problem and then a smaller one called twice in a row, and checks
each result against the handle-based entry point running the same
FP64-accumulated M pass, within the 1e-10 relative bar (per column of Y,
per row of X) of the other FP64 parity tests.  It is collected last on
purpose.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from _parity import colmax_rel

pytestmark = pytest.mark.gpu


def _handle_sweeps(n, m, k, M32, X, Y, nsweeps):
    """The handle-based entry point, FP64-accumulated pass: the iterates after
    each of nsweeps sweeps from (X, Y)."""
    from paper_2101_08431_gb300 import NMF_PREC_MIXED, StreamingNMF
    out = []
    with StreamingNMF(n, k, m, prec=NMF_PREC_MIXED, kkt_target=0.0) as h:
        h.append_columns(M32)
        h.set_factors(X, Y)
        h.set_pass_mode(1)
        for _ in range(nsweeps):
            h.sweep(1)
            Xg, Yg, _, _ = h.get_factors()
            out.append((Xg, Yg))
    return out


def _device_problem(torch, M32, X, Y):
    """Caller-owned device buffers in the entry point's layouts."""
    n, m = M32.shape
    ldm = (n + 31) // 32 * 32
    dev = torch.device("cuda", 0)
    Md = torch.zeros((m, ldm), dtype=torch.float32, device=dev)      # column-major n x m, ld = ldm
    Md[:, :n] = torch.from_numpy(np.ascontiguousarray(M32.T))
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)            # n x k row-major
    Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).to(dev)          # k x m column-major
    st = torch.zeros(16, dtype=torch.float64, device=dev)
    return Md, Xd, Yd, st, ldm


def _call(L, torch, Md, n, m, ldm, k, Xd, Yd, st):
    stream = torch.cuda.current_stream(Md.device).cuda_stream
    s = L.nmf_sweep_noalloc(C.c_void_p(Md.data_ptr()), n, m, ldm, k, C.c_void_p(Xd.data_ptr()),
                            C.c_void_p(Yd.data_ptr()), C.c_void_p(st.data_ptr()), C.c_void_p(stream))
    assert s == 0
    torch.cuda.synchronize(Md.device)
    return Xd.cpu().numpy().copy(), Yd.cpu().numpy().T.copy(), st.cpu().numpy().copy()


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import _native, build
    build.build()
    return torch, _native.load()


def test_noalloc_sweep_matches_handle_sweep_twice():
    torch, L = _setup()
    # a larger problem of another rank first, so that the smaller problem
    # after it runs on an array that still holds a bigger call's contents
    # (masks, the subset table of G, the FP32 split of X, the partials)
    cases = [(2000, 4000, 8, 22, 1), (1000, 300, 4, 21, 2)]
    for n, m, k, seed, calls in cases:
        M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=seed)
        X, Y = synth.init_factors(n, m, k, seed=seed)
        X, Y, _, _, _, _, _ = oracle.anls(M, X, Y, max_sweeps=6)
        M32 = np.asfortranarray(M.astype(np.float32))
        ref = _handle_sweeps(n, m, k, M32, X, Y, calls)
        Md, Xd, Yd, st, ldm = _device_problem(torch, M32, X, Y)
        Xin, Yin = X, Y
        for c in range(calls):
            Xa, Ya, sa = _call(L, torch, Md, n, m, ldm, k, Xd, Yd, st)
            Xr, Yr = ref[c]
            assert colmax_rel(Ya, Yr, axis=0) <= 1e-10 and colmax_rel(Xa, Xr, axis=1) <= 1e-10, (n, m, k, c)
            assert sa[15] == 0.0                        # no device error
            # the record of the incoming iterate: its objective
            assert sa[1] == pytest.approx(oracle.objective(M, Xin, Yin), rel=1e-9)
            Xin, Yin = Xa, Ya


def test_noalloc_reports_nonfinite_data_and_keeps_the_iterate():
    torch, L = _setup()
    n, m, k = 500, 120, 3
    M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=23)
    X, Y = synth.init_factors(n, m, k, seed=23)
    M32 = np.asfortranarray(M.astype(np.float32))
    M32[17, 40] = np.nan
    Md, Xd, Yd, st, ldm = _device_problem(torch, M32, X, Y)
    Xa, Ya, sa = _call(L, torch, Md, n, m, ldm, k, Xd, Yd, st)
    assert int(sa[15]) & 2                              # the non-finite bit
    np.testing.assert_array_equal(Xa, X)
    np.testing.assert_array_equal(Ya, Y)


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
