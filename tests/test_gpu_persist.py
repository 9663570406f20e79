"""nmf_save / nmf_load through the C ABI: a stream's resident window, iterate
and sweep state written to a file and read back into a new handle (Sec. 1's
streaming setting keeps a problem resident for as long as its columns keep
arriving; persistence lets that state outlive the process).  Sweeps of the
loaded handle must give bitwise the iterates, passive sets and statistics of
the saved handle, including a window that wraps around the ring and the
mixed-precision schedule part-way through."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import StreamingNMF, build
    build.build()
    return StreamingNMF


def _same(ha, hb):
    Xa, Ya, xa, ya = ha.get_factors()
    Xb, Yb, xb, yb = hb.get_factors()
    assert np.array_equal(Xa, Xb) and np.array_equal(Ya, Yb)
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)


@pytest.mark.parametrize("n,k,cap,prec,mode", [
    (900, 4, 300, 1, -1),      # mixed form, automatic schedule
    (640, 6, 200, 0, None),    # FP64 form
    (700, 16, 150, 1, 0),      # rank 16, tensor-core pass
])
def test_sweeps_after_load_are_bitwise_those_without(tmp_path, n, k, cap, prec, mode):
    S = _lib()
    import torch
    M, _, _ = synth.pdf_like(n, cap + 40, k, noise=1e-3, relative=True, seed=n + k)
    cols = np.asfortranarray(M.astype(np.float32) if prec == 1 else M)
    X, Y = synth.init_factors(n, cap, k, seed=n + k)
    a = S(n, k, cap, prec=prec, kkt_target=0.0)
    a.append_columns(np.asfortranarray(cols[:, :cap - 20]))
    a.append_columns(np.asfortranarray(cols[:, cap - 20:cap + 40]))   # evicts 40: the window wraps
    assert a.m == cap
    a.set_factors(X, Y)
    if mode is not None:
        a.set_pass_mode(mode)
    a.sweep(50)
    path = tmp_path / "state.nmf"
    a.save(path)
    stream = torch.cuda.Stream()
    b = S.load(path, stream=stream.cuda_stream)
    assert (b.n, b.k, b.m_capacity, b.m) == (n, k, cap, cap)
    _same(a, b)
    sa, sb = a.sweep(70), b.sweep(70)          # 32-sweep chunks: plain, captured, replayed
    assert sa == sb
    _same(a, b)
    assert a.objective_kkt() == b.objective_kkt()
    a.close()
    b.close()


def test_load_rejects_a_damaged_file(tmp_path):
    S = _lib()
    from paper_2101_08431_gb300 import NMFError
    n, k, m = 300, 3, 40
    M, _, _ = synth.pdf_like(n, m, k, seed=1)
    X, Y = synth.init_factors(n, m, k, seed=1)
    with S(n, k, m, prec=0) as a:
        a.append_columns(np.asfortranarray(M))
        a.set_factors(X, Y)
        a.sweep(3)
        path = tmp_path / "s.nmf"
        a.save(path)
    raw = path.read_bytes()
    for bad in (raw[:-1], raw + b"\0", b"XXXXXXXX" + raw[8:]):
        p = tmp_path / "bad.nmf"
        p.write_bytes(bad)
        with pytest.raises(NMFError) as e:
            S.load(p)
        assert e.value.status == 1
    b = S.load(path)                    # the intact file still loads
    assert b.m == m
    b.close()
