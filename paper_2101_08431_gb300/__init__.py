"""GB300 (sm_103a) library for the stage-1 ANLS sweep of two-stage streaming
NMF (Gu, Du & Billinge, arXiv 2101.08431).

The Python layer marshals arguments to the C ABI of ``include/nmf.h``; every
step of the method runs in the library's CUDA kernels.  ``StreamingNMF`` is a
convenience wrapper around one handle; ``_native`` exposes the raw functions
under their C names.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native
from ._native import (NMF_DTYPE_F32, NMF_DTYPE_F64, NMF_PREC_FP64, NMF_PREC_MIXED, NMF_WARM_COLD,
                      NMF_WARM_CHAIN, NMF_WARM_PREV, NMFError, check, load, nmf_config, nmf_stats)

__all__ = ["StreamingNMF", "StreamingNMFBatch", "StreamingServer", "NMFError", "load", "nmf_config", "nmf_stats",
           "measure_fma_peaks", "NMF_PREC_FP64",
           "NMF_PREC_MIXED", "NMF_DTYPE_F32", "NMF_DTYPE_F64", "NMF_WARM_COLD", "NMF_WARM_PREV", "NMF_WARM_CHAIN"]


def _ptr(a):
    """(address, on_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError("expected a numpy array or a torch tensor")


def _cols_arg(cols):
    """(address, ncols, ld, dtype, on_device, keep-alive) of n x c columns."""
    if isinstance(cols, np.ndarray):
        a = np.asfortranarray(cols)
        dtype = NMF_DTYPE_F32 if a.dtype == np.float32 else NMF_DTYPE_F64
        if a.dtype not in (np.float32, np.float64):
            a = np.asfortranarray(a, dtype=np.float64)
            dtype = NMF_DTYPE_F64
        return a.ctypes.data, int(a.shape[1]), int(max(a.shape[0], 1)), dtype, 0, a
    t = cols   # torch tensor, column-major view expected: stride (1, ld)
    if t.stride(0) != 1:
        t = t.t().contiguous().t()
    dtype = NMF_DTYPE_F32 if str(t.dtype) == "torch.float32" else NMF_DTYPE_F64
    return t.data_ptr(), int(t.shape[1]), int(max(t.stride(1), 1)), dtype, int(t.is_cuda), t


def _config(lib, n, k, m_capacity, prec, kkt_target, stol, mixed_switch, max_sweeps, warm_start, stream):
    cfg = nmf_config()
    lib.nmf_config_init(C.byref(cfg))
    cfg.n, cfg.m_capacity, cfg.k, cfg.prec = int(n), int(m_capacity), int(k), int(prec)
    cfg.kkt_target, cfg.stol, cfg.mixed_switch = float(kkt_target), float(stol), float(mixed_switch)
    cfg.max_sweeps, cfg.warm_start = int(max_sweeps), int(warm_start)
    cfg.cuda_stream = stream
    return cfg


class StreamingNMF:
    """One problem: min 1/2||XY - M||^2, X, Y >= 0, columns of M appended over time."""

    def __init__(self, n, k, m_capacity, prec=NMF_PREC_MIXED, kkt_target=1e-8, stol=0.0,
                 mixed_switch=1e-6, max_sweeps=100000, warm_start=NMF_WARM_PREV, stream=None, kkt_abs_target=0.0):
        self.lib = load()
        cfg = nmf_config()
        self.lib.nmf_config_init(C.byref(cfg))
        cfg.n, cfg.m_capacity, cfg.k, cfg.prec = int(n), int(m_capacity), int(k), int(prec)
        cfg.kkt_target, cfg.stol, cfg.mixed_switch = float(kkt_target), float(stol), float(mixed_switch)
        cfg.max_sweeps, cfg.warm_start = int(max_sweeps), int(warm_start)
        cfg.cuda_stream = stream
        cfg.kkt_abs_target = float(kkt_abs_target)
        h = C.c_void_p()
        check(self.lib.nmf_create(C.byref(cfg), C.byref(h)))
        self.h = h
        self.n, self.k, self.m_capacity = int(n), int(k), int(m_capacity)

    # -- data -------------------------------------------------------------------
    def append_columns(self, cols):
        """cols: n x c (numpy or torch, float32/float64); any strides with unit row stride."""
        ptr, ncols, ld, dtype, dev, keep = _cols_arg(cols)
        st = self.lib.nmf_append_columns(self.h, C.c_void_p(ptr), ncols, ld, dtype, dev)
        del keep
        return check(st, self.h)

    @property
    def m(self):
        return int(self.lib.nmf_num_columns(self.h))

    def set_factors(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.asfortranarray(Y, dtype=np.float64)
        check(self.lib.nmf_set_factors(self.h, C.c_void_p(X.ctypes.data), C.c_void_p(Y.ctypes.data), 0),
              self.h)

    def get_factors(self):
        m = self.m
        X = np.zeros((self.n, self.k))
        Y = np.zeros((self.k, m), order="F")
        xm = np.zeros(self.n, dtype=np.uint32)
        ym = np.zeros(m, dtype=np.uint32)
        check(self.lib.nmf_get_factors(self.h, C.c_void_p(X.ctypes.data), C.c_void_p(Y.ctypes.data),
                                       C.c_void_p(xm.ctypes.data), C.c_void_p(ym.ctypes.data), 0), self.h)
        return X, np.ascontiguousarray(Y), xm, ym

    # -- iteration --------------------------------------------------------------
    def set_pass_mode(self, mode):
        check(self.lib.nmf_set_pass_mode(self.h, int(mode)), self.h)

    def sweep(self, nsweeps=1, want_stats=True, allow_notconv=False):
        st = nmf_stats()
        s = self.lib.nmf_sweep(self.h, int(nsweeps), C.byref(st) if want_stats else None)
        if allow_notconv and s == _native.NMF_ENOTCONV:
            return st.as_dict()
        check(s, self.h)
        return st.as_dict() if want_stats else None

    def objective_kkt(self):
        f, e, r = C.c_double(), C.c_double(), C.c_double()
        check(self.lib.nmf_objective_kkt(self.h, C.byref(f), C.byref(e), C.byref(r)), self.h)
        return {"f": f.value, "kkt_abs": e.value, "kkt_rel": r.value}

    def set_timing(self, on=True):
        check(self.lib.nmf_set_timing(self.h, int(bool(on))), self.h)

    def get_timing(self):
        ym, xm = C.c_double(), C.c_double()
        yl, xl = C.c_int64(), C.c_int64()
        check(self.lib.nmf_get_timing(self.h, C.byref(ym), C.byref(yl), C.byref(xm), C.byref(xl)), self.h)
        return {"ypass_ms": ym.value, "ypass_launches": yl.value, "xpass_ms": xm.value,
                "xpass_launches": xl.value}

    PASSES = {"f32": 0, "ref": 1, "df": 2, "inc": 3, "f64": 4}

    def get_pass_timing(self, name):
        """Device time of one pass variant's M and row passes since
        set_timing(True): {"ypass_ms", "xpass_ms", "sweeps"}."""
        ym, xm, n = C.c_double(), C.c_double(), C.c_int64()
        check(self.lib.nmf_get_pass_timing(self.h, self.PASSES[name], C.byref(ym), C.byref(xm), C.byref(n)),
              self.h)
        return {"ypass_ms": ym.value, "xpass_ms": xm.value, "sweeps": n.value}

    @property
    def launches(self):
        return int(self.lib.nmf_launch_count(self.h))

    # -- column sharding (one rank's share of a multi-GPU sweep) ----------------
    def shard_y_half(self):
        """The Y half on this handle's columns; returns (sum_buf, max_buf),
        host arrays to be all-reduced (sum, max) across the ranks."""
        n = int(self.lib.nmf_shard_buffer_len(self.n, self.k))
        sb, mb = np.zeros(n), np.zeros(1)
        check(self.lib.nmf_shard_y_half(self.h, C.c_void_p(sb.ctypes.data), C.c_void_p(mb.ctypes.data), 0), self.h)
        return sb, mb

    def shard_x_half(self, sum_buf, max_buf):
        """The X half from the all-reduced buffers; returns the statistics of
        the incoming iterate over the whole problem."""
        sb = np.ascontiguousarray(sum_buf, dtype=np.float64)
        mb = np.ascontiguousarray(max_buf, dtype=np.float64)
        st = nmf_stats()
        check(self.lib.nmf_shard_x_half(self.h, C.c_void_p(sb.ctypes.data), C.c_void_p(mb.ctypes.data), 0,
                                        C.byref(st)), self.h)
        return st.as_dict()

    # -- stage 2 (Sec. 3-4) --------------------------------------------------------
    IPM_STATS = ("E0", "f", "newton", "outer", "mu", "full_hessian_steps", "armijo_failures")

    def ipm(self, eps_tol=1e-6, max_newton=500, allow_notconv=False):
        """Stage 2 from the current iterate; returns its statistics (the
        result becomes the handle's iterate)."""
        st = np.zeros(7)
        s = self.lib.nmf_ipm(self.h, float(eps_tol), int(max_newton), st.ctypes.data_as(C.POINTER(C.c_double)))
        if not (allow_notconv and s == _native.NMF_ENOTCONV):
            check(s, self.h)
        d = dict(zip(self.IPM_STATS, st.tolist()))
        d["status"] = s
        return d

    def ipm_direction(self, R, S, mu, rho, full):
        """One Newton direction of stage 2 at the current iterate for duals
        R (n x k) and S (k x m): (dX, dY, dR, dS)."""
        m = self.m
        R = np.ascontiguousarray(R, dtype=np.float64)
        S = np.asfortranarray(S, dtype=np.float64)
        dX, dR = np.zeros((self.n, self.k)), np.zeros((self.n, self.k))
        dY, dS = np.zeros((self.k, m), order="F"), np.zeros((self.k, m), order="F")
        ptr = lambda a: C.c_void_p(a.ctypes.data)
        check(self.lib.nmf_ipm_direction(self.h, ptr(R), ptr(S), float(mu), float(rho), int(bool(full)), ptr(dX),
                                         ptr(dY), ptr(dR), ptr(dS), 0), self.h)
        return dX, np.ascontiguousarray(dY), dR, np.ascontiguousarray(dS)

    # -- persistence ------------------------------------------------------------
    def save(self, path):
        """Write the handle's window, iterate and sweep state to path."""
        check(self.lib.nmf_save(self.h, str(path).encode()), self.h)

    @classmethod
    def load(cls, path, stream=None):
        """A new handle holding the state saved at path (on `stream`)."""
        self = cls.__new__(cls)
        self.lib = load()
        h = C.c_void_p()
        check(self.lib.nmf_load(str(path).encode(), stream, C.byref(h)))
        self.h = h
        cfg = nmf_config()
        check(self.lib.nmf_get_config(h, C.byref(cfg)), h)
        self.n, self.k, self.m_capacity = int(cfg.n), int(cfg.k), int(cfg.m_capacity)
        return self

    def close(self):
        if getattr(self, "h", None):
            self.lib.nmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class StreamingNMFBatch:
    """Many independent problems (n_j, k_j, m_capacity_j) swept together by the
    batched persistent launches of the library (FP32 M, mixed precision)."""

    def __init__(self, shapes, kkt_target=1e-8, stol=0.0, mixed_switch=1e-6, max_sweeps=100000,
                 warm_start=NMF_WARM_PREV, stream=None):
        self.lib = load()
        self.shapes = [(int(n), int(k), int(mc)) for n, k, mc in shapes]
        arr = (nmf_config * len(self.shapes))()
        for j, (n, k, mc) in enumerate(self.shapes):
            arr[j] = _config(self.lib, n, k, mc, NMF_PREC_MIXED, kkt_target, stol, mixed_switch, max_sweeps,
                             warm_start, None)
        b = C.c_void_p()
        check(self.lib.nmf_batch_create(arr, len(self.shapes), stream, C.byref(b)))
        self.b = b

    def __len__(self):
        return len(self.shapes)

    def _chk(self, st):
        return check(st, batch=self.b)

    def append_columns(self, j, cols):
        ptr, ncols, ld, dtype, dev, keep = _cols_arg(cols)
        st = self.lib.nmf_batch_append_columns(self.b, int(j), C.c_void_p(ptr), ncols, ld, dtype, dev)
        del keep
        return self._chk(st)

    def m(self, j):
        return int(self.lib.nmf_num_columns(self.lib.nmf_batch_problem(self.b, int(j))))

    def set_factors(self, j, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.asfortranarray(Y, dtype=np.float64)
        self._chk(self.lib.nmf_batch_set_factors(self.b, int(j), C.c_void_p(X.ctypes.data),
                                                 C.c_void_p(Y.ctypes.data), 0))

    def get_factors(self, j):
        n, k, _ = self.shapes[j]
        m = self.m(j)
        X = np.zeros((n, k))
        Y = np.zeros((k, m), order="F")
        xm = np.zeros(n, dtype=np.uint32)
        ym = np.zeros(m, dtype=np.uint32)
        self._chk(self.lib.nmf_batch_get_factors(self.b, int(j), C.c_void_p(X.ctypes.data),
                                                 C.c_void_p(Y.ctypes.data), C.c_void_p(xm.ctypes.data),
                                                 C.c_void_p(ym.ctypes.data), 0))
        return X, np.ascontiguousarray(Y), xm, ym

    def set_pass_mode(self, mode):
        self._chk(self.lib.nmf_batch_set_pass_mode(self.b, int(mode)))

    def set_schedule(self, cols_per_item, stage_cap=8):
        self._chk(self.lib.nmf_batch_set_schedule(self.b, int(cols_per_item), int(stage_cap)))

    def sweep(self, max_sweeps=0, allow_notconv=False):
        """Returns (per-problem statistics, batch sweeps launched)."""
        sts = (nmf_stats * len(self.shapes))()
        nrun = C.c_int32()
        s = self.lib.nmf_batch_sweep(self.b, int(max_sweeps), sts, C.byref(nrun))
        if not (allow_notconv and s == _native.NMF_ENOTCONV):
            self._chk(s)
        return [sts[j].as_dict() for j in range(len(self.shapes))], int(nrun.value)

    def autotune(self, trial_sweeps=3):
        c, sc, ms = C.c_int32(), C.c_int32(), C.c_double()
        self._chk(self.lib.nmf_batch_autotune(self.b, int(trial_sweeps), C.byref(c), C.byref(sc), C.byref(ms)))
        return {"cols_per_item": c.value, "stage_cap": sc.value, "ms_per_sweep": ms.value}

    def objective_kkt(self, j):
        h = self.lib.nmf_batch_problem(self.b, int(j))
        f, e, r = C.c_double(), C.c_double(), C.c_double()
        check(self.lib.nmf_objective_kkt(h, C.byref(f), C.byref(e), C.byref(r)), h)
        return {"f": f.value, "kkt_abs": e.value, "kkt_rel": r.value}

    @property
    def launches(self):
        return int(self.lib.nmf_batch_launch_count(self.b))

    def close(self):
        if getattr(self, "b", None):
            self.lib.nmf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class StreamingServer:
    """The library's streaming server: streams of time columns arriving in
    chunks, served by a worker thread with continuous batching."""

    def __init__(self, hbm_budget_bytes=0, max_streams=64, kkt_target=1e-6, mixed_switch=1e-6,
                 max_sweeps_per_chunk=500, sweeps_per_round=8, stream=None):
        self.lib = load()
        cfg = _native.nmf_server_config()
        self.lib.nmf_server_config_init(C.byref(cfg))
        cfg.hbm_budget_bytes, cfg.max_streams = int(hbm_budget_bytes), int(max_streams)
        cfg.kkt_target, cfg.mixed_switch = float(kkt_target), float(mixed_switch)
        cfg.max_sweeps_per_chunk, cfg.sweeps_per_round = int(max_sweeps_per_chunk), int(sweeps_per_round)
        cfg.cuda_stream = stream
        s = C.c_void_p()
        check(self.lib.nmf_server_create(C.byref(cfg), C.byref(s)))
        self.s = s
        self.shape = {}

    def _chk(self, st):
        if st != _native.NMF_OK:
            detail = self.lib.nmf_server_last_error(self.s).decode() if self.s else ""
            raise NMFError(st, "%s%s" % (self.lib.nmf_status_string(st).decode(), (": " + detail) if detail else ""))
        return st

    def open_stream(self, n, k, m_capacity, seed=0):
        i = C.c_int32()
        self._chk(self.lib.nmf_server_open_stream(self.s, int(n), int(k), int(m_capacity), int(seed), C.byref(i)))
        self.shape[i.value] = (int(n), int(k), int(m_capacity))
        return i.value

    def submit(self, sid, cols):
        """cols: n x c float32 (numpy); returns the chunk's ticket."""
        a = np.asfortranarray(cols, dtype=np.float32)
        t = C.c_uint64()
        self._chk(self.lib.nmf_server_submit(self.s, int(sid), C.c_void_p(a.ctypes.data), int(a.shape[1]),
                                             int(a.shape[0]), C.byref(t)))
        return int(t.value)

    def close_stream(self, sid):
        self._chk(self.lib.nmf_server_close_stream(self.s, int(sid)))

    def poll(self, wait_ms=0, cap=1024):
        out = (_native.nmf_chunk_result * cap)()
        n = C.c_int32()
        self._chk(self.lib.nmf_server_poll(self.s, out, int(cap), C.byref(n), int(wait_ms)))
        return [out[i].as_dict() for i in range(n.value)]

    def get_factors(self, sid):
        n, k, mcap = self.shape[sid]
        X = np.zeros((n, k))
        Y = np.zeros((k, mcap), order="F")
        xm = np.zeros(n, dtype=np.uint32)
        ym = np.zeros(mcap, dtype=np.uint32)
        m = C.c_int64()
        self._chk(self.lib.nmf_server_get_factors(self.s, int(sid), C.c_void_p(X.ctypes.data),
                                                  C.c_void_p(Y.ctypes.data), C.c_void_p(xm.ctypes.data),
                                                  C.c_void_p(ym.ctypes.data), C.byref(m)))
        mm = int(m.value)
        return X, np.ascontiguousarray(Y[:, :mm]), xm, ym[:mm]

    def stats(self):
        st = _native.nmf_server_stats()
        self._chk(self.lib.nmf_server_get_stats(self.s, C.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "s", None):
            self.lib.nmf_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def measure_fma_peaks(stream=None):
    """Measured FMA throughput of the current device in TFLOP/s (2 flops per
    FMA): {"fp64_tflops", "fp32_tflops"} (``nmf_measure_fma_peaks``)."""
    lib = load()
    out = (C.c_double * 2)()
    check(lib.nmf_measure_fma_peaks(out, C.c_void_p(stream or 0)))
    return {"fp64_tflops": out[0], "fp32_tflops": out[1]}
