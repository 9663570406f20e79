"""ctypes front end of the CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library never
does.  The C file is compiled here with the system C compiler into
``oracle/_build/liboracle.so`` (plain ``-O2``, single-threaded).

Array conventions follow Sec. 3.1 of the paper: M is n x m column-major, X is
n x k row-major (so its buffer is x = vec(X^T)), Y is k x m column-major (its
buffer is y = vec(Y)).  The wrappers take and return numpy arrays in the
natural (n, m) / (n, k) / (k, m) shapes and handle the layouts.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

OK, EINVAL, NOTCONV, ENUMERIC, NOTPD = 0, 1, 4, 6, 7

_lib = None
_dp = C.POINTER(C.c_double)
_up = C.POINTER(C.c_uint32)


_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle shared library (idempotent).  openmp=True builds the
    same source with -fopenmp into a second library, whose sweep shares the
    independent column and row problems among the host's threads (for the
    all-cores CPU baseline); every value it computes is the serial build's."""
    os.makedirs(_BUILD, exist_ok=True)
    lib_path = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < os.path.getmtime(_SRC):
        tmp = lib_path + ".tmp.%d" % os.getpid()
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11"] + flags + ["-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib_path)
    return lib_path


_lib_omp = None


def lib(openmp: bool = False):
    global _lib, _lib_omp
    if openmp:
        if _lib_omp is None:
            _lib_omp = _declare(C.CDLL(build(openmp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(L):
    """Argument types of the oracle's C functions on the loaded library L."""
    i64, i32, d = C.c_int64, C.c_int, C.c_double
    L.oracle_nnls.argtypes = [i32, _dp, _dp, _dp, _up, C.POINTER(C.c_int)]
    L.oracle_nnls_warm.argtypes = [i32, _dp, _dp, _dp, _up, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.oracle_sweep.argtypes = [i64, i64, i32, _dp, i64, _dp, _dp, _up, _up, C.POINTER(C.c_int64)]
    L.oracle_grad.argtypes = [i64, i64, i32, _dp, i64, _dp, _dp, _dp, _dp]
    L.oracle_grad.restype = d
    L.oracle_objective.argtypes = [i64, i64, i32, _dp, i64, _dp, _dp]
    L.oracle_objective.restype = d
    L.oracle_kkt.argtypes = [i64, i64, i32, _dp, i64, _dp, _dp, _dp]
    L.oracle_anls.argtypes = [i64, i64, i32, _dp, i64, _dp, _dp, _up, _up, i32, d, d, _dp,
                              C.POINTER(C.c_int)]
    L.oracle_ipm_direction.argtypes = [i64, i64, i32, _dp, i64, _dp, _dp, _dp, _dp, d, d, i32,
                                       _dp, _dp, _dp, _dp]
    L.oracle_ipm.argtypes = [i64, i64, i32, _dp, i64, _dp, _dp, d, i32, _dp, _dp, i32,
                             C.POINTER(C.c_int)]
    L.oracle_two_stage.argtypes = [i64, i64, i32, _dp, i64, _dp, _dp, d, i32, d, i32, _dp]
    return L


def _p(a):
    return a.ctypes.data_as(_dp)


def _colmajor(M):
    return np.asfortranarray(np.asarray(M, dtype=np.float64))


def _xbuf(X):
    """Fresh row-major float64 copy (safe to hand to C for writing)."""
    return np.array(X, dtype=np.float64, order="C", copy=True)


def _ybuf(Y):
    """Fresh column-major float64 copy (safe to hand to C for writing)."""
    return np.array(Y, dtype=np.float64, order="F", copy=True)


def nnls(G, b):
    """Cold-start Lawson-Hanson NNLS of min 1/2 y'Gy - b'y, y >= 0.

    Returns (y, passive mask, outer iterations, status)."""
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    k = b.shape[0]
    y = np.zeros(k)
    mask = C.c_uint32(0)
    it = C.c_int(0)
    st = lib().oracle_nnls(k, _p(G), _p(b), _p(y), C.byref(mask), C.byref(it))
    return y, mask.value, it.value, st


def nnls_warm(G, b, y0):
    """Warm-started Lawson-Hanson from the support of y0 (Sec. 2's reuse of the
    previous problem's solution).  Returns (y, passive mask, entering steps,
    passive-set changes, status)."""
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    y = np.ascontiguousarray(np.maximum(np.asarray(y0, dtype=np.float64), 0.0)).copy()
    k = b.shape[0]
    mask = C.c_uint32(0)
    it = C.c_int(0)
    ch = C.c_int(0)
    st = lib().oracle_nnls_warm(k, _p(G), _p(b), _p(y), C.byref(mask), C.byref(it), C.byref(ch))
    return y, mask.value, it.value, ch.value, st


def sweep(M, X, Y, openmp=False):
    """One ANLS sweep (Y-update, then X-update). Returns (X, Y, xmask, ymask, status).
    openmp=True runs the -fopenmp build (columns and rows on all host threads)."""
    Mf = _colmajor(M)
    n, m = Mf.shape
    X = _xbuf(X)
    Y = _ybuf(Y)
    k = X.shape[1]
    xm = np.zeros(n, dtype=np.uint32)
    ym = np.zeros(m, dtype=np.uint32)
    nc = C.c_int64(0)
    st = lib(openmp).oracle_sweep(n, m, k, _p(Mf), n, _p(X), _p(Y), xm.ctypes.data_as(_up),
                                  ym.ctypes.data_as(_up), C.byref(nc))
    return X, Y, xm, ym, st


def grad(M, X, Y):
    """(f, graX, graY) with f = 1/2||XY-M||^2, graX = (XY-M)Y^T, graY = X^T(XY-M)."""
    Mf = _colmajor(M)
    n, m = Mf.shape
    Xb, Yb = _xbuf(X), _ybuf(Y)
    k = Xb.shape[1]
    gX = np.zeros((n, k))
    gY = np.zeros((k, m), order="F")
    f = lib().oracle_grad(n, m, k, _p(Mf), n, _p(Xb), _p(Yb), _p(gX), _p(gY))
    return f, gX, np.ascontiguousarray(gY)


def objective(M, X, Y):
    Mf = _colmajor(M)
    n, m = Mf.shape
    Xb, Yb = _xbuf(X), _ybuf(Y)
    return lib().oracle_objective(n, m, Xb.shape[1], _p(Mf), n, _p(Xb), _p(Yb))


KKT_FIELDS = ("E_abs", "rel", "neg", "comp", "s_g", "xymax", "f")


def kkt(M, X, Y):
    """KKT violation of an ANLS point; dict with the fields of KKT_FIELDS."""
    Mf = _colmajor(M)
    n, m = Mf.shape
    Xb, Yb = _xbuf(X), _ybuf(Y)
    out = np.zeros(7)
    st = lib().oracle_kkt(n, m, Xb.shape[1], _p(Mf), n, _p(Xb), _p(Yb), _p(out))
    if st != OK:
        raise ValueError("oracle_kkt status %d" % st)
    return dict(zip(KKT_FIELDS, out.tolist()))


def anls(M, X, Y, max_sweeps=100, stol=0.0, kkt_target=0.0, want_trace=False):
    """Stage-1 ANLS driver.  Returns (X, Y, xmask, ymask, sweeps, trace, status);
    trace rows are (f, E_abs, rel KKT, relative step) per evaluated point."""
    Mf = _colmajor(M)
    n, m = Mf.shape
    X = _xbuf(X)
    Y = _ybuf(Y)
    k = X.shape[1]
    xm = np.zeros(n, dtype=np.uint32)
    ym = np.zeros(m, dtype=np.uint32)
    trace = np.zeros((max_sweeps + 1, 4)) if want_trace else None
    sw = C.c_int(0)
    st = lib().oracle_anls(n, m, k, _p(Mf), n, _p(X), _p(Y), xm.ctypes.data_as(_up),
                           ym.ctypes.data_as(_up), int(max_sweeps), float(stol), float(kkt_target),
                           _p(trace) if want_trace else C.cast(None, _dp), C.byref(sw))
    if want_trace:
        trace = trace[: sw.value + 1]
    return X, Y, xm, ym, sw.value, trace, st


def ipm_direction(M, X, Y, R, S, mu, rho, full):
    """Primal-dual direction of eq. "eqn:equation" via the Schur complement of Sec. 3.2.

    R is the dual of X (n x k), S the dual of Y (k x m).  Returns
    (dX, dY, dR, dS, status) in the natural shapes."""
    Mf = _colmajor(M)
    n, m = Mf.shape
    Xb, Yb, Rb, Sb = _xbuf(X), _ybuf(Y), _xbuf(R), _ybuf(S)
    k = Xb.shape[1]
    dX = np.zeros((n, k))
    dR = np.zeros((n, k))
    dY = np.zeros((k, m), order="F")
    dS = np.zeros((k, m), order="F")
    st = lib().oracle_ipm_direction(n, m, k, _p(Mf), n, _p(Xb), _p(Yb), _p(Rb), _p(Sb),
                                    float(mu), float(rho), int(full), _p(dX), _p(dY), _p(dR), _p(dS))
    return dX, np.ascontiguousarray(dY), dR, np.ascontiguousarray(dS), st


IPM_STATS = ("E0", "f", "newton", "outer", "mu", "full_hessian_steps", "armijo_failures")


def ipm(M, X, Y, eps_tol=1e-6, max_newton=500, trace_cap=0):
    """Stage 2 from the point (X, Y).  Returns (X, Y, stats dict, trace, status);
    trace rows are (outer index, mu, phi before, phi after, full Hessian used,
    alpha_1, alpha_2, E(.;mu) before the step)."""
    Mf = _colmajor(M)
    n, m = Mf.shape
    X = _xbuf(X)
    Y = _ybuf(Y)
    k = X.shape[1]
    stats = np.zeros(8)
    tr = np.zeros((max(trace_cap, 1), 8))
    nt = C.c_int(0)
    st = lib().oracle_ipm(n, m, k, _p(Mf), n, _p(X), _p(Y), float(eps_tol), int(max_newton),
                          _p(stats), _p(tr), int(trace_cap), C.byref(nt))
    return (X, np.ascontiguousarray(Y), dict(zip(IPM_STATS, stats[:7].tolist())),
            tr[: nt.value], st)


def two_stage(M, X, Y, stol=1e-4, max_sweeps=2000, eps_tol=1e-6, max_newton=500):
    """Alg. "alg:fast".  Returns (X, Y, stats dict incl. 'sweeps', status)."""
    Mf = _colmajor(M)
    n, m = Mf.shape
    X = _xbuf(X)
    Y = _ybuf(Y)
    k = X.shape[1]
    stats = np.zeros(8)
    st = lib().oracle_two_stage(n, m, k, _p(Mf), n, _p(X), _p(Y), float(stol), int(max_sweeps),
                                float(eps_tol), int(max_newton), _p(stats))
    d = dict(zip(IPM_STATS, stats[:7].tolist()))
    d["sweeps"] = int(stats[7])
    return X, np.ascontiguousarray(Y), d, st
