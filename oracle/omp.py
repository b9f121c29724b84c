"""Multicolour OpenMP form of the oracle's V-cycle (all-cores CPU baseline).

TEST INFRASTRUCTURE ONLY: used by the CPU-baseline leg of `bench.py` and by
the tests that pin it to the serial oracle.  The product library never calls
it.  App. "Multi-Color Gauss Seidel" is the paper's own CPU parallelisation:
the rows of one colour class do not couple, so a class is updated in parallel;
this module runs the oracle's cycle (Alg. 2, same hierarchy, same colour order,
same readings) with that parallel sweep and parallel transfers, over
`smg_omp.c`.  The coarsest direct solve is the oracle's serial one.
"""
import ctypes

import numpy as np

from . import build as _build
from . import chol_solve

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build_omp())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.omp_threads.restype = i64
        lib.omp_threads.argtypes = []
        lib.omp_gs_sweep.restype = i64
        lib.omp_gs_sweep.argtypes = [i64, p, p, p, p, p, p, p, i64, i64]
        lib.omp_residual.restype = None
        lib.omp_residual.argtypes = [i64, p, p, p, p, p, p, i64]
        lib.omp_spmv.restype = None
        lib.omp_spmv.argtypes = [i64, p, p, p, p, p, i64, i64]
        _LIB = lib
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads():
    """Threads the OpenMP loops use (OMP_NUM_THREADS, else all host cores)."""
    return int(_lib().omp_threads())


class _Csr:
    def __init__(self, M):
        M = M.tocsr()
        M.sort_indices()
        self.n = M.shape[0]
        self.ptr = np.ascontiguousarray(M.indptr, dtype=np.int64)
        self.col = np.ascontiguousarray(M.indices, dtype=np.int64)
        self.val = np.ascontiguousarray(M.data, dtype=np.float64)


class OmpLevels:
    """The oracle's levels (oracle.build_levels) in the arrays the loops take."""

    def __init__(self, levels):
        self.levels = []
        for lv in levels:
            d = {"A": _Csr(lv.A), "L": lv.L}
            if lv.P is not None:
                d["P"] = _Csr(lv.P)
                d["PT"] = _Csr(lv.P.T)
                k = int(lv.colour.max()) + 1
                d["cptr"] = np.concatenate([[0], np.cumsum(np.bincount(lv.colour, minlength=k))]).astype(np.int64)
                d["rows"] = np.ascontiguousarray(lv.fwd, dtype=np.int64)  # colour classes, ascending rows
                d["ncol"] = k
            self.levels.append(d)


def _relax(d, x, b, sweeps, reverse, nrhs):
    A = d["A"]
    for _ in range(sweeps):
        st = _lib().omp_gs_sweep(d["ncol"], _p(d["cptr"]), _p(d["rows"]), _p(A.ptr), _p(A.col), _p(A.val),
                                 _p(b), _p(x), nrhs, 1 if reverse else 0)
        if st != 0:
            raise ZeroDivisionError("zero diagonal in row %d" % (-st - 1))


def vcycle(ol, h, x, b, opt):
    """Alg. 2 from level h (the oracle's `vcycle`, binary64, Gauss-Seidel)."""
    d = ol.levels[h]
    if h == len(ol.levels) - 1:
        return chol_solve(d["L"], b)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    nrhs = 1 if b.ndim == 1 else b.shape[1]
    _relax(d, x, b, opt.mu_pre, False, nrhs)
    A, PT, P = d["A"], d["PT"], d["P"]
    r = np.empty_like(b)
    _lib().omp_residual(A.n, _p(A.ptr), _p(A.col), _p(A.val), _p(b), _p(x), _p(r), nrhs)
    rc = np.empty((PT.n,) + b.shape[1:])
    _lib().omp_spmv(PT.n, _p(PT.ptr), _p(PT.col), _p(PT.val), _p(r), _p(rc), nrhs, 0)
    c = np.ascontiguousarray(vcycle(ol, h + 1, np.zeros_like(rc), rc, opt))
    _lib().omp_spmv(P.n, _p(P.ptr), _p(P.col), _p(P.val), _p(c), _p(x), nrhs, 1)
    _relax(d, x, b, opt.mu_post, opt.post_reverse, nrhs)
    return x
