"""CPU oracle for sparse Cholesky: ctypes wrapper around oracle.c.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it; the library never does.  It shares no code with the CUDA
path.  Every function is a plain, slow, FP64, single-thread restatement of a definition:

* ``permute``     B = P^T A P (Sec. 2: the analysis phase reorders rows and columns)
* ``symbolic``    column-union pattern of L and the elimination tree (Sec. 2)
* ``supernodes``  fundamental supernodes cut to a width cap, and their level sets
                  (Sec. 2 amalgamation; Sec. 3 and Fig. 1 for the level sets)
* ``factor``      left-looking column Cholesky A = L L^T (Sec. 1; Sec. 3, Listing 1)
* ``solve``       L y = b, L^T x = y (Sec. 1, Sec. 2)
* ``residual``    max_c ||b - A x||_inf / (||A||_inf ||x||_inf)
* ``llt_error``   ||B - L L^T||_F / ||B||_F
* flop count      sum_j c_j^2 (c_j = rows of column j of L, diagonal included); the
                  factor loop counts its own operations so tests can check the model.

Parity status: every function is pinned by tests/test_oracle.py (dense brute force,
closed forms, invariants, the Fig. 1 level sets); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain -O2, no -ffast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        p = C.c_void_p
        i64 = C.c_int64
        L.orc_permute.argtypes = [i64, p, p, p, p, p, p, p]
        L.orc_symbolic.argtypes = [i64, p, p, p, p, p, C.POINTER(C.c_void_p)]
        L.orc_free.argtypes = [p]
        L.orc_supernodes.argtypes = [i64, p, p, i64, p, p, p, p]
        L.orc_factor.argtypes = [i64, p, p, p, p, p, p, p]
        L.orc_factor.restype = i64
        L.orc_solve.argtypes = [i64, p, p, p, p, i64, p, i64, p, i64]
        L.orc_spmv.argtypes = [i64, p, p, p, p, p]
        L.orc_residual.argtypes = [i64, p, p, p, i64, p, i64, p, i64, p]
        L.orc_llt_error.argtypes = [i64, p, p, p, p, p, p, p, p]
        L.orc_opt_d.argtypes = [i64, C.c_int32, p, p]
        L.orc_hybrid_uses_blas.argtypes = [i64, C.c_int32, i64]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class NotSPD(Exception):
    def __init__(self, col: int):
        super().__init__(f"matrix is not positive definite: pivot of column {col} <= 0")
        self.col = col


def permute(n, colptr, rowind, vals, perm):
    colptr, rowind, vals, perm = (_c(colptr, np.int64), _c(rowind, np.int32),
                                  _c(vals, np.float64), _c(perm, np.int32))
    nnz = int(colptr[n])
    bp = np.zeros(n + 1, np.int64)
    bi = np.zeros(max(nnz, 1), np.int32)
    bx = np.zeros(max(nnz, 1), np.float64)
    rc = lib().orc_permute(n, _ptr(colptr), _ptr(rowind), _ptr(vals), _ptr(perm),
                           _ptr(bp), _ptr(bi), _ptr(bx))
    if rc:
        raise ValueError(f"orc_permute: invalid input ({rc})")
    return bp, bi[:nnz], bx[:nnz]


def symbolic(n, bp, bi):
    """Returns parent[n], colcount[n], Lp[n+1], Li[nnzL]."""
    bp, bi = _c(bp, np.int64), _c(bi, np.int32)
    parent = np.zeros(n, np.int32)
    cc = np.zeros(n, np.int64)
    lp = np.zeros(n + 1, np.int64)
    li_ptr = C.c_void_p()
    rc = lib().orc_symbolic(n, _ptr(bp), _ptr(bi), _ptr(parent), _ptr(cc), _ptr(lp),
                            C.byref(li_ptr))
    if rc:
        raise MemoryError("orc_symbolic")
    nnz = int(lp[n])
    li = np.ctypeslib.as_array(C.cast(li_ptr, C.POINTER(C.c_int32)), shape=(max(nnz, 1),))
    li = li[:nnz].copy()
    lib().orc_free(li_ptr)
    return parent, cc, lp, li


def supernodes(parent, colcount, width_cap):
    """Returns sn_start[ns+1], sn_parent[ns], level[ns]."""
    n = len(parent)
    parent, colcount = _c(parent, np.int32), _c(colcount, np.int64)
    start = np.zeros(n + 1, np.int32)
    sp = np.zeros(max(n, 1), np.int32)
    lv = np.zeros(max(n, 1), np.int32)
    ns = C.c_int64()
    rc = lib().orc_supernodes(n, _ptr(parent), _ptr(colcount), int(width_cap), _ptr(start),
                              _ptr(sp), _ptr(lv), C.byref(ns))
    if rc:
        raise ValueError("orc_supernodes")
    k = ns.value
    return start[:k + 1].copy(), sp[:k].copy(), lv[:k].copy()


def factor(n, bp, bi, bx, lp, li):
    """Returns (Lx, flops counted by the loop).  Raises NotSPD."""
    bp, bi, bx, lp, li = (_c(bp, np.int64), _c(bi, np.int32), _c(bx, np.float64),
                          _c(lp, np.int64), _c(li, np.int32))
    lx = np.zeros(max(int(lp[n]), 1), np.float64)
    fl = C.c_double()
    bad = lib().orc_factor(n, _ptr(bp), _ptr(bi), _ptr(bx), _ptr(lp), _ptr(li), _ptr(lx),
                           C.byref(fl))
    if bad == -2:
        raise MemoryError("orc_factor")
    if bad >= 0:
        raise NotSPD(int(bad))
    return lx[:int(lp[n])], fl.value


def solve(n, lp, li, lx, perm, B):
    B = np.asfortranarray(np.asarray(B, dtype=np.float64).reshape(n, -1))
    X = np.zeros_like(B, order="F")
    lp, li, lx, perm = _c(lp, np.int64), _c(li, np.int32), _c(lx, np.float64), _c(perm, np.int32)
    lib().orc_solve(n, _ptr(lp), _ptr(li), _ptr(lx), _ptr(perm), B.shape[1], _ptr(B), n,
                    _ptr(X), n)
    return X


def spmv(n, colptr, rowind, vals, x):
    x = _c(x, np.float64)
    y = np.zeros(n)
    colptr, rowind, vals = _c(colptr, np.int64), _c(rowind, np.int32), _c(vals, np.float64)
    lib().orc_spmv(n, _ptr(colptr), _ptr(rowind), _ptr(vals), _ptr(x), _ptr(y))
    return y


def residual(n, colptr, rowind, vals, B, X):
    B = np.asfortranarray(np.asarray(B, dtype=np.float64).reshape(n, -1))
    X = np.asfortranarray(np.asarray(X, dtype=np.float64).reshape(n, -1))
    colptr, rowind, vals = _c(colptr, np.int64), _c(rowind, np.int32), _c(vals, np.float64)
    rel = C.c_double()
    lib().orc_residual(n, _ptr(colptr), _ptr(rowind), _ptr(vals), B.shape[1], _ptr(B), n,
                       _ptr(X), n, C.byref(rel))
    return rel.value


def opt_d(n, counts) -> int:
    """Threshold D of the OPT-D heuristic (Sec. 4.1, Algorithm 1) for outer tasks with the
    given numbers of inner tasks."""
    c = _c(np.asarray(counts, dtype=np.int32), np.int32)
    d = C.c_int32()
    rc = lib().orc_opt_d(int(n), len(c), _ptr(c) if len(c) else None, C.byref(d))
    if rc != 0:
        raise ValueError(f"orc_opt_d: {rc}")
    return d.value


def hybrid_uses_blas(n, nsuper, nnz) -> bool:
    """The hybrid switch of Sec. 4.3: True selects multi-threaded BLAS per supernode."""
    return bool(lib().orc_hybrid_uses_blas(int(n), int(nsuper), int(nnz)))


def llt_error(n, bp, bi, bx, lp, li, lx):
    """Returns ||B - L L^T||_F / ||B||_F."""
    args = [_c(bp, np.int64), _c(bi, np.int32), _c(bx, np.float64), _c(lp, np.int64),
            _c(li, np.int32), _c(lx, np.float64)]
    e, b = C.c_double(), C.c_double()
    lib().orc_llt_error(n, *[_ptr(a) for a in args], C.byref(e), C.byref(b))
    return e.value / b.value if b.value > 0 else e.value


@dataclass
class OracleFactor:
    n: int
    perm: np.ndarray
    bp: np.ndarray
    bi: np.ndarray
    bx: np.ndarray
    parent: np.ndarray
    colcount: np.ndarray
    lp: np.ndarray
    li: np.ndarray
    lx: np.ndarray
    flops_counted: float

    @property
    def nnz_l(self) -> int:
        return int(self.lp[-1])

    @property
    def flops(self) -> float:
        """Flop model sum_j c_j^2."""
        return float(np.sum(self.colcount.astype(np.float64) ** 2))

    def solve(self, B):
        return solve(self.n, self.lp, self.li, self.lx, self.perm, B)

    def supernodes(self, width_cap):
        return supernodes(self.parent, self.colcount, width_cap)


def cholesky(A, perm=None) -> OracleFactor:
    """Full oracle pipeline on an ``inputs.SpdMatrix``: permute, symbolic, factor."""
    n = A.n
    if perm is None:
        perm = np.arange(n, dtype=np.int32)
    bp, bi, bx = permute(n, A.colptr, A.rowind, A.vals, perm)
    parent, cc, lp, li = symbolic(n, bp, bi)
    lx, fl = factor(n, bp, bi, bx, lp, li)
    return OracleFactor(n, np.asarray(perm, np.int32), bp, bi, bx, parent, cc, lp, li, lx, fl)
