"""Multi-core CPU baseline of the paper's own method: left-looking supernodal Cholesky as
OpenMP tasks under the task-granularity policies of Sec. 4 (NONESTED, NESTED, OPT-D,
OPT-D-COST).  A comparison point timed on the host cores; it shares no code with the library
or the oracle.  The supernode partition and panel row lists come from the library's analysis
through the C ABI (``chol_sym_export``, ``chol_sym_rows``)."""
import ctypes as C
import os
import subprocess
import time

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "cpu_tasks.c")
_SO = os.path.join(_DIR, "libcputasks.so")

NONESTED, NESTED, OPTD, OPTD_COST = 0, 1, 2, 3
POLICIES = {"nonested": NONESTED, "nested": NESTED, "optd": OPTD, "optd_cost": OPTD_COST}

_lib = None


def build(force: bool = False) -> str:
    """Compile cpu_tasks.c with gcc and OpenMP (-O3, no -march flags: the same source builds
    on x86-64 and Arm hosts)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        p, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.ct_factor.argtypes = [i64, p, p, p, p, i32, p, p, p, C.c_int, C.c_int, p, p, p, p]
        L.ct_factor.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Panels:
    """The factor as supernode panels (partition, row lists, column-major values)."""

    def __init__(self, start, rowptr, rows, lx, D, inner, seconds):
        self.start, self.rowptr, self.rows, self.lx = start, rowptr, rows, lx
        self.D, self.inner_tasks, self.seconds = D, inner, seconds

    def on_pattern(self, lp, li):
        """The panel values at the entries of a CSC pattern of L (permuted numbering), and the
        largest magnitude among the panel entries outside it (explicit zeros of relaxed
        supernodes, which must stay zero up to rounding)."""
        ns = len(self.start) - 1
        w = np.diff(self.start).astype(np.int64)
        m = np.diff(self.rowptr)
        off = np.concatenate([[0], np.cumsum(w * m)])
        out = np.zeros(len(li))
        extra = 0.0
        for s in range(ns):
            r = self.rows[self.rowptr[s]:self.rowptr[s + 1]]
            for j in range(self.start[s], self.start[s + 1]):
                col = self.lx[off[s] + (j - self.start[s]) * m[s]:off[s] + (j - self.start[s] + 1) * m[s]]
                pat = li[lp[j]:lp[j + 1]]
                pos = np.searchsorted(r, pat)
                out[lp[j]:lp[j + 1]] = col[pos]
                mask = np.ones(m[s], dtype=bool)
                mask[pos] = False
                mask[:j - self.start[s]] = False  # above the diagonal: unused
                if mask.any():
                    extra = max(extra, float(np.abs(col[mask]).max()))
        return out, extra


def factor(A, perm, start, rowptr, rows, policy="optd_cost", threads=None) -> Panels:
    """Factors A (inputs.SpdMatrix: lower CSC) with the given panel structure."""
    threads = threads or os.cpu_count() or 1
    start = np.ascontiguousarray(start, dtype=np.int32)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    colptr = np.ascontiguousarray(A.colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(A.rowind, dtype=np.int32)
    vals = np.ascontiguousarray(A.vals, dtype=np.float64)
    w = np.diff(start).astype(np.int64)
    m = np.diff(rowptr)
    lx = np.empty(int(np.sum(w * m)), dtype=np.float64)
    D, inner, bad = C.c_int32(), C.c_int64(), C.c_int32()
    t0 = time.perf_counter()
    rc = lib().ct_factor(A.n, _ptr(colptr), _ptr(rowind), _ptr(vals), _ptr(perm),
                         len(start) - 1, _ptr(start), _ptr(rowptr), _ptr(rows),
                         POLICIES[policy], int(threads), _ptr(lx), C.byref(D), C.byref(inner),
                         C.byref(bad))
    secs = time.perf_counter() - t0
    if rc != 0:
        raise RuntimeError(f"ct_factor: {rc} (column {bad.value})")
    return Panels(start, rowptr, rows, lx, D.value, inner.value, secs)
