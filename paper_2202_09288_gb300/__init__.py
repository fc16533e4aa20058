"""GB300 (sm_103a) supernodal sparse Cholesky: a thin ctypes binding of include/chol.h.

Every function here only marshals arguments to the C ABI of ``libchol.so``; all work runs
in the library (host analysis in C++, the numeric phases in CUDA kernels).  If the
library is missing, importing works but every call raises: there is no fallback.

Host arrays are numpy arrays; device arrays are torch CUDA tensors (PyTorch is used only
for device memory and streams).  Function names follow the C ABI.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchol.so")

CHOL_OK, CHOL_PENDING = 0, 1
CHOL_E_INVALID, CHOL_E_NOT_SPD, CHOL_E_OOM, CHOL_E_CUDA = -1, -2, -3, -4
CHOL_E_TIMEOUT, CHOL_E_NODEVICE, CHOL_E_STALL, CHOL_E_SCRATCH = -5, -6, -7, -8
CHOL_HOST, CHOL_DEVICE = 0, 1
CHOL_ASSEMBLY_ATOMIC, CHOL_ASSEMBLY_OWNER = 0, 1
CHOL_FP64, CHOL_MIXED = 0, 1
CHOL_SCHUR_OZAKI, CHOL_SCHUR_DMMA = 0, 1
CHOL_GRAN_TILES, CHOL_GRAN_OPTD, CHOL_GRAN_OPTD_COST, CHOL_GRAN_HYBRID = 0, 1, 2, 3


class CholError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        msg = lib().chol_strerror(status).decode()
        super().__init__(f"{where}: {msg} ({status})" if where else f"{msg} ({status})")
        self.status = status


class chol_opts(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("width_cap", C.c_int),
                ("assembly", C.c_int), ("hbm_budget", C.c_size_t), ("pivot_tau", C.c_double),
                ("relax", C.c_double), ("fp64_schur", C.c_int)]


class chol_sym_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz_a", C.c_int64), ("nnz_l", C.c_int64),
                ("l_storage", C.c_int64), ("nsuper", C.c_int64), ("nlevels", C.c_int64),
                ("flops", C.c_double), ("max_width", C.c_int64), ("max_rows", C.c_int64),
                ("flops_panel", C.c_double), ("nfundamental", C.c_int64),
                ("ntrsm_tc", C.c_int64)]


class chol_refine_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("fell_back", C.c_int), ("residual", C.c_double),
                ("pivot_redos", C.c_int64)]


class chol_tile_policy(C.Structure):
    _fields_ = [("min_rows_tile64", C.c_int), ("min_rows_tile32", C.c_int),
                ("min_level_tiles64", C.c_int), ("min_rows_tile128", C.c_int),
                ("min_level_tiles128", C.c_int),
                ("granularity", C.c_int), ("min_rows_trsm_tc", C.c_int)]


class chol_server_opts(C.Structure):
    _fields_ = [("device", C.c_int), ("slots", C.c_int), ("max_batch", C.c_int),
                ("hbm_budget", C.c_size_t), ("width_cap", C.c_int), ("assembly", C.c_int),
                ("sym_cache", C.c_int), ("analyzers", C.c_int)]


class chol_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("colptr", C.c_void_p), ("rowind", C.c_void_p),
                ("vals", C.c_void_p), ("perm", C.c_void_p), ("nrhs", C.c_int64),
                ("B", C.c_void_p), ("ldb", C.c_int64), ("X", C.c_void_p), ("ldx", C.c_int64),
                ("precision", C.c_int), ("tol", C.c_double)]


class chol_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("fell_back", C.c_int),
                ("residual", C.c_double), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double), ("batch_size", C.c_int)]


class chol_prof_entry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("ms", C.c_double),
                ("timed", C.c_int64), ("flops", C.c_double), ("bytes", C.c_double)]


# name -> (restype, argtypes)
_P, _I, _I64 = C.c_void_p, C.c_int, C.c_int64
EXPORTS = {
    "chol_default_opts": (None, [C.POINTER(chol_opts)]),
    "chol_version": (_I, []),
    "chol_strerror": (C.c_char_p, [_I]),
    "chol_create": (_I, [C.POINTER(chol_opts), C.POINTER(_P)]),
    "chol_destroy": (None, [_P]),
    "chol_analyze": (_I, [C.POINTER(chol_opts), _I64, _P, _P, _P, C.POINTER(_P)]),
    "chol_sym_info": (_I, [_P, C.POINTER(chol_sym_stats)]),
    "chol_sym_export": (_I, [_P, _P, _P, _P, _P]),
    "chol_sym_rows": (_I, [_P, _P, _P]),
    "chol_free_sym": (None, [_P]),
    "chol_factorize": (_I, [_P, _P, _P, _I, _I, C.POINTER(_P)]),
    "chol_refactorize": (_I, [_P, _P, _P, _I]),
    "chol_factor_status": (_I, [_P, _P, C.POINTER(_I64)]),
    "chol_factor_export": (_I, [_P, _P, _P, _P, _P]),
    "chol_factor_panels": (_I, [_P, _P, _I64, _I64, _P, _I]),
    "chol_free_num": (None, [_P]),
    "chol_solve": (_I, [_P, _P, _I64, _P, _I64, _P, _I64, _I]),
    "chol_refine": (_I, [_P, _P, _I64, _P, _I64, _P, _I64, _I, C.c_double, _I,
                         C.POINTER(chol_refine_info)]),
    "chol_refine_gmres": (_I, [_P, _P, _I64, _P, _I64, _P, _I64, _I, C.c_double, _I, _I,
                               C.POINTER(chol_refine_info)]),
    "chol_solve_noalloc": (_I, [_P, _P, _I64, _P, _I64, _P, _I64]),
    "chol_noalloc_scratch_bytes": (C.c_size_t, []),
    "chol_batch_create": (_I, [_P, _I, C.POINTER(_P), C.POINTER(_P)]),
    "chol_batch_factorize": (_I, [_P, _P, C.POINTER(_P), _I, _I]),
    "chol_batch_free": (None, [_P]),
    "chol_sym_get_tile_policy": (_I, [_P, C.POINTER(chol_tile_policy)]),
    "chol_sym_set_tile_policy": (_I, [_P, C.POINTER(chol_tile_policy)]),
    "chol_autotune": (_I, [_P, _P, _I, C.POINTER(chol_tile_policy), C.POINTER(C.c_double)]),
    "chol_opt_d": (_I, [C.c_int64, C.c_int32, _P, C.POINTER(C.c_int32)]),
    "chol_sym_granularity": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "chol_sym_schur_tiles": (_I, [_P, _P, _P, _P, _P, C.POINTER(C.c_int64)]),
    "chol_partition_tree": (_I, [C.c_int32, _P, _P, _I, C.c_double, _P,
                                 C.POINTER(C.c_double)]),
    "chol_sym_partition": (_I, [_P, _I, C.c_double, _P, C.POINTER(C.c_double),
                                C.POINTER(C.c_double)]),
    "chol_default_server_opts": (None, [C.POINTER(chol_server_opts)]),
    "chol_server_create": (_I, [C.POINTER(chol_server_opts), C.POINTER(_P)]),
    "chol_submit": (_I, [_P, C.POINTER(chol_request), C.POINTER(C.c_uint64)]),
    "chol_poll": (_I, [_P, C.c_uint64, C.POINTER(chol_result)]),
    "chol_wait": (_I, [_P, C.c_uint64, C.POINTER(chol_result)]),
    "chol_server_clock": (C.c_double, [_P]),
    "chol_server_destroy": (None, [_P]),
    "chol_profile_enable": (_I, [_P, _I]),
    "chol_profile_only": (_I, [_P, C.c_char_p]),
    "chol_set_device_wait": (_I, [_P, C.c_longlong]),
    "chol_profile_read": (_I, [_P, C.POINTER(chol_prof_entry), _I, C.POINTER(_I)]),
    "chol_profile_reset": (_I, [_P]),
}

_lib = None


def lib():
    """Loads libchol.so (raises if it has not been built: no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                               "`python -m paper_2202_09288_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != CHOL_OK:
        raise CholError(rc, where)


def _ptr(a):
    """(pointer, where) of a numpy array (host) or a torch CUDA tensor (device)."""
    if a is None:
        return None, CHOL_HOST
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous and not a.flags.f_contiguous:
            raise ValueError("array must be contiguous")
        return a.ctypes.data, CHOL_HOST
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), (CHOL_DEVICE if a.is_cuda else CHOL_HOST)
    raise TypeError(f"unsupported array type {type(a)}")


# ---- C ABI, one Python function per entry point -----------------------------------------
def chol_default_opts() -> chol_opts:
    o = chol_opts()
    lib().chol_default_opts(C.byref(o))
    return o


def chol_version() -> int:
    return lib().chol_version()


# device ordinal of every live context (for the argument checks of the device-pointer calls)
_CTX_DEVICE: dict[int, int] = {}


def chol_create(opts: chol_opts | None = None) -> int:
    h = C.c_void_p()
    _check(lib().chol_create(C.byref(opts) if opts is not None else None, C.byref(h)),
           "chol_create")
    _CTX_DEVICE[h.value] = opts.device if opts is not None else 0
    return h.value


def chol_destroy(ctx: int) -> None:
    _CTX_DEVICE.pop(ctx, None)
    lib().chol_destroy(ctx)


def _host_block(B, n_hint=None):
    """A float64 host block as (array, n, k) laid out column-major (a 1-D vector is n x 1)."""
    if B.dtype != np.float64:
        raise ValueError(f"host arrays must be float64, not {B.dtype}")
    B2 = B.reshape(B.shape[0], -1)
    if not B2.flags.f_contiguous:
        raise ValueError("host blocks must be column-major (Fortran) contiguous")
    return B2, B2.shape[0], B2.shape[1]


def _check_device_pair(ctx, B, X, where: str):
    """Device tensors B, X for a solve on ctx: float64, contiguous, X shaped like B, both on
    the context's GPU.  Returns (k, n): tensor rows are right-hand sides (shape (k, n)), a
    1-D tensor is one right-hand side."""
    import torch

    for name, T in (("B", B), ("X", X)):
        if not isinstance(T, torch.Tensor) or not T.is_cuda:
            raise ValueError(f"{where}: {name} must be a CUDA tensor")
        if T.dtype != torch.float64:
            raise ValueError(f"{where}: {name} must be float64, not {T.dtype}")
        if not T.is_contiguous():
            raise ValueError(f"{where}: {name} must be contiguous")
        if T.dim() not in (1, 2):
            raise ValueError(f"{where}: {name} must have shape (n,) or (k, n)")
    if tuple(X.shape) != tuple(B.shape):
        raise ValueError(f"{where}: X has shape {tuple(X.shape)}, B has {tuple(B.shape)}")
    dev = _CTX_DEVICE.get(ctx)
    for name, T in (("B", B), ("X", X)):
        if dev is not None and T.device.index != dev:
            raise ValueError(f"{where}: {name} is on cuda:{T.device.index}, the context on "
                             f"cuda:{dev}")
    return (1, B.shape[0]) if B.dim() == 1 else (B.shape[0], B.shape[1])


def chol_analyze(opts, n, colptr, rowind, perm) -> int:
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int32)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    h = C.c_void_p()
    _check(lib().chol_analyze(C.byref(opts) if opts is not None else None, int(n),
                              colptr.ctypes.data, rowind.ctypes.data,
                              perm.ctypes.data, C.byref(h)), "chol_analyze")
    return h.value


def chol_sym_info(sym) -> dict:
    st = chol_sym_stats()
    _check(lib().chol_sym_info(sym, C.byref(st)), "chol_sym_info")
    return {name: getattr(st, name) for name, _ in chol_sym_stats._fields_}


def chol_sym_export(sym) -> dict:
    info = chol_sym_info(sym)
    n, ns = info["n"], info["nsuper"]
    parent = np.zeros(n, np.int32)
    cc = np.zeros(n, np.int64)
    start = np.zeros(ns + 1, np.int32)
    level = np.zeros(ns, np.int32)
    _check(lib().chol_sym_export(sym, parent.ctypes.data, cc.ctypes.data, start.ctypes.data,
                                 level.ctypes.data), "chol_sym_export")
    return {"parent": parent, "colcount": cc, "sn_start": start, "sn_level": level}


def chol_sym_rows(sym) -> tuple:
    """(rowptr, rows): the row list of every supernode panel."""
    ns = chol_sym_info(sym)["nsuper"]
    rowptr = np.zeros(ns + 1, np.int64)
    _check(lib().chol_sym_rows(sym, rowptr.ctypes.data, None), "chol_sym_rows")
    rows = np.zeros(int(rowptr[-1]), np.int32)
    _check(lib().chol_sym_rows(sym, None, rows.ctypes.data), "chol_sym_rows")
    return rowptr, rows


def chol_free_sym(sym) -> None:
    lib().chol_free_sym(sym)


def chol_factorize(ctx, sym, vals, precision=CHOL_FP64) -> int:
    p, where = _ptr(vals)
    h = C.c_void_p()
    _check(lib().chol_factorize(ctx, sym, p, where, precision, C.byref(h)), "chol_factorize")
    return h.value


def chol_refactorize(ctx, num, vals) -> None:
    p, where = _ptr(vals)
    _check(lib().chol_refactorize(ctx, num, p, where), "chol_refactorize")


def chol_factor_status(ctx, num) -> tuple[int, int]:
    bad = C.c_int64(-1)
    rc = lib().chol_factor_status(ctx, num, C.byref(bad))
    if rc not in (CHOL_OK, CHOL_E_NOT_SPD):
        _check(rc, "chol_factor_status")
    return rc, bad.value


def chol_factor_export(ctx, num, n, nnz_l):
    lp = np.zeros(n + 1, np.int64)
    li = np.zeros(nnz_l, np.int32)
    lx = np.zeros(nnz_l, np.float64)
    _check(lib().chol_factor_export(ctx, num, lp.ctypes.data, li.ctypes.data, lx.ctypes.data),
           "chol_factor_export")
    return lp, li, lx


def chol_factor_panels(ctx, num, first, count, out):
    """Copies the raw panels of supernodes first .. first+count-1 into out (a float64 numpy
    array or CUDA tensor holding sum m_s n_s entries, contiguous)."""
    if isinstance(out, np.ndarray):
        if out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError("chol_factor_panels: out must be contiguous float64")
        p, where = out.ctypes.data, CHOL_HOST
    else:
        import torch

        if out.dtype != torch.float64 or not out.is_contiguous() or not out.is_cuda:
            raise ValueError("chol_factor_panels: out must be a contiguous float64 CUDA tensor")
        p, where = out.data_ptr(), CHOL_DEVICE
    _check(lib().chol_factor_panels(ctx, num, int(first), int(count), p, where),
           "chol_factor_panels")
    return out


def chol_free_num(num) -> None:
    lib().chol_free_num(num)


def chol_solve(ctx, num, B, X=None):
    """Solves A X = B.  B: numpy (n,) / (n, k) Fortran-ordered, or a torch CUDA tensor laid
    out column-major (shape (k, n) contiguous, i.e. column c is row c of the tensor).  A
    given X must match B (float64, same shape and layout, same device)."""
    if isinstance(B, np.ndarray):
        B2 = np.asfortranarray(B.reshape(B.shape[0], -1), dtype=np.float64)
        n, k = B2.shape
        if X is None:
            X = np.zeros((n, k), dtype=np.float64, order="F")
        elif not isinstance(X, np.ndarray) or X.size != n * k:
            raise ValueError("chol_solve: X must be a host array with as many entries as B")
        X2, xn, xk = _host_block(X)
        if (xn, xk) != (n, k):
            raise ValueError(f"chol_solve: X is {xn} x {xk}, B is {n} x {k}")
        _check(lib().chol_solve(ctx, num, k, B2.ctypes.data, n, X2.ctypes.data, n, CHOL_HOST),
               "chol_solve")
        return X.reshape(B.shape) if B.ndim == 1 else X
    # torch device tensor: (k, n) contiguous = n x k column-major, ld = n
    if X is None:
        X = B.new_empty(B.shape)
    k, n = _check_device_pair(ctx, B, X, "chol_solve")
    _check(lib().chol_solve(ctx, num, k, B.data_ptr(), n, X.data_ptr(), n, CHOL_DEVICE),
           "chol_solve")
    return X


def chol_refine(ctx, num, B, X=None, tol=1e-12, maxit=10, check=True):
    """Iterative refinement to ||b - A x||_inf / (||A||_inf ||x||_inf) <= tol.  B: numpy
    (n,) / (n, k) or a torch CUDA tensor of shape (k, n) / (n,) (as chol_solve).  Returns
    (X, info dict); raises CholError on failure (CHOL_E_STALL only if check is True)."""
    info = chol_refine_info()
    if isinstance(B, np.ndarray):
        B2 = np.asfortranarray(B.reshape(B.shape[0], -1), dtype=np.float64)
        n, k = B2.shape
        X2 = np.zeros((n, k), dtype=np.float64, order="F")
        rc = lib().chol_refine(ctx, num, k, B2.ctypes.data, n, X2.ctypes.data, n, CHOL_HOST,
                               tol, maxit, C.byref(info))
        out = X2.reshape(B.shape) if B.ndim == 1 else X2
    else:
        out = B.new_empty(B.shape) if X is None else X
        k, n = _check_device_pair(ctx, B, out, "chol_refine")
        rc = lib().chol_refine(ctx, num, k, B.data_ptr(), n, out.data_ptr(), n, CHOL_DEVICE,
                               tol, maxit, C.byref(info))
    d = {"iterations": info.iterations, "fell_back": bool(info.fell_back),
         "residual": info.residual, "pivot_redos": info.pivot_redos, "status": rc}
    if rc != CHOL_OK and (check or rc != CHOL_E_STALL):
        raise CholError(rc, "chol_refine")
    return out, d


def chol_refine_gmres(ctx, num, B, X=None, tol=1e-12, restart=0, maxit=0, check=True):
    """GMRES-based iterative refinement (FGMRES preconditioned with the factor) to
    ||b - A x||_inf / (||A||_inf ||x||_inf) <= tol; arguments and result as chol_refine."""
    info = chol_refine_info()
    if isinstance(B, np.ndarray):
        B2 = np.asfortranarray(B.reshape(B.shape[0], -1), dtype=np.float64)
        n, k = B2.shape
        X2 = np.zeros((n, k), dtype=np.float64, order="F")
        rc = lib().chol_refine_gmres(ctx, num, k, B2.ctypes.data, n, X2.ctypes.data, n,
                                     CHOL_HOST, tol, restart, maxit, C.byref(info))
        out = X2.reshape(B.shape) if B.ndim == 1 else X2
    else:
        out = B.new_empty(B.shape) if X is None else X
        k, n = _check_device_pair(ctx, B, out, "chol_refine_gmres")
        rc = lib().chol_refine_gmres(ctx, num, k, B.data_ptr(), n, out.data_ptr(), n,
                                     CHOL_DEVICE, tol, restart, maxit, C.byref(info))
    d = {"iterations": info.iterations, "fell_back": bool(info.fell_back),
         "residual": info.residual, "pivot_redos": info.pivot_redos, "status": rc}
    if rc != CHOL_OK and (check or rc != CHOL_E_STALL):
        raise CholError(rc, "chol_refine_gmres")
    return out, d


def chol_solve_noalloc(ctx, num, B, X):
    """Device-pointer solve without any device allocation (torch CUDA tensors laid out as
    in chol_solve: shape (k, n) contiguous, or (n,) for one right-hand side)."""
    k, n = _check_device_pair(ctx, B, X, "chol_solve_noalloc")
    _check(lib().chol_solve_noalloc(ctx, num, k, B.data_ptr(), n, X.data_ptr(), n),
           "chol_solve_noalloc")
    return X


def chol_noalloc_scratch_bytes() -> int:
    return lib().chol_noalloc_scratch_bytes()


def chol_batch_create(ctx, nums) -> int:
    arr = (C.c_void_p * len(nums))(*nums)
    h = C.c_void_p()
    _check(lib().chol_batch_create(ctx, len(nums), arr, C.byref(h)), "chol_batch_create")
    return h.value


def chol_batch_factorize(ctx, batch, vals=None, use_graph=True) -> None:
    """vals: None, or a list with one entry per member (None, a numpy array or a torch CUDA
    tensor of that member's values; all entries host or all device)."""
    arr, where = None, CHOL_HOST
    if vals is not None:
        ptrs = []
        for v in vals:
            p, w = _ptr(v)
            ptrs.append(p)
            if v is not None:
                where = w
        arr = (C.c_void_p * len(ptrs))(*ptrs)
    _check(lib().chol_batch_factorize(ctx, batch, arr, where, 1 if use_graph else 0),
           "chol_batch_factorize")


def chol_batch_free(batch) -> None:
    lib().chol_batch_free(batch)


def chol_sym_get_tile_policy(sym) -> dict:
    p = chol_tile_policy()
    _check(lib().chol_sym_get_tile_policy(sym, C.byref(p)), "chol_sym_get_tile_policy")
    return {f: getattr(p, f) for f, _ in chol_tile_policy._fields_}


def chol_sym_set_tile_policy(sym, policy: dict) -> None:
    p = chol_tile_policy()
    _check(lib().chol_sym_get_tile_policy(sym, C.byref(p)), "chol_sym_get_tile_policy")
    for f, v in policy.items():  # fields not given keep their current value
        setattr(p, f, v)
    _check(lib().chol_sym_set_tile_policy(sym, C.byref(p)), "chol_sym_set_tile_policy")


def chol_opt_d(n: int, counts) -> int:
    """Threshold D of the OPT-D heuristic (Sec. 4.1, Algorithm 1) for outer tasks with the
    given numbers of inner tasks."""
    c = np.ascontiguousarray(counts, dtype=np.int32)
    d = C.c_int32()
    _check(lib().chol_opt_d(int(n), len(c), c.ctypes.data_as(C.c_void_p) if len(c) else None,
                            C.byref(d)), "chol_opt_d")
    return d.value


def chol_sym_granularity(sym) -> dict:
    """The granularity rule of sym's task lists: {"rule", "D", "nsplit"}."""
    rule, d, nsplit = C.c_int(), C.c_int32(), C.c_int32()
    _check(lib().chol_sym_granularity(sym, C.byref(rule), C.byref(d), C.byref(nsplit)),
           "chol_sym_granularity")
    return {"rule": rule.value, "D": d.value, "nsplit": nsplit.value}


def chol_sym_schur_tiles(sym) -> dict:
    """Every Schur tile task of sym's current task lists: arrays s, i0, k0, tile."""
    cnt = C.c_int64()
    _check(lib().chol_sym_schur_tiles(sym, None, None, None, None, C.byref(cnt)),
           "chol_sym_schur_tiles")
    out = {k: np.zeros(cnt.value, dtype=np.int32) for k in ("s", "i0", "k0", "tile")}
    _check(lib().chol_sym_schur_tiles(sym, *[out[k].ctypes.data_as(C.c_void_p)
                                             for k in ("s", "i0", "k0", "tile")],
                                      C.byref(cnt)), "chol_sym_schur_tiles")
    return out


def chol_partition_tree(parent, work, nparts, tol=0.05):
    """(owner, imbalance): subtree-to-device partition of a forest (see chol.h)."""
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    work = np.ascontiguousarray(work, dtype=np.float64)
    owner = np.zeros(parent.size, dtype=np.int32)
    imb = C.c_double()
    _check(lib().chol_partition_tree(parent.size, parent.ctypes.data, work.ctypes.data,
                                     int(nparts), float(tol), owner.ctypes.data, C.byref(imb)),
           "chol_partition_tree")
    return owner, imb.value


def chol_sym_partition(sym, nparts, tol=0.05):
    """(owner per supernode, imbalance, top flops) of sym's supernodal tree."""
    ns = chol_sym_info(sym)["nsuper"]
    owner = np.zeros(ns, dtype=np.int32)
    imb, top = C.c_double(), C.c_double()
    _check(lib().chol_sym_partition(sym, int(nparts), float(tol), owner.ctypes.data,
                                    C.byref(imb), C.byref(top)), "chol_sym_partition")
    return owner, imb.value, top.value


def chol_autotune(ctx, num, reps=1) -> tuple[dict, float]:
    p = chol_tile_policy()
    ms = C.c_double()
    _check(lib().chol_autotune(ctx, num, reps, C.byref(p), C.byref(ms)), "chol_autotune")
    return {f: getattr(p, f) for f, _ in chol_tile_policy._fields_}, ms.value


def chol_profile_enable(ctx, on: bool) -> None:
    _check(lib().chol_profile_enable(ctx, 1 if on else 0), "chol_profile_enable")


def chol_profile_only(ctx, name=None) -> None:
    """Brackets only the launches of kernel kind `name` with events (None: every kind)."""
    _check(lib().chol_profile_only(ctx, name.encode() if name else None), "chol_profile_only")


def chol_set_device_wait(ctx, cycles: int) -> None:
    """Test hook: bound of the tensor-core Schur consumers' accumulator wait (0: default)."""
    _check(lib().chol_set_device_wait(ctx, int(cycles)), "chol_set_device_wait")


def chol_profile_read(ctx) -> dict:
    arr = (chol_prof_entry * 32)()
    cnt = C.c_int()
    _check(lib().chol_profile_read(ctx, arr, 32, C.byref(cnt)), "chol_profile_read")
    return {arr[k].name.decode(): {"launches": arr[k].launches, "ms": arr[k].ms,
                                   "timed": arr[k].timed, "flops": arr[k].flops,
                                   "bytes": arr[k].bytes} for k in range(cnt.value)}


def chol_profile_reset(ctx) -> None:
    _check(lib().chol_profile_reset(ctx), "chol_profile_reset")


# ---- small object wrappers used by the tests and the bench -------------------------------
def make_opts(device: int = 0, width_cap: int = 64, assembly: int = CHOL_ASSEMBLY_ATOMIC,
              stream: int | None = None, hbm_budget: int = 0, relax: float = 0.0,
              fp64_schur: int = CHOL_SCHUR_OZAKI) -> chol_opts:
    """relax: 0 = the library default, < 0 = fundamental supernodes only."""
    o = chol_default_opts()
    o.device, o.width_cap, o.assembly, o.hbm_budget = device, width_cap, assembly, hbm_budget
    o.stream = stream
    o.fp64_schur = fp64_schur
    if relax:
        o.relax = relax
    return o


class Context:
    def __init__(self, device: int = 0, width_cap: int = 64, assembly: int = CHOL_ASSEMBLY_ATOMIC,
                 stream: int | None = None, hbm_budget: int = 0, relax: float = 0.0,
                 fp64_schur: int = CHOL_SCHUR_OZAKI):
        self.opts = make_opts(device, width_cap, assembly, stream, hbm_budget, relax, fp64_schur)
        self.handle = chol_create(self.opts)

    def close(self):
        if self.handle:
            chol_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Symbolic:
    """Host symbolic analysis; ``opts`` is a Context, a chol_opts, or None (W = 64)."""

    def __init__(self, opts, A, perm):
        if isinstance(opts, Context):
            opts = opts.opts
        self.n = A.n
        self.handle = chol_analyze(opts, A.n, A.colptr, A.rowind, perm)
        self.info = chol_sym_info(self.handle)

    def export(self):
        return chol_sym_export(self.handle)

    def __del__(self):
        try:
            if self.handle:
                chol_free_sym(self.handle)
        except Exception:
            pass


class Factor:
    def __init__(self, ctx: Context, sym: Symbolic, vals, precision=CHOL_FP64):
        self.ctx, self.sym = ctx, sym
        self.handle = chol_factorize(ctx.handle, sym.handle, vals, precision)

    def refactor(self, vals):
        chol_refactorize(self.ctx.handle, self.handle, vals)

    def status(self):
        return chol_factor_status(self.ctx.handle, self.handle)

    def export(self):
        return chol_factor_export(self.ctx.handle, self.handle, self.sym.n,
                                  self.sym.info["nnz_l"])

    def solve(self, B, X=None):
        return chol_solve(self.ctx.handle, self.handle, B, X)

    def autotune(self, reps=1):
        return chol_autotune(self.ctx.handle, self.handle, reps)

    def refine(self, B, X=None, tol=1e-12, maxit=10, check=True):
        return chol_refine(self.ctx.handle, self.handle, B, X, tol, maxit, check)

    def refine_gmres(self, B, X=None, tol=1e-12, restart=0, maxit=0, check=True):
        return chol_refine_gmres(self.ctx.handle, self.handle, B, X, tol, restart, maxit, check)

    def __del__(self):
        try:
            if self.handle:
                chol_free_num(self.handle)
        except Exception:
            pass


class Batch:
    """Batched factorization of several factors (same context, precision, assembly)."""

    def __init__(self, ctx: Context, factors):
        self.ctx, self.factors = ctx, list(factors)
        self.handle = chol_batch_create(ctx.handle, [f.handle for f in self.factors])

    def factorize(self, vals=None, use_graph=True):
        chol_batch_factorize(self.ctx.handle, self.handle, vals, use_graph)

    def close(self):
        if self.handle:
            chol_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _result_dict(r: chol_result) -> dict:
    return {f: getattr(r, f) for f, _ in chol_result._fields_}


class Server:
    """Request server with continuous batching (chol_server_create / chol_submit /
    chol_poll / chol_wait).  Host arrays of a request are copied at submit, except X, which
    the server fills: the Server keeps it alive until the result has been collected."""

    def __init__(self, device=0, slots=2, max_batch=16, hbm_budget=0, width_cap=64,
                 assembly=CHOL_ASSEMBLY_ATOMIC, sym_cache=64):
        o = chol_server_opts()
        lib().chol_default_server_opts(C.byref(o))
        o.device, o.slots, o.max_batch, o.hbm_budget = device, slots, max_batch, hbm_budget
        o.width_cap, o.assembly, o.sym_cache = width_cap, assembly, sym_cache
        h = C.c_void_p()
        _check(lib().chol_server_create(C.byref(o), C.byref(h)), "chol_server_create")
        self.handle = h.value
        self._outputs = {}

    def submit(self, A, perm, B, precision=CHOL_FP64, tol=1e-12) -> int:
        B2 = np.asfortranarray(np.asarray(B, dtype=np.float64).reshape(A.n, -1))
        X = np.zeros_like(B2, order="F")
        colptr = np.ascontiguousarray(A.colptr, np.int64)
        rowind = np.ascontiguousarray(A.rowind, np.int32)
        vals = np.ascontiguousarray(A.vals, np.float64)
        perm = np.ascontiguousarray(perm, np.int32)
        q = chol_request(A.n, colptr.ctypes.data, rowind.ctypes.data, vals.ctypes.data,
                         perm.ctypes.data, B2.shape[1], B2.ctypes.data, A.n, X.ctypes.data,
                         A.n, precision, tol)
        t = C.c_uint64()
        _check(lib().chol_submit(self.handle, C.byref(q), C.byref(t)), "chol_submit")
        self._outputs[t.value] = X
        return t.value

    def poll(self, ticket):
        r = chol_result()
        rc = lib().chol_poll(self.handle, ticket, C.byref(r))
        if rc == CHOL_PENDING:
            return None
        _check(rc, "chol_poll")
        return self._outputs.pop(ticket), _result_dict(r)

    def wait(self, ticket):
        r = chol_result()
        _check(lib().chol_wait(self.handle, ticket, C.byref(r)), "chol_wait")
        return self._outputs.pop(ticket), _result_dict(r)

    def clock(self) -> float:
        return lib().chol_server_clock(self.handle)

    def close(self):
        if self.handle:
            lib().chol_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
