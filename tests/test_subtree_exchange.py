"""The one exchange step of a subtree-to-device factorization, on two gloo ranks (CPU): with
the supernodal tree partitioned by chol_sym_partition, B = P^T A P has no entry coupling
two ranks' subtree columns, so each rank factors its subtrees alone and sends the
update of its subtrees to the top-part columns T, S_r = B[T, R_r] B[R_r, R_r]^-1 B[R_r, T];
the sum over ranks (all_reduce) gives the top part's Schur complement, whose Cholesky
factor equals the rows and columns T of the single-device factor L (every topological
order of the elimination tree gives the same L) -- compared with the oracle's L.  The
per-rank arithmetic here is dense FP64 numpy standing in for the device factorization; the
exchange is measured on no hardware (one GPU per run)."""
import os
import socket

import numpy as np
import pytest
import scipy.linalg as sl

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import paper_2202_09288_gb300 as P  # noqa: E402
from paper_2202_09288_gb300 import inputs  # noqa: E402

NAME = "st27x3_6"


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup():
    A, perm = inputs.workload(NAME)
    sym = P.Symbolic(P.make_opts(width_cap=64), A, perm)
    owner, _, _ = P.chol_sym_partition(sym.handle, 2, tol=0.2)
    start = sym.export()["sn_start"]
    col_owner = np.repeat(owner, np.diff(start))
    bp, bi, bx = oracle.permute(A.n, A.colptr, A.rowind, A.vals, perm)
    B = np.zeros((A.n, A.n))
    for j in range(A.n):
        B[bi[bp[j]:bp[j + 1]], j] = bx[bp[j]:bp[j + 1]]
    B = B + np.tril(B, -1).T
    return A, perm, col_owner, B


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A, perm, col_owner, B = _setup()
    R = np.nonzero(col_owner == rank)[0]
    T = np.nonzero(col_owner < 0)[0]
    # this rank's subtrees: factor B[R, R], then its update to the top columns
    Lr = np.linalg.cholesky(B[np.ix_(R, R)])
    Y = sl.solve_triangular(Lr, B[np.ix_(R, T)], lower=True)
    S = torch.from_numpy(Y.T @ Y)
    dist.all_reduce(S)  # the exchange: sum of the ranks' updates to the top part
    if rank == 0:
        Lt = np.linalg.cholesky(B[np.ix_(T, T)] - S.numpy())
        out["Lt"] = Lt
        out["T"] = T
    dist.barrier()
    dist.destroy_process_group()


def test_partition_makes_subtrees_independent():
    A, perm, col_owner, B = _setup()
    R0, R1 = np.nonzero(col_owner == 0)[0], np.nonzero(col_owner == 1)[0]
    assert R0.size and R1.size and (col_owner < 0).any()
    assert not B[np.ix_(R0, R1)].any()  # no coupling between the ranks' subtrees in B ...
    f = oracle.cholesky(A, perm)        # ... nor in L
    L = np.zeros((A.n, A.n))
    for j in range(A.n):
        L[f.li[f.lp[j]:f.lp[j + 1]], j] = f.lx[f.lp[j]:f.lp[j + 1]]
    assert not L[np.ix_(R0, R1)].any() and not L[np.ix_(R1, R0)].any()


def test_two_rank_exchange_gives_the_top_factor():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        Lt, T = out["Lt"], out["T"]
    A, perm = inputs.workload(NAME)
    f = oracle.cholesky(A, perm)
    L = np.zeros((A.n, A.n))
    for j in range(A.n):
        L[f.li[f.lp[j]:f.lp[j + 1]], j] = f.lx[f.lp[j]:f.lp[j + 1]]
    ref = L[np.ix_(T, T)]
    assert np.linalg.norm(Lt - ref) / np.linalg.norm(ref) <= 1e-12
