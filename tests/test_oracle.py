"""Pins of the CPU oracle against facts that do not come from the oracle itself:
library routines (numpy.linalg.cholesky), a textbook row-oriented Cholesky in pure
Python, graph elimination by brute force, closed forms (1D Laplacian), the paper's
Fig. 1 level sets (Sec. 3) and exact invariants."""
import math
import os

import numpy as np
import pytest

import oracle
from conftest import fig1_matrix, fig1_tree
from paper_2202_09288_gb300 import inputs


def dense_L(f):
    L = np.zeros((f.n, f.n))
    for j in range(f.n):
        L[f.li[f.lp[j]:f.lp[j + 1]], j] = f.lx[f.lp[j]:f.lp[j + 1]]
    return L


def seeded_perm(n, seed):
    return np.argsort(inputs.uniform(seed, 9, n), kind="stable").astype(np.int32)


def textbook_cholesky(a):
    """Row-by-row (Cholesky-Banachiewicz) dense factorization, pure Python loops."""
    n = len(a)
    L = [[0.0] * n for _ in range(n)]
    for i in range(n):
        for j in range(i + 1):
            s = sum(L[i][k] * L[j][k] for k in range(j))
            if i == j:
                L[i][j] = math.sqrt(a[i][i] - s)
            else:
                L[i][j] = (a[i][j] - s) / L[j][j]
    return np.array(L)


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (7, 3), (40, 4), (120, 5)])
def test_dense_vs_numpy(n, seed):
    A = inputs.random_spd_dense(n, seed)
    for perm in (np.arange(n, dtype=np.int32), seeded_perm(n, seed)):
        f = oracle.cholesky(A, perm)
        Ad = A.to_dense()[np.ix_(perm, perm)]
        ref = np.linalg.cholesky(Ad)
        err = np.linalg.norm(dense_L(f) - ref) / np.linalg.norm(ref)
        assert err <= 1e-14, err
        assert f.nnz_l == n * (n + 1) // 2


@pytest.mark.parametrize("n", [3, 9, 12])
def test_dense_vs_textbook_loops(n):
    A = inputs.random_spd_dense(n, 11 + n)
    f = oracle.cholesky(A)
    ref = textbook_cholesky(A.to_dense().tolist())
    assert np.linalg.norm(dense_L(f) - ref) <= 1e-14 * np.linalg.norm(ref)


def test_lap1d_closed_form():
    n = 60
    f = oracle.cholesky(inputs.laplacian_1d(n))
    L = dense_L(f)
    j = np.arange(n)
    diag = np.sqrt((j + 2.0) / (j + 1.0))
    sub = -np.sqrt((j[:-1] + 1.0) / (j[:-1] + 2.0))
    assert np.max(np.abs(np.diag(L) - diag) / diag) <= 1e-15
    assert np.max(np.abs(np.diag(L, -1) - sub) / np.abs(sub)) <= 1e-15
    assert f.nnz_l == 2 * n - 1
    assert list(f.parent) == list(range(1, n)) + [-1]
    start, sp, lv = f.supernodes(10 ** 6)
    # only the last two columns have nested structure (c = 2, 1): supernodes
    # {0}, {1}, ..., {n-3}, {n-2, n-1}, forming one chain
    assert list(start) == list(range(n - 1)) + [n]
    assert list(sp) == list(range(1, n - 1)) + [-1]
    assert list(lv) == list(range(n - 1))


def graph_elimination_pattern(adj, n):
    """Fill pattern by eliminating vertices in order: the later neighbours of vertex k
    become a clique (brute force on a dense boolean matrix)."""
    M = np.array(adj, dtype=bool)
    for k in range(n):
        nb = [i for i in range(k + 1, n) if M[i, k]]
        for a in nb:
            for b in nb:
                M[a, b] = True
    return np.tril(M | np.eye(n, dtype=bool))


@pytest.mark.parametrize("seed", range(6))
def test_symbolic_vs_graph_elimination(seed):
    n = 30
    u = inputs.uniform(100 + seed, 7, n * n).reshape(n, n)
    adj = (u > 0.85) | (u.T > 0.85)
    a = np.where(adj, 0.1 * np.sign(u + u.T), 0.0)
    a = a + a.T
    a[np.arange(n), np.arange(n)] = np.abs(a).sum(1) + 1.0
    A = inputs.from_dense(a)
    perm = seeded_perm(n, seed)
    f = oracle.cholesky(A, perm)
    pat = graph_elimination_pattern((a != 0)[np.ix_(perm, perm)], n)
    got = np.zeros((n, n), bool)
    for j in range(n):
        got[f.li[f.lp[j]:f.lp[j + 1]], j] = True
    assert (got == pat).all()
    # elimination tree: parent(j) = first off-diagonal row of column j
    for j in range(n):
        rows = np.nonzero(pat[j + 1:, j])[0]
        assert f.parent[j] == (rows[0] + j + 1 if rows.size else -1)
    assert (f.colcount == pat.sum(0)).all()
    # numeric L has no entry outside the symbolic pattern
    Lref = np.linalg.cholesky(a[np.ix_(perm, perm)])
    assert np.all(np.abs(Lref[~pat]) < 1e-300)


def test_fig1_level_sets():
    """Sec. 3, Fig. 1 (tests/golden/fig1_tree.txt): the oracle's elimination tree and level
    sets of a matrix built on the printed tree equal the printed tree and schedule."""
    edges, levels = fig1_tree()
    f = oracle.cholesky(fig1_matrix())
    assert sorted((j + 1, int(p) + 1) for j, p in enumerate(f.parent) if p >= 0) == sorted(edges)
    start, sp, lv = f.supernodes(64)
    assert list(start) == list(range(f.n + 1))  # no two of them form a supernode
    sets = [sorted(int(s) + 1 for s in np.nonzero(lv == l)[0]) for l in range(lv.max() + 1)]
    assert sets == levels


def test_dense_supernode_and_width_cap():
    n = 30
    f = oracle.cholesky(inputs.random_spd_dense(n, 3))
    start, sp, lv = f.supernodes(10 ** 6)
    assert list(start) == [0, n]
    start, sp, lv = f.supernodes(8)
    assert list(start) == [0, 8, 16, 24, 30]
    assert list(sp) == [1, 2, 3, -1]
    assert list(lv) == [0, 1, 2, 3]


@pytest.mark.parametrize("name", ["lap2d_12", "lap3d_5", "st27x3_3", "dense"])
def test_flop_model_counts(name):
    if name == "dense":
        A, perm = inputs.random_spd_dense(25, 8), None
    else:
        A, perm = inputs.workload(name)
    f = oracle.cholesky(A, perm)
    assert f.flops_counted == f.flops  # every counted op equals sum_j c_j^2
    assert f.flops == float(np.sum(f.colcount.astype(np.int64) ** 2))


@pytest.mark.parametrize("name", ["lap2d_32", "st27x3_5", "diff3d7_8"])
def test_llt_invariant(name):
    A, perm = inputs.workload(name)
    f = oracle.cholesky(A, perm)
    e = oracle.llt_error(A.n, f.bp, f.bi, f.bx, f.lp, f.li, f.lx)
    assert e <= 1e-13, e


def test_diagonal_and_block_diagonal():
    d = 1.0 + np.arange(10.0)
    f = oracle.cholesky(inputs.from_dense(np.diag(d)))
    assert np.array_equal(f.lx, np.sqrt(d))
    b1 = inputs.random_spd_dense(6, 1).to_dense()
    b2 = inputs.random_spd_dense(9, 2).to_dense()
    a = np.zeros((15, 15))
    a[:6, :6], a[6:, 6:] = b1, b2
    L = dense_L(oracle.cholesky(inputs.from_dense(a)))
    assert np.allclose(L[:6, :6], np.linalg.cholesky(b1), rtol=1e-14, atol=1e-14)
    assert np.allclose(L[6:, 6:], np.linalg.cholesky(b2), rtol=1e-14, atol=1e-14)
    assert np.all(L[6:, :6] == 0.0)


def test_not_spd_detected():
    d = 1.0 + np.arange(10.0)
    d[7] = -1.0
    with pytest.raises(oracle.NotSPD) as e:
        oracle.cholesky(inputs.from_dense(np.diag(d)))
    assert e.value.col == 7
    a = inputs.laplacian_2d_5pt(6)
    vals = a.vals.copy()
    vals[a.colptr[20]] = -4.0
    bad = inputs.SpdMatrix(a.n, a.colptr, a.rowind, vals)
    with pytest.raises(oracle.NotSPD):
        oracle.cholesky(bad)


def test_permute_matches_dense_indexing():
    A = inputs.laplacian_3d_7pt(4)
    perm = seeded_perm(A.n, 3)
    bp, bi, bx = oracle.permute(A.n, A.colptr, A.rowind, A.vals, perm)
    B = inputs.SpdMatrix(A.n, bp, bi, bx).to_dense()
    assert np.array_equal(B, A.to_dense()[np.ix_(perm, perm)])
    with pytest.raises(ValueError):
        oracle.permute(A.n, A.colptr, A.rowind, A.vals, np.zeros(A.n, np.int32))


def test_solve_1d_and_residual():
    n = 200
    A = inputs.laplacian_1d(n)
    f = oracle.cholesky(A)
    xt = inputs.uniform(1, 5, n)
    b = A.to_dense() @ xt
    x = f.solve(b)[:, 0]
    kappa = (2.0 / (1 - math.cos(math.pi / (n + 1))))  # lambda_max / lambda_min bound
    assert np.max(np.abs(x - xt)) <= 10 * kappa * 2.2e-16 * np.max(np.abs(xt))
    assert oracle.residual(n, A.colptr, A.rowind, A.vals, b, x) <= 1e-15


def test_solve_multi_rhs_permuted():
    A, perm = inputs.workload("st27x3_4")
    f = oracle.cholesky(A, perm)
    X_true = inputs.rhs_block(4, A.n, 3)
    Bm = A.to_scipy_full() @ X_true
    X = f.solve(Bm)
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, Bm, X) <= 1e-15
    np.testing.assert_allclose(X, np.linalg.solve(A.to_dense(), Bm), rtol=1e-11, atol=1e-13)


def test_residual_and_spmv_definitions():
    d = np.array([1.0, 2.0, 4.0])
    A = inputs.from_dense(np.diag(d))
    x = np.array([1.0, -1.0, 0.5])
    assert np.array_equal(oracle.spmv(3, A.colptr, A.rowind, A.vals, x), d * x)
    b = d * x
    b[1] += 0.25  # ||r||_inf = 0.25, ||A||_inf = 4, ||x||_inf = 1
    assert oracle.residual(3, A.colptr, A.rowind, A.vals, b, x) == 0.25 / 4.0
    A2 = inputs.laplacian_2d_5pt(5)
    x2 = inputs.uniform(3, 5, 25)
    assert np.allclose(oracle.spmv(25, A2.colptr, A2.rowind, A2.vals, x2), A2.to_dense() @ x2,
                       rtol=0, atol=1e-14)


# ---- OPT-D threshold (Sec. 4.1, Algorithm 1) and the hybrid switch (Sec. 4.3) -------------

def _opt_d_cases():
    path = os.path.join(os.path.dirname(__file__), "golden", "opt_d_cases.txt")
    cases = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        n, counts, d, why = [f.strip() for f in line.split(";")]
        c = []
        for item in counts.split(","):
            v, rep = item.split("*")
            c += [int(v)] * int(rep)
        cases.append((int(n), c, int(d), why))
    return cases


@pytest.mark.parametrize("case", _opt_d_cases(), ids=lambda c: c[3])
def test_opt_d_hand_computed(case):
    n, counts, d, _ = case
    assert oracle.opt_d(n, counts) == d


def test_opt_d_bounds_and_empty():
    rng = np.random.default_rng(7)
    for _ in range(50):
        ns = int(rng.integers(1, 400))
        c = rng.integers(0, 60, size=ns)
        d = oracle.opt_d(int(rng.integers(1, 100000)), c)
        assert 0 <= d <= c.max() + 1
    assert oracle.opt_d(100, []) == 0
    with pytest.raises(ValueError):
        oracle.opt_d(10, [1, -1])


def test_hybrid_switch_cases():
    # average supernode size n / nsuper and density nnz / n^2, by hand
    assert oracle.hybrid_uses_blas(1000, 10, 10**6)          # avg 100 > 50
    assert oracle.hybrid_uses_blas(1000, 40, 50)             # avg 25 > 20, density 5e-5 < 1e-4
    assert not oracle.hybrid_uses_blas(1000, 40, 1000)       # avg 25, density 1e-3
    assert not oracle.hybrid_uses_blas(1000, 100, 10)        # avg 10
    assert not oracle.hybrid_uses_blas(1000, 20, 10**5)      # avg exactly 50 (not above), density 0.1
    assert oracle.hybrid_uses_blas(1000, 20, 10)             # avg 50 > 20 and density 1e-5 < 1e-4


def _dense_b(f):
    """B = P^T A P as a full dense symmetric matrix, from the oracle's lower CSC."""
    B = np.zeros((f.n, f.n))
    for j in range(f.n):
        rows = f.bi[f.bp[j]:f.bp[j + 1]]
        B[rows, j] = f.bx[f.bp[j]:f.bp[j + 1]]
        B[j, rows] = f.bx[f.bp[j]:f.bp[j + 1]]
    return B


@pytest.mark.parametrize("name", ["lap2d_9", "st27x3_3", "diff3d7_5", "dense"])
def test_llt_error_matches_dense_norm(name):
    """||B - L L^T||_F / ||B||_F against the same quantity formed densely with numpy, on a
    factor perturbed in every stored entry (so the error is far above rounding and a dropped
    term, a missing factor 2 on the off-diagonal entries or a skipped diagonal shows)."""
    if name == "dense":
        A, perm = inputs.random_spd_dense(20, 4), None
    else:
        A, perm = inputs.workload(name)
    f = oracle.cholesky(A, perm)
    lx = f.lx * (1.0 + 1e-3 * inputs.uniform(21, 2, f.lx.size))
    L = np.zeros((f.n, f.n))
    for j in range(f.n):
        L[f.li[f.lp[j]:f.lp[j + 1]], j] = lx[f.lp[j]:f.lp[j + 1]]
    B = _dense_b(f)
    want = np.linalg.norm(B - L @ L.T) / np.linalg.norm(B)
    got = oracle.llt_error(f.n, f.bp, f.bi, f.bx, f.lp, f.li, lx)
    assert want > 1e-6
    assert abs(got - want) <= 1e-10 * want, (got, want)


@pytest.mark.parametrize("which", ["offdiag", "diag"])
def test_llt_error_single_entry_closed_form(which):
    """L' = L + delta e_i e_j^T (entry (i, j) of the pattern) gives
    L' L'^T - L L^T = delta (c e_i^T + e_i c^T) + delta^2 e_i e_i^T with c = L[:, j], whose
    Frobenius norm squared is 2 delta^2 sum_{k != i} c_k^2 + (2 delta c_i + delta^2)^2.
    L L^T equals B to rounding, so the oracle's ||B - L' L'^T||_F must be that value."""
    A, perm = inputs.workload("lap2d_8")
    f = oracle.cholesky(A, perm)
    j = 17
    q = f.lp[j] + (1 if which == "offdiag" else 0)  # first off-diagonal entry, or the pivot
    i = int(f.li[q])
    assert (i > j) == (which == "offdiag")
    delta = 1e-4
    lx = f.lx.copy()
    lx[q] += delta
    c = np.zeros(f.n)
    c[f.li[f.lp[j]:f.lp[j + 1]]] = f.lx[f.lp[j]:f.lp[j + 1]]
    e2 = 2 * delta ** 2 * (np.sum(c ** 2) - c[i] ** 2) + (2 * delta * c[i] + delta ** 2) ** 2
    bnorm = np.sqrt(np.sum(np.where(f.bi == np.repeat(np.arange(f.n), np.diff(f.bp)), 1.0, 2.0)
                           * f.bx ** 2))
    want = np.sqrt(e2) / bnorm
    got = oracle.llt_error(f.n, f.bp, f.bi, f.bx, f.lp, f.li, lx)
    assert abs(got - want) <= 1e-9 * want, (got, want)
    # the unperturbed factor sits at rounding level, far below the perturbation
    assert oracle.llt_error(f.n, f.bp, f.bi, f.bx, f.lp, f.li, f.lx) <= 1e-6 * want
