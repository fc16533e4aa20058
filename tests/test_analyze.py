"""Host symbolic analysis of the library (through the C ABI) against the oracle's brute
force: elimination tree, column counts, supernode partition and level sets must match
bit for bit (Sec. 2 analysis; Sec. 3 / Fig. 1 level sets).  CPU only."""
import numpy as np
import pytest

import oracle
import paper_2202_09288_gb300 as P
from conftest import fig1_matrix, fig1_tree
from paper_2202_09288_gb300 import inputs

CASES = ["lap2d_16", "lap2d_64", "lap3d_9", "st27x3_6", "diff3d7_10"]


def both(A, perm, W):
    # the oracle's partition is the fundamental one: no relaxed amalgamation here
    sym = P.Symbolic(P.make_opts(width_cap=W, relax=-1.0), A, perm)
    got = sym.export()
    bp, bi, bx = oracle.permute(A.n, A.colptr, A.rowind, A.vals, perm)
    parent, cc, lp, li = oracle.symbolic(A.n, bp, bi)
    start, sp, lv = oracle.supernodes(parent, cc, W)
    return sym, got, (parent, cc, start, lv)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("W", [64, 16, 1, 128])
def test_symbolic_matches_oracle(name, W):
    A, perm = inputs.workload(name)
    sym, got, (parent, cc, start, lv) = both(A, perm, W)
    assert np.array_equal(got["parent"], parent)
    assert np.array_equal(got["colcount"], cc)
    assert np.array_equal(got["sn_start"], start)
    assert np.array_equal(got["sn_level"], lv)
    info = sym.info
    assert info["nnz_l"] == int(cc.sum())
    assert info["flops"] == float(np.sum(cc.astype(np.float64) ** 2))
    assert info["nsuper"] == len(start) - 1
    assert info["nlevels"] == int(lv.max()) + 1
    assert info["max_width"] <= W


def test_random_patterns_and_perms():
    for seed in range(5):
        n = 80
        u = inputs.uniform(200 + seed, 7, n * n).reshape(n, n)
        adj = (u > 0.93) | (u.T > 0.93)
        a = np.where(adj, -0.05, 0.0)
        a = np.tril(a) + np.tril(a, -1).T
        a[np.arange(n), np.arange(n)] = 1.0
        A = inputs.from_dense(a)
        perm = np.argsort(inputs.uniform(seed, 9, n), kind="stable").astype(np.int32)
        for W in (3, 64):
            sym, got, (parent, cc, start, lv) = both(A, perm, W)
            assert np.array_equal(got["parent"], parent)
            assert np.array_equal(got["colcount"], cc)
            assert np.array_equal(got["sn_start"], start)
            assert np.array_equal(got["sn_level"], lv)


def test_fig1_tree_levels():
    """Sec. 3, Fig. 1 (tests/golden/fig1_tree.txt): the library's level sets."""
    edges, levels = fig1_tree()
    A = fig1_matrix()
    sym = P.Symbolic(P.make_opts(relax=-1.0), A, np.arange(A.n, dtype=np.int32))
    e = sym.export()
    assert sorted((j + 1, int(p) + 1) for j, p in enumerate(e["parent"]) if p >= 0) == sorted(edges)
    lv = e["sn_level"]
    assert [sorted(int(s) + 1 for s in np.nonzero(lv == l)[0]) for l in range(lv.max() + 1)] == levels


def test_empty_and_one():
    A = inputs.from_dense(np.array([[2.0]]))
    sym = P.Symbolic(None, A, np.zeros(1, np.int32))
    assert sym.info["nnz_l"] == 1 and sym.info["nsuper"] == 1
    A0 = inputs.SpdMatrix(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    sym0 = P.Symbolic(None, A0, np.zeros(0, np.int32))
    assert sym0.info["nnz_l"] == 0 and sym0.info["nsuper"] == 0


def _bad(n, colptr, rowind, perm):
    with pytest.raises(P.CholError) as e:
        P.chol_analyze(None, n, np.array(colptr), np.array(rowind), np.array(perm))
    assert e.value.status == P.CHOL_E_INVALID


def test_invalid_inputs_rejected():
    _bad(2, [0, 1, 2], [1, 0], [0, 1])          # entry above the diagonal in column 1
    _bad(2, [0, 2, 3], [1, 0, 1], [0, 1])       # unsorted rows
    _bad(2, [0, 2, 3], [0, 0, 1], [0, 1])       # duplicate row
    _bad(2, [0, 2, 3], [0, 2, 1], [0, 1])       # row out of range
    _bad(2, [0, 1, 2], [0, 1], [0, 0])          # perm not a permutation
    _bad(2, [0, 1, 2], [0, 1], [0, 2])          # perm out of range
    _bad(-1, [0], [], [])                       # negative order
    with pytest.raises(P.CholError):
        P.chol_analyze(P.make_opts(width_cap=512), 1, np.array([0, 1]), np.array([0]),
                       np.array([0]))


def test_abi_exports_every_declared_symbol():
    import re
    import ctypes
    hdr = open(P.LIB_PATH.replace("paper_2202_09288_gb300/libchol.so", "include/chol.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(chol_[a-z_0-9]+)\s*\(", hdr))
    assert names, "no declarations parsed"
    L = ctypes.CDLL(P.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert set(P.EXPORTS) >= names


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.CholError) as e:
        P.Context()
    assert e.value.status == P.CHOL_E_NODEVICE


def check_panels_cover_l(sym, A, perm, exact):
    """Every column's rows in L (the oracle's symbolic pattern) lie in its panel's rows from
    the column's own position on; with fundamental supernodes they are equal."""
    got = sym.export()
    rowptr, rows = P.chol_sym_rows(sym.handle)
    bp, bi, bx = oracle.permute(A.n, A.colptr, A.rowind, A.vals, perm)
    parent, cc, lp, li = oracle.symbolic(A.n, bp, bi)
    start = got["sn_start"]
    for s in range(len(start) - 1):
        r = rows[rowptr[s]:rowptr[s + 1]]
        assert np.all(np.diff(r) > 0)
        w = start[s + 1] - start[s]
        assert np.array_equal(r[:w], np.arange(start[s], start[s + 1]))
        for jj in range(w):
            j = start[s] + jj
            col = li[lp[j]:lp[j + 1]]
            if exact:
                assert np.array_equal(r[jj:], col)
            else:
                assert np.all(np.isin(col, r[jj:]))
    return got, parent, cc


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("W", [64, 128, 5])
def test_relaxed_amalgamation(name, W):
    """Relaxed supernodes (Sec. 2: explicit zeros buy wider dense blocks): the panels
    cover L, the etree and counts are untouched, the reported flops stay those of the
    exact L, the explicit zeros stay within the merge rule's largest share (1/2), and the
    level sets follow the definition over the relaxed tree (Fig. 1)."""
    A, perm = inputs.workload(name)
    sym = P.Symbolic(P.make_opts(width_cap=W), A, perm)
    got, parent, cc = check_panels_cover_l(sym, A, perm, exact=False)
    assert np.array_equal(got["parent"], parent) and np.array_equal(got["colcount"], cc)
    info = sym.info
    assert info["flops"] == float(np.sum(cc.astype(np.float64) ** 2))
    assert info["nnz_l"] == int(cc.sum())
    fund = P.Symbolic(P.make_opts(width_cap=W, relax=-1.0), A, perm).info
    assert info["nfundamental"] == fund["nfundamental"]
    assert info["nsuper"] <= fund["nsuper"]
    assert info["flops_panel"] >= info["flops"]
    assert fund["flops_panel"] == fund["flops"]
    start = got["sn_start"]
    wdt = np.diff(start).astype(np.int64)
    m = cc[start[:-1]].astype(np.int64)  # rows of a panel = count of its first column...
    rowptr, _ = P.chol_sym_rows(sym.handle)
    m = np.diff(rowptr)                  # ...only without padding: take the panel's own
    lower = int(np.sum(m * wdt - wdt * (wdt - 1) // 2))
    assert info["l_storage"] >= lower >= info["nnz_l"]
    assert lower - info["nnz_l"] <= 0.5 * lower
    assert info["max_width"] <= W
    # levels: 0 without children, else 1 + the children's largest
    col2sn = np.repeat(np.arange(len(start) - 1), wdt)
    lv = np.zeros(len(start) - 1, np.int64)
    for s in range(len(start) - 1):
        par = parent[start[s + 1] - 1]
        if par >= 0:
            t = col2sn[par]
            lv[t] = max(lv[t], lv[s] + 1)
    assert np.array_equal(got["sn_level"], lv)


def test_relaxed_amalgamation_merges_narrow_supernodes():
    A, perm = inputs.workload("diff3d7_10")
    relaxed = P.Symbolic(P.make_opts(), A, perm).info
    fund = P.Symbolic(P.make_opts(relax=-1.0), A, perm).info
    assert relaxed["nsuper"] < fund["nsuper"] / 2
    assert relaxed["flops_panel"] <= 1.5 * relaxed["flops"]  # small fronts: up to 1/2 zeros


def test_fundamental_panels_equal_l():
    A, perm = inputs.workload("lap3d_9")
    sym = P.Symbolic(P.make_opts(relax=-1.0), A, perm)
    check_panels_cover_l(sym, A, perm, exact=True)


# ---- task granularity (Sec. 4: OPT-D, OPT-D-COST, hybrid) applied to Schur tiles ---------

def test_opt_d_library_matches_oracle():
    rng = np.random.default_rng(11)
    for _ in range(100):
        ns = int(rng.integers(0, 400))
        c = rng.integers(0, int(rng.integers(1, 5000)), size=ns)
        n = int(rng.integers(0, 10 ** 6))
        assert P.chol_opt_d(n, c) == oracle.opt_d(n, c)
    # skewed counts (mostly zero or one, a few large), as supernodal trees give: every
    # stopping criterion of the algorithm becomes the binding one somewhere in this sweep
    for _ in range(300):
        ns = int(rng.integers(1, 6000))
        c = np.where(rng.random(ns) < 0.9, rng.integers(0, 2, size=ns),
                     rng.integers(0, int(rng.integers(2, 3000)), size=ns))
        n = int(rng.integers(0, 2 * 10 ** 5))
        assert P.chol_opt_d(n, c) == oracle.opt_d(n, c)
    assert P.chol_opt_d(100, []) == oracle.opt_d(100, []) == 0
    with pytest.raises(P.CholError):
        P.chol_opt_d(10, [3, -1])


SIZE_ONLY = {"min_rows_tile64": 64, "min_rows_tile32": 17, "min_level_tiles64": 0,
             "min_rows_tile128": 128, "min_level_tiles128": 0}


@pytest.mark.parametrize("name", ["st27x3_8", "lap3d_12", "diff3d7_12", "lap2d_64"])
def test_granularity_rules(name):
    A, perm = inputs.workload(name)
    sym = P.Symbolic(P.make_opts(width_cap=64), A, perm)
    start = sym.export()["sn_start"]
    rowptr, _ = P.chol_sym_rows(sym.handle)
    w = np.diff(start).astype(np.int64)
    u = np.diff(rowptr).astype(np.int64) - w
    # inner tasks of each outer task under the size thresholds alone (level counts off)
    T = np.where(u >= 128, 128, np.where(u >= 64, 64, np.where(u >= 17, 32, 16)))
    nt = (u + T - 1) // T
    inner = np.where(u > 0, nt * (nt + 1) // 2, 0)
    D = oracle.opt_d(A.n, inner)
    P.chol_sym_set_tile_policy(sym.handle, {**SIZE_ONLY, "granularity": P.CHOL_GRAN_TILES})
    assert P.chol_sym_granularity(sym.handle) == {"rule": 0, "D": -1, "nsplit": 0}
    P.chol_sym_set_tile_policy(sym.handle, {**SIZE_ONLY, "granularity": P.CHOL_GRAN_OPTD})
    assert P.chol_sym_granularity(sym.handle) == {"rule": P.CHOL_GRAN_OPTD, "D": D,
                                                  "nsplit": int(np.sum((inner >= D) & (inner > 0)))}
    P.chol_sym_set_tile_policy(sym.handle, {**SIZE_ONLY, "granularity": P.CHOL_GRAN_OPTD_COST})
    costly = 2.0 * T * T * w >= 50000.0
    assert P.chol_sym_granularity(sym.handle) == {"rule": P.CHOL_GRAN_OPTD_COST, "D": D,
                                                  "nsplit": int(np.sum((inner >= D) & (inner > 0)
                                                                       & costly))}
    P.chol_sym_set_tile_policy(sym.handle, {**SIZE_ONLY, "granularity": P.CHOL_GRAN_HYBRID})
    blas = oracle.hybrid_uses_blas(A.n, len(w), 2 * sym.info["nnz_a"] - A.n)
    got = P.chol_sym_granularity(sym.handle)
    assert got["rule"] == (P.CHOL_GRAN_TILES if blas else P.CHOL_GRAN_OPTD_COST)
    with pytest.raises(P.CholError):
        P.chol_sym_set_tile_policy(sym.handle, {"granularity": 4})


@pytest.mark.parametrize("name", ["st27x3_8", "lap3d_12", "diff3d7_12", "lap2d_64"])
@pytest.mark.parametrize("rule", [0, 1, 2, 3])
def test_schur_tiles_cover_each_update_once(name, rule):
    """Under every granularity rule, the Schur tiles of each supernode cover the lower
    triangle of its update U_s = L21 L21^T exactly once (tiles clipped at its order)."""
    A, perm = inputs.workload(name)
    sym = P.Symbolic(P.make_opts(width_cap=64), A, perm)
    P.chol_sym_set_tile_policy(sym.handle, {"granularity": rule})
    start = sym.export()["sn_start"]
    rowptr, _ = P.chol_sym_rows(sym.handle)
    u = np.diff(rowptr) - np.diff(start)
    t = P.chol_sym_schur_tiles(sym.handle)
    cover = {s: np.zeros((u[s], u[s]), dtype=np.int32) for s in range(len(u)) if u[s] > 0}
    for s, i0, k0, T in zip(t["s"], t["i0"], t["k0"], t["tile"]):
        assert k0 <= i0 and i0 % T == 0 and k0 % T == 0
        cover[s][i0:i0 + T, k0:k0 + T] += 1
    for s, c in cover.items():
        low = c[np.tril_indices(len(c))]
        assert low.min() == 1 and low.max() == 1, s


@pytest.mark.parametrize("name", ["st27x3_11", "diff3d7_14", "lap2d_64"])
def test_tensor_core_trsm_levels(name):
    """The tensor-core TRSM (FP64 factors) takes a level's 128-tile supernodes when their
    off-diagonal rows add up to min_rows_trsm_tc: with the size thresholds alone deciding the
    128-tile class (u >= 128, no level counts), the count of such supernodes follows from the
    level sets."""
    A, perm = inputs.workload(name)
    sym = P.Symbolic(P.make_opts(width_cap=64), A, perm)
    ex = sym.export()
    lvl = ex["sn_level"]
    rowptr, _ = P.chol_sym_rows(sym.handle)
    w = np.diff(ex["sn_start"]).astype(np.int64)
    u = np.diff(rowptr).astype(np.int64) - w
    c128 = u >= 128
    rows = np.bincount(lvl[c128], weights=u[c128], minlength=int(lvl.max()) + 1)
    for thr in (1, 128, 300, 1000, 16384):
        P.chol_sym_set_tile_policy(sym.handle, {**SIZE_ONLY, "min_rows_trsm_tc": thr})
        expect = int(np.sum(c128 & (rows[lvl] >= thr)))
        assert P.chol_sym_info(sym.handle)["ntrsm_tc"] == expect, thr
    with pytest.raises(P.CholError):
        P.chol_sym_set_tile_policy(sym.handle, {"min_rows_trsm_tc": 0})
