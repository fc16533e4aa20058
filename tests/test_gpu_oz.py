"""GPU parity of the FP64 Schur tiles computed on the bf16 tensor cores by operand
splitting: every L21 row scaled by a power of two and cut into 8 exact 7-bit slices whose
products accumulate exactly.  The FP64 factor must still match the oracle to 1e-12
(relative Frobenius) with residual <= 1e-13 (Sec. 3, Listing 1: the SYRK + GEMM update,
here on 128 x 128 tiles), agree with the FP64 DMMA tiles to far below that, and stay
bitwise reproducible with owner-ordered assembly, alone and batched."""
import numpy as np
import pytest

import oracle
import paper_2202_09288_gb300 as P
from paper_2202_09288_gb300 import inputs
from conftest import column_error

pytestmark = pytest.mark.gpu

# every supernode in the 128-tile class, and every level's TRSM on the tensor cores
ALL128 = {"min_rows_tile64": 1, "min_rows_tile32": 1, "min_level_tiles64": 0,
          "min_rows_tile128": 1, "min_level_tiles128": 0, "min_rows_trsm_tc": 1}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def problem(name):
    if name.startswith("dense_"):
        A = inputs.random_spd_dense(int(name.split("_")[1]), 6)
        return A, np.arange(A.n, dtype=np.int32)
    if name == "scaled_st27x3_9":
        # D A D with row scales spread over 16 decades: the per-row exponents of the
        # slices must carry them; the factor is D L
        A, perm = inputs.workload("st27x3_9")
        d = 10.0 ** (8.0 * inputs.uniform(17, 3, A.n))
        cols = np.repeat(np.arange(A.n), np.diff(A.colptr))
        vals = A.vals * d[A.rowind] * d[cols]
        return inputs.SpdMatrix(A.n, A.colptr, A.rowind, vals, A.grid, A.dofs), perm
    return inputs.workload(name)


def factor(A, perm, mode=P.CHOL_SCHUR_OZAKI, assembly=P.CHOL_ASSEMBLY_ATOMIC, policy=ALL128):
    ctx = P.Context(assembly=assembly, fp64_schur=mode)
    sym = P.Symbolic(ctx, A, perm)
    P.chol_sym_set_tile_policy(sym.handle, policy)
    P.chol_profile_enable(ctx.handle, True)
    num = P.Factor(ctx, sym, A.vals)
    prof = P.chol_profile_read(ctx.handle)
    return ctx, sym, num, prof


@pytest.mark.parametrize("name", ["lap2d_64", "st27x3_11", "dense_300", "diff3d7_14",
                                  "scaled_st27x3_9"])
@pytest.mark.parametrize("assembly", [P.CHOL_ASSEMBLY_ATOMIC, P.CHOL_ASSEMBLY_OWNER])
def test_oz_tiles_match_oracle(torch, name, assembly):
    A, perm = problem(name)
    ref = oracle.cholesky(A, perm)
    ctx, sym, num, prof = factor(A, perm, assembly=assembly)
    assert num.status()[0] == P.CHOL_OK
    # the 128-tile supernodes of levels with several supernodes take the tensor-core TRSM
    # (A21's slices, then the product with the inverse's slices); every 128-tile level
    # slices its L21 for the tiles
    assert prof["schur128_oz"]["launches"] > 0
    assert prof["oz_slice"]["launches"] == (prof["schur128_oz"]["launches"] +
                                            prof["trsm_oz"]["launches"])
    assert prof["trsm_oz"]["launches"] > 0
    lp, li, lx = num.export()
    assert np.array_equal(li, ref.li)
    err = np.linalg.norm(lx - ref.lx) / np.linalg.norm(ref.lx)
    assert err <= 1e-12, err
    # column by column too: the slices' error is relative to each row's largest entry, and
    # in the row-scaled case an error confined to the small rows would not move the norm
    # of the whole factor
    cerr = column_error(lp, lx, ref.lx)
    assert cerr <= 1e-12, cerr
    b = A.to_scipy_full() @ inputs.rhs_block(5, A.n, 1)[:, 0]
    x = num.solve(b)
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, x) <= 1e-13


@pytest.mark.parametrize("name", ["st27x3_11", "dense_300"])
def test_oz_agrees_with_dmma(torch, name):
    A, perm = problem(name)
    _, _, oz, prof = factor(A, perm)
    _, _, dm, prof_dm = factor(A, perm, mode=P.CHOL_SCHUR_DMMA)
    assert prof_dm["schur128_oz"]["launches"] == 0 and prof_dm["schur128_f64"]["launches"] > 0
    # the tensor-core TRSM against the FP64 one too
    assert prof["trsm_oz"]["launches"] > 0 and prof_dm["trsm_oz"]["launches"] == 0
    lp, _, a = oz.export()
    b = dm.export()[2]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-14
    assert column_error(lp, a, b) <= 1e-13


def test_oz_owner_bitwise_alone_and_batched(torch):
    probs = [problem(nm) for nm in ["st27x3_11", "dense_300", "lap2d_40"]]
    ctx = P.Context(assembly=P.CHOL_ASSEMBLY_OWNER)
    syms = [P.Symbolic(ctx, A, perm) for A, perm in probs]
    for s in syms:
        P.chol_sym_set_tile_policy(s.handle, ALL128)
    alone = []
    for s, (A, _) in zip(syms, probs):
        f = P.Factor(ctx, s, A.vals)
        first = f.export()[2].copy()
        f.refactor(A.vals)
        assert np.array_equal(f.export()[2], first)  # run to run
        alone.append(first)
        del f
    P.chol_profile_enable(ctx.handle, True)
    nums = [P.Factor(ctx, s, 2.0 * A.vals) for s, (A, _) in zip(syms, probs)]
    batch = P.Batch(ctx, nums)
    for use_graph in (False, True):
        batch.factorize([A.vals for A, _ in probs], use_graph=use_graph)
        for num, lx in zip(nums, alone):
            assert np.array_equal(num.export()[2], lx)
    assert P.chol_profile_read(ctx.handle)["schur128_oz"]["launches"] > 0
    batch.close()


def test_oz_width_128_uses_dmma(torch):
    """W = 128 is beyond the slices' K = 64: the FP64 factor falls back to DMMA tiles."""
    A, perm = problem("st27x3_11")
    ref = oracle.cholesky(A, perm)
    ctx = P.Context(width_cap=128)
    sym = P.Symbolic(ctx, A, perm)
    P.chol_sym_set_tile_policy(sym.handle, ALL128)
    P.chol_profile_enable(ctx.handle, True)
    num = P.Factor(ctx, sym, A.vals)
    prof = P.chol_profile_read(ctx.handle)
    assert prof["schur128_oz"]["launches"] == 0
    lx = num.export()[2]
    assert np.linalg.norm(lx - ref.lx) / np.linalg.norm(ref.lx) <= 1e-12
    assert column_error(ref.lp, lx, ref.lx) <= 1e-12
