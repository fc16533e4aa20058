"""GPU parity of the mixed-precision factor (FP32 panels of the equilibrated matrix, FP64
pivot redo) and of FP64 iterative refinement.

The paper factors in double precision; the mixed factor must reach the same answer after
refinement: relative residual ||b - A x||_inf / (||A||_inf ||x||_inf) <= 1e-12 for 1 and 16
right-hand sides, and the same solution as the FP64 factor up to the conditioning.  The
FP32 factor itself is compared with the oracle's factor of the same equilibrated matrix."""
import numpy as np
import pytest

import oracle
import paper_2202_09288_gb300 as P
from paper_2202_09288_gb300 import inputs
from conftest import column_error

pytestmark = pytest.mark.gpu

REFINE_TOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def scaled_matrix(A):
    """S A S with S = diag(A)^{-1/2} (the equilibration the mixed factor applies)."""
    d = np.zeros(A.n)
    for j in range(A.n):
        assert A.rowind[A.colptr[j]] == j
        d[j] = A.vals[A.colptr[j]]
    s = 1.0 / np.sqrt(d)
    cols = np.repeat(np.arange(A.n), np.diff(A.colptr))
    vals = A.vals * s[A.rowind] * s[cols]
    return inputs.SpdMatrix(A.n, A.colptr, A.rowind, vals)


@pytest.mark.parametrize("name", ["lap2d_64", "st27x3_11", "diff3d7_14", "diff3d7_24"])
@pytest.mark.parametrize("nrhs", [1, 16])
def test_mixed_refinement_reaches_fp64(torch, name, nrhs):
    A, perm = inputs.workload(name)
    ctx = P.Context()
    sym = P.Symbolic(ctx, A, perm)
    mixed = P.Factor(ctx, sym, A.vals, precision=P.CHOL_MIXED)
    fp64 = P.Factor(ctx, sym, A.vals, precision=P.CHOL_FP64)
    assert mixed.status()[0] == P.CHOL_OK
    Xt = inputs.rhs_block(8, A.n, nrhs)
    Bm = np.asfortranarray(A.to_scipy_full() @ Xt)
    X, info = mixed.refine(Bm, tol=REFINE_TOL)
    res = oracle.residual(A.n, A.colptr, A.rowind, A.vals, Bm, X)
    assert res <= REFINE_TOL, (res, info)
    assert info["residual"] <= REFINE_TOL
    assert abs(info["residual"] - res) <= 0.5 * res + 1e-16  # device and oracle agree
    X64 = fp64.solve(Bm)
    scale = np.abs(X64).max()
    # both solutions are backward stable to 1e-12; their difference is bounded by the
    # condition number, which the log-normal diffusion makes large
    kappa_bound = {"lap2d_64": 1e4, "st27x3_11": 1e2, "diff3d7_14": 1e4, "diff3d7_24": 1e4}[name]
    assert np.abs(X - X64).max() <= kappa_bound * 1e-12 * scale


@pytest.mark.parametrize("name", ["lap2d_64", "st27x3_6"])
def test_mixed_factor_matches_oracle_of_scaled_matrix(torch, name):
    A, perm = inputs.workload(name)
    As = scaled_matrix(A)
    ref = oracle.cholesky(As, perm)
    ctx = P.Context()
    sym = P.Symbolic(ctx, A, perm)
    num = P.Factor(ctx, sym, A.vals, precision=P.CHOL_MIXED)
    lp, li, lx = num.export()
    assert np.array_equal(li, ref.li)
    err = np.linalg.norm(lx - ref.lx) / np.linalg.norm(ref.lx)
    assert err <= 2e-6, err  # FP32 rounding of a well-conditioned factor
    cerr = column_error(lp, lx, ref.lx)
    assert cerr <= 1e-5, cerr


def test_refine_with_fp64_factor(torch):
    A, perm = inputs.workload("st27x3_11")
    ctx = P.Context()
    num = P.Factor(ctx, P.Symbolic(ctx, A, perm), A.vals)
    b = A.to_scipy_full() @ inputs.rhs_block(3, A.n, 1)[:, 0]
    x, info = num.refine(b, tol=REFINE_TOL)
    assert info["residual"] <= REFINE_TOL and not info["fell_back"]
    assert info["iterations"] <= 1
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, x) <= REFINE_TOL


def test_fallback_to_fp64_when_refinement_stalls(torch):
    """maxit = 0 leaves the mixed factor no refinement step: the residual of its direct
    solve is far above 1e-12, so the call must fall back to the FP64 factor."""
    A, perm = inputs.workload("diff3d7_14")
    ctx = P.Context()
    num = P.Factor(ctx, P.Symbolic(ctx, A, perm), A.vals, precision=P.CHOL_MIXED)
    b = A.to_scipy_full() @ inputs.rhs_block(4, A.n, 1)[:, 0]
    x, info = num.refine(b, tol=REFINE_TOL, maxit=0)
    assert info["fell_back"]
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, x) <= REFINE_TOL
    # the FP64 factor is kept: a second call goes straight to it
    x2, info2 = num.refine(b, tol=REFINE_TOL, maxit=0)
    assert info2["fell_back"]
    # atomic assembly: equal up to the rounding of the forward-solve scatter order
    np.testing.assert_allclose(x2, x, rtol=0, atol=1e-12 * np.abs(x).max())


def test_small_pivot_redone_in_fp64(torch):
    """Blocks [[1, 1-e], [1-e, 1]] with e = 1e-7 have a second pivot of about 2e-7, below
    the FP32 threshold 1e-5: the diagonal block is refactored in FP64."""
    nb = 20
    e = 1e-7
    a = np.zeros((2 * nb, 2 * nb))
    for q in range(nb):
        a[2 * q:2 * q + 2, 2 * q:2 * q + 2] = [[1.0, 1.0 - e], [1.0 - e, 1.0]]
    A = inputs.from_dense(a)
    perm = np.arange(A.n, dtype=np.int32)
    ctx = P.Context()
    num = P.Factor(ctx, P.Symbolic(ctx, A, perm), A.vals, precision=P.CHOL_MIXED)
    assert num.status()[0] == P.CHOL_OK
    b = a @ inputs.rhs_block(5, A.n, 1)[:, 0]
    x, info = num.refine(b, tol=REFINE_TOL)
    assert info["pivot_redos"] >= 1
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, x) <= REFINE_TOL


def test_mixed_device_pointers_and_owner_determinism(torch):
    A, perm = inputs.workload("st27x3_8")
    ctx = P.Context(assembly=P.CHOL_ASSEMBLY_OWNER)
    sym = P.Symbolic(ctx, A, perm)
    num = P.Factor(ctx, sym, torch.from_numpy(A.vals).cuda(), precision=P.CHOL_MIXED)
    l1 = num.export()[2].copy()
    num.refactor(A.vals)
    assert np.array_equal(num.export()[2], l1)
    Bm = np.asfortranarray(A.to_scipy_full() @ inputs.rhs_block(6, A.n, 4))
    Bd = torch.from_numpy(np.ascontiguousarray(Bm.T)).cuda()
    Xd, info = num.refine(Bd, tol=REFINE_TOL)
    torch.cuda.synchronize()
    X = Xd.cpu().numpy().T
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, Bm, X) <= REFINE_TOL
    Xd2, _ = num.refine(Bd, tol=REFINE_TOL)
    torch.cuda.synchronize()
    assert np.array_equal(Xd2.cpu().numpy().T, X)


TC_ON = {"min_rows_tile128": 1, "min_level_tiles128": 0}
TC_OFF = {"min_rows_tile128": 1 << 30}


def mixed_factor(A, perm, policy, assembly=P.CHOL_ASSEMBLY_ATOMIC):
    ctx = P.Context(assembly=assembly)
    sym = P.Symbolic(ctx, A, perm)
    P.chol_sym_set_tile_policy(sym.handle, policy)
    P.chol_profile_enable(ctx.handle, True)
    num = P.Factor(ctx, sym, A.vals, precision=P.CHOL_MIXED)
    prof = P.chol_profile_read(ctx.handle)
    return ctx, sym, num, prof


def dense_problem(n):
    A = inputs.random_spd_dense(n, 4)
    return A, np.arange(A.n, dtype=np.int32)


@pytest.mark.parametrize("name", ["lap2d_64", "st27x3_11", "dense_300"])
@pytest.mark.parametrize("assembly", [P.CHOL_ASSEMBLY_ATOMIC, P.CHOL_ASSEMBLY_OWNER])
def test_tensor_core_tiles_match_oracle(torch, name, assembly):
    """128 x 128 Schur tiles on the tcgen05 tensor cores (3xTF32, FP32 accumulation): the
    FP32 factor of S A S matches the oracle's FP64 factor to FP32 rounding, the tasks ran
    on the tensor-core kernel, and the ragged tails (tile rows past the update's end,
    supernode widths that are not multiples of the MMA's K = 8) are covered."""
    A, perm = dense_problem(300) if name == "dense_300" else inputs.workload(name)
    ref = oracle.cholesky(scaled_matrix(A), perm)
    ctx, sym, num, prof = mixed_factor(A, perm, TC_ON, assembly)
    assert num.status()[0] == P.CHOL_OK
    assert prof["schur128_tc"]["launches"] > 0
    lp, li, lx = num.export()
    assert np.array_equal(li, ref.li)
    err = np.linalg.norm(lx - ref.lx) / np.linalg.norm(ref.lx)
    assert err <= 2e-6, err
    cerr = column_error(lp, lx, ref.lx)
    assert cerr <= 1e-5, cerr
    # and the tensor-core factor agrees with the SIMT FP32 factor to FP32 rounding
    _, _, simt, prof_simt = mixed_factor(A, perm, TC_OFF, assembly)
    assert prof_simt["schur128_tc"]["launches"] == 0
    lx2 = simt.export()[2]
    assert np.linalg.norm(lx - lx2) / np.linalg.norm(lx2) <= 2e-6


@pytest.mark.parametrize("name", ["diff3d7_14", "st27x3_11"])
def test_tensor_core_factor_refines_to_fp64(torch, name):
    A, perm = inputs.workload(name)
    ctx, sym, num, prof = mixed_factor(A, perm, TC_ON)
    assert prof["schur128_tc"]["launches"] > 0
    B = np.asfortranarray(A.to_scipy_full() @ inputs.rhs_block(12, A.n, 4))
    X, info = num.refine(B, tol=REFINE_TOL)
    assert not info["fell_back"]
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, B, X) <= REFINE_TOL


def test_tensor_core_owner_mode_is_bitwise_reproducible(torch):
    A, perm = inputs.workload("st27x3_11")
    _, _, a, _ = mixed_factor(A, perm, TC_ON, P.CHOL_ASSEMBLY_OWNER)
    _, _, b, _ = mixed_factor(A, perm, TC_ON, P.CHOL_ASSEMBLY_OWNER)
    lx = a.export()[2]
    assert np.array_equal(lx, b.export()[2])
    a.refactor(A.vals)
    assert np.array_equal(lx, a.export()[2])
