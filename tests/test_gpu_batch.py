"""GPU parity of batched factorization (one launch per level and kernel kind across many
matrices, CUDA-graph replay), of Schur tile policies and of the autotuner.  Every member must match the oracle as when factored alone (Sec. 3, Fig. 1:
independent supernodes run together; here across matrices), and with owner-ordered
assembly a member's factor must be bitwise identical alone and in the mix."""
import numpy as np
import pytest

import oracle
import paper_2202_09288_gb300 as P
from paper_2202_09288_gb300 import inputs
from conftest import column_error

pytestmark = pytest.mark.gpu

FACTOR_TOL = 1e-12
RESID_TOL = 1e-13


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def problem(name):
    if name.startswith("dense_"):
        A = inputs.random_spd_dense(int(name.split("_")[1]), 9)
        return A, np.arange(A.n, dtype=np.int32)
    if name.startswith("lap1d_"):
        A = inputs.laplacian_1d(int(name.split("_")[1]))
        return A, np.arange(A.n, dtype=np.int32)
    return inputs.workload(name)


MIX = ["lap2d_23", "st27x3_6", "diff3d7_10", "dense_100", "lap1d_50", "lap3d_9"]


def check_member(ctx, num, A, perm, ref):
    assert num.status()[0] == P.CHOL_OK
    lp, li, lx = num.export()
    assert np.array_equal(li, ref.li)
    err = np.linalg.norm(lx - ref.lx) / np.linalg.norm(ref.lx)
    assert err <= FACTOR_TOL, err
    cerr = column_error(lp, lx, ref.lx)
    assert cerr <= FACTOR_TOL, cerr
    b = A.to_scipy_full() @ inputs.rhs_block(2, A.n, 1)[:, 0]
    x = num.solve(b)
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, x) <= RESID_TOL


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_of_different_matrices(torch, use_graph):
    ctx = P.Context()
    probs = [problem(nm) for nm in MIX]
    refs = [oracle.cholesky(A, perm) for A, perm in probs]
    syms = [P.Symbolic(ctx, A, perm) for A, perm in probs]
    # members start factored from other values (3 A); the batch factors A itself
    nums = [P.Factor(ctx, s, 3.0 * A.vals) for s, (A, _) in zip(syms, probs)]
    batch = P.Batch(ctx, nums)
    batch.factorize([A.vals for A, _ in probs], use_graph=use_graph)
    for num, (A, perm), ref in zip(nums, probs, refs):
        check_member(ctx, num, A, perm, ref)
    # replay with new values: 4 A has factor 2 L
    batch.factorize([4.0 * A.vals for A, _ in probs], use_graph=use_graph)
    for num, ref in zip(nums, refs):
        lx = num.export()[2]
        assert np.linalg.norm(lx - 2 * ref.lx) / np.linalg.norm(2 * ref.lx) <= FACTOR_TOL
        assert column_error(ref.lp, lx, 2 * ref.lx) <= FACTOR_TOL
    batch.close()


def test_batch_device_values_and_mixed(torch):
    ctx = P.Context()
    probs = [problem(nm) for nm in ["st27x3_6", "diff3d7_10", "lap2d_23"]]
    syms = [P.Symbolic(ctx, A, perm) for A, perm in probs]
    nums = [P.Factor(ctx, s, A.vals, precision=P.CHOL_MIXED) for s, (A, _) in zip(syms, probs)]
    batch = P.Batch(ctx, nums)
    batch.factorize([torch.from_numpy(A.vals).cuda() for A, _ in probs])
    for num, (A, perm) in zip(nums, probs):
        assert num.status()[0] == P.CHOL_OK
        b = A.to_scipy_full() @ inputs.rhs_block(3, A.n, 1)[:, 0]
        x, info = num.refine(b, tol=1e-12)
        assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, x) <= 1e-12
    batch.close()


def test_owner_batch_is_bitwise_equal_to_alone(torch):
    """Alone vs in the mix: with owner-ordered assembly the member's factor and solution
    do not depend on the other members."""
    ctx = P.Context(assembly=P.CHOL_ASSEMBLY_OWNER)
    probs = [problem(nm) for nm in MIX]
    syms = [P.Symbolic(ctx, A, perm) for A, perm in probs]
    alone = []
    for s, (A, _) in zip(syms, probs):
        f = P.Factor(ctx, s, A.vals)
        b = A.to_scipy_full() @ inputs.rhs_block(4, A.n, 1)[:, 0]
        alone.append((f.export()[2].copy(), f.solve(b).copy(), b))
        del f
    nums = [P.Factor(ctx, s, 2.0 * A.vals) for s, (A, _) in zip(syms, probs)]
    batch = P.Batch(ctx, nums)
    batch.factorize([A.vals for A, _ in probs], use_graph=True)
    for num, (lx, x, b) in zip(nums, alone):
        assert np.array_equal(num.export()[2], lx)
        assert np.array_equal(num.solve(b), x)
    batch.close()


NO128 = {"min_rows_tile128": 1 << 30, "min_level_tiles128": 0}
POLICIES = [
    {"min_rows_tile64": 1, "min_rows_tile32": 1, "min_level_tiles64": 0, **NO128},  # all 64
    {"min_rows_tile64": 10 ** 6, "min_rows_tile32": 10 ** 6, "min_level_tiles64": 0,
     **NO128},                                                                    # all 16
    {"min_rows_tile64": 10 ** 6, "min_rows_tile32": 1, "min_level_tiles64": 0, **NO128},  # 32
    {"min_rows_tile64": 1, "min_rows_tile32": 1, "min_level_tiles64": 0,
     "min_rows_tile128": 1, "min_level_tiles128": 0, "min_rows_trsm_tc": 1},      # all 128
]


@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("assembly", [P.CHOL_ASSEMBLY_ATOMIC, P.CHOL_ASSEMBLY_OWNER])
def test_tile_policies_are_correct(torch, policy, assembly):
    ctx = P.Context(assembly=assembly)
    A, perm = problem("st27x3_11")
    ref = oracle.cholesky(A, perm)
    sym = P.Symbolic(ctx, A, perm)
    P.chol_sym_set_tile_policy(sym.handle, policy)
    got = P.chol_sym_get_tile_policy(sym.handle)
    assert {k: got[k] for k in policy} == policy and got["granularity"] == P.CHOL_GRAN_TILES
    P.chol_profile_enable(ctx.handle, True)
    num = P.Factor(ctx, sym, A.vals)
    prof = P.chol_profile_read(ctx.handle)
    if policy["min_rows_tile128"] == 1:  # 128-wide FP64 tasks: bf16 tensor-core slices
        assert prof["schur128_oz"]["launches"] > 0 and prof["trsm_oz"]["launches"] > 0
        assert prof["schur64_f64"]["launches"] == 0
    check_member(ctx, num, A, perm, ref)


def test_tile_policy_rejects_bad_thresholds(torch):
    ctx = P.Context()
    A, perm = problem("lap2d_23")
    sym = P.Symbolic(ctx, A, perm)
    before = P.chol_sym_get_tile_policy(sym.handle)
    for bad in [{"min_rows_tile64": 0}, {"min_rows_tile128": 0}, {"min_level_tiles128": -1}]:
        with pytest.raises(P.CholError):
            P.chol_sym_set_tile_policy(sym.handle, bad)
    assert P.chol_sym_get_tile_policy(sym.handle) == before


def test_autotuner(torch):
    ctx = P.Context()
    A, perm = problem("st27x3_14")
    ref = oracle.cholesky(A, perm)
    sym = P.Symbolic(ctx, A, perm)
    num = P.Factor(ctx, sym, A.vals)
    policy, ms = num.autotune(reps=1)
    assert ms > 0 and set(policy) == {"min_rows_tile64", "min_rows_tile32", "min_level_tiles64",
                                      "min_rows_tile128", "min_level_tiles128", "granularity",
                                      "min_rows_trsm_tc"}
    assert P.chol_sym_get_tile_policy(sym.handle) == policy
    check_member(ctx, num, A, perm, ref)


@pytest.mark.parametrize("rule", [P.CHOL_GRAN_OPTD, P.CHOL_GRAN_OPTD_COST, P.CHOL_GRAN_HYBRID])
@pytest.mark.parametrize("precision", [P.CHOL_FP64, P.CHOL_MIXED])
def test_granularity_rules_are_correct(torch, rule, precision):
    """The OPT-D / OPT-D-COST / hybrid task granularity (Sec. 4) only regroups the Schur
    tiles: the factor matches the oracle (FP64) or refines to 1e-12 (mixed)."""
    ctx = P.Context()
    A, perm = problem("st27x3_11")
    sym = P.Symbolic(ctx, A, perm)
    P.chol_sym_set_tile_policy(sym.handle, {"granularity": rule})
    g = P.chol_sym_granularity(sym.handle)
    assert g["D"] >= 0 or g["rule"] == P.CHOL_GRAN_TILES
    num = P.Factor(ctx, sym, A.vals, precision)
    if precision == P.CHOL_FP64:
        check_member(ctx, num, A, perm, oracle.cholesky(A, perm))
    else:
        B = np.asfortranarray(A.to_scipy_full() @ inputs.rhs_block(8, A.n, 1))
        X, info = num.refine(B, tol=1e-12)
        assert info["residual"] <= 1e-12
        assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, B, X) <= 1e-12
