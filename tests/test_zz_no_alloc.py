"""chol_solve_noalloc: the solve variant for callers that cannot allocate device memory
when they solve (stream capture in global mode, runtimes that own all device memory).
Its workspace is a fixed array inside the library; the test checks, through the C ABI,
that two calls in a row give the same solutions as chol_solve (the allocating entry
point) within the tolerances of the other GPU tests; that the first solve of a fresh factor
through it changes the device's free memory by nothing (with more right-hand sides than one
pass takes, so the array is reused by two passes); that it serves an FP32 (mixed-precision)
factor as chol_solve does; and that a request larger than the fixed array is refused with
CHOL_E_SCRATCH.  It sits in a file of its own that pytest collects last."""
import numpy as np
import pytest

import oracle
import paper_2202_09288_gb300 as P
from paper_2202_09288_gb300 import inputs

pytestmark = pytest.mark.gpu

RESID_TOL = 1e-13
AGREE_TOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("assembly", [P.CHOL_ASSEMBLY_ATOMIC, P.CHOL_ASSEMBLY_OWNER])
def test_noalloc_matches_chol_solve_twice(torch, assembly):
    ctx = P.Context(assembly=assembly)
    A, perm = inputs.workload("st27x3_10")
    sym = P.Symbolic(ctx, A, perm)
    num = P.Factor(ctx, sym, A.vals)
    assert num.status()[0] == P.CHOL_OK
    Afull = A.to_scipy_full()
    for call, k in enumerate((3, 5)):  # two calls in a row, different right-hand sides
        Bm = np.asfortranarray(Afull @ inputs.rhs_block(40 + call, A.n, k))
        Bd = torch.from_numpy(np.ascontiguousarray(Bm.T)).cuda()
        ref = torch.empty_like(Bd)
        got = torch.full_like(Bd, float("nan"))
        num.solve(Bd, ref)
        P.chol_solve_noalloc(ctx.handle, num.handle, Bd, got)
        torch.cuda.synchronize()
        ref_h, got_h = ref.cpu().numpy().T, got.cpu().numpy().T
        assert np.all(np.isfinite(got_h))
        res = oracle.residual(A.n, A.colptr, A.rowind, A.vals, Bm, got_h)
        assert res <= RESID_TOL, res
        np.testing.assert_allclose(got_h, ref_h, rtol=0, atol=AGREE_TOL * np.abs(ref_h).max())
        if assembly == P.CHOL_ASSEMBLY_OWNER:
            assert np.array_equal(got_h, ref_h)  # same deterministic launch sequence


def test_noalloc_rejects_oversized_request(torch):
    ctx = P.Context()
    A, perm = inputs.workload("lap2d_320")  # n = 102,400: 32 columns need > 32 MiB
    sym = P.Symbolic(ctx, A, perm)
    num = P.Factor(ctx, sym, A.vals)
    assert 2 * A.n * 32 * 8 > P.chol_noalloc_scratch_bytes()
    Bd = torch.ones((32, A.n), dtype=torch.float64, device="cuda")
    Xd = torch.zeros_like(Bd)
    with pytest.raises(P.CholError) as e:
        P.chol_solve_noalloc(ctx.handle, num.handle, Bd, Xd)
    assert e.value.status == P.CHOL_E_SCRATCH
    # a single right-hand side of the same system fits and is solved
    b = A.to_scipy_full() @ inputs.rhs_block(7, A.n, 1)[:, 0]
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    P.chol_solve_noalloc(ctx.handle, num.handle, bd, xd)
    torch.cuda.synchronize()
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, xd.cpu().numpy()) <= RESID_TOL


def _solve_both(torch, ctx, num, A, k, seed):
    """(chol_solve result, chol_solve_noalloc result, B) for k right-hand sides."""
    Bm = np.asfortranarray(A.to_scipy_full() @ inputs.rhs_block(seed, A.n, k))
    Bd = torch.from_numpy(np.ascontiguousarray(Bm.T)).cuda()
    got = torch.full_like(Bd, float("nan"))
    P.chol_solve_noalloc(ctx.handle, num.handle, Bd, got)
    ref = torch.empty_like(Bd)
    num.solve(Bd, ref)
    torch.cuda.synchronize()
    return ref.cpu().numpy().T, got.cpu().numpy().T, Bm


def test_noalloc_first_solve_of_fresh_factor_allocates_nothing(torch):
    """40 right-hand sides (a pass of 32, then one of 8, through the same array) on a factor
    that has never been solved: the device's free memory is the same before and after the
    call.  A warm-up call on another factor first loads the solve kernels and the array (the
    CUDA runtime loads module code and device variables on first use), which is memory the
    runtime takes once per process, not per call."""
    ctx = P.Context()
    W, wperm = inputs.workload("lap2d_40")
    wsym = P.Symbolic(ctx, W, wperm)
    warm = P.Factor(ctx, wsym, W.vals)
    _solve_both(torch, ctx, warm, W, 40, 60)
    A, perm = inputs.workload("lap2d_150")  # n = 22,500: 32 columns need ~12 MB of the array
    sym = P.Symbolic(ctx, A, perm)
    num = P.Factor(ctx, sym, A.vals)
    assert num.status()[0] == P.CHOL_OK
    Bm = np.asfortranarray(A.to_scipy_full() @ inputs.rhs_block(61, A.n, 40))
    Bd = torch.from_numpy(np.ascontiguousarray(Bm.T)).cuda()
    got = torch.full_like(Bd, float("nan"))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    P.chol_solve_noalloc(ctx.handle, num.handle, Bd, got)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    got_h = got.cpu().numpy().T
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, Bm, got_h) <= RESID_TOL
    ref_h = num.solve(Bm)
    np.testing.assert_allclose(got_h, ref_h, rtol=0, atol=AGREE_TOL * np.abs(ref_h).max())


def test_noalloc_serves_a_mixed_factor(torch):
    """An FP32 factor of the equilibrated matrix (CHOL_MIXED): its solves compute in FP32 on
    FP64 vectors and scale by the equilibration; with owner-ordered assembly both entry
    points run the same deterministic launch sequence, so they agree bit for bit, twice."""
    ctx = P.Context(assembly=P.CHOL_ASSEMBLY_OWNER)
    A, perm = inputs.workload("diff3d7_12")
    sym = P.Symbolic(ctx, A, perm)
    num = P.Factor(ctx, sym, A.vals, precision=P.CHOL_MIXED)
    assert num.status()[0] == P.CHOL_OK
    for call, k in enumerate((1, 4)):
        ref_h, got_h, Bm = _solve_both(torch, ctx, num, A, k, 70 + call)
        assert np.all(np.isfinite(got_h))
        assert np.array_equal(got_h, ref_h)
        # an FP32 factor's direct solve is accurate to FP32 level (refinement does the rest)
        assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, Bm, got_h) <= 1e-5
