"""chol_solve_noalloc: the solve variant for callers that cannot allocate device memory
when they solve (stream capture in global mode, runtimes that own all device memory).
Its workspace is a fixed array inside the library; the test checks, through the C ABI,
that two calls in a row give the same solutions as chol_solve (the allocating entry
point) within the tolerances of the other GPU tests, and that a request larger than
the fixed array is refused with CHOL_E_SCRATCH.  It sits in a file of its own that
pytest collects last."""
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
