"""GMRES-based iterative refinement (chol_refine_gmres): the FP64 residual's correction
equation solved by flexible GMRES preconditioned with the factor.  On a matrix whose
condition number after diagonal scaling is ~2e10 (a floating diffusion operator plus a
1e-10 relative diagonal shift), refinement with the FP32 factor alone stalls (kappa times
FP32's accuracy is far above 1) and falls back to an FP64 factorization, while GMRES-IR with
the same FP32 factor reaches a relative residual of 1e-12 without it.  Residuals are
checked with the oracle's residual; both paths' times are printed for the record."""
import time

import numpy as np
import pytest

import oracle
import paper_2202_09288_gb300 as P
from paper_2202_09288_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_gmres_ir_converges_where_refinement_stalls(torch):
    A, perm = inputs.workload("floatdiff_16")
    ctx = P.Context()
    sym = P.Symbolic(ctx, A, perm)
    b = A.to_scipy_full() @ inputs.rhs_block(3, A.n, 1)[:, 0]
    plain = P.Factor(ctx, sym, A.vals, precision=P.CHOL_MIXED)
    assert plain.status()[0] == P.CHOL_OK
    t0 = time.perf_counter()
    x1, info1 = plain.refine(b, tol=1e-12, check=False)
    t_plain = time.perf_counter() - t0
    assert info1["fell_back"], info1  # refinement with the FP32 factor alone stalled
    gm = P.Factor(ctx, sym, A.vals, precision=P.CHOL_MIXED)
    t0 = time.perf_counter()
    x2, info2 = gm.refine_gmres(b, tol=1e-12)
    t_gmres = time.perf_counter() - t0
    assert not info2["fell_back"], info2
    assert info2["residual"] <= 1e-12
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, x2) <= 1e-12
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, x1) <= 1e-12
    print(f"\nfloatdiff_16: refinement {info1['iterations']} steps + FP64 fallback "
          f"{1e3 * t_plain:.1f} ms; GMRES-IR {info2['iterations']} GMRES iterations "
          f"{1e3 * t_gmres:.1f} ms (FP32 factor only)")


@pytest.mark.parametrize("precision", [P.CHOL_FP64, P.CHOL_MIXED])
def test_gmres_ir_several_rhs_host_and_device(torch, precision):
    A, perm = inputs.workload("diff3d7_14")
    ctx = P.Context()
    sym = P.Symbolic(ctx, A, perm)
    num = P.Factor(ctx, sym, A.vals, precision=precision)
    Bm = np.asfortranarray(A.to_scipy_full() @ inputs.rhs_block(8, A.n, 3))
    X, info = num.refine_gmres(Bm, tol=1e-13, restart=8)
    assert info["residual"] <= 1e-13 and not info["fell_back"]
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, Bm, X) <= 1e-13
    Bd = torch.from_numpy(np.ascontiguousarray(Bm.T)).cuda()
    Xd, info_d = num.refine_gmres(Bd, tol=1e-13, restart=8)
    torch.cuda.synchronize()
    assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, Bm, Xd.cpu().numpy().T) <= 1e-13
    with pytest.raises(P.CholError):
        num.refine_gmres(Bm, restart=65)
