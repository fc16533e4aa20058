"""Failure path of the bounded device waits of the tensor-core Schur kernels (the waits on
mbarriers between their load, MMA and consumer roles).  A test hook makes the consumers wait
on a barrier that nothing completes, for 1,000 clock cycles, in place of an accumulator
that never finishes (no fault, trap or endless loop is involved): they give up, the
kernel's other waits then expire in turn (each bounded in time), every role waits for its
own copies and MMAs in flight, the tensor memory is freed, later launches of the
factorization skip their work, and chol_factor_status reports CHOL_E_TIMEOUT within
seconds.  With the default bound restored
the same context, the same factor and a new factor give the oracle's L -- which also shows
the failed launch released its tensor memory (a later launch allocates all of it)."""
import time

import numpy as np
import pytest

import oracle
import paper_2202_09288_gb300 as P
from paper_2202_09288_gb300 import inputs
from conftest import column_error

pytestmark = pytest.mark.gpu

ALL128 = {"min_rows_tile64": 1, "min_rows_tile32": 1, "min_level_tiles64": 0,
          "min_rows_tile128": 1, "min_level_tiles128": 0}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("precision", [P.CHOL_FP64, P.CHOL_MIXED])
def test_accumulator_wait_timeout_is_reported_and_context_recovers(torch, precision):
    A, perm = inputs.workload("st27x3_11")
    ctx = P.Context()
    sym = P.Symbolic(ctx, A, perm)
    P.chol_sym_set_tile_policy(sym.handle, ALL128)
    P.chol_set_device_wait(ctx.handle, 1000)  # consumers give up after 1,000 cycles
    P.chol_profile_enable(ctx.handle, True)
    t0 = time.time()
    num = P.Factor(ctx, sym, A.vals, precision=precision)
    rc = P.lib().chol_factor_status(ctx.handle, num.handle, None)
    elapsed = time.time() - t0
    kind = "schur128_oz" if precision == P.CHOL_FP64 else "schur128_tc"
    assert P.chol_profile_read(ctx.handle)[kind]["launches"] > 0
    assert rc == P.CHOL_E_TIMEOUT, rc
    assert elapsed < 60.0, elapsed
    # default bound again: the same factor, then a new one, on the same context
    P.chol_set_device_wait(ctx.handle, 0)
    num.refactor(A.vals)
    assert num.status()[0] == P.CHOL_OK
    fresh = P.Factor(ctx, sym, A.vals, precision=precision)
    assert fresh.status()[0] == P.CHOL_OK
    b = A.to_scipy_full() @ inputs.rhs_block(9, A.n, 1)[:, 0]
    if precision == P.CHOL_FP64:
        ref = oracle.cholesky(A, perm)
        for f in (num, fresh):
            lp, _, lx = f.export()
            assert column_error(lp, lx, ref.lx) <= 1e-12
            x = f.solve(b)
            assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, b, x) <= 1e-13
    else:
        for f in (num, fresh):
            x, info = f.refine(b, tol=1e-12)
            assert info["residual"] <= 1e-12
    with pytest.raises(P.CholError):
        P.chol_set_device_wait(ctx.handle, -1)
