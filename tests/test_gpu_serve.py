"""GPU tests of the request server (continuous batching under an HBM budget): every
request is answered to its residual target, results do not depend on what else was in
flight (owner-ordered assembly: bitwise), admission respects the budget, and a request
larger than the budget fails cleanly while the server keeps serving."""
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


def shifted(A, sigma):
    """A + sigma diag(A): a new numeric matrix on the same pattern."""
    vals = A.vals.copy()
    vals[A.colptr[:-1]] *= 1.0 + sigma
    return inputs.SpdMatrix(A.n, A.colptr, A.rowind, vals, A.grid, A.dofs)


def request_mix(count, seed):
    u = (inputs.uniform(seed, 11, 4 * count) + 1.0) / 2.0
    out = []
    for r in range(count):
        if u[4 * r] < 0.5:
            A, perm = inputs.workload(f"lap2d_{int(10 + 30 * u[4 * r + 1])}")
        else:
            A, perm = inputs.workload(f"diff3d7_{int(5 + 9 * u[4 * r + 1])}")
        A = shifted(A, u[4 * r + 2])
        nrhs = 1 + int(8 * u[4 * r + 3]) % 8
        B = A.to_scipy_full() @ inputs.rhs_block(seed + r, A.n, nrhs)
        out.append((A, perm, np.asfortranarray(B)))
    return out


def test_served_requests_meet_tolerance(torch):
    reqs = request_mix(40, 1)
    srv = P.Server(slots=2, max_batch=8)
    tickets = []
    for i, (A, perm, B) in enumerate(reqs):
        prec = P.CHOL_MIXED if i % 2 else P.CHOL_FP64
        tickets.append(srv.submit(A, perm, B, precision=prec, tol=1e-12))
    for t, (A, perm, B) in zip(tickets, reqs):
        X, res = srv.wait(t)
        assert res["status"] == P.CHOL_OK, res
        assert res["residual"] <= 1e-12
        assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, B, X) <= 1e-12
        assert res["t_submit"] <= res["t_start"] <= res["t_done"]
        assert 1 <= res["batch_size"] <= 8
    srv.close()


def test_poll_reports_once(torch):
    (A, perm, B), = request_mix(1, 5)
    srv = P.Server(slots=1, max_batch=1)
    t = srv.submit(A, perm, B)
    got = None
    while got is None:
        got = srv.poll(t)
    X, res = got
    assert res["status"] == P.CHOL_OK
    with pytest.raises(P.CholError):
        srv.poll(t)  # a ticket is reported once
    srv.close()


def test_alone_and_in_the_mix_are_bitwise_equal(torch):
    reqs = request_mix(12, 2)
    alone = P.Server(slots=1, max_batch=1, assembly=P.CHOL_ASSEMBLY_OWNER)
    ref = [alone.wait(alone.submit(A, perm, B, precision=P.CHOL_MIXED)) for A, perm, B in reqs]
    alone.close()
    mix = P.Server(slots=2, max_batch=6, assembly=P.CHOL_ASSEMBLY_OWNER)
    tickets = [mix.submit(A, perm, B, precision=P.CHOL_MIXED) for A, perm, B in reqs]
    results = [mix.wait(t) for t in tickets]
    mix.close()
    assert max(res["batch_size"] for _, res in results) > 1  # groups really were shared
    for (X_mix, res_mix), (X_alone, res_alone) in zip(results, ref):
        assert res_alone["batch_size"] == 1
        assert np.array_equal(X_mix, X_alone)
        assert res_mix["iterations"] == res_alone["iterations"]


def test_admission_under_a_small_budget(torch):
    reqs = request_mix(10, 3)
    # room for about one of the larger requests at a time
    srv = P.Server(slots=2, max_batch=8, hbm_budget=96 << 20)
    tickets = [srv.submit(A, perm, B) for A, perm, B in reqs]
    big = inputs.laplacian_2d_5pt(700)  # needs far more than the budget
    bp = inputs.nested_dissection(big.grid)
    t_big = srv.submit(big, bp, np.ones((big.n, 1)))
    for t, (A, perm, B) in zip(tickets, reqs):
        X, res = srv.wait(t)
        assert res["status"] == P.CHOL_OK
        assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, B, X) <= 1e-12
    X, res = srv.wait(t_big)
    assert res["status"] == P.CHOL_E_OOM
    # the server still serves after the refusal
    A, perm, B = reqs[0]
    X, res = srv.wait(srv.submit(A, perm, B))
    assert res["status"] == P.CHOL_OK
    srv.close()


def test_request_arriving_mid_group_is_admitted_at_once(torch):
    """Continuous batching: a small request submitted while a long group occupies one slot
    is admitted by the other slot at once -- it starts after the long group started and
    finishes before that group ends -- and its solution is bit for bit the one it gets
    when served alone (owner-ordered assembly)."""
    import time

    L, lperm = inputs.workload("st27x3_40")
    LB = np.asfortranarray(L.to_scipy_full() @ inputs.rhs_block(21, L.n, 32))
    S, sperm = inputs.workload("lap2d_24")
    SB = np.asfortranarray(S.to_scipy_full() @ inputs.rhs_block(22, S.n, 2))
    srv = P.Server(slots=2, max_batch=4, assembly=P.CHOL_ASSEMBLY_OWNER)
    srv.wait(srv.submit(L, lperm, LB))          # analysis of the long pattern cached
    srv.wait(srv.submit(S, sperm, SB))          # and of the small one
    t_long = srv.submit(L, lperm, LB)
    time.sleep(0.03)                            # the long group is on the GPU by now
    t_short = srv.submit(S, sperm, SB)
    Xs, rs = srv.wait(t_short)
    Xl, rl = srv.wait(t_long)
    srv.close()
    assert rs["status"] == P.CHOL_OK and rl["status"] == P.CHOL_OK
    assert rl["batch_size"] == 1 and rs["batch_size"] == 1
    assert rl["t_start"] < rs["t_start"] < rl["t_done"], (rl, rs)
    assert rs["t_done"] < rl["t_done"], (rl, rs)
    assert oracle.residual(S.n, S.colptr, S.rowind, S.vals, SB, Xs) <= 1e-12
    assert oracle.residual(L.n, L.colptr, L.rowind, L.vals, LB, Xl) <= 1e-12
    alone = P.Server(slots=1, max_batch=1, assembly=P.CHOL_ASSEMBLY_OWNER)
    Xa, ra = alone.wait(alone.submit(S, sperm, SB))
    alone.close()
    assert np.array_equal(Xs, Xa)


def test_group_refinement_with_a_stalling_member_and_many_rhs(torch):
    """A group's requests refine together (one synchronization per iteration for the group).
    One member's FP32 factor cannot reach the tolerance (floating diffusion, condition ~1e10:
    its refinement stalls and falls back to the FP64 factor), one has 40 right-hand sides
    (more than one pass), the others are ordinary: every result meets its tolerance and
    equals, bit for bit, the same request served alone (owner-ordered assembly)."""
    reqs = request_mix(4, 7)
    F, fperm = inputs.workload("floatdiff_16")
    reqs.append((F, fperm, np.asfortranarray(F.to_scipy_full() @ inputs.rhs_block(91, F.n, 2))))
    A40, p40 = inputs.workload("lap2d_20")
    reqs.append((A40, p40, np.asfortranarray(A40.to_scipy_full() @ inputs.rhs_block(92, A40.n, 40))))
    alone = P.Server(slots=1, max_batch=1, assembly=P.CHOL_ASSEMBLY_OWNER)
    ref = [alone.wait(alone.submit(A, perm, B, precision=P.CHOL_MIXED)) for A, perm, B in reqs]
    alone.close()
    mix = P.Server(slots=1, max_batch=8, assembly=P.CHOL_ASSEMBLY_OWNER)
    tickets = [mix.submit(A, perm, B, precision=P.CHOL_MIXED) for A, perm, B in reqs]
    got = [mix.wait(t) for t in tickets]
    mix.close()
    assert max(r["batch_size"] for _, r in got) > 1
    for (A, perm, B), (X0, r0), (X, r) in zip(reqs, ref, got):
        assert r["status"] == P.CHOL_OK and r0["status"] == P.CHOL_OK, (r, r0)
        assert r["residual"] <= 1e-12
        assert oracle.residual(A.n, A.colptr, A.rowind, A.vals, B, X) <= 1e-12
        assert np.array_equal(X, X0)
    assert got[-2][1]["fell_back"] and ref[-2][1]["fell_back"]
    assert not got[0][1]["fell_back"]
