"""The multi-core CPU baseline of the paper's tasking (Sec. 3 left-looking supernodal
factorization with the Sec. 4 granularity policies) reaches the oracle's L.  CPU only."""
import numpy as np
import pytest

import cpu_tasks
import oracle
import paper_2202_09288_gb300 as P
from paper_2202_09288_gb300 import inputs


@pytest.mark.parametrize("name", ["lap2d_16", "lap3d_9", "st27x3_6", "diff3d7_10"])
@pytest.mark.parametrize("policy", list(cpu_tasks.POLICIES))
@pytest.mark.parametrize("relax", [-1.0, 0.0])
def test_cpu_tasks_match_oracle(name, policy, relax):
    A, perm = inputs.workload(name)
    sym = P.Symbolic(P.make_opts(width_cap=64, relax=relax), A, perm)
    rowptr, rows = P.chol_sym_rows(sym.handle)
    pan = cpu_tasks.factor(A, perm, sym.export()["sn_start"], rowptr, rows, policy, threads=4)
    ref = oracle.cholesky(A, perm)
    got, extra = pan.on_pattern(ref.lp, ref.li)
    scale = np.abs(ref.lx).max()
    assert np.abs(got - ref.lx).max() <= 1e-12 * scale
    assert extra <= 1e-13 * scale  # explicit zeros of relaxed supernodes stay zero
    if policy in ("optd", "optd_cost"):
        assert pan.D >= 0
    else:
        assert pan.D == -1
    if policy == "nonested":
        assert pan.inner_tasks == 0


def test_cpu_tasks_threshold_is_algorithm_1():
    """The D it applies is Algorithm 1 over the number of updates of each supernode."""
    A, perm = inputs.workload("st27x3_8")
    sym = P.Symbolic(P.make_opts(width_cap=64), A, perm)
    start = sym.export()["sn_start"]
    rowptr, rows = P.chol_sym_rows(sym.handle)
    col2sn = np.repeat(np.arange(len(start) - 1), np.diff(start))
    counts = np.zeros(len(start) - 1, dtype=np.int64)
    for s in range(len(start) - 1):
        r = rows[rowptr[s] + (start[s + 1] - start[s]):rowptr[s + 1]]
        t = col2sn[r]
        counts[np.unique(t)] += 1  # one update of each target by s (its rows are sorted)
    pan = cpu_tasks.factor(A, perm, start, rowptr, rows, "optd", threads=2)
    assert pan.D == oracle.opt_d(A.n, counts)


def test_cpu_tasks_not_spd():
    A, perm = inputs.workload("lap2d_16")
    A.vals[A.colptr[5]] = -1.0  # a negative diagonal entry (column 5 stores its diagonal first)
    sym = P.Symbolic(P.make_opts(width_cap=64), A, perm)
    rowptr, rows = P.chol_sym_rows(sym.handle)
    with pytest.raises(RuntimeError):
        cpu_tasks.factor(A, perm, sym.export()["sn_start"], rowptr, rows, "nested", threads=2)
