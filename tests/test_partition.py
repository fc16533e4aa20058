"""Subtree-to-device partition of the supernodal elimination tree (chol_partition_tree,
chol_sym_partition): subtrees of different parts never update one another (Sec. 3, Fig. 1:
supernodes are independent unless one is an ancestor of the other), the top part is closed
under parents, and the parts' work is balanced as far as the tree allows."""
import numpy as np
import pytest

import paper_2202_09288_gb300 as P
from paper_2202_09288_gb300 import inputs
from conftest import fig1_tree


def test_fig1_tree_by_hand():
    """The Fig. 1 tree, unit work, two parts, tol 0.  Roots {6}: one subtree for two parts,
    so 6 splits into {4 (work 3), 5 (work 2)}; dealt 3 | 2, not even, so the heavier 4
    splits: {5 (2), 1 (1), 2 (1)} dealt 5 | 1 + 2 = 2 | 2.  Top part {4, 6}."""
    edges, _ = fig1_tree()
    nv = 1 + max(max(e) for e in edges)  # labels 1..6 -> vertices 0..5
    parent = np.full(nv - 1, -1, np.int32)
    for c, p in edges:
        parent[c - 1] = p - 1
    owner, imb = P.chol_partition_tree(parent, np.ones(nv - 1), 2, tol=0.0)
    assert list(owner) == [1, 1, 0, -1, 0, -1]
    assert imb == 1.0


def check_partition(parent, owner, nparts):
    for v, p in enumerate(parent):
        if owner[v] >= 0 and p >= 0:
            assert owner[p] in (owner[v], -1)  # a subtree's parent is in it or on top
        if owner[v] < 0 and p >= 0:
            assert owner[p] < 0                 # the top part is closed under parents
    # children of a top vertex are top or subtree roots; a subtree's vertices share a part
    assert set(np.unique(owner)) <= set(range(-1, nparts))


@pytest.mark.parametrize("name", ["st27x3_8", "lap3d_12", "diff3d7_12", "lap2d_40"])
@pytest.mark.parametrize("nparts", [2, 3, 4])
def test_partition_of_workloads(name, nparts):
    A, perm = inputs.workload(name)
    sym = P.Symbolic(P.make_opts(width_cap=64), A, perm)
    owner, imb, top = P.chol_sym_partition(sym.handle, nparts, tol=0.1)
    ex = sym.export()
    start = ex["sn_start"]
    # the supernodal parent of s: the supernode of the elimination-tree parent of its last column
    cp = ex["parent"]
    col2sn = np.repeat(np.arange(len(start) - 1), np.diff(start))
    last = start[1:] - 1
    sp = np.where(cp[last] >= 0, col2sn[np.maximum(cp[last], 0)], -1).astype(np.int32)
    check_partition(sp, owner, nparts)
    assert all((owner == p).any() for p in range(nparts))
    # the same through the generic tree entry point
    work = np.array([np.sum(ex["colcount"][start[s]:start[s + 1]].astype(float) ** 2)
                     for s in range(len(start) - 1)])
    owner2, imb2 = P.chol_partition_tree(sp, work, nparts, tol=0.1)
    assert np.array_equal(owner, owner2) and imb == imb2
    assert top == pytest.approx(work[owner < 0].sum())
    # balance: within tolerance, unless only single supernodes were left to split
    loads = np.array([work[owner == p].sum() for p in range(nparts)])
    assert imb == pytest.approx(loads.max() / loads.mean())
    assert imb <= 1.1 + 1e-12 or not any(
        (sp == s).any() for s in np.nonzero(owner >= 0)[0] if sp[s] < 0 or owner[sp[s]] < 0)


def test_partition_rejects_bad_forests():
    with pytest.raises(P.CholError):
        P.chol_partition_tree([1, 0], [1.0, 1.0], 2)      # cycle
    with pytest.raises(P.CholError):
        P.chol_partition_tree([5, -1], [1.0, 1.0], 2)     # parent out of range
    with pytest.raises(P.CholError):
        P.chol_partition_tree([-1, 0], [1.0, -1.0], 2)    # negative work
    with pytest.raises(P.CholError):
        P.chol_partition_tree([-1], [1.0], 0)             # no parts
    owner, imb = P.chol_partition_tree([-1, 0, 0], [0.0, 1.0, 1.0], 1)
    assert list(owner) == [0, 0, 0] and imb == 1.0
