import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def fig1_tree():
    """The Fig. 1 example (Sec. 3) from tests/golden/fig1_tree.txt: (edges, level sets),
    supernode labels 1-based as printed."""
    edges, levels = [], []
    with open(os.path.join(GOLDEN, "fig1_tree.txt")) as f:
        for line in f:
            parts = line.split()
            if not parts or parts[0].startswith("#"):
                continue
            if parts[0] == "edge":
                edges.append((int(parts[1]), int(parts[2])))
            elif parts[0] == "level":
                levels.append(sorted(int(x) for x in parts[1:]))
    return edges, levels


def fig1_matrix():
    """An SPD matrix whose elimination tree is the Fig. 1 tree (one column per
    supernode): A_ij != 0 for every edge (child i, parent j), diagonally dominant."""
    import numpy as np
    from paper_2202_09288_gb300 import inputs
    edges, _ = fig1_tree()
    n = 1 + max(max(e) for e in edges)
    a = np.eye(n - 1) * 4.0
    for c, p in edges:
        a[c - 1, p - 1] = a[p - 1, c - 1] = -1.0
    return inputs.from_dense(a)


def column_error(lp, lx, ref_lx):
    """max_j ||L[:, j] - L_ref[:, j]||_2 / ||L_ref[:, j]||_2 over the columns of two factors
    stored on the same CSC pattern (lp): the relative-error tolerance applied to every
    column, so that an error confined to small-magnitude entries cannot hide behind the
    norm of the whole factor."""
    import numpy as np
    lp = np.asarray(lp, dtype=np.int64)
    counts = np.diff(lp)
    if counts.size == 0:
        return 0.0
    nz = counts > 0
    starts = lp[:-1][nz]
    d2 = np.add.reduceat((np.asarray(lx) - np.asarray(ref_lx)) ** 2, starts)
    r2 = np.add.reduceat(np.asarray(ref_lx) ** 2, starts)
    return float(np.sqrt(np.max(d2 / np.maximum(r2, np.finfo(float).tiny))))
