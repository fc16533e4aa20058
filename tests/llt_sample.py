"""Entry-level check of a supernodal factor at sizes the oracle cannot factor: rows of L are
read from the raw supernode panels (layout of chol_factor_panels) and entries of L L^T at
sampled (i, j) are compared with B = P^T A P.  Shared by the full-size GPU tests; the panel
values come in through a gather function, so the logic also runs on the CPU against panels
built from the oracle's factor."""
import numpy as np


def panel_layout(start, rowptr):
    """Per supernode: width w, rows m and the offset of its panel in the panel array."""
    w = np.diff(np.asarray(start, dtype=np.int64))
    m = np.diff(np.asarray(rowptr, dtype=np.int64))
    valptr = np.concatenate([[0], np.cumsum(m * w)])
    return w, m, valptr


def rows_of_l(want, start, rowptr, rows, gather):
    """{i: (k, L_ik)} for every row i in `want`: the columns k <= i of the panels whose row
    lists hold i, and their values.  gather(idx) returns the panel entries at int64 offsets."""
    start = np.asarray(start, dtype=np.int64)
    rowptr = np.asarray(rowptr, dtype=np.int64)
    w, m, valptr = panel_layout(start, rowptr)
    want = np.unique(np.asarray(want, dtype=np.int64))
    pos = np.nonzero(np.isin(rows, want))[0]
    s = np.searchsorted(rowptr, pos, side="right") - 1
    r = pos - rowptr[s]                       # position of the row inside panel s
    i = rows[pos].astype(np.int64)
    ncols = np.where(r < w[s], r + 1, w[s])   # a row inside the diagonal block: k <= i only
    rep = np.repeat(np.arange(pos.size), ncols)
    c = np.arange(int(ncols.sum())) - np.repeat(np.cumsum(ncols) - ncols, ncols)
    idx = valptr[s][rep] + c * m[s][rep] + r[rep]
    vals = np.asarray(gather(idx))
    k = start[s][rep] + c
    row = i[rep]
    order = np.lexsort((k, row))
    row, k, vals = row[order], k[order], vals[order]
    cut = np.searchsorted(row, want)
    cut_end = np.searchsorted(row, want, side="right")
    return {int(q): (k[a:b], vals[a:b]) for q, a, b in zip(want, cut, cut_end)}


def llt_entry(Li, Lj, j):
    """(L L^T)_ij = sum_{k <= j} L_ik L_jk from two rows of L given as (k, value)."""
    ki, vi = Li
    kj, vj = Lj
    sel = kj <= j
    common, a, b = np.intersect1d(ki, kj[sel], assume_unique=True, return_indices=True)
    return float(np.dot(vi[a], vj[sel][b]))


def b_entry(bp, bi, bx, i, j):
    """B_ij (i >= j) from the lower CSC of B; 0 outside its pattern."""
    a, b = bp[j], bp[j + 1]
    q = a + np.searchsorted(bi[a:b], i)
    return float(bx[q]) if q < b and bi[q] == i else 0.0


def sample_pairs(js, bp, bi, start, rowptr, rows, col2sn, per_col, fill_per_col, seed):
    """(i, j) pairs: for each sampled column j, up to per_col rows of B's column j (the
    diagonal included) and up to fill_per_col rows of j's panel outside B's pattern (fill,
    where L L^T must cancel to 0)."""
    rng = np.random.default_rng(seed)
    pairs = []
    for j in js:
        j = int(j)
        bro = bi[bp[j]:bp[j + 1]]
        pick = bro if bro.size <= per_col else np.concatenate(
            [[j], rng.choice(bro[1:], per_col - 1, replace=False)])
        pairs += [(int(i), j) for i in pick]
        s = col2sn[j]
        prow = rows[rowptr[s]:rowptr[s + 1]]
        fill = np.setdiff1d(prow[prow > j], bro)
        if fill.size:
            pairs += [(int(i), j) for i in rng.choice(fill, min(fill_per_col, fill.size),
                                                      replace=False)]
    return pairs


def max_llt_error(pairs, Lrows, bp, bi, bx):
    """max over the pairs of |(L L^T)_ij - B_ij| / sqrt(B_ii B_jj)."""
    worst = 0.0
    for i, j in pairs:
        got = llt_entry(Lrows[i], Lrows[j], j)
        want = b_entry(bp, bi, bx, i, j)
        scale = np.sqrt(b_entry(bp, bi, bx, i, i) * b_entry(bp, bi, bx, j, j))
        worst = max(worst, abs(got - want) / scale)
    return worst
