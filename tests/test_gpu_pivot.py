"""The FP64 POTRF's pivot scaling: column j of a diagonal block is multiplied by
y = p^(-1/2) (p the pivot) computed from an FP32 estimate and a third-order correction,
with the exponent handled by integer arithmetic.  Tested through the C ABI on a block-
diagonal matrix of 2 x 2 blocks [[p, a], [a, q]] (a = 2^k, q = 1 + 2 a^2 / p, SPD): the
first column of each block is its supernode's first pivot, so L21 = a y exactly and
L11 = p y.  Against 1/sqrt(p) and sqrt(p) correctly rounded (Python decimal, 60 digits)
over pivots spanning the whole FP64 exponent range, including subnormals (which take the
library's division and square root)."""
import decimal

import numpy as np
import pytest

import paper_2202_09288_gb300 as P
from paper_2202_09288_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def pivots():
    m = 1.0 + (inputs.uniform(31, 1, 2100) + 1.0) / 2.0  # mantissas in [1, 2)
    e = np.arange(-1021, 1021, dtype=np.int64)
    p = np.ldexp(m[: e.size], e)
    sub = np.ldexp(m[-20:], np.arange(-1070, -1050))      # subnormal pivots
    return np.concatenate([p, sub, [1.0, 2.0, 4.0, 0.25]])


def exact(x, f):
    decimal.getcontext().prec = 60
    return float(f(decimal.Decimal(float(x))))


def ulps(a, b):
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_pivot_rsqrt_within_two_ulps(torch):
    p = pivots()
    k = np.round(np.log2(p) / 2.0).astype(np.int64)
    a = np.ldexp(1.0, k)                      # exact powers of two
    q = 1.0 + 2.0 * (a * a / p)               # a^2 / p in [0.5, 2]: SPD, no overflow
    nb = p.size
    n = 2 * nb
    rows, vals, cp = [], [], [0]
    for b in range(nb):
        rows += [2 * b, 2 * b + 1]
        vals += [p[b], a[b]]
        cp.append(len(rows))
        rows += [2 * b + 1]
        vals += [q[b]]
        cp.append(len(rows))
    A = inputs.SpdMatrix(n, np.array(cp, np.int64), np.array(rows, np.int32),
                         np.array(vals, np.float64), (), 1)
    ctx = P.Context()
    sym = P.Symbolic(ctx, A, np.arange(n, dtype=np.int32))
    num = P.Factor(ctx, sym, A.vals)
    assert num.status()[0] == P.CHOL_OK
    lp, li, lx = num.export()
    first = lp[0:n:2]                          # column 2b: entries L11 (row 2b), L21 (row 2b+1)
    assert np.all(li[first] == 2 * np.arange(nb)) and np.all(li[first + 1] == 2 * np.arange(nb) + 1)
    y = lx[first + 1] / a                      # exact: a is a power of two
    y_ref = np.array([exact(x, lambda d: 1 / d.sqrt()) for x in p])
    s_ref = np.array([exact(x, lambda d: d.sqrt()) for x in p])
    assert ulps(y, y_ref).max() <= 2, (p[np.argmax(ulps(y, y_ref))], ulps(y, y_ref).max())
    assert ulps(lx[first], s_ref).max() <= 3, ulps(lx[first], s_ref).max()
