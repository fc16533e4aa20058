"""Generators: sizes from the closed forms, SPD-ness, the ordering is a permutation
with the separator structure the nested-dissection rule states."""
import numpy as np
import pytest

from paper_2202_09288_gb300 import inputs


def test_splitmix64_reference_value():
    # SplitMix64 with state 0: first output after one increment (published sequence
    # of the Steele-Lea-Flood generator seeded with 0)
    z = inputs._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    u = inputs.uniform(1, 2, 1000)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert np.array_equal(inputs.uniform(1, 2, 10, offset=5), inputs.uniform(1, 2, 15)[5:])


@pytest.mark.parametrize("k", [1, 2, 5, 64])
def test_2d_5pt_counts(k):
    a = inputs.laplacian_2d_5pt(k)
    assert a.nnz_full == 5 * k * k - 4 * k


@pytest.mark.parametrize("k", [1, 3, 6])
def test_3d_7pt_counts(k):
    a = inputs.diffusion_3d_7pt(k, 3)
    assert a.nnz_full == 7 * k ** 3 - 6 * k * k


@pytest.mark.parametrize("k", [2, 4, 5])
def test_27pt_counts_and_dominance(k):
    a = inputs.stencil27_3dof(k, 2)
    assert a.n == 3 * k ** 3
    assert a.nnz_full == 9 * (3 * k - 2) ** 3
    d = a.to_dense()
    assert np.array_equal(d, d.T)
    off = np.abs(d).sum(1) - np.abs(np.diag(d))
    assert np.all(np.diag(d) > off)


def test_diffusion_is_spd_and_lognormal():
    a = inputs.diffusion_3d_7pt(5, 3, sigma=1.5)
    d = a.to_dense()
    assert np.linalg.eigvalsh(d).min() > 0
    z = inputs.normal(3, 1, 20000)
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1) < 0.03


@pytest.mark.parametrize("grid,dofs", [((8, 8, 1), 1), ((7, 5, 1), 1), ((6, 6, 6), 3),
                                       ((9, 4, 3), 1)])
def test_nd_is_permutation(grid, dofs):
    p = inputs.nested_dissection(grid, dofs, leaf=4)
    n = grid[0] * grid[1] * grid[2] * dofs
    assert np.array_equal(np.sort(p), np.arange(n))


def test_nd_root_separator_2d():
    k = 8
    p = inputs.nested_dissection((k, k, 1), 1, leaf=4)
    # the root cut is perpendicular to x (tie between x and y goes to x) at x = 4;
    # its k nodes are numbered last, in natural order
    last = p[-k:]
    assert np.array_equal(last % k, np.full(k, 4))
    assert np.array_equal(last // k, np.arange(k))
    # the lower half (x < 4) is numbered before the upper half (x > 4)
    first = p[:4 * k]
    assert np.all(first % k < 4)


def test_nd_dofs_consecutive():
    p = inputs.nested_dissection((4, 4, 4), 3, leaf=8)
    assert np.array_equal(p[1::3] - p[0::3], np.ones(64, np.int32))
    assert np.all(p[0::3] % 3 == 0)


def test_floating_diffusion_is_spd_and_ill_conditioned():
    """Rows of the floating operator sum to delta times the diagonal over (1 + delta); the
    off-diagonal entries are those of the Dirichlet operator; after diagonal scaling the
    condition number is ~2 / delta (eigenvalues of a small case)."""
    k = 6
    F = inputs.floating_diffusion_3d_7pt(k, 3, 1.5, 1e-6).to_scipy_full().toarray()
    D = inputs.diffusion_3d_7pt(k, 3, 1.5).to_scipy_full().toarray()
    off = ~np.eye(F.shape[0], dtype=bool)
    assert np.array_equal(F[off], D[off])
    d = np.diag(F)
    np.testing.assert_allclose(F.sum(axis=1), d * 1e-6 / (1 + 1e-6), rtol=1e-6, atol=1e-12)
    s = 1 / np.sqrt(d)
    ev = np.linalg.eigvalsh(F * s[:, None] * s[None, :])
    assert ev[0] > 0
    assert 0.5 * 2e6 < ev[-1] / ev[0] < 2 * 2e6
