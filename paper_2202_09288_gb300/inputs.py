"""Seeded synthetic SPD inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the factorization: it only builds matrices, right-hand
sides and grid orderings.  The matrices stand in for the SuiteSparse SPD collections the
paper evaluates on (Sec. 5, Tables 1-4: structural, 2D/3D and thermal problems), which are
not available here: 2D/3D stencils with 1 or 3 unknowns per grid node.

Conventions
-----------
* A matrix is returned as the LOWER triangle (diagonal included) in CSC form:
  ``colptr`` int64[n+1], ``rowind`` int32[nnz], ``vals`` float64[nnz]; rows sorted
  ascending inside each column.  The full matrix is A = L_A + L_A^T - diag.
* A permutation ``perm`` is int32[n] with ``perm[new] = old``: the permuted matrix is
  B = P^T A P with B[i, j] = A[perm[i], perm[j]].
* Random numbers come from SplitMix64 (Steele, Lea, Flood 2014): state advances by the
  golden-ratio increment 0x9E3779B97F4A7C15 and each output is the finaliser
  z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB; z ^= z>>31.
  A stream is keyed by (seed, stream id); draw i of a stream is the finaliser applied to
  key + (i+1) * increment, so any draw can be made independently of the others.
  Uniform u in [-1, 1) = ((x >> 11) * 2^-53) * 2 - 1; normals by Box-Muller in float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = _mix(np.array([np.uint64(seed) ^ (np.uint64(stream) * _M2)], dtype=np.uint64))[0]
    return k


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of SplitMix64 stream (seed, stream) as uint64."""
    key = _stream_key(seed, stream)
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + idx * _GOLDEN)


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform float64 in [-1, 1)."""
    x = splitmix64(seed, stream, count, offset)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller from pairs of draws u1, u2 in (0, 1]."""
    m = (count + 1) // 2
    x = splitmix64(seed, stream, 2 * m)
    u = ((x >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


@dataclass
class SpdMatrix:
    """Lower-triangular CSC of an SPD matrix plus the grid it came from (if any)."""

    n: int
    colptr: np.ndarray  # int64[n+1]
    rowind: np.ndarray  # int32[nnz]
    vals: np.ndarray  # float64[nnz]
    grid: tuple = ()  # (kx, ky, kz) nodes per axis; () for non-grid matrices
    dofs: int = 1
    name: str = ""

    @property
    def nnz_lower(self) -> int:
        return int(self.colptr[-1])

    @property
    def nnz_full(self) -> int:
        return 2 * self.nnz_lower - self.n

    def to_scipy_full(self):
        """Full symmetric scipy.sparse CSC matrix (for computing b = A x in tests)."""
        import scipy.sparse as sp

        low = sp.csc_matrix((self.vals, self.rowind, self.colptr), shape=(self.n, self.n))
        return (low + low.T - sp.diags(low.diagonal())).tocsc()

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        for j in range(self.n):
            lo, hi = self.colptr[j], self.colptr[j + 1]
            a[self.rowind[lo:hi], j] = self.vals[lo:hi]
        return a + np.tril(a, -1).T


def _from_slots(rows: np.ndarray, vals: np.ndarray, valid: np.ndarray, n: int):
    """Compress a dense (column, slot) table whose slots are already row-sorted."""
    counts = valid.sum(axis=1)
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=colptr[1:])
    return colptr, rows[valid].astype(np.int32), vals[valid].astype(np.float64)


def from_dense(a: np.ndarray, name: str = "dense") -> SpdMatrix:
    """Lower CSC of the structurally nonzero entries of a dense symmetric matrix."""
    n = a.shape[0]
    colptr = [0]
    rows, vals = [], []
    for j in range(n):
        idx = np.nonzero(a[j:, j])[0] + j
        if a[j, j] == 0.0 and (idx.size == 0 or idx[0] != j):
            idx = np.concatenate([[j], idx])
        rows.append(idx)
        vals.append(a[idx, j])
        colptr.append(colptr[-1] + idx.size)
    return SpdMatrix(n, np.asarray(colptr, dtype=np.int64),
                     np.concatenate(rows).astype(np.int32),
                     np.concatenate(vals).astype(np.float64), name=name)


def laplacian_1d(n: int) -> SpdMatrix:
    """tridiag(-1, 2, -1): the 1D Dirichlet Laplacian."""
    rows = np.stack([np.arange(n), np.arange(1, n + 1)], axis=1)
    vals = np.tile(np.array([2.0, -1.0]), (n, 1))
    valid = rows < n
    colptr, ri, v = _from_slots(rows, vals, valid, n)
    return SpdMatrix(n, colptr, ri, v, grid=(n, 1, 1), name=f"lap1d_{n}")


def laplacian_2d_5pt(k: int) -> SpdMatrix:
    """2D 5-point Laplacian on a k x k grid: diagonal 4, neighbours -1, Dirichlet
    (neighbours outside the grid are absent).  Node p = x + k*y."""
    n = k * k
    p = np.arange(n)
    x, y = p % k, p // k
    rows = np.stack([p, p + 1, p + k], axis=1)
    vals = np.tile(np.array([4.0, -1.0, -1.0]), (n, 1))
    valid = np.stack([np.ones(n, bool), x < k - 1, y < k - 1], axis=1)
    colptr, ri, v = _from_slots(rows, vals, valid, n)
    return SpdMatrix(n, colptr, ri, v, grid=(k, k, 1), name=f"lap2d5_{k}")


def laplacian_3d_7pt(k: int) -> SpdMatrix:
    """3D 7-point Laplacian on k^3: diagonal 6, neighbours -1, Dirichlet."""
    return diffusion_3d_7pt(k, seed=0, sigma=0.0)


def diffusion_3d_7pt(k: int, seed: int, sigma: float = 1.5) -> SpdMatrix:
    """3D 7-point variable-coefficient diffusion on k^3 nodes.

    Cell (= node) coefficient kappa_p = exp(sigma * z_p) with z_p standard normal
    (stream 1).  Face coefficient = harmonic mean 2 kp kq / (kp + kq); A_pq = -face;
    A_pp = sum of its faces + kappa_p for every face on the Dirichlet boundary.
    sigma = 0 gives the constant-coefficient 7-point Laplacian (diagonal 6).
    """
    n = k ** 3
    kap = np.exp(sigma * normal(seed, 1, n)) if sigma != 0.0 else np.ones(n)
    p = np.arange(n)
    x, y, z = p % k, (p // k) % k, p // (k * k)
    diag = np.zeros(n)
    offs = [(1, x < k - 1), (k, y < k - 1), (k * k, z < k - 1)]
    lower_vals = []
    for off, ok in offs:
        q = np.where(ok, p + off, p)
        face = 2.0 * kap * kap[q] / (kap + kap[q])
        face = np.where(ok, face, 0.0)
        lower_vals.append(-face)
        diag += face
        diag[q[ok]] += face[ok]
    # Dirichlet boundary faces: 6 - (number of interior neighbours)
    nb = ((x > 0).astype(int) + (x < k - 1) + (y > 0) + (y < k - 1) + (z > 0) + (z < k - 1))
    diag += (6 - nb) * kap
    rows = np.stack([p, p + 1, p + k, p + k * k], axis=1)
    vals = np.stack([diag] + lower_vals, axis=1)
    valid = np.stack([np.ones(n, bool)] + [ok for _, ok in offs], axis=1)
    colptr, ri, v = _from_slots(rows, vals, valid, n)
    return SpdMatrix(n, colptr, ri, v, grid=(k, k, k), name=f"diff3d7_{k}_s{sigma}")


def floating_diffusion_3d_7pt(k: int, seed: int, sigma: float = 1.5,
                              delta: float = 1e-10) -> SpdMatrix:
    """The diffusion operator of diffusion_3d_7pt without its boundary terms (a floating,
    Neumann body: every row sums to zero), plus delta times its diagonal.  SPD; its smallest
    eigenvalue is ~delta relative to the largest, also after diagonal scaling, so the
    condition number of diag(A)^-1/2 A diag(A)^-1/2 is ~2 / delta."""
    a = diffusion_3d_7pt(k, seed, sigma)
    vals = a.vals.copy()
    first = a.colptr[:-1]
    off = np.ones(vals.size, bool)
    off[first] = False
    cols = np.repeat(np.arange(a.n), np.diff(a.colptr))
    # sum of the faces of every node: -(off-diagonal row sum of the full symmetric matrix)
    faces = np.zeros(a.n)
    np.add.at(faces, cols[off], -vals[off])
    np.add.at(faces, a.rowind[off], -vals[off])
    vals[first] = faces * (1.0 + delta)
    return SpdMatrix(a.n, a.colptr, a.rowind, vals, grid=a.grid,
                     name=f"floatdiff_{k}_s{sigma}_d{delta:g}")


def _offsets27_forward():
    """The 13 neighbour offsets (dx, dy, dz) that point to a larger node index."""
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz > 0 or (dz == 0 and dy > 0) or (dz == 0 and dy == 0 and dx > 0):
                    out.append((dx, dy, dz))
    return out


def stencil27_3dof(k: int, seed: int) -> SpdMatrix:
    """3D 27-point stencil on k^3 nodes with 3 unknowns per node (elasticity-like).

    For every neighbour pair p < q a 3x3 block B_pq with entries U[-1, 1) (stream 2);
    A[q-block, p-block] = B_pq^T (so A[p, q] = B_pq).  The diagonal block of node p is
    sym(R_p) + delta_p I, R_p entries U[-1,1) (stream 3), with
    delta_p = sum over neighbours q of ||A_pq||_inf + ||sym(R_p)||_inf + 1,
    ||.||_inf the max absolute row sum of the block as it sits in p's block row.  Every
    row is then strictly diagonally dominant with a positive diagonal, so A is SPD.
    Unknown 3p + a belongs to node p.
    """
    N = k ** 3
    n = 3 * N
    p = np.arange(N)
    x, y, z = p % k, (p // k) % k, p // (k * k)
    offs = _offsets27_forward()
    offs.sort(key=lambda o: o[0] + k * o[1] + k * k * o[2])  # row order inside a column
    nb_valid, nb_q, blocks = [], [], []
    rowsum_in = np.zeros(N)  # sum_q ||A_pq||_inf over the blocks in p's block row
    for oi, (dx, dy, dz) in enumerate(offs):
        ok = ((x + dx >= 0) & (x + dx < k) & (y + dy >= 0) & (y + dy < k)
              & (z + dz >= 0) & (z + dz < k))
        q = np.where(ok, p + dx + k * dy + k * k * dz, p)
        b = uniform(seed, 2, 9 * N, offset=9 * N * oi).reshape(N, 3, 3)  # B_pq[a, c]
        b = np.where(ok[:, None, None], b, 0.0)
        # block in p's row is B_pq (rows a); block in q's row is B_pq^T (rows c)
        rowsum_in += np.abs(b).sum(axis=2).max(axis=1)
        np.add.at(rowsum_in, q[ok], np.abs(b[ok]).sum(axis=1).max(axis=1))
        nb_valid.append(ok)
        nb_q.append(q)
        blocks.append(b)
    r = uniform(seed, 3, 9 * N).reshape(N, 3, 3)
    s = 0.5 * (r + r.transpose(0, 2, 1))
    delta = rowsum_in + np.abs(s).sum(axis=2).max(axis=1) + 1.0
    dblk = s + delta[:, None, None] * np.eye(3)[None]
    # slots per column j = 3p + a: diag block rows 3p+c (c >= a), then each forward
    # neighbour q (in increasing q order) rows 3q+c, value A[3q+c, 3p+a] = B_pq[a, c]
    nslot = 3 + 3 * len(offs)
    rows = np.zeros((N, 3, nslot), dtype=np.int64)
    vals = np.zeros((N, 3, nslot))
    valid = np.zeros((N, 3, nslot), dtype=bool)
    for a in range(3):
        for c in range(3):
            rows[:, a, c] = 3 * p + c
            vals[:, a, c] = dblk[:, c, a]
            valid[:, a, c] = c >= a
        for oi in range(len(offs)):
            for c in range(3):
                sl = 3 + 3 * oi + c
                rows[:, a, sl] = 3 * nb_q[oi] + c
                vals[:, a, sl] = blocks[oi][:, a, c]
                valid[:, a, sl] = nb_valid[oi]
    colptr, ri, v = _from_slots(rows.reshape(n, nslot), vals.reshape(n, nslot),
                                valid.reshape(n, nslot), n)
    return SpdMatrix(n, colptr, ri, v, grid=(k, k, k), dofs=3, name=f"st27x3_{k}")


def random_spd_dense(n: int, seed: int) -> SpdMatrix:
    """Dense SPD B B^T + n I with B entries U[-1, 1) (stream 4)."""
    b = uniform(seed, 4, n * n).reshape(n, n)
    return from_dense(b @ b.T + n * np.eye(n), name=f"dense_{n}")


def nested_dissection(grid: tuple, dofs: int = 1, leaf: int = 64) -> np.ndarray:
    """Geometric nested-dissection ordering of a kx x ky x kz grid (perm[new] = old).

    A box with more than ``leaf`` nodes is cut by the grid plane through the middle of
    its longest axis (ties go to the lowest axis, x before y before z) at
    lo + len // 2.  The lower half is numbered first, then the upper half, then the
    separator plane; a box of at most ``leaf`` nodes is numbered in natural order
    (x fastest, then y, then z), as is every separator plane.  The unknowns of a node
    stay consecutive.  A one-plane separator disconnects the two halves for 5-, 7- and
    27-point stencils, whose couplings differ by at most one step per axis.
    The ordering step is not part of the paper's method (CHOLMOD takes it from METIS or
    AMD, Sec. 2); this deterministic stand-in only serves grid inputs.
    """
    kx, ky, kz = (tuple(grid) + (1, 1))[:3]
    pieces = []

    def natural(lo, hi):
        xs = np.arange(lo[0], hi[0])
        ys = np.arange(lo[1], hi[1]) * kx
        zs = np.arange(lo[2], hi[2]) * (kx * ky)
        return (zs[:, None, None] + ys[None, :, None] + xs[None, None, :]).ravel()

    def rec(lo, hi):
        ext = [hi[a] - lo[a] for a in range(3)]
        if min(ext) <= 0:
            return
        if ext[0] * ext[1] * ext[2] <= leaf:
            pieces.append(natural(lo, hi))
            return
        a = int(np.argmax(ext))
        mid = lo[a] + ext[a] // 2
        lo1, hi1 = list(lo), list(hi)
        hi1[a] = mid
        lo2, hi2 = list(lo), list(hi)
        lo2[a] = mid + 1
        los, his = list(lo), list(hi)
        los[a], his[a] = mid, mid + 1
        rec(lo1, hi1)
        rec(lo2, hi2)
        pieces.append(natural(los, his))

    rec([0, 0, 0], [kx, ky, kz])
    node_perm = np.concatenate(pieces).astype(np.int64)
    if dofs == 1:
        return node_perm.astype(np.int32)
    return (dofs * node_perm[:, None] + np.arange(dofs)[None, :]).ravel().astype(np.int32)


def rhs_block(seed: int, n: int, nrhs: int, stream: int = 5) -> np.ndarray:
    """n x nrhs column-major (Fortran-order) block with entries U[-1, 1)."""
    return np.asfortranarray(uniform(seed, stream, n * nrhs).reshape(nrhs, n).T)


# Named workloads: the five configurations this library is measured on.
def workload(name: str) -> tuple[SpdMatrix, np.ndarray]:
    """Matrix and nested-dissection ordering of a named workload.

    lap2d_64      2D 5-point Laplacian, 64 x 64 grid (n = 4,096)
    st27x3_48     3D 27-point, 3 dofs/node, 48^3 grid (n = 331,776), seed 2
    diff3d7_96    3D 7-point log-normal (sigma 1.5) diffusion, 96^3 (n = 884,736), seed 3
    st27x3_80     3D 27-point, 3 dofs/node, 80^3 (n = 1,536,000), seed 5
    Scaled-down members of the same families: ``st27x3_<k>``, ``diff3d7_<k>``,
    ``lap2d_<k>``, ``lap3d_<k>``; ``floatdiff_<k>``: the floating diffusion operator
    (floating_diffusion_3d_7pt, sigma 1.5, delta 1e-10, seed 3), condition ~2e10 after
    diagonal scaling.
    """
    fam, k = name.rsplit("_", 1)
    k = int(k)
    if fam == "lap2d":
        a = laplacian_2d_5pt(k)
    elif fam == "lap3d":
        a = laplacian_3d_7pt(k)
    elif fam == "st27x3":
        a = stencil27_3dof(k, seed={48: 2, 80: 5}.get(k, 2))
    elif fam == "diff3d7":
        a = diffusion_3d_7pt(k, seed=3)
    elif fam == "floatdiff":
        a = floating_diffusion_3d_7pt(k, seed=3)
    else:
        raise ValueError(f"unknown workload {name}")
    return a, nested_dissection(a.grid, a.dofs)
