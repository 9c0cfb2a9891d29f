"""Seeded synthetic inputs: complex symmetric sparse matrices (CSR) and right-hand sides.

This module builds problems only.  It holds none of the solver's arithmetic, so both
the CPU oracle (through the tests) and the CUDA path read the very same arrays.

Problem family (Sec. 1, Eq. 1.1): ``A X = B`` with ``A = A^T != A^H`` sparse n x n and
``B`` n x p.  The paper's own matrices (Matrix Market young*c, dense RCS sets of
Sec. 3, Tables 2-3) are not available, so these Helmholtz-shaped and random complex
symmetric matrices stand in for them.

Conventions (fixed here, used by every caller):

* grid spacing ``h = 1/(N+1)`` on the unit square/cube, homogeneous Dirichlet boundary;
  ``-Delta_h`` has ``2d/h^2`` on the diagonal and ``-1/h^2`` for each grid neighbour;
* node ``(ix, iy[, iz])`` has row index ``ix*N*N + iy*N + iz`` (C order);
* CSR arrays are ``int32 row_ptr[n+1]``, ``int32 col_idx[nnz]`` (sorted within each
  row, both triangles stored) and ``complex128 vals[nnz]``;
* "complex normal" is ``(N(0,1) + i N(0,1)) / sqrt(2)`` from
  ``numpy.random.default_rng(seed)``: the real parts of the whole n x p block are drawn
  first, then the imaginary parts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class CSR:
    """A sparse n x n matrix in CSR form with both triangles stored."""
    n: int
    row_ptr: np.ndarray   # int32 [n+1]
    col_idx: np.ndarray   # int32 [nnz]
    vals: np.ndarray      # complex128 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.vals, self.col_idx, self.row_ptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        return self.to_scipy().toarray()

    def nbytes(self, value_bytes: int = 16) -> int:
        """Bytes of one full read of the matrix: values + column indices + row pointers."""
        return self.nnz * (value_bytes + 4) + 4 * (self.n + 1)


def csr_from_scipy(M) -> CSR:
    M = sp.csr_matrix(M, dtype=np.complex128)
    M.sum_duplicates()
    M.sort_indices()
    return CSR(n=M.shape[0], row_ptr=M.indptr.astype(np.int32), col_idx=M.indices.astype(np.int32),
               vals=M.data.astype(np.complex128))


def _neg_laplacian_1d(N: int) -> sp.csr_matrix:
    h = 1.0 / (N + 1)
    return sp.diags([-np.ones(N - 1), 2.0 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1], format="csr") / h**2


def neg_laplacian(N: int, dim: int) -> sp.csr_matrix:
    """5-point (dim=2) or 7-point (dim=3) finite-difference -Delta_h on an N^dim grid."""
    T = _neg_laplacian_1d(N)
    I = sp.identity(N, format="csr")
    if dim == 2:
        return (sp.kron(T, I) + sp.kron(I, T)).tocsr()
    if dim == 3:
        return (sp.kron(sp.kron(T, I), I) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(I, I), T)).tocsr()
    raise ValueError("dim must be 2 or 3")


def helmholtz_2d(N: int, k: float, damping: float) -> CSR:
    """``A = -Delta_h - k^2 (1 + i*damping) I`` on an N x N grid (complex symmetric)."""
    L = neg_laplacian(N, 2).astype(np.complex128)
    A = L - (k * k) * (1.0 + 1j * damping) * sp.identity(N * N, format="csr")
    return csr_from_scipy(A)


def border_depth(N: int, border: int) -> np.ndarray:
    """Per-axis depth (in cells) into an absorbing border of width ``border``:
    ``border`` at the outermost cell, 1 at the innermost border cell, 0 inside."""
    i = np.arange(N)
    return np.maximum(np.maximum(border - i, i - (N - 1 - border)), 0).astype(np.float64)


def helmholtz_3d_absorbing(N: int, k: float, border: int = 6, sigma_max: float = 1.0) -> CSR:
    """``A = -Delta_h - k^2 (1 + i*sigma(x)) I`` on an N^3 grid.

    ``sigma = sigma_max * (d / border)^2`` with ``d`` the largest per-axis depth into the
    border, so the damping rises quadratically over the last ``border`` cells and is 0 in
    the interior.  A is complex symmetric and not Hermitian.
    """
    d1 = border_depth(N, border)
    d = np.maximum(np.maximum(d1[:, None, None], d1[None, :, None]), d1[None, None, :])
    sigma = sigma_max * (d / border) ** 2
    L = neg_laplacian(N, 3).astype(np.complex128)
    A = L - sp.diags((k * k) * (1.0 + 1j * sigma.ravel()), 0, format="csr")
    return csr_from_scipy(A)


def fibonacci_sphere(m: int) -> np.ndarray:
    """m unit vectors spread over the sphere (Fibonacci lattice), shape (m, 3)."""
    j = np.arange(m, dtype=np.float64)
    z = 1.0 - (2.0 * j + 1.0) / m
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = j * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def plane_waves_3d(N: int, k: float, m: int) -> np.ndarray:
    """``B[:, j] = exp(i k d_j . x)`` at the grid nodes ``x = (i+1) h``; shape (N^3, m)."""
    h = 1.0 / (N + 1)
    x = (np.arange(N, dtype=np.float64) + 1.0) * h
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    dirs = fibonacci_sphere(m)
    return np.ascontiguousarray(np.exp(1j * k * (pts @ dirs.T)))


def complex_normal(n: int, p: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n, p))
    im = rng.standard_normal((n, p))
    return np.ascontiguousarray((re + 1j * im) / math.sqrt(2.0))


def random_complex_symmetric(n: int, nnz_per_row: int, seed: int, diag=4.0 + 0.5j,
                             scale: float = 0.1) -> CSR:
    """Random sparse complex symmetric matrix with a strong complex diagonal.

    Off-diagonal pairs (i, j), i < j, are drawn uniformly; each gets one complex normal
    value times ``scale`` mirrored to (j, i).  With ``diag = 4 + 0.5i`` and small
    ``scale`` the matrix is well conditioned (used for the small pin and parity cases).
    """
    rng = np.random.default_rng(seed)
    m = max(0, (nnz_per_row - 1) * n // 2)
    i = rng.integers(0, n, size=m)
    j = rng.integers(0, n, size=m)
    keep = i != j
    i, j = i[keep], j[keep]
    v = scale * (rng.standard_normal(i.shape[0]) + 1j * rng.standard_normal(i.shape[0])) / math.sqrt(2.0)
    U = sp.coo_matrix((v, (np.minimum(i, j), np.maximum(i, j))), shape=(n, n)).tocsr()
    U.sum_duplicates()
    A = U + U.T + sp.diags(np.full(n, diag, dtype=np.complex128), 0)
    return csr_from_scipy(A)


def random_symmetric_27pt(nx: int, ny: int, nz: int, seed: int, drop: float = 0.1,
                          diag=4.0 + 0.5j, scale: float = 0.1) -> CSR:
    """3D 27-point pattern with a fraction ``drop`` of the off-diagonal pairs removed
    symmetrically; off-diagonal values ``scale * complex normal`` (mirrored), diagonal
    ``diag``.  Pairs are dropped first, then the values are drawn, from one generator."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    idx = np.arange(n).reshape(nx, ny, nz)
    rows, cols = [], []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                # keep each unordered pair once: lexicographically positive offsets
                if (dx, dy, dz) <= (0, 0, 0):
                    continue
                a = idx[max(0, -dx):nx - max(0, dx), max(0, -dy):ny - max(0, dy), max(0, -dz):nz - max(0, dz)]
                b = idx[max(0, dx):nx + min(0, dx), max(0, dy):ny + min(0, dy), max(0, dz):nz + min(0, dz)]
                rows.append(a.ravel())
                cols.append(b.ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    order = np.lexsort((c, r))
    r, c = r[order], c[order]
    keep = rng.random(r.shape[0]) >= drop
    r, c = r[keep], c[keep]
    v = scale * (rng.standard_normal(r.shape[0]) + 1j * rng.standard_normal(r.shape[0])) / math.sqrt(2.0)
    U = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    A = U + U.T + sp.diags(np.full(n, diag, dtype=np.complex128), 0)
    return csr_from_scipy(A)


@dataclass
class Problem:
    name: str
    A: CSR
    B: np.ndarray
    method: str          # "cocg_rq" | "cocr_rq"
    tol: float
    maxit: int
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.n

    @property
    def p(self) -> int:
        return int(self.B.shape[1])


def helmholtz2d_n1024_p4(method: str = "cocr_rq") -> Problem:
    """2D 5-point Helmholtz, 32x32 grid (n=1024), k=6, damping 0.05; B n x 4 complex
    normal (seed 0); X0 = 0; tol 1e-10; maxit 500."""
    return Problem("helmholtz2d_32x32_k6_p4", helmholtz_2d(32, 6.0, 0.05), complex_normal(1024, 4, 0),
                   method, 1e-10, 500)


def helmholtz3d_n262144_p16(method: str = "cocr_rq", maxit: int = 20000) -> Problem:
    """3D 7-point Helmholtz, 64^3 grid (n=262,144), k=20, quadratic absorbing ramp over a
    6-cell border (sigma_max = 1); B = 16 plane waves on a Fibonacci sphere; tol 1e-10."""
    N, k = 64, 20.0
    return Problem("helmholtz3d_64cube_k20_p16_planewaves", helmholtz_3d_absorbing(N, k), plane_waves_3d(N, k, 16),
                   method, 1e-10, maxit)


def helmholtz3d_n2097152_p32(method: str = "cocr_rq", maxit: int = 50000) -> Problem:
    """3D 7-point Helmholtz, 128^3 grid (n=2,097,152), k=40, same absorbing ramp; B n x 32
    complex normal (seed 1); tol 1e-10."""
    N = 128
    return Problem("helmholtz3d_128cube_k40_p32", helmholtz_3d_absorbing(N, 40.0), complex_normal(N**3, 32, 1),
                   method, 1e-10, maxit)


def helmholtz2d_batch(count: int = 64, seed: int = 3, side_range=(64, 512), k_range=(5.0, 30.0),
                      damping_range=(0.02, 0.1), p_choices=(1, 2, 4, 8, 16)):
    """Independent 2D 5-point Helmholtz systems of uneven size: for each system, from one
    ``default_rng(seed)`` stream in this order, grid side ~ U{side_range}, k ~ U[k_range],
    damping ~ U[damping_range], p ~ choice(p_choices); then B is complex normal with seed
    ``1000 * seed + i``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.integers(side_range[0], side_range[1] + 1))
        k = float(rng.uniform(*k_range))
        damping = float(rng.uniform(*damping_range))
        p = int(rng.choice(p_choices))
        A = helmholtz_2d(side, k, damping)
        out.append(Problem(f"helmholtz2d_{side}x{side}_k{k:.1f}_p{p}", A, complex_normal(A.n, p, 1000 * seed + i),
                           "cocr_rq", 1e-10, 20000, extra={"side": side, "k": k, "damping": damping}))
    return out
