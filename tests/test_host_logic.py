"""Host-side logic that needs no GPU: the seeded input generators (their sizes, structure
and symmetry, against the closed forms of the 5- and 7-point stencils), the bench's
algorithmic byte and flop counts, and its comment-insensitive hash of the row-pass
sources."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1601_05362_gb300 import problems as P  # noqa: E402


def _symmetric(A):
    S = A.to_scipy()
    return abs(S - S.T).max() == 0.0


def test_helmholtz_2d_size_and_symmetry():
    A = P.helmholtz_2d(32, 6.0, 0.05)
    N = 32
    assert A.n == N * N
    assert A.nnz == 5 * N * N - 4 * N          # 5-point stencil, Dirichlet borders
    assert _symmetric(A)
    S = A.to_scipy()
    assert np.allclose(S.diagonal().imag, -36.0 * 0.05)   # -k^2 (1 + 0.05 i) shift


def test_helmholtz_3d_bench_workload():
    pr = P.helmholtz3d_n262144_p16()
    N = 64
    assert pr.n == N ** 3 == 262144 and pr.p == 16
    assert pr.A.nnz == 7 * N ** 3 - 6 * N ** 2 == 1810432
    assert _symmetric(pr.A)
    # plane waves exp(i k d.x): unit modulus
    assert np.allclose(np.abs(pr.B), 1.0)
    # absorbing border: the imaginary part of the diagonal is zero inside, largest at the faces
    d = pr.A.to_scipy().diagonal()
    assert d.imag.min() < 0.0 and np.count_nonzero(d.imag) < pr.n


def test_fibonacci_directions_are_unit_and_distinct():
    D = P.fibonacci_sphere(16)
    assert D.shape == (16, 3)
    assert np.allclose(np.linalg.norm(D, axis=1), 1.0)
    G = D @ D.T
    assert np.max(G - 2 * np.eye(16)) < 1.0 - 1e-6    # no two directions coincide


def test_random_families_are_complex_symmetric():
    A = P.random_complex_symmetric(500, 8, seed=3)
    assert _symmetric(A) and A.n == 500
    R = P.random_symmetric_27pt(8, 8, 6, seed=2)
    assert _symmetric(R)
    assert R.nnz < 27 * R.n                         # 10% of the off-diagonal pairs dropped


def test_generators_are_seeded():
    a = P.complex_normal(100, 3, 7)
    b = P.complex_normal(100, 3, 7)
    c = P.complex_normal(100, 3, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # (N(0,1) + i N(0,1)) / sqrt(2): unit variance per entry
    big = P.complex_normal(20000, 4, 1)
    assert abs(np.mean(np.abs(big) ** 2) - 1.0) < 0.05


def test_batch_recipe():
    probs = P.helmholtz2d_batch(64)
    assert len(probs) == 64
    assert {pr.p for pr in probs} <= {1, 2, 4, 8, 16}
    sides = [int(round(np.sqrt(pr.n))) for pr in probs]
    assert min(sides) >= 64 and max(sides) <= 512
    assert sum(pr.n for pr in probs) == 5868820
    again = P.helmholtz2d_batch(64)
    assert all(np.array_equal(a.B, b.B) for a, b in zip(probs, again))


def test_bench_algorithmic_counts():
    import types
    import bench
    pr = P.helmholtz3d_n262144_p16()
    n, p, nnz = pr.n, pr.p, pr.A.nnz
    ops = bench.fp64_ops(pr)
    # pass C at p = 16: Q = W T (136 complex MACs), X, S, U updates (256 each), U^T U (136):
    # 1040 MACs of three FMAs; adds: 24 input sums + 32 output combines (T), 3 x (32 + 32)
    # (full applies), 32 (the Gram's companion tile)
    assert ops["cocr_passC"] == (3 * 1040 * n, 280 * n)
    # pass A: W = Q - U alpha' (256 MACs), W^H W (136); the SpMM: gather (four products),
    # V = Y T (136, three), W^T Y (136, four)
    assert ops["cocr_passA"] == (3 * 392 * n, 96 * n)
    assert ops["spmm_gram"] == (4 * nnz * p + 3 * 136 * n + 4 * 136 * n, 56 * n)
    flops, bytes_, it_bytes, it_flops = bench.algorithmic(pr)
    assert flops["cocr_passC"] == 2.0 * 3120 * n + 280 * n
    assert bytes_["cocr_passC"] == 9 * n * p * 16
    assert it_bytes == pr.A.nbytes(16) + 14 * n * p * 16
    assert abs(it_bytes / 1e6 - 976.78) < 0.01
    assert abs(it_flops / 1e9 - 3.0964) < 0.001
    # kernel widths below 8 keep four products everywhere
    small = types.SimpleNamespace(n=1000, p=4, A=types.SimpleNamespace(nnz=5000))
    o4 = bench.fp64_ops(small)
    assert o4["cocr_passC"] == (4 * 1000 * (4 * 5 + 3 * 16), 0)
    assert o4["cocr_passA"] == (4 * 1000 * (16 + 10), 0)


def test_source_hash_ignores_comments(tmp_path):
    import bench
    code = "int f(int a) {  // add one\n  /* a block\n     comment */\n  return a + 1;\n}\n\n"
    same = "int f(int a) {\n  return a + 1;\n}\n"
    other = "int f(int a) {\n  return a + 2;\n}\n"
    assert bench.code_of(code) == bench.code_of(same)
    assert bench.code_of(code) != bench.code_of(other)
    assert len(bench.source_hash()) == 16
