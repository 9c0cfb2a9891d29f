"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself:

* Petrov-Galerkin brute force (Eqs. 1.2-1.3, Table 1): the m-th iterate of block COCG is
  the unique ``X_m = X_0 + K_m y`` with ``K_m^T (B - A X_m) = 0``; of block COCR the one
  with ``(A K_m)^T (B - A X_m) = 0``.  Solved here by a dense least-squares-free linear
  solve over an explicitly built block Krylov basis.
* dense LU (``numpy.linalg.solve`` on the dense matrix) for the converged solution;
* p = 1 reduction to the scalar COCG / COCR methods the block methods extend (Sec. 1);
* equality of the rq forms (Algorithms 2-3) with the plain forms (Algorithm 1 and the
  derived block COCG) in exact arithmetic, and ``||R_m||_F = ||xi_m||_F`` (Sec. 2.2);
* the bilinear orthogonality relations of Table 1 on stored iterates;
* finite termination of a block Krylov method within ceil(n/p) steps;
* the real SPD case, where Algorithm 2 reduces to block CG (computed separately here in
  real arithmetic).
* planted mistakes in the oracle (on the CPU) are caught by the Galerkin pin.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle.blcoc_oracle as O
from paper_1601_05362_gb300 import problems as P


def dense_cs(n, seed, spread=6.0, offscale=0.15, shift=1.0 + 0.3j):
    """Dense complex symmetric, non-Hermitian test matrix with a spread spectrum."""
    rng = np.random.default_rng(seed)
    G = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2)
    A = offscale * (G + G.T) / 2 + np.diag(shift + np.linspace(0.0, spread, n) * (1 + 0.1j))
    assert np.allclose(A, A.T) and not np.allclose(A, A.conj().T)
    return A


def galerkin_iterate(A, B, X0, m, kind):
    """Brute-force m-th iterate from the subspace + orthogonality definition."""
    R0 = B - A @ X0
    blocks = [R0]
    for _ in range(m - 1):
        blocks.append(A @ blocks[-1])
    K = np.concatenate(blocks, axis=1)
    K, _ = np.linalg.qr(K)          # any basis of the same span gives the same iterate
    AK = A @ K
    Lt = K.T if kind == "cocg" else AK.T   # L = K_m (COCG) or A K_m (COCR), bilinear form
    y = np.linalg.solve(Lt @ AK, Lt @ R0)
    return X0 + K @ y


# --------------------------------------------------------------------------- basics

def test_thin_qr_normalised():
    rng = np.random.default_rng(5)
    W = rng.standard_normal((40, 5)) + 1j * rng.standard_normal((40, 5))
    Q, R = O.thin_qr(W)
    assert np.allclose(Q.conj().T @ Q, np.eye(5), atol=1e-14)
    assert np.allclose(Q @ R, W, atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0)
    d = np.diag(R)
    assert np.all(np.abs(d.imag) == 0) and np.all(d.real >= 0)


def test_generators_symmetric_not_hermitian():
    for A in (P.helmholtz_2d(12, 6.0, 0.05), P.helmholtz_3d_absorbing(14, 20.0),
              P.random_complex_symmetric(200, 7, 3), P.random_symmetric_27pt(6, 5, 4, 2)):
        M = A.to_scipy()
        assert abs(M - M.T).max() == 0
        assert abs(M - M.conj().T).max() > 0
        assert np.all(np.diff(A.row_ptr) >= 1)
        for i in range(0, A.n, max(1, A.n // 7)):
            cols = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
            assert np.all(np.diff(cols) > 0)


def test_helmholtz_sizes():
    A1 = P.helmholtz_2d(32, 6.0, 0.05)
    assert (A1.n, A1.nnz) == (1024, 5 * 1024 - 4 * 32)
    A2 = P.helmholtz_3d_absorbing(20, 20.0)
    assert (A2.n, A2.nnz) == (8000, 7 * 8000 - 6 * 400)
    d = P.border_depth(64, 6)
    assert d[0] == 6 and d[5] == 1 and d[6] == 0 and d[57] == 0 and d[58] == 1 and d[63] == 6


# --------------------------------------------------------------------------- Galerkin pin

@pytest.mark.parametrize("kind", ["cocg", "cocr"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_rq_iterates_equal_petrov_galerkin(kind, p):
    n = 40
    A = dense_cs(n, seed=11 + p)
    rng = np.random.default_rng(100 + p)
    B = rng.standard_normal((n, p)) + 1j * rng.standard_normal((n, p))
    X0 = 0.1 * (rng.standard_normal((n, p)) + 1j * rng.standard_normal((n, p)))
    solver = O.bl_cocg_rq if kind == "cocg" else O.bl_cocr_rq
    plain = O.bl_cocg if kind == "cocg" else O.bl_cocr
    for m in range(1, 5):
        Xg = galerkin_iterate(A, B, X0, m, kind)
        for f in (solver, plain):
            r = f(A, B, X0=X0, tol=0.0, maxit=m)
            assert r.iters == m
            err = np.linalg.norm(r.X - Xg) / np.linalg.norm(Xg)
            assert err < 1e-9, (f.__name__, m, err)


def test_galerkin_pin_separates_the_two_methods():
    """The COCG and COCR iterates differ, so the pin distinguishes the two conditions."""
    n, p = 40, 2
    A = dense_cs(n, seed=3)
    B = np.random.default_rng(1).standard_normal((n, p)) + 0j
    X0 = np.zeros_like(B)
    a = galerkin_iterate(A, B, X0, 2, "cocg")
    b = galerkin_iterate(A, B, X0, 2, "cocr")
    assert np.linalg.norm(a - b) / np.linalg.norm(a) > 1e-3


# --------------------------------------------------------------------------- planted mistakes

def _galerkin_error(kind, m=3, p=2):
    n = 40
    A = dense_cs(n, seed=21)
    rng = np.random.default_rng(22)
    B = rng.standard_normal((n, p)) + 1j * rng.standard_normal((n, p))
    X0 = np.zeros_like(B)
    f = O.bl_cocg_rq if kind == "cocg" else O.bl_cocr_rq
    r = f(A, B, X0=X0, tol=0.0, maxit=m)
    Xg = galerkin_iterate(A, B, X0, m, kind)
    return np.linalg.norm(r.X - Xg) / np.linalg.norm(Xg)


@pytest.mark.parametrize("kind", ["cocg", "cocr"])
def test_planted_conjugated_inner_product_is_caught(kind, monkeypatch):
    assert _galerkin_error(kind) < 1e-9
    monkeypatch.setattr(O, "bt", lambda Y, Z: Y.conj().T @ Z)
    assert _galerkin_error(kind) > 1e-4


@pytest.mark.parametrize("kind", ["cocg", "cocr"])
def test_planted_transposed_solve_is_caught(kind, monkeypatch):
    real_solve = O.small_solve
    monkeypatch.setattr(O, "small_solve", lambda M, R: real_solve(M, R).T)
    assert _galerkin_error(kind) > 1e-4


@pytest.mark.parametrize("kind", ["cocg", "cocr"])
def test_planted_unnormalised_qr_is_harmless(kind, monkeypatch):
    """Sec. 2.2: the iterates do not depend on the phase freedom of the QR factor."""
    def qr_neg(W):
        Q, R = np.linalg.qr(W, mode="reduced")
        ph = np.exp(1j * np.arange(W.shape[1]))
        return Q * ph[None, :], np.conj(ph)[:, None] * R
    monkeypatch.setattr(O, "thin_qr", qr_neg)
    assert _galerkin_error(kind) < 1e-9


# --------------------------------------------------------------------------- dense LU

@pytest.mark.parametrize("method", ["cocg_rq", "cocr_rq"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_converged_solution_matches_dense_lu(method, p):
    n = 64
    A = dense_cs(n, seed=40 + p, spread=3.0)
    rng = np.random.default_rng(7 + p)
    B = rng.standard_normal((n, p)) + 1j * rng.standard_normal((n, p))
    f = O.bl_cocg_rq if method == "cocg_rq" else O.bl_cocr_rq
    r = f(A, B, tol=1e-10, maxit=4 * n)
    assert r.status == "converged"
    X = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(r.X - X) / np.linalg.norm(X) < 10 * kappa * 1e-10
    assert O.true_relres(A, B, r.X) < 10 * 1e-10


def test_sparse_helmholtz_matches_dense_lu():
    A = P.helmholtz_2d(12, 3.0, 0.05)
    M = A.to_scipy()
    B = P.complex_normal(A.n, 3, 0)
    for f in (O.bl_cocg_rq, O.bl_cocr_rq):
        r = f(M, B, tol=1e-11, maxit=2000)
        assert r.status == "converged"
        X = np.linalg.solve(A.to_dense(), B)
        assert np.linalg.norm(r.X - X) / np.linalg.norm(X) < 1e-7
        assert O.true_relres(M, B, r.X) < 1e-10


# --------------------------------------------------------------------------- p = 1

@pytest.mark.parametrize("kind", ["cocg", "cocr"])
def test_p1_reduces_to_scalar_method(kind):
    A = P.random_complex_symmetric(300, 9, 4, diag=2.0 + 0.4j, scale=0.3).to_scipy()
    b = P.complex_normal(300, 1, 9)
    f_block = O.bl_cocg_rq if kind == "cocg" else O.bl_cocr_rq
    f_scalar = O.cocg if kind == "cocg" else O.cocr
    rb = f_block(A, b, tol=0.0, maxit=20, record=True)
    rs = f_scalar(A, b[:, 0], tol=0.0, maxit=20)
    hb, hs = np.array(rb.hist), np.array(rs.hist)
    assert np.max(np.abs(hb - hs) / hs) < 1e-10
    # xi_m = ||r_m||_2 (a positive real number) under the positive-diagonal normalisation
    for m in (0, 5, 10):
        xi = rb.record["xi"][m]
        assert xi.shape == (1, 1) and xi[0, 0].imag == 0 and xi[0, 0].real > 0
    assert np.linalg.norm(rb.X - rs.X) / np.linalg.norm(rs.X) < 1e-10


# --------------------------------------------------------------------------- rq vs plain

@pytest.mark.parametrize("kind", ["cocg", "cocr"])
def test_rq_equals_plain_form_early_iterations(kind):
    A = P.random_complex_symmetric(400, 8, 12, diag=2.5 + 0.5j, scale=0.3).to_scipy()
    B = P.complex_normal(400, 4, 13)
    rq = (O.bl_cocg_rq if kind == "cocg" else O.bl_cocr_rq)(A, B, tol=0.0, maxit=10, record=True)
    pl = (O.bl_cocg if kind == "cocg" else O.bl_cocr)(A, B, tol=0.0, maxit=10, record=True)
    for m in range(11):
        # ||R_m||_F = ||xi_m||_F (Sec. 2.2) and identical iterates
        assert abs(rq.hist[m] - pl.hist[m]) <= 1e-10 * pl.hist[m]
        Xa, Xb = rq.record["X"][m], pl.record["X"][m]
        if m > 0:
            assert np.linalg.norm(Xa - Xb) / np.linalg.norm(Xb) < 1e-10
        # R_m = Q_m xi_m
        Rm = rq.record["Q"][m] @ rq.record["xi"][m]
        assert np.linalg.norm(Rm - pl.record["R"][m]) <= 1e-10 * np.linalg.norm(pl.record["R"][m])


def test_recursive_residual_tracks_true_residual():
    A = P.helmholtz_2d(16, 4.0, 0.05).to_scipy()
    B = P.complex_normal(256, 3, 2)
    for f in (O.bl_cocg_rq, O.bl_cocr_rq):
        r = f(A, B, tol=1e-10, maxit=2000, record=True)
        assert r.status == "converged"
        for m in range(0, r.iters + 1, max(1, r.iters // 8)):
            t = O.true_relres(A, B, r.record["X"][m])
            assert abs(t - r.hist[m]) <= 1e-6 * r.hist[m] + 1e-12
        assert O.true_relres(A, B, r.X) <= 10 * 1e-10


# --------------------------------------------------------------------------- Table 1

def _offdiag_max(blocks, form):
    worst = 0.0
    for i in range(len(blocks)):
        for j in range(max(0, i - 10), i):
            G = form(blocks[i], blocks[j])
            worst = max(worst, np.linalg.norm(G) / (np.linalg.norm(blocks[i]) * np.linalg.norm(blocks[j])))
    return worst


def test_table1_invariants_cocg_rq():
    Ad = dense_cs(120, seed=8)
    B = P.complex_normal(120, 3, 4)
    r = O.bl_cocg_rq(Ad, B, tol=0.0, maxit=14, record=True)
    Qs, Ss = r.record["Q"], r.record["S"]
    assert _offdiag_max(Qs, lambda a, b: a.T @ b) < 1e-8          # R_i^T R_j = 0
    assert _offdiag_max(Ss, lambda a, b: a.T @ (Ad @ b)) < 1e-8   # P_i^T A P_j = 0
    for Q in Qs:
        assert np.allclose(Q.conj().T @ Q, np.eye(3), atol=1e-13)
    # sanity: the conjugated form is NOT orthogonal (the pin is not vacuous)
    assert _offdiag_max(Qs, lambda a, b: a.conj().T @ b) > 1e-3


def test_table1_invariants_cocr_rq():
    Ad = dense_cs(120, seed=9)
    B = P.complex_normal(120, 3, 5)
    r = O.bl_cocr_rq(Ad, B, tol=0.0, maxit=14, record=True)
    Qs, Us, Ss = r.record["Q"], r.record["U"], r.record["S"]
    assert _offdiag_max(Qs, lambda a, b: a.T @ (Ad @ b)) < 1e-8   # R_i^T A R_j = 0
    assert _offdiag_max(Us, lambda a, b: a.T @ b) < 1e-8          # (AP_i)^T (AP_j) = 0
    for S, U in zip(Ss, Us):
        assert np.linalg.norm(U - Ad @ S) <= 1e-11 * np.linalg.norm(U)   # U_m = A S_m
    assert _offdiag_max(Qs, lambda a, b: a.T @ b) > 1e-3


# --------------------------------------------------------------------------- termination

@pytest.mark.parametrize("kind", ["cocg", "cocr"])
def test_finite_termination(kind):
    n, p = 24, 4
    A = dense_cs(n, seed=31, spread=2.0)
    B = np.random.default_rng(3).standard_normal((n, p)) + 0.5j
    f = O.bl_cocg_rq if kind == "cocg" else O.bl_cocr_rq
    r = f(A, B, tol=1e-12, maxit=n)
    assert r.status == "converged" and r.iters <= n // p + 2


def test_identity_scaled_converges_in_one_step():
    n, p = 30, 3
    c = 2.0 - 0.7j
    A = c * np.eye(n)
    B = P.complex_normal(n, p, 1)
    for f in (O.bl_cocg_rq, O.bl_cocr_rq):
        r = f(A, B, tol=1e-14, maxit=5)
        assert r.iters == 1
        assert np.allclose(r.X, B / c, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------- real SPD

def block_cg_real(A, B, m):
    """O'Leary's block CG in real arithmetic (independent reference)."""
    X = np.zeros_like(B)
    R = B.copy()
    P_ = R.copy()
    for _ in range(m):
        AP = A @ P_
        a = np.linalg.solve(P_.T @ AP, R.T @ R)
        X = X + P_ @ a
        Rn = R - AP @ a
        b = np.linalg.solve(R.T @ R, Rn.T @ Rn)
        P_ = Rn + P_ @ b
        R = Rn
    return X


def test_real_spd_reduces_to_block_cg():
    Lap = P.neg_laplacian(9, 2).toarray() * (1.0 / 100.0) + 0.5 * np.eye(81)
    B = np.random.default_rng(6).standard_normal((81, 3))
    for m in (1, 3, 6):
        r = O.bl_cocg_rq(Lap.astype(np.complex128), B.astype(np.complex128), tol=0.0, maxit=m)
        assert np.max(np.abs(r.X.imag)) == 0.0
        Xr = block_cg_real(Lap, B, m)
        assert np.linalg.norm(r.X.real - Xr) / np.linalg.norm(Xr) < 1e-11


# --------------------------------------------------------------------------- breakdown

@pytest.mark.parametrize("kind", ["cocg", "cocr"])
def test_rank_deficient_rhs_is_a_breakdown(kind):
    """Duplicated columns of B make R_0 rank deficient (the loss of independence that
    Sec. 2.2 names); the paper has no rule, the oracle reports a breakdown."""
    A = dense_cs(30, seed=2)
    b = P.complex_normal(30, 1, 3)
    B = np.concatenate([b, b, P.complex_normal(30, 1, 4)], axis=1)
    f = O.bl_cocg_rq if kind == "cocg" else O.bl_cocr_rq
    r = f(A, B, tol=1e-10, maxit=30)
    assert r.status == "breakdown" and r.iters == 0


@pytest.mark.parametrize("kind", ["cocg", "cocr"])
def test_exhausted_krylov_space_ends_in_breakdown_or_convergence(kind):
    """n = 64, p = 3: the block Krylov space is exhausted after about n/p steps; with a
    tolerance below the attainable accuracy the oracle must stop cleanly."""
    A = dense_cs(64, seed=43, spread=3.0)
    rng = np.random.default_rng(10)
    B = rng.standard_normal((64, 3)) + 1j * rng.standard_normal((64, 3))
    f = O.bl_cocg_rq if kind == "cocg" else O.bl_cocr_rq
    r = f(A, B, tol=1e-15, maxit=256)
    assert r.status in ("breakdown", "converged")
    assert r.iters <= 64 // 3 + 4
    assert O.true_relres(A, B, r.X) < 1e-9


# --------------------------------------------------------------------------- alpha' reading

def test_cocr_rq_alpha_rhs_reading():
    """Algorithm 3 prints ``Q_m^T U_m`` as the alpha' right-hand side; Algorithm 1's
    ``R_m^T V_m`` under Sec. 2.2's substitutions gives ``Q_m^T V_m``.  Equal in exact
    arithmetic; in floating point the printed form diverges on this 2D Helmholtz case,
    while the derived form follows Algorithm 1 to convergence."""
    A = P.helmholtz_2d(12, 3.0, 0.05).to_scipy()
    B = P.complex_normal(144, 3, 0)
    plain = O.bl_cocr(A, B, tol=1e-10, maxit=144)
    derived = O.bl_cocr_rq(A, B, tol=1e-10, maxit=144)
    printed = O.bl_cocr_rq(A, B, tol=1e-10, maxit=144, alpha_rhs="QU")
    assert plain.status == "converged" and derived.status == "converged"
    assert abs(derived.iters - plain.iters) <= 2
    assert O.true_relres(A, B, derived.X) < 1e-9
    assert printed.status != "converged" or O.true_relres(A, B, printed.X) > 1e-6
    # both readings agree in the early iterations (exact-arithmetic equality)
    a = O.bl_cocr_rq(A, B, tol=0.0, maxit=8)
    b = O.bl_cocr_rq(A, B, tol=0.0, maxit=8, alpha_rhs="QU")
    assert np.linalg.norm(a.X - b.X) / np.linalg.norm(a.X) < 1e-10


# --------------------------------------------------------------------------- stored fixture

def test_golden_fixture_is_reproduced():
    """tests/golden/helmholtz2d_n1024_p4.json was written by tests/golden/make_golden.py
    (oracle only); the oracle must still reproduce it."""
    import json, os
    path = os.path.join(os.path.dirname(__file__), "golden", "helmholtz2d_n1024_p4.json")
    g = json.load(open(path))
    for method, f in (("cocg_rq", O.bl_cocg_rq), ("cocr_rq", O.bl_cocr_rq)):
        pr = P.helmholtz2d_n1024_p4(method)
        r = f(pr.A.to_scipy(), pr.B, tol=pr.tol, maxit=pr.maxit)
        ref = g["runs"][method]
        assert r.iters == ref["iters"] and r.status == ref["status"]
        h = np.array(r.hist[:20]); hr = np.array(ref["hist"][:20])
        assert np.max(np.abs(h - hr) / hr) < 1e-12


def test_cocr_rq_explicit_u_equals_galerkin():
    """U_{m+1} = A S_{m+1} instead of the recurrence gives the same iterates (Sec. 2.1)."""
    n, p = 40, 2
    A = dense_cs(n, seed=17)
    rng = np.random.default_rng(18)
    B = rng.standard_normal((n, p)) + 1j * rng.standard_normal((n, p))
    X0 = np.zeros_like(B)
    for m in range(1, 5):
        r = O.bl_cocr_rq(A, B, X0=X0, tol=0.0, maxit=m, u_explicit=True)
        Xg = galerkin_iterate(A, B, X0, m, "cocr")
        assert np.linalg.norm(r.X - Xg) / np.linalg.norm(Xg) < 1e-9
