"""bl_cocg_rq and bl_cocr_rq in a chosen floating-point precision (test infrastructure).

Only the tests and the golden-value script use this module; the library never calls it.

The FP64 oracle (``blcoc_oracle``) calls LAPACK for its QR and p x p solves, which exist
only in double precision.  This module writes those steps out with plain numpy arithmetic
so that the same iteration can run in ``numpy.clongdouble``: 80-bit extended precision on
x86 (64-bit significand, unit roundoff 5.4e-20) and IEEE binary128 on aarch64 (113-bit
significand, 9.6e-35).  Against it, the FP64 oracle's own rounding error is measured
instead of argued: the difference between the FP64 and the extended-precision residual
histories is the FP64 run's rounding error to within the extended precision's, which is
what bounds how closely any FP64 implementation (the CUDA path included) can be expected
to follow the oracle.

Steps (the same as ``blcoc_oracle``, in the paper's order, Sec. 2.2):

* sparse product: ``Y[i] = sum_j a_ij X[j]`` over the stored entries of row i;
* thin QR (Sec. 2.2; MATLAB's ``qr(W,0)`` is Householder): Householder reflectors
  (Golub and Van Loan, Alg. 5.2.1, complex form) applied column by column, Q formed by
  applying them to the first p columns of the identity, the diagonal of R then made real
  and non-negative as in ``blcoc_oracle.thin_qr``;
* p x p solves: Gaussian elimination with partial pivoting on the largest modulus
  (Golub and Van Loan, Alg. 3.4.1), then back substitution;
* Algorithm 2 (bl_cocg_rq) and Algorithm 3 (bl_cocr_rq, right-hand side ``Q_m^T V_m`` of
  the alpha' system, the oracle's default reading) for a fixed number of iterations.

Called with ``dtype=np.complex128`` the functions reproduce ``blcoc_oracle`` up to the
different rounding of the library routines (pinned in tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np

__all__ = ["csr_apply", "householder_qr", "lu_solve", "bl_cocr_rq_xp", "bl_cocg_rq_xp", "EXTENDED"]

EXTENDED = np.clongdouble


def csr_apply(row_ptr, col_idx, vals, X):
    """Y = A X for CSR arrays (values already in X's dtype): Y[i] = sum_j a_ij X[col_j]."""
    n = len(row_ptr) - 1
    prod = vals[:, None] * X[col_idx]
    Y = np.zeros((n, X.shape[1]), dtype=X.dtype)
    starts = np.asarray(row_ptr[:-1])
    nonempty = np.asarray(row_ptr[1:]) > starts
    if np.any(nonempty):
        sums = np.add.reduceat(prod, starts[nonempty], axis=0)
        Y[nonempty] = sums
    return Y


def householder_qr(W):
    """Thin QR W = Q R with Q^H Q = I (Householder), diag(R) real and non-negative."""
    W = np.array(W, copy=True)
    n, p = W.shape
    dt = W.dtype
    real = np.zeros(1, dtype=dt).real.dtype
    vs = []
    for k in range(p):
        x = W[k:, k].copy()
        normx = np.sqrt(np.sum((x.real * x.real + x.imag * x.imag)))
        if normx == 0:
            vs.append(None)
            continue
        x0 = x[0]
        ax0 = np.sqrt(x0.real * x0.real + x0.imag * x0.imag)
        phase = x0 / ax0 if ax0 != 0 else dt.type(1)
        alpha = -phase * normx                     # reflect x onto alpha e_1 (no cancellation)
        v = x
        v[0] = x0 - alpha
        vnorm2 = np.sum(v.real * v.real + v.imag * v.imag)
        if vnorm2 == 0:
            vs.append(None)
            continue
        # W[k:, k:] <- (I - 2 v v^H / (v^H v)) W[k:, k:]
        coef = (2 / vnorm2) * (np.conj(v) @ W[k:, k:])
        W[k:, k:] -= np.outer(v, coef)
        vs.append((k, v, vnorm2))
    R = np.triu(W[:p, :p])
    Q = np.zeros((n, p), dtype=dt)
    Q[np.arange(p), np.arange(p)] = 1
    for item in reversed(vs):                      # Q = H_0 H_1 ... H_{p-1} I[:, :p]
        if item is None:
            continue
        k, v, vnorm2 = item
        coef = (2 / vnorm2) * (np.conj(v) @ Q[k:, :])
        Q[k:, :] -= np.outer(v, coef)
    d = np.diag(R).copy()
    mag = np.sqrt(d.real * d.real + d.imag * d.imag)
    phase = np.where(mag > 0, d / np.where(mag > 0, mag, real.type(1)), dt.type(1))
    Q = Q * phase[None, :]
    R = np.conj(phase)[:, None] * R
    R[np.arange(p), np.arange(p)] = mag          # |r_kk| exactly (the product above rounds)
    return Q, R


def lu_solve(M, RHS):
    """Solve M Z = RHS by Gaussian elimination with partial pivoting (largest modulus)."""
    M = np.array(M, copy=True)
    Z = np.array(RHS, copy=True)
    p = M.shape[0]
    for k in range(p):
        col = M[k:, k]
        mags = col.real * col.real + col.imag * col.imag
        r = k + int(np.argmax(mags))
        if mags[r - k] == 0:
            raise ZeroDivisionError("singular p x p system")
        if r != k:
            M[[k, r]] = M[[r, k]]
            Z[[k, r]] = Z[[r, k]]
        for i in range(k + 1, p):
            l = M[i, k] / M[k, k]
            M[i, k:] -= l * M[k, k:]
            Z[i] -= l * Z[k]
    for k in range(p - 1, -1, -1):
        Z[k] = (Z[k] - M[k, k + 1:] @ Z[k + 1:]) / M[k, k]
    return Z


def _prep(A, B, dtype):
    row_ptr = np.asarray(A.row_ptr)
    col_idx = np.asarray(A.col_idx)
    vals = np.asarray(A.vals).astype(dtype)
    return row_ptr, col_idx, vals, np.asarray(B).astype(dtype)


def _fro(M):
    return np.sqrt(np.sum(M.real * M.real + M.imag * M.imag))


def bl_cocr_rq_xp(A, B, iters, dtype=EXTENDED):
    """Algorithm 3 for `iters` iterations from X0 = 0 in `dtype`; A is a CSR with
    ``row_ptr``, ``col_idx``, ``vals``.  Returns (hist, X, xi): hist[m] = ||xi_m||_F/||B||_F
    for m = 0..iters."""
    rp, ci, va, B = _prep(A, B, dtype)
    def mul(Y):
        return csr_apply(rp, ci, va, Y)
    nb = _fro(B)
    X = np.zeros_like(B)
    Q, xi = householder_qr(B)                      # Q_0 xi_0 = B - A X_0 (X_0 = 0)
    S = Q.copy()
    V = mul(Q)                                     # U_0 = V_0 = A Q_0
    U = V.copy()
    hist = [_fro(xi) / nb]
    for _ in range(iters):
        alpha = lu_solve(U.T @ U, Q.T @ V)         # (U^T U) alpha' = Q^T V
        X = X + S @ (alpha @ xi)                   # X += S alpha' xi
        Qn, tau = householder_qr(Q - U @ alpha)    # Q_{m+1} tau = Q_m - U_m alpha'
        xi = tau @ xi
        Vn = mul(Qn)
        beta = lu_solve(Q.T @ V, tau.T @ (Qn.T @ Vn))   # (Q^T V) beta' = tau^T Q+^T V+
        S = Qn + S @ beta
        U = Vn + U @ beta
        Q, V = Qn, Vn
        hist.append(_fro(xi) / nb)
    return hist, X, xi


def bl_cocg_rq_xp(A, B, iters, dtype=EXTENDED):
    """Algorithm 2 for `iters` iterations from X0 = 0 in `dtype` (see bl_cocr_rq_xp)."""
    rp, ci, va, B = _prep(A, B, dtype)
    nb = _fro(B)
    X = np.zeros_like(B)
    Q, xi = householder_qr(B)
    S = Q.copy()
    hist = [_fro(xi) / nb]
    for _ in range(iters):
        AS = csr_apply(rp, ci, va, S)
        alpha = lu_solve(S.T @ AS, Q.T @ Q)        # (S^T A S) alpha' = Q^T Q
        X = X + S @ (alpha @ xi)
        Qn, tau = householder_qr(Q - AS @ alpha)
        xi = tau @ xi
        beta = lu_solve(Q.T @ Q, tau.T @ (Qn.T @ Qn))
        S = Qn + S @ beta
        Q = Qn
        hist.append(_fro(xi) / nb)
    return hist, X, xi
