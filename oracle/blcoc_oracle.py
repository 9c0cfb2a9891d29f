"""Plain, slow, FP64 CPU oracle for bl_cocg_rq and bl_cocr_rq (test infrastructure).

This module is the correctness authority for the CUDA solver.  It is test
infrastructure: only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
leg of ``bench.py`` use it; the library never calls it.

Everything is complex128 numpy.  Library primitives used as single steps: the sparse
product ``A @ V`` (scipy CSR), the thin Householder QR ``numpy.linalg.qr`` and the
LU-with-partial-pivoting solve ``numpy.linalg.solve``.  There is no blocking, fusion or
reordering beyond what the algorithms in the paper state.

Notation follows the paper (Gu, Carpentieri, Huang, Meng, "Block variants of the COCG
and COCR methods for solving complex symmetric linear systems with multiple right-hand
sides"):

* ``Y.T @ Z`` is the unconjugated bilinear form used by every coefficient (Table 1:
  conjugate orthogonality against ``bar(A)``, ``bar(R_0)`` is the plain transpose);
  only the QR factorisation is orthonormal in the Hermitian sense, ``Q^H Q = I_p``
  (Sec. 2.2).
* Readings of the paper where its text is garbled (all in Sec. 2.2):
  - ``S_m = P_m xi_m^{-1}``, ``tau_{m+1} = xi_{m+1} xi_m^{-1}``,
    ``alpha'_m = xi_m alpha_m xi_m^{-1}``, ``beta'_m = xi_m beta_m xi_{m+1}^{-1}``;
  - Algorithm 3's ``X_{m+1} = X_m + P_m alpha'_m`` is read as ``X_m + S_m alpha'_m xi_m``
    (the form of Algorithm 2; ``P_m`` does not exist in the rq iteration);
  - Algorithm 3 solves for ``beta'_m`` (its text writes ``beta_m``);
  - the right-hand side of Algorithm 3's alpha' system is ``Q_m^T V_m``.  Algorithm 3
    prints ``Q_m^T U_m``, which equals it only in exact arithmetic; ``Q_m^T V_m`` is what
    Algorithm 1's ``R_m^T V_m`` becomes under Sec. 2.2's substitutions
    (``R_m = Q_m xi_m``, ``P_m = S_m xi_m``, ``alpha'_m = xi_m alpha_m xi_m^{-1}``), and the
    printed form diverges in floating point on a small 2D Helmholtz problem where
    Algorithm 1 converges (tests/test_oracle_pins.py).  ``alpha_rhs="QU"`` keeps the
    printed form;
  - the QR factor is normalised so that ``diag(xi)`` is real and non-negative (MATLAB's
    ``qr(W,0)`` leaves a diagonal unitary freedom that the iterates do not depend on);
  - stopping rule: ``||xi_m||_F / ||B||_F <= tol`` tested before iteration m; the
    returned iteration count is m (the test at the top of each iteration of Algorithms 2-3).

Every public solver returns a :class:`Result`.  ``hist[m]`` is the recursive relative
residual at the top of iteration m (``||xi_m||_F/||B||_F`` for the rq forms,
``||R_m||_F/||B||_F`` for the plain forms).

Pins (tests/test_oracle_pins.py): Petrov-Galerkin brute force of Eqs. 1.2-1.3 with
Table 1, dense LU, p = 1 reduction to scalar COCG/COCR, rq vs plain forms, Table 1
orthogonality invariants, ``||R_m||_F = ||xi_m||_F``, finite termination, and the real
SPD reduction to block CG.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "Result", "Breakdown", "bt", "fro", "thin_qr", "small_solve", "rank_deficient",
    "bl_cocg_rq", "bl_cocr_rq", "bl_cocg", "bl_cocr", "cocg", "cocr",
    "true_relres", "csr_operator",
]

CONVERGED, NOT_CONVERGED, BREAKDOWN = "converged", "not_converged", "breakdown"


@dataclass
class Result:
    X: np.ndarray
    hist: list
    iters: int
    status: str
    xi: Optional[np.ndarray] = None
    record: dict = field(default_factory=dict)


def csr_operator(row_ptr, col_idx, vals, n):
    """scipy CSR matrix from raw CSR arrays (the oracle's sparse product is scipy's)."""
    import scipy.sparse as sp
    return sp.csr_matrix((np.asarray(vals, dtype=np.complex128), np.asarray(col_idx), np.asarray(row_ptr)),
                         shape=(n, n))


def bt(Y, Z):
    """Unconjugated bilinear block product ``Y^T Z`` (Table 1's orthogonality form)."""
    return Y.T @ Z


def fro(M) -> float:
    return float(np.linalg.norm(M))


def thin_qr(W):
    """Thin QR ``W = Q R`` with ``Q^H Q = I`` (Sec. 2.2 and its footnote: MATLAB ``qr(W,0)``,
    i.e. Householder).  The diagonal of R is made real and non-negative."""
    Q, R = np.linalg.qr(W, mode="reduced")
    d = np.diag(R).copy()
    mag = np.abs(d)
    phase = np.where(mag > 0, d / np.where(mag > 0, mag, 1.0), 1.0)
    Q = Q * phase[None, :]
    R = np.conj(phase)[:, None] * R
    return Q, R


def rank_deficient(R) -> bool:
    """Breakdown test for a QR factor (the paper has no rule; Sec. 2.2 only motivates the
    rq form by loss of linear independence): a non-finite entry, or a diagonal entry below
    ``1e-14`` times the largest one, means the block has lost rank."""
    d = np.abs(np.diag(R))
    return (not np.all(np.isfinite(R))) or d.min() <= 1e-14 * d.max()


class Breakdown(Exception):
    pass


def small_solve(M, RHS):
    """Solve the p x p complex system ``M Z = RHS`` by LU with partial pivoting (what MATLAB's
    backslash does for a general square matrix; the paper does not state its solver)."""
    if not np.all(np.isfinite(M)) or not np.all(np.isfinite(RHS)):
        raise Breakdown("non-finite p x p system")
    try:
        return np.linalg.solve(M, RHS)
    except np.linalg.LinAlgError as e:   # exactly singular pivot
        raise Breakdown(str(e)) from e


def _x0(B, X0):
    return np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.complex128, copy=True)


def true_relres(A, B, X) -> float:
    """``||B - A X||_F / ||B||_F`` (the TRR of Sec. 3, before the log10)."""
    return fro(B - A @ X) / fro(B)


def bl_cocg_rq(A, B, X0=None, tol=1e-10, maxit=None, record=False) -> Result:
    """Block COCG with residual orthonormalization, Algorithm 2 (Sec. 2.2)."""
    B = np.asarray(B, dtype=np.complex128)
    n, p = B.shape
    maxit = n if maxit is None else maxit
    X = _x0(B, X0)
    nb = fro(B)
    Q, xi = thin_qr(B - A @ X)                 # Q_0 xi_0 = B - A X_0
    S = Q.copy()                               # S_0 = Q_0
    hist, rec = [], {"Q": [], "S": [], "X": [], "xi": [], "AS": []}
    status, m = NOT_CONVERGED, 0
    if rank_deficient(xi) and fro(xi) > 0:
        return Result(X=X, hist=[fro(xi) / nb], iters=0, status=BREAKDOWN, xi=xi)
    for m in range(maxit + 1):
        res = fro(xi) / nb
        hist.append(res)
        if record:
            rec["Q"].append(Q.copy()); rec["S"].append(S.copy()); rec["X"].append(X.copy()); rec["xi"].append(xi.copy())
        if res <= tol:                         # stop when ||xi_m||_F/||B||_F <= eps
            status = CONVERGED
            break
        if m == maxit:
            break
        AS = A @ S
        if record:
            rec["AS"].append(AS.copy())
        try:
            alpha = small_solve(bt(S, AS), bt(Q, Q))      # (S^T A S) alpha' = Q^T Q
        except Breakdown:
            status = BREAKDOWN
            break
        X = X + S @ (alpha @ xi)                          # X += S alpha' xi
        Qn, tau = thin_qr(Q - AS @ alpha)                 # Q_{m+1} tau_{m+1} = Q_m - A S_m alpha'
        if rank_deficient(tau):
            status, m = BREAKDOWN, m + 1
            break
        xi = tau @ xi                                     # xi_{m+1} = tau_{m+1} xi_m
        try:
            beta = small_solve(bt(Q, Q), tau.T @ bt(Qn, Qn))  # (Q_m^T Q_m) beta' = tau^T Q^T Q
        except Breakdown:
            status, m = BREAKDOWN, m + 1
            break
        S = Qn + S @ beta                                 # S_{m+1} = Q_{m+1} + S_m beta'
        Q = Qn
    return Result(X=X, hist=hist, iters=m, status=status, xi=xi, record=rec if record else {})


def bl_cocr_rq(A, B, X0=None, tol=1e-10, maxit=None, record=False, alpha_rhs="QV", u_explicit=False) -> Result:
    """Block COCR with residual orthonormalization, Algorithm 3 (Sec. 2.2).

    ``alpha_rhs`` selects the right-hand side of the alpha' system: ``"QV"``
    (``Q_m^T V_m``, derived from Algorithm 1, default) or ``"QU"`` (``Q_m^T U_m``, as
    printed).  ``u_explicit`` replaces the recurrence ``U_{m+1} = V_{m+1} + U_m beta'_m``
    by the product ``U_{m+1} = A S_{m+1}`` it stands for (Sec. 2.1 introduces the
    recurrence only to save that product)."""
    if alpha_rhs not in ("QV", "QU"):
        raise ValueError("alpha_rhs must be 'QV' or 'QU'")
    B = np.asarray(B, dtype=np.complex128)
    n, p = B.shape
    maxit = n if maxit is None else maxit
    X = _x0(B, X0)
    nb = fro(B)
    Q, xi = thin_qr(B - A @ X)                 # Q_0 xi_0 = B - A X_0
    S = Q.copy()                               # S_0 = Q_0, U_0 = V_0 = A Q_0
    V = A @ Q
    U = V.copy()
    hist, rec = [], {"Q": [], "S": [], "U": [], "V": [], "X": [], "xi": []}
    status, m = NOT_CONVERGED, 0
    if rank_deficient(xi) and fro(xi) > 0:
        return Result(X=X, hist=[fro(xi) / nb], iters=0, status=BREAKDOWN, xi=xi)
    for m in range(maxit + 1):
        res = fro(xi) / nb
        hist.append(res)
        if record:
            for key, val in (("Q", Q), ("S", S), ("U", U), ("V", V), ("X", X), ("xi", xi)):
                rec[key].append(val.copy())
        if res <= tol:
            status = CONVERGED
            break
        if m == maxit:
            break
        try:
            rhs = bt(Q, V) if alpha_rhs == "QV" else bt(Q, U)
            alpha = small_solve(bt(U, U), rhs)            # (U^T U) alpha' = Q^T V
        except Breakdown:
            status = BREAKDOWN
            break
        X = X + S @ (alpha @ xi)                          # X += S alpha' xi (the reading of the X update)
        Qn, tau = thin_qr(Q - U @ alpha)                  # Q_{m+1} tau_{m+1} = Q_m - U_m alpha'
        if rank_deficient(tau):
            status, m = BREAKDOWN, m + 1
            break
        xi = tau @ xi
        Vn = A @ Qn                                       # V_{m+1} = A Q_{m+1}
        try:
            beta = small_solve(bt(Q, V), tau.T @ bt(Qn, Vn))  # (Q^T V) beta' = tau^T Q^T V
        except Breakdown:
            status, m = BREAKDOWN, m + 1
            break
        S = Qn + S @ beta                                 # S_{m+1} = Q_{m+1} + S_m beta'
        U = (A @ S) if u_explicit else (Vn + U @ beta)    # U_{m+1} = V_{m+1} + U_m beta'
        Q, V = Qn, Vn
    return Result(X=X, hist=hist, iters=m, status=status, xi=xi, record=rec if record else {})


def bl_cocr(A, B, X0=None, tol=1e-10, maxit=None, record=False) -> Result:
    """Plain block COCR, Algorithm 1 (Sec. 2.1).  The stopping test uses ``||B||_F``
    (equal to Algorithm 1's ``||R_0||_F`` when X0 = 0) so its history compares with
    the rq form."""
    B = np.asarray(B, dtype=np.complex128)
    n, p = B.shape
    maxit = n if maxit is None else maxit
    X = _x0(B, X0)
    nb = fro(B)
    R = B - A @ X                               # R_0 = B - A X_0
    P = R.copy()                                # P_0 = R_0, U_0 = V_0 = A R_0
    V = A @ R
    U = V.copy()
    hist, rec = [], {"R": [], "P": [], "X": []}
    status, m = NOT_CONVERGED, 0
    for m in range(maxit + 1):
        res = fro(R) / nb
        hist.append(res)
        if record:
            rec["R"].append(R.copy()); rec["P"].append(P.copy()); rec["X"].append(X.copy())
        if res <= tol:
            status = CONVERGED
            break
        if m == maxit:
            break
        alpha = small_solve(bt(U, U), bt(R, V))       # (U^T U) alpha = R^T V
        X = X + P @ alpha                             # X += P alpha
        Rn = R - U @ alpha                            # R_{m+1} = R_m - U_m alpha
        Vn = A @ Rn
        beta = small_solve(bt(R, V), bt(Rn, Vn))      # (R_m^T V_m) beta = R_{m+1}^T V_{m+1}
        P = Rn + P @ beta                             # P_{m+1} = R_{m+1} + P_m beta
        U = Vn + U @ beta                             # U_{m+1} = V_{m+1} + U_m beta
        R, V = Rn, Vn
    return Result(X=X, hist=hist, iters=m, status=status, record=rec if record else {})


def bl_cocg(A, B, X0=None, tol=1e-10, maxit=None, record=False) -> Result:
    """Plain block COCG (the paper cites it but does not print it).  The coefficients
    follow from Eqs. (2.1)-(2.2) with Table 1's COCG conditions ``R_{m+1}^T R_m = 0``
    and ``P_{m+1}^T A P_m = 0``: ``alpha = (P^T A P)^{-1} R^T R``,
    ``beta = (R_m^T R_m)^{-1} R_{m+1}^T R_{m+1}``."""
    B = np.asarray(B, dtype=np.complex128)
    n, p = B.shape
    maxit = n if maxit is None else maxit
    X = _x0(B, X0)
    nb = fro(B)
    R = B - A @ X
    P = R.copy()
    hist, rec = [], {"R": [], "P": [], "X": []}
    status, m = NOT_CONVERGED, 0
    for m in range(maxit + 1):
        res = fro(R) / nb
        hist.append(res)
        if record:
            rec["R"].append(R.copy()); rec["P"].append(P.copy()); rec["X"].append(X.copy())
        if res <= tol:
            status = CONVERGED
            break
        if m == maxit:
            break
        AP = A @ P
        alpha = small_solve(bt(P, AP), bt(R, R))
        X = X + P @ alpha
        Rn = R - AP @ alpha
        beta = small_solve(bt(R, R), bt(Rn, Rn))
        P = Rn + P @ beta
        R = Rn
    return Result(X=X, hist=hist, iters=m, status=status, record=rec if record else {})


def cocg(A, b, x0=None, tol=1e-10, maxit=None) -> Result:
    """Scalar COCG (van der Vorst and Melissen): conjugate gradients with the
    unconjugated form ``x^T y`` for a complex symmetric A.  Written independently of the
    block code; it is the p = 1 reference for bl_cocg_rq."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    n = b.shape[0]
    maxit = n if maxit is None else maxit
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    nb = float(np.sqrt(np.sum(np.abs(b) ** 2)))
    r = b - A @ x
    pvec = r.copy()
    rho = np.sum(r * r)
    hist = []
    status, m = NOT_CONVERGED, 0
    for m in range(maxit + 1):
        res = float(np.sqrt(np.sum(np.abs(r) ** 2))) / nb
        hist.append(res)
        if res <= tol:
            status = CONVERGED
            break
        if m == maxit:
            break
        q = A @ pvec
        a = rho / np.sum(pvec * q)
        x = x + a * pvec
        r = r - a * q
        rho_new = np.sum(r * r)
        pvec = r + (rho_new / rho) * pvec
        rho = rho_new
    return Result(X=x.reshape(-1, 1), hist=hist, iters=m, status=status)


def cocr(A, b, x0=None, tol=1e-10, maxit=None) -> Result:
    """Scalar COCR (Sogabe and Zhang): conjugate residuals with the unconjugated form.
    Written independently of the block code; the p = 1 reference for bl_cocr_rq."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    n = b.shape[0]
    maxit = n if maxit is None else maxit
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    nb = float(np.sqrt(np.sum(np.abs(b) ** 2)))
    r = b - A @ x
    pvec = r.copy()
    Ar = A @ r
    Ap = Ar.copy()
    rAr = np.sum(r * Ar)
    hist = []
    status, m = NOT_CONVERGED, 0
    for m in range(maxit + 1):
        res = float(np.sqrt(np.sum(np.abs(r) ** 2))) / nb
        hist.append(res)
        if res <= tol:
            status = CONVERGED
            break
        if m == maxit:
            break
        a = rAr / np.sum(Ap * Ap)
        x = x + a * pvec
        r = r - a * Ap
        Ar = A @ r
        rAr_new = np.sum(r * Ar)
        beta = rAr_new / rAr
        pvec = r + beta * pvec
        Ap = Ar + beta * Ap
        rAr = rAr_new
    return Result(X=x.reshape(-1, 1), hist=hist, iters=m, status=status)
