"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
* residual history ||xi_m||_F/||B||_F: <= 1e-8 relative for m <= 20 (two FP64 runs of the
  recurrence with different summation orders, well-conditioned inputs; observed ~1e-11);
* X_m at a fixed iteration count: <= 1e-10 relative (well-conditioned inputs);
* xi_m elementwise: <= 1e-8 relative to ||xi_m||_F;
* the sparse product A X: <= 1e-14 relative (one reordering of a sum of at most 27 terms).
"""
import numpy as np
import pytest

import oracle.blcoc_oracle as O
from paper_1601_05362_gb300 import problems as P
from gpu_common import need_gpu, to_dev, rel, oracle_iters_range

pytestmark = pytest.mark.gpu

HIST_TOL = 1e-8
X_TOL = 1e-10


def _handle(A):
    from paper_1601_05362_gb300 import blcoc
    return blcoc.Handle.from_csr(A)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 8, 13, 16, 17, 32])
def test_spmm_matches_scipy(p):
    torch = need_gpu()
    A = P.random_complex_symmetric(1000 + p, 9, seed=p)
    Xh = P.complex_normal(A.n, p, 7)
    h = _handle(A)
    X = to_dev(torch, Xh)
    Y = torch.zeros_like(X)
    h.spmm(X, Y)
    Yref = A.to_scipy() @ Xh
    assert rel(Y.cpu().numpy(), Yref) < 1e-14


def test_residual_norm():
    torch = need_gpu()
    A = P.helmholtz_2d(37, 5.0, 0.05)
    B = P.complex_normal(A.n, 6, 1)
    Xh = P.complex_normal(A.n, 6, 2)
    h = _handle(A)
    r = h.residual_norm(to_dev(torch, B), to_dev(torch, Xh))
    ref = np.linalg.norm(B - A.to_scipy() @ Xh)
    assert abs(r - ref) <= 1e-13 * ref


@pytest.mark.parametrize("method", ["cocg_rq", "cocr_rq"])
def test_helmholtz2d_n1024_p4_full_solve(method):
    """The 32x32 2D Helmholtz problem (n=1024, p=4, tol 1e-10, maxit 500)."""
    torch = need_gpu()
    pr = P.helmholtz2d_n1024_p4(method)
    A = pr.A.to_scipy()
    f = O.bl_cocg_rq if method == "cocg_rq" else O.bl_cocr_rq
    ref = f(A, pr.B, tol=pr.tol, maxit=pr.maxit)
    h = _handle(pr.A)
    B = to_dev(torch, pr.B)
    X = torch.zeros_like(B)
    st = h.solve(B, X, method=method, tol=pr.tol, maxit=pr.maxit)
    info = h.info()
    assert st == 0, h.last_error()
    # the residual of this indefinite problem is erratic, so where it first crosses tol
    # moves by a few iterations under different rounding (BLAS, reduction order): the
    # count must lie within max(3, 5%) of the oracle's own spread under 1e-16
    # perturbations of B
    lo, hi = oracle_iters_range(f, A, pr.B, pr.tol, pr.maxit)
    slack = max(3, ref.iters // 20)
    assert lo - slack <= info["iters"] <= hi + slack, (info["iters"], lo, hi)
    hist = info["hist"]
    m = min(21, len(hist), len(ref.hist))
    assert np.max(np.abs(hist[:m] - np.array(ref.hist[:m])) / np.array(ref.hist[:m])) < HIST_TOL
    assert info["relres_true"] <= 10 * pr.tol
    assert abs(info["relres_true"] - O.true_relres(A, pr.B, X.cpu().numpy())) < 1e-12
    if info["iters"] == ref.iters:
        assert rel(X.cpu().numpy(), ref.X) < 1e-8


@pytest.mark.parametrize("method", ["cocg_rq", "cocr_rq"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 8, 16, 32])
def test_fixed_iterations_match_oracle(method, p):
    """X_m, xi_m and the history after exactly m iterations (tol = 0), ragged n and p."""
    torch = need_gpu()
    n = 1500 + 3 * p  # not a multiple of the 32-row chunk
    A = P.random_complex_symmetric(n, 8, seed=100 + p, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(n, p, 200 + p)
    X0 = 0.1 * P.complex_normal(n, p, 300 + p)
    m = 12
    f = O.bl_cocg_rq if method == "cocg_rq" else O.bl_cocr_rq
    ref = f(A.to_scipy(), Bh, X0=X0, tol=0.0, maxit=m)
    h = _handle(A)
    B = to_dev(torch, Bh)
    X = to_dev(torch, X0)
    st = h.solve(B, X, method=method, tol=0.0, maxit=m)
    info = h.info()
    assert st == 5, h.last_error()          # not converged: ran exactly m iterations
    assert info["iters"] == m
    hist = info["hist"]
    assert np.max(np.abs(hist - np.array(ref.hist)) / np.array(ref.hist)) < HIST_TOL
    assert rel(X.cpu().numpy(), ref.X) < X_TOL
    xi = h.xi(p)
    assert np.max(np.abs(xi - ref.xi)) / np.linalg.norm(ref.xi) < HIST_TOL


@pytest.mark.parametrize("method", ["cocg_rq", "cocr_rq"])
def test_host_pointers_equal_device_pointers(method):
    torch = need_gpu()
    pr = P.helmholtz2d_n1024_p4(method)
    h = _handle(pr.A)
    Xh = np.zeros_like(pr.B)
    st = h.solve(pr.B, Xh, method=method, tol=1e-10, maxit=500)
    info_h = h.info()
    B = to_dev(torch, pr.B)
    X = torch.zeros_like(B)
    st2 = h.solve(B, X, method=method, tol=1e-10, maxit=500)
    assert st == st2 == 0
    assert np.array_equal(Xh, X.cpu().numpy())          # bitwise: deterministic reductions
    assert info_h["iters"] == h.info()["iters"]


def test_host_staging_follows_its_own_capacity():
    """Host-memory B and X go through handle-owned staging buffers.  A device-pointer solve
    with a wider block in between must not let a later host solve reuse buffers sized for
    a narrower one: host p = 4, device p = 16, host p = 8 on one handle, the last checked
    bitwise against the same solve from device pointers."""
    torch = need_gpu()
    A = P.helmholtz_2d(40, 5.0, 0.05)
    h = _handle(A)
    out = {}
    for p, where in ((4, "host"), (16, "device"), (8, "host"), (8, "device")):
        Bh = P.complex_normal(A.n, p, 70 + p)
        if where == "host":
            X = np.zeros_like(Bh)
            st = h.solve(Bh, X, method="cocr_rq", tol=1e-10, maxit=400)
        else:
            Xd = torch.zeros((A.n, p), dtype=torch.complex128, device="cuda")
            st = h.solve(to_dev(torch, Bh), Xd, method="cocr_rq", tol=1e-10, maxit=400)
            X = Xd.cpu().numpy()
        assert st == 0, (p, where, h.last_error())
        assert h.info()["relres_true"] <= 1e-9
        out[(p, where)] = X
    assert np.array_equal(out[(8, "host")], out[(8, "device")])
    h.close()


def test_graph_and_direct_launches_agree_bitwise():
    torch = need_gpu()
    pr = P.helmholtz2d_n1024_p4("cocr_rq")
    h = _handle(pr.A)
    B = to_dev(torch, pr.B)
    out = []
    for g, poll in ((1, 16), (0, 16), (1, 5)):
        h.set_option("graph", g)
        h.set_option("poll", poll)
        X = torch.zeros_like(B)
        assert h.solve(B, X, tol=1e-10, maxit=500) == 0
        out.append((X.cpu().numpy(), h.info()["iters"]))
    for X, it in out[1:]:
        assert it == out[0][1] and np.array_equal(X, out[0][0])


def test_edge_cases():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.random_complex_symmetric(300, 6, seed=1)
    h = _handle(A)
    Bh = P.complex_normal(300, 3, 1)
    B = to_dev(torch, Bh)
    # maxit = 0: X unchanged, not converged
    X0 = to_dev(torch, P.complex_normal(300, 3, 2))
    X = X0.clone()
    assert h.solve(B, X, tol=1e-10, maxit=0) == blcoc.BLCOC_NOT_CONVERGED
    assert torch.equal(X, X0) and h.info()["iters"] == 0
    # zero right-hand side: X = 0, converged at once
    Z = torch.zeros_like(B)
    X = X0.clone()
    assert h.solve(Z, X, tol=1e-10, maxit=10) == 0
    assert float(X.abs().max()) == 0.0
    # exact initial guess converges at iteration 0
    Xs = np.linalg.solve(A.to_dense(), Bh)
    X = to_dev(torch, Xs)
    assert h.solve(B, X, tol=1e-8, maxit=10) == 0 and h.info()["iters"] == 0
    # duplicated columns: the residual block has no full rank -> breakdown
    Bd = Bh.copy()
    Bd[:, 1] = Bd[:, 0]
    X = torch.zeros_like(B)
    assert h.solve(to_dev(torch, Bd), X, tol=1e-10, maxit=50) == blcoc.BLCOC_BREAKDOWN
    # invalid arguments
    with pytest.raises(blcoc.BlcocError):
        h.solve(B, torch.zeros_like(B), tol=-1.0)
    st = h._lib.blcoc_solve(h._h, B.data_ptr(), X.data_ptr(), 33, 1, 1e-10, 10)
    assert st == blcoc.BLCOC_ERR_INVALID_ARG
    st = h._lib.blcoc_solve(h._h, B.data_ptr(), X.data_ptr(), 3, 7, 1e-10, 10)
    assert st == blcoc.BLCOC_ERR_INVALID_ARG


@pytest.mark.parametrize("method", ["cocg_rq", "cocr_rq"])
@pytest.mark.parametrize("gap,expect", [(1e-15, "breakdown"), (1e-4, "ok")])
def test_breakdown_on_nearly_dependent_columns_agrees_with_oracle(method, gap, expect):
    """Right-hand sides whose last column equals the first up to a relative `gap`.  At
    1e-15 the block has lost rank to working accuracy: the oracle's Householder factor has a
    diagonal below 1e-14 of its largest and the GPU's Cholesky pivot is below 64 eps of the
    column's squared norm, so both report a breakdown at the setup QR (rounding alone leaves
    that pivot a tiny positive number, which a test on its sign lets through).  At 1e-4
    neither does and the solve converges."""
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.random_complex_symmetric(600, 8, seed=41, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(A.n, 4, 42)
    Bh[:, 3] = Bh[:, 0] * (1.0 + gap * P.complex_normal(A.n, 1, 43)[:, 0])
    f = O.bl_cocg_rq if method == "cocg_rq" else O.bl_cocr_rq
    ref = f(A.to_scipy(), Bh, tol=1e-10, maxit=500)
    h = _handle(A)
    B = to_dev(torch, Bh)
    X = torch.zeros_like(B)
    st = h.solve(B, X, method=method, tol=1e-10, maxit=500)
    if expect == "breakdown":
        assert ref.status == O.BREAKDOWN and ref.iters == 0
        assert st == blcoc.BLCOC_BREAKDOWN and h.info()["iters"] == 0, blcoc.status_string(st)
        assert float(X.abs().max()) == 0.0            # X_0 is returned unchanged
    else:
        assert ref.status == O.CONVERGED
        assert st == blcoc.BLCOC_OK, h.last_error()
        assert h.info()["relres_true"] <= 1e-9
    h.close()


def test_shifted_cholqr3_fallback_on_ill_conditioned_right_hand_sides():
    """Columns dependent to 1e-10: a Cholesky QR cannot resolve them (cond^2 eps >> 1), a
    Householder QR can.  The oracle (Householder) converges.  Both rq methods with the
    shifted CholQR3 fallback (default) converge to the tolerance as well and their QR factor
    xi_0 matches the oracle's where it is resolved; without the fallback the solve reports
    a breakdown at the setup QR."""
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.random_complex_symmetric(600, 8, seed=41, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(A.n, 4, 42)
    Bh[:, 3] = Bh[:, 0] * (1.0 + 1e-10 * P.complex_normal(A.n, 1, 43)[:, 0])
    for f in (O.bl_cocr_rq, O.bl_cocg_rq):
        assert f(A.to_scipy(), Bh, tol=1e-10, maxit=500).status == O.CONVERGED
    ref0 = O.bl_cocr_rq(A.to_scipy(), Bh, tol=0.0, maxit=0)
    B = to_dev(torch, Bh)
    h = _handle(A)
    for method in ("cocr_rq", "cocg_rq"):
        h.set_option("qr_fallback", 1)
        X = torch.zeros_like(B)
        assert h.solve(B, X, method=method, tol=0.0, maxit=0) == blcoc.BLCOC_NOT_CONVERGED, h.last_error()
        d_gpu, d_ref = np.abs(np.diag(h.xi(4))), np.abs(np.diag(ref0.xi))
        assert np.max(np.abs(d_gpu - d_ref) / d_ref) < 1e-4, (method, d_gpu, d_ref)
        X.zero_()
        assert h.solve(B, X, method=method, tol=1e-10, maxit=500) == blcoc.BLCOC_OK, (method, h.last_error())
        assert O.true_relres(A.to_scipy(), Bh, X.cpu().numpy()) <= 1e-9
        h.set_option("qr_fallback", 0)
        X.zero_()
        assert h.solve(B, X, method=method, tol=1e-10, maxit=500) == blcoc.BLCOC_BREAKDOWN
    h.close()


def test_create_rejects_bad_matrices():
    need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.random_complex_symmetric(200, 6, seed=3)
    v = A.vals.copy()
    v[5] += 0.5  # breaks a_ij = a_ji
    with pytest.raises(blcoc.BlcocError) as e:
        blcoc.Handle(A.n, A.row_ptr, A.col_idx, v)
    assert e.value.status == blcoc.BLCOC_ERR_NOT_SYMMETRIC
    ci = A.col_idx.copy()
    ci[3] = A.n + 5  # out of range column
    with pytest.raises(blcoc.BlcocError) as e:
        blcoc.Handle(A.n, A.row_ptr, ci, A.vals)
    assert e.value.status == blcoc.BLCOC_ERR_INVALID_ARG
    rp = A.row_ptr.copy()
    rp[10], rp[11] = rp[11], rp[10]  # non-monotone row pointers
    with pytest.raises(blcoc.BlcocError) as e:
        blcoc.Handle(A.n, rp, A.col_idx, A.vals)
    assert e.value.status == blcoc.BLCOC_ERR_INVALID_ARG


def test_device_csr_input():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.helmholtz_2d(20, 4.0, 0.05)
    h = blcoc.Handle(A.n, to_dev(torch, A.row_ptr), to_dev(torch, A.col_idx), to_dev(torch, A.vals))
    Xh = P.complex_normal(A.n, 2, 0)
    X = to_dev(torch, Xh)
    Y = torch.zeros_like(X)
    h.spmm(X, Y)
    assert rel(Y.cpu().numpy(), A.to_scipy() @ Xh) < 1e-14


@pytest.mark.parametrize("p", [1, 4, 16])
def test_cocr_explicit_u_option_matches_oracle(p):
    """Option u_explicit = 1 forms U_{m+1} = A S_{m+1} by a sparse product instead of
    Algorithm 3's recurrence; the iterates are the same in exact arithmetic."""
    torch = need_gpu()
    n = 1500 + 3 * p
    A = P.random_complex_symmetric(n, 8, seed=100 + p, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(n, p, 200 + p)
    ref = O.bl_cocr_rq(A.to_scipy(), Bh, tol=0.0, maxit=12)
    h = _handle(A)
    h.set_option("u_explicit", 1)
    B = to_dev(torch, Bh)
    X = torch.zeros_like(B)
    assert h.solve(B, X, tol=0.0, maxit=12) == 5
    hist = h.info()["hist"]
    assert np.max(np.abs(hist - np.array(ref.hist)) / np.array(ref.hist)) < HIST_TOL
    assert rel(X.cpu().numpy(), ref.X) < X_TOL
    X.zero_()
    assert h.solve(B, X, tol=1e-10, maxit=2000) == 0
    assert h.info()["relres_true"] < 1e-9


@pytest.mark.parametrize("method", ["cocg", "cocr"])
@pytest.mark.parametrize("p", [1, 3, 8, 16])
def test_plain_block_methods_match_oracle(method, p):
    """Plain block COCR (Algorithm 1) and plain block COCG against the oracle's plain forms."""
    torch = need_gpu()
    n = 1500 + 3 * p
    A = P.random_complex_symmetric(n, 8, seed=300 + p, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(n, p, 400 + p)
    f = O.bl_cocg if method == "cocg" else O.bl_cocr
    ref = f(A.to_scipy(), Bh, tol=0.0, maxit=10)
    h = _handle(A)
    B = to_dev(torch, Bh)
    X = torch.zeros_like(B)
    assert h.solve(B, X, method=method, tol=0.0, maxit=10) == 5
    hist = h.info()["hist"]
    assert np.max(np.abs(hist - np.array(ref.hist)) / np.array(ref.hist)) < HIST_TOL
    assert rel(X.cpu().numpy(), ref.X) < X_TOL


@pytest.mark.parametrize("method", ["cocg", "cocr"])
def test_plain_block_methods_full_solve(method):
    """The plain forms are the less robust ones (Sec. 3: without residual
    orthonormalization bl_cocg fails on young3c); on this indefinite problem their history
    amplifies rounding differences faster, so the bounds are 10x the oracle's own response
    to a 1e-16 relative perturbation of B (history, m <= 20) and twice its iteration-count
    change plus 5%."""
    torch = need_gpu()
    pr = P.helmholtz2d_n1024_p4(method)
    A = pr.A.to_scipy()
    f = O.bl_cocg if method == "cocg" else O.bl_cocr
    ref = f(A, pr.B, tol=1e-10, maxit=pr.maxit)
    Bp = pr.B * (1.0 + 1e-16 * np.random.default_rng(0).standard_normal(pr.B.shape))
    refp = f(A, Bp, tol=1e-10, maxit=pr.maxit)
    m = min(21, len(ref.hist), len(refp.hist))
    hist_sens = np.max(np.abs(np.array(refp.hist[:m]) - np.array(ref.hist[:m])) / np.array(ref.hist[:m]))
    h = _handle(pr.A)
    B = to_dev(torch, pr.B)
    X = torch.zeros_like(B)
    st = h.solve(B, X, method=method, tol=1e-10, maxit=pr.maxit)
    info = h.info()
    assert st == 0 and ref.status == "converged"
    assert abs(info["iters"] - ref.iters) <= 2 * abs(refp.iters - ref.iters) + max(3, ref.iters // 20)
    dev = np.max(np.abs(info["hist"][:m] - np.array(ref.hist[:m])) / np.array(ref.hist[:m]))
    assert dev < max(HIST_TOL, 10 * hist_sens), (dev, hist_sens)
    assert info["relres_true"] < 1e-8


@pytest.mark.parametrize("method,p", [("cocr_rq", p) for p in (5, 8, 13, 16, 17, 24, 32)] +
                         [("cocg_rq", p) for p in (5, 8, 16, 21, 32)])
def test_fp64_tc_option_matches_oracle(method, p):
    """Option fp64_tc: the p x p block updates run on the bf16 tensor cores by exact
    integer slicing; the iterates must match the FP64 oracle like the FP64-FMA path.
    Widths 17-32 run the kernels whose slice digits are staged in shared memory (K = 64
    real columns, level sums still exact in fp32)."""
    torch = need_gpu()
    n = 1500 + 3 * p
    A = P.random_complex_symmetric(n, 8, seed=100 + p, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(n, p, 200 + p)
    X0 = 0.1 * P.complex_normal(n, p, 300 + p)
    f = O.bl_cocr_rq if method == "cocr_rq" else O.bl_cocg_rq
    ref = f(A.to_scipy(), Bh, X0=X0, tol=0.0, maxit=12)
    h = _handle(A)
    h.set_option("fp64_tc", 1)
    B = to_dev(torch, Bh)
    X = to_dev(torch, X0)
    assert h.solve(B, X, method=method, tol=0.0, maxit=12) == 5
    hist = h.info()["hist"]
    assert np.max(np.abs(hist - np.array(ref.hist)) / np.array(ref.hist)) < HIST_TOL
    assert rel(X.cpu().numpy(), ref.X) < X_TOL
    xi = h.xi(p)
    assert np.max(np.abs(xi - ref.xi)) / np.linalg.norm(ref.xi) < HIST_TOL


def test_fp64_tc_full_solve_helmholtz2d():
    torch = need_gpu()
    pr = P.helmholtz2d_n1024_p4("cocr_rq")
    Bh = P.complex_normal(pr.n, 16, 9)
    ref = O.bl_cocr_rq(pr.A.to_scipy(), Bh, tol=1e-10, maxit=500)
    h = _handle(pr.A)
    h.set_option("fp64_tc", 1)
    B = to_dev(torch, Bh)
    X = torch.zeros_like(B)
    assert h.solve(B, X, tol=1e-10, maxit=500) == 0
    info = h.info()
    # the residual stagnates near 1e-10 before crossing it: the oracle's own count spreads
    # over several iterations under 1e-16 perturbations of B (47 to 54 on two machines)
    lo, hi = oracle_iters_range(O.bl_cocr_rq, pr.A.to_scipy(), Bh, 1e-10, 500)
    slack = max(3, ref.iters // 20)
    assert lo - slack <= info["iters"] <= hi + slack, (info["iters"], lo, hi)
    m = min(21, len(ref.hist))
    assert np.max(np.abs(info["hist"][:m] - np.array(ref.hist[:m])) / np.array(ref.hist[:m])) < HIST_TOL
    assert info["relres_true"] <= 1e-9


@pytest.mark.parametrize("method", ["cocg_rq", "cocr_rq"])
@pytest.mark.parametrize("p,tc", [(1, 0), (4, 0), (7, 0), (16, 0), (7, 1), (16, 1), (32, 1)])
def test_cholqr2_option_matches_oracle(method, p, tc):
    """Option qr_passes = 2 (CholQR2: a second pass W <- W T1 and a second Cholesky factor
    after every Cholesky QR, setup included) against the oracle's Householder QR, also with
    the block updates on the tensor cores (the second factor's slices feed the passes)."""
    torch = need_gpu()
    n = 1500 + 3 * p
    A = P.random_complex_symmetric(n, 8, seed=100 + p, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(n, p, 200 + p)
    X0 = 0.1 * P.complex_normal(n, p, 300 + p)
    m = 12
    f = O.bl_cocg_rq if method == "cocg_rq" else O.bl_cocr_rq
    ref = f(A.to_scipy(), Bh, X0=X0, tol=0.0, maxit=m)
    h = _handle(A)
    h.set_option("qr_passes", 2)
    h.set_option("fp64_tc", tc)
    B = to_dev(torch, Bh)
    X = to_dev(torch, X0)
    assert h.solve(B, X, method=method, tol=0.0, maxit=m) == 5, h.last_error()
    info = h.info()
    assert info["iters"] == m
    assert np.max(np.abs(info["hist"] - np.array(ref.hist)) / np.array(ref.hist)) < HIST_TOL
    assert rel(X.cpu().numpy(), ref.X) < X_TOL
    xi = h.xi(p)
    assert np.max(np.abs(xi - ref.xi)) / np.linalg.norm(ref.xi) < HIST_TOL
    X.copy_(to_dev(torch, X0))
    assert h.solve(B, X, method=method, tol=1e-10, maxit=500) == 0
    assert h.info()["relres_true"] <= 1e-9
    h.close()


@pytest.mark.parametrize("method", ["cocg_rq", "cocr_rq"])
def test_cholqr2_on_nearly_dependent_right_hand_sides(method):
    """B with nearly dependent columns (condition ~2.6e6, Gram condition ~7e12).  The QR
    factor xi_0 (maxit = 0) against the oracle's Householder factor: single-pass Cholesky QR
    loses about cond^2 eps in the small diagonal entries, CholQR2 keeps about cond eps
    (both forms give the same iterates X, which do not depend on the basis)."""
    torch = need_gpu()
    n, p = 2000, 6
    A = P.random_complex_symmetric(n, 8, seed=31, diag=3.0 + 0.6j, scale=0.25)
    b = P.complex_normal(n, 1, 32)
    Bh = np.repeat(b, p, axis=1) + 1e-6 * P.complex_normal(n, p, 33)
    assert np.linalg.cond(Bh) > 1e6
    f = O.bl_cocg_rq if method == "cocg_rq" else O.bl_cocr_rq
    ref = np.diag(f(A.to_scipy(), Bh, tol=0.0, maxit=0).xi)
    errs = {}
    for qr in (1, 2):
        h = _handle(A)
        h.set_option("qr_passes", qr)
        B = to_dev(torch, Bh)
        X = torch.zeros_like(B)
        assert h.solve(B, X, method=method, tol=0.0, maxit=0) == 5
        errs[qr] = float(np.max(np.abs(np.diag(h.xi(p)) - ref) / np.abs(ref)))
        h.close()
    assert errs[2] < 1e-8, errs
    assert errs[1] > 100 * errs[2], errs


@pytest.mark.parametrize("p,split", [(1, 2), (1, 4), (2, 4), (4, 2), (4, 4), (8, 2), (8, 4), (16, 2)])
def test_spmm_row_bundle_splits_match_oracle(p, split):
    """SpMM row bundles with 2 or 4 lane groups splitting each row's nonzeros (option
    spmm_split): the iterates match the oracle like the default bundle."""
    torch = need_gpu()
    n = 1500 + 3 * p
    A = P.random_complex_symmetric(n, 9, seed=700 + p, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(n, p, 800 + p)
    m = 12
    ref = O.bl_cocr_rq(A.to_scipy(), Bh, tol=0.0, maxit=m)
    h = _handle(A)
    h.set_option("spmm_split", split)
    B = to_dev(torch, Bh)
    X = torch.zeros_like(B)
    assert h.solve(B, X, tol=0.0, maxit=m) == 5, h.last_error()
    assert h.stat("spmm_split") == split
    info = h.info()
    assert np.max(np.abs(info["hist"] - np.array(ref.hist)) / np.array(ref.hist)) < HIST_TOL
    assert rel(X.cpu().numpy(), ref.X) < X_TOL
    h.close()


def test_spmm_row_bundle_autotune_is_cached_and_reproducible():
    """spmm_split = 0: a timed sweep picks the bundle once per (n, nnz/row, p); the solve
    then equals a solve with that bundle forced, bit for bit."""
    torch = need_gpu()
    A = P.random_complex_symmetric(3000, 9, seed=77, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(3000, 4, 78)
    h = _handle(A)
    B = to_dev(torch, Bh)
    h.set_option("spmm_split", 0)
    X1 = torch.zeros_like(B)
    assert h.solve(B, X1, tol=1e-10, maxit=500) == 0
    chosen = h.stat("spmm_split")
    assert chosen in (1, 2, 4)
    X2 = torch.zeros_like(B)
    assert h.solve(B, X2, tol=1e-10, maxit=500) == 0
    assert h.stat("spmm_split") == chosen
    h.set_option("spmm_split", chosen)
    X3 = torch.zeros_like(B)
    assert h.solve(B, X3, tol=1e-10, maxit=500) == 0
    assert np.array_equal(X1.cpu().numpy(), X3.cpu().numpy())
    assert np.array_equal(X2.cpu().numpy(), X3.cpu().numpy())
    h.close()


def test_history_after_a_longer_solve_on_the_same_handle():
    """A second solve with a larger maxit grows the history buffer; the iterations' CUDA
    graph captured by the first solve must not keep writing to the old buffer: the second
    history equals that of a fresh handle, bit for bit."""
    torch = need_gpu()
    pr = P.helmholtz2d_n1024_p4("cocr_rq")
    B = to_dev(torch, pr.B)
    h = _handle(pr.A)
    X = torch.zeros_like(B)
    h.solve(B, X, tol=0.0, maxit=5)
    X.zero_()
    h.solve(B, X, tol=0.0, maxit=400)
    grown = np.asarray(h.info()["hist"])
    h2 = _handle(pr.A)
    X2 = torch.zeros_like(B)
    h2.solve(B, X2, tol=0.0, maxit=400)
    fresh = np.asarray(h2.info()["hist"])
    assert len(grown) == len(fresh) == 401
    assert np.array_equal(grown, fresh)
    assert torch.equal(X, X2)
