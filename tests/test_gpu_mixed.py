"""Mixed-precision form (iterative refinement around bl_cocr_rq / bl_cocg_rq with
complex64 inner solves; FP64 residual, p x p solves and QR).

The tests check what the method promises: the FP64 true relative residual
||B - A X||_F/||B||_F recomputed here on the CPU reaches the tolerance, and the solution
agrees with a dense LU solve (small, well-conditioned cases) and with the oracle's FP64
solution; at n = 262,144 on the 27-point random complex symmetric family it reaches a
true residual of 1e-10.  On the indefinite 64^3 Helmholtz problem the complex64 inner
solves diverge (its residual grows ~16x before it falls, and in single precision the
iteration loses its bilinear orthogonality first); the refinement must then stop with a
status instead of looping.
"""
import numpy as np
import pytest

import oracle.blcoc_oracle as O
from paper_1601_05362_gb300 import problems as P
from gpu_common import need_gpu, to_dev, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", ["cocr_rq_mixed", "cocg_rq_mixed"])
@pytest.mark.parametrize("p", [1, 3, 4, 8, 16, 32])
def test_mixed_reaches_fp64_tolerance_small(method, p):
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.random_complex_symmetric(900 + p, 8, seed=7 + p, diag=3.0 + 0.6j, scale=0.25)
    Bh = P.complex_normal(A.n, p, 70 + p)
    with blcoc.Handle.from_csr(A) as h:
        B = to_dev(torch, Bh)
        X = torch.zeros_like(B)
        st = h.solve(B, X, method=method, tol=1e-12, maxit=5000)
        assert st == blcoc.BLCOC_OK, h.last_error()
        outer = h.stat("outer_iters")
        info = h.info(hist_len=outer + 1)
    Xg = X.cpu().numpy()
    trr = O.true_relres(A.to_scipy(), Bh, Xg)
    assert trr <= 1e-12
    assert abs(info["relres_true"] - trr) <= 1e-3 * trr + 1e-16
    Xd = np.linalg.solve(A.to_dense(), Bh)
    assert rel(Xg, Xd) < 1e-10
    assert outer >= 2      # complex64 inner solves need refinement to get here
    assert np.all(np.diff(info["hist"][: outer + 1]) < 0)   # each refinement step reduces the residual


def test_mixed_helmholtz2d_n1024_p4():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    pr = P.helmholtz2d_n1024_p4("cocr_rq")
    ref = O.bl_cocr_rq(pr.A.to_scipy(), pr.B, tol=1e-12, maxit=2000)
    with blcoc.Handle.from_csr(pr.A) as h:
        B = to_dev(torch, pr.B)
        X = torch.zeros_like(B)
        assert h.solve(B, X, method="cocr_rq_mixed", tol=1e-10, maxit=5000) == blcoc.BLCOC_OK
    Xg = X.cpu().numpy()
    assert O.true_relres(pr.A.to_scipy(), pr.B, Xg) <= 1e-10
    assert rel(Xg, ref.X) < 1e-7


def test_mixed_random27pt_n262144_p16_true_residual():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.random_symmetric_27pt(64, 64, 64, seed=2)
    Bh = P.complex_normal(A.n, 16, 5)
    with blcoc.Handle.from_csr(A) as h:
        B = to_dev(torch, Bh)
        X = torch.zeros_like(B)
        st = h.solve(B, X, method="cocr_rq_mixed", tol=1e-10, maxit=20000)
        assert st == blcoc.BLCOC_OK, h.last_error()
    trr = O.true_relres(A.to_scipy(), Bh, X.cpu().numpy())
    assert trr <= 1e-10


def test_mixed_helmholtz3d_stops_with_status():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    pr = P.helmholtz3d_n262144_p16("cocr_rq")
    with blcoc.Handle.from_csr(pr.A) as h:
        h.set_option("inner_maxit", 200)
        h.set_option("outer_maxit", 6)
        B = to_dev(torch, pr.B)
        X = torch.zeros_like(B)
        st = h.solve(B, X, method="cocr_rq_mixed", tol=1e-10, maxit=5000)
        assert st in (blcoc.BLCOC_NOT_CONVERGED, blcoc.BLCOC_BREAKDOWN)
        assert h.stat("outer_iters") <= 6


def test_mixed_zero_rhs_and_bad_args():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.random_complex_symmetric(200, 6, seed=1)
    with blcoc.Handle.from_csr(A) as h:
        B = torch.zeros((200, 3), dtype=torch.complex128, device="cuda")
        X = to_dev(torch, P.complex_normal(200, 3, 1))
        assert h.solve(B, X, method="cocr_rq_mixed", tol=1e-10, maxit=100) == blcoc.BLCOC_OK
        assert float(X.abs().max()) == 0.0
        with pytest.raises(blcoc.BlcocError):
            h.set_option("inner_tol_exp", 0)
