"""Differentiable solve (paper_1601_05362_gb300.autograd) on the 27-point random complex
symmetric family with 10% of the pairs dropped, diagonal 4+0.5i; loss L = sum |C^T X|^2.

* gradients against a dense FP64 reference (torch.linalg.solve with autograd) at n = 1024;
* central finite differences on symmetric pairs (a_ij, a_ji), real and imaginary steps;
* at n = 1,048,576 (128 x 128 x 64, p = 8): the adjoint solution satisfies its equation,
  checked through the library's residual norm (a property that holds at any size).
"""
import numpy as np
import pytest

from paper_1601_05362_gb300 import problems as P
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _setup(torch, nx, ny, nz, p=8):
    from paper_1601_05362_gb300.autograd import SymmetricCSR
    A = P.random_symmetric_27pt(nx, ny, nz, seed=2)
    op = SymmetricCSR(A.row_ptr, A.col_idx, A.n, A.vals)
    B = torch.from_numpy(P.complex_normal(A.n, p, 3)).cuda()
    Cm = torch.from_numpy(P.complex_normal(A.n, p, 4)).cuda()
    return A, op, B, Cm


def _loss(X, Cm):
    return (Cm.transpose(0, 1) @ X).abs().pow(2).sum()


def test_gradient_matches_dense_reference():
    torch = need_gpu()
    from paper_1601_05362_gb300.autograd import blcoc_solve
    A, op, B, Cm = _setup(torch, 16, 8, 8)
    vals = torch.from_numpy(A.vals).cuda().requires_grad_(True)
    Bv = B.clone().requires_grad_(True)
    L = _loss(blcoc_solve(vals, Bv, op, tol=1e-13, maxit=2000), Cm)
    L.backward()
    # dense FP64 reference on the CPU
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    vr = torch.from_numpy(A.vals).requires_grad_(True)
    Br = B.cpu().clone().requires_grad_(True)
    Ad = torch.zeros((A.n, A.n), dtype=torch.complex128).index_put(
        (torch.from_numpy(rows), torch.from_numpy(A.col_idx.astype(np.int64))), vr)
    Lr = _loss(torch.linalg.solve(Ad, Br), Cm.cpu())
    Lr.backward()
    assert abs(L.item() - Lr.item()) <= 1e-10 * Lr.item()
    gv, gvr = vals.grad.cpu().numpy(), vr.grad.numpy()
    gb, gbr = Bv.grad.cpu().numpy(), Br.grad.numpy()
    assert np.linalg.norm(gv - gvr) / np.linalg.norm(gvr) < 1e-8
    assert np.linalg.norm(gb - gbr) / np.linalg.norm(gbr) < 1e-8
    op.close()


def test_gradient_matches_central_differences():
    torch = need_gpu()
    from paper_1601_05362_gb300.autograd import blcoc_solve
    A, op, B, Cm = _setup(torch, 16, 8, 8)
    vals0 = torch.from_numpy(A.vals).cuda()
    vals = vals0.clone().requires_grad_(True)
    L = _loss(blcoc_solve(vals, B, op, tol=1e-13, maxit=2000), Cm)
    L.backward()
    g = vals.grad.cpu().numpy()
    # position of each (i, j) entry
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    pos = {(int(i), int(j)): e for e, (i, j) in enumerate(zip(rows, A.col_idx))}
    rng = np.random.default_rng(0)
    picks = [pos[(k, k)] for k in (0, 517)] + [int(e) for e in rng.integers(0, A.nnz, 6)]
    h = 1e-6
    for e in picks:
        i, j = int(rows[e]), int(A.col_idx[e])
        pair = [e] if i == j else [e, pos[(j, i)]]
        gsum = sum(g[q] for q in pair)
        for step, part in ((h, "re"), (1j * h, "im")):
            vals_p = vals0.clone()
            vals_m = vals0.clone()
            for q in pair:
                vals_p[q] += step
                vals_m[q] -= step
            with torch.no_grad():
                Lp = _loss(blcoc_solve(vals_p, B, op, tol=1e-13, maxit=2000), Cm).item()
                Lm = _loss(blcoc_solve(vals_m, B, op, tol=1e-13, maxit=2000), Cm).item()
            fd = (Lp - Lm) / (2 * h)
            an = gsum.real if part == "re" else gsum.imag
            assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-3 * np.abs(g).max()), (e, part, fd, an)
    op.close()


def test_adjoint_at_n1048576():
    torch = need_gpu()
    from paper_1601_05362_gb300.autograd import blcoc_solve
    A, op, B, Cm = _setup(torch, 128, 128, 64)
    vals = torch.from_numpy(A.vals).cuda().requires_grad_(True)
    Bv = B.clone().requires_grad_(True)
    X = blcoc_solve(vals, Bv, op, tol=1e-10, maxit=2000)
    L = _loss(X, Cm)
    L.backward()
    # forward: B - A X small; adjoint: A conj(Lambda) = conj(G) with G = dL/dconj(X)
    rf = op.handle.residual_norm(B, X.detach())
    assert rf <= 1e-9 * torch.linalg.norm(B).item()
    G = (Cm.conj() @ (Cm.transpose(0, 1) @ X.detach())) * 2.0
    Lam = Bv.grad
    ra = op.handle.residual_norm(G.conj_physical(), Lam.conj_physical())
    assert ra <= 1e-9 * torch.linalg.norm(G).item()
    assert torch.isfinite(vals.grad).all()
    op.close()


@pytest.mark.parametrize("p", [1, 5, 8])
def test_sampled_grad_kernel(p):
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.random_symmetric_27pt(10, 9, 8, seed=4)
    Lam = P.complex_normal(A.n, p, 1)
    X = P.complex_normal(A.n, p, 2)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    ref = -np.sum(Lam[rows] * np.conj(X[A.col_idx]), axis=1)
    with blcoc.Handle.from_csr(A) as h:
        out = torch.zeros(A.nnz, dtype=torch.complex128, device="cuda")
        h.sampled_grad(torch.from_numpy(Lam).cuda(), torch.from_numpy(X).cuda(), out)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-14 * np.max(np.abs(ref))
