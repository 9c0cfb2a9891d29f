"""Differentiable solve X = A^{-1} B for a sparse complex symmetric A (torch.autograd).

Forward: bl_cocr_rq (Algorithm 3) through the C ABI.  Backward, for the upstream
gradient G = dL/dconj(X) of a real loss L (PyTorch's conjugate-Wirtinger convention):

* grad_B = A^{-H} G.  Because A = A^T, A^{-H} G = conj(A^{-1} conj(G)): one more block
  solve with the same A and the same handle;
* grad_vals[e] = -sum_k Lambda_ik conj(X_jk) for the stored entry e = (i, j), with
  Lambda = grad_B (the sampled outer product, computed by blcoc_sampled_grad).

Both triangles of A are stored, so the values are independent parameters; a symmetric
perturbation of the pair (a_ij, a_ji) changes L by Re(conj(g_ij + g_ji) * delta).

Usage::

    op = SymmetricCSR(row_ptr, col_idx, n)          # pattern, device-resident
    X = blcoc_solve(vals, B, op)                     # vals: (nnz,) complex128, requires_grad
"""
from __future__ import annotations

import torch

from . import blcoc


class SymmetricCSR:
    """A fixed CSR pattern plus one solver handle whose values follow the tensor passed
    to each forward call."""

    def __init__(self, row_ptr, col_idx, n, vals0):
        self.n = int(n)
        self.nnz = int(len(col_idx))
        rp = torch.as_tensor(row_ptr, dtype=torch.int32).cuda().contiguous()
        ci = torch.as_tensor(col_idx, dtype=torch.int32).cuda().contiguous()
        v0 = torch.as_tensor(vals0, dtype=torch.complex128).cuda().contiguous()
        self.handle = blcoc.Handle(self.n, rp, ci, v0)
        self._keep = (rp, ci)

    def set_values(self, vals: torch.Tensor):
        self.handle.set_values(vals.detach().contiguous())

    def close(self):
        self.handle.close()


class _BlcocSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, B, op, method, tol, maxit):
        op.set_values(vals)
        Bc = B.detach().contiguous()
        X = torch.zeros_like(Bc)
        st = op.handle.solve(Bc, X, method=method, tol=tol, maxit=maxit)
        if st != blcoc.BLCOC_OK:
            raise blcoc.BlcocError(st, "forward solve: " + op.handle.last_error())
        ctx.op = op
        ctx.params = (method, tol, maxit)
        ctx.save_for_backward(vals, X)
        return X

    @staticmethod
    def backward(ctx, G):
        vals, X = ctx.saved_tensors
        op = ctx.op
        method, tol, maxit = ctx.params
        op.set_values(vals)
        Gc = G.conj_physical().contiguous()   # materialised: the C ABI reads raw memory
        Y = torch.zeros_like(Gc)
        st = op.handle.solve(Gc, Y, method=method, tol=tol, maxit=maxit)
        if st != blcoc.BLCOC_OK:
            raise blcoc.BlcocError(st, "adjoint solve: " + op.handle.last_error())
        Lam = Y.conj_physical().contiguous()
        grad_vals = None
        if ctx.needs_input_grad[0]:
            grad_vals = torch.empty_like(vals, memory_format=torch.contiguous_format)
            op.handle.sampled_grad(Lam, X, grad_vals)
        grad_B = Lam if ctx.needs_input_grad[1] else None
        return grad_vals, grad_B, None, None, None, None


def blcoc_solve(vals: torch.Tensor, B: torch.Tensor, op: SymmetricCSR, method: str = "cocr_rq", tol: float = 1e-12,
                maxit: int | None = None) -> torch.Tensor:
    """Differentiable X = A(vals)^{-1} B (device tensors, complex128)."""
    return _BlcocSolve.apply(vals, B, op, method, tol, op.n if maxit is None else int(maxit))
