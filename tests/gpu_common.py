"""Helpers shared by the GPU tests (not collected as tests)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_05362_gb300 import build
    build.build()
    return torch


def to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_iters_range(solve, A, B, tol, maxit, seeds=6):
    """Iteration counts the oracle itself reaches on B and on B perturbed by 1e-16
    relative (seeded): where the residual of an indefinite problem stagnates near tol,
    the step at which it first crosses moves by several iterations under rounding-level
    changes, so a GPU count is judged against this spread."""
    its = [solve(A, B, tol=tol, maxit=maxit).iters]
    for s in range(seeds):
        Bp = B * (1.0 + 1e-16 * np.random.default_rng(s).standard_normal(B.shape))
        its.append(solve(A, Bp, tol=tol, maxit=maxit).iters)
    return min(its), max(its)
