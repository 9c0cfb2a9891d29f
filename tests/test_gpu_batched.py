"""Batched solves (blcoc_solve_batched): many independent systems of uneven n and p.

* without autotuning the launch shape equals the single solve's, so every system's
  iterate, iteration count and history must equal a separate blcoc_solve bit for bit;
* with autotuning (grids sized for fewer SMs: the cross-CTA reduction order changes)
  every system must still converge to the tolerance with the oracle-parity history
  bound (1e-8 for m <= 20) against its separate solve.
"""
import numpy as np
import pytest

from paper_1601_05362_gb300 import problems as P
from gpu_common import need_gpu, to_dev

pytestmark = pytest.mark.gpu


def _batch(torch, count=10):
    from paper_1601_05362_gb300 import blcoc
    probs = P.helmholtz2d_batch(count, seed=5, side_range=(20, 72), k_range=(3.0, 9.0))
    hs = [blcoc.Handle.from_csr(pr.A) for pr in probs]
    Bs = [to_dev(torch, pr.B) for pr in probs]
    return probs, hs, Bs


def _separate(torch, hs, Bs):
    out = []
    for h, B in zip(hs, Bs):
        X = torch.zeros_like(B)
        assert h.solve(B, X, tol=1e-10, maxit=5000) == 0
        out.append((X.cpu().numpy(), h.info()))
    return out


def test_batched_equals_separate_solves_bitwise():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    probs, hs, Bs = _batch(torch)
    ref = _separate(torch, hs, Bs)
    Xs = [torch.zeros_like(B) for B in Bs]
    st, ms, msg = blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=5000, autotune=False)
    assert st == blcoc.BLCOC_OK
    assert ms > 0
    for (Xr, ir), X, h in zip(ref, Xs, hs):
        info = h.info()
        assert info["iters"] == ir["iters"]
        assert np.array_equal(X.cpu().numpy(), Xr)
        assert np.array_equal(info["hist"], ir["hist"])
    for h in hs:
        h.close()


def test_batched_autotuned_converges():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    probs, hs, Bs = _batch(torch, 12)
    ref = _separate(torch, hs, Bs)
    Xs = [torch.zeros_like(B) for B in Bs]
    st, ms, msg = blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=5000, autotune=True)
    assert st == blcoc.BLCOC_OK
    assert msg.startswith("autotuned launch shape")
    for (Xr, ir), X, h in zip(ref, Xs, hs):
        info = h.info()
        assert info["relres_true"] <= 1e-9
        m = min(21, len(ir["hist"]), len(info["hist"]))
        assert np.max(np.abs(info["hist"][:m] - ir["hist"][:m]) / ir["hist"][:m]) < 1e-8
        assert abs(info["iters"] - ir["iters"]) <= max(3, ir["iters"] // 20)
    for h in hs:
        h.close()


def test_batched_rejects_shared_handles():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    probs, hs, Bs = _batch(torch, 2)
    Xs = [torch.zeros_like(B) for B in Bs]
    with pytest.raises(blcoc.BlcocError):
        blcoc.solve_batched([hs[0], hs[0]], [Bs[0], Bs[0]], Xs[:1] * 2)
    for h in hs:
        h.close()


def test_batched_cholqr2_equals_separate_solves_bitwise():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    probs, hs, Bs = _batch(torch, 6)
    for h in hs:
        h.set_option("qr_passes", 2)
    ref = _separate(torch, hs, Bs)
    Xs = [torch.zeros_like(B) for B in Bs]
    st, ms, msg = blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=5000, autotune=False)
    assert st == blcoc.BLCOC_OK
    for (Xr, ir), X, h in zip(ref, Xs, hs):
        assert h.info()["iters"] == ir["iters"]
        assert np.array_equal(X.cpu().numpy(), Xr)
    with pytest.raises(blcoc.BlcocError):   # the persistent form runs single-pass Cholesky QR only
        blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=5000, autotune=False, persistent=True)
    for h in hs:
        h.close()


def test_batched_honours_tensor_core_and_explicit_u_options():
    """Per-handle options (fp64_tc, u_explicit) apply to that system in a batch exactly as
    in a separate blcoc_solve: the batch equals separate solves bit for bit."""
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    probs = P.helmholtz2d_batch(8, seed=7, side_range=(20, 60), k_range=(3.0, 9.0), p_choices=(4, 8, 16))
    hs = [blcoc.Handle.from_csr(pr.A) for pr in probs]
    Bs = [to_dev(torch, pr.B) for pr in probs]
    for i, h in enumerate(hs):
        h.set_option("fp64_tc", 1)
        h.set_option("u_explicit", i % 2)
    ref = _separate(torch, hs, Bs)
    Xs = [torch.zeros_like(B) for B in Bs]
    st, ms, msg = blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=5000, autotune=False)
    assert st == blcoc.BLCOC_OK
    for (Xr, ir), X, h in zip(ref, Xs, hs):
        assert h.info()["iters"] == ir["iters"]
        assert np.array_equal(X.cpu().numpy(), Xr)
        assert h.info()["relres_true"] <= 1e-9
    with pytest.raises(blcoc.BlcocError):
        blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=5000, autotune=False, persistent=True)
    for h in hs:
        h.close()


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_of_config_sized_systems_matches_oracle(persistent):
    """Systems of the 64-system batch workload itself (2D Helmholtz, seed 3): the largest
    grid sides it draws (up to 512, n up to 262,144) together with small ones, through
    the CUDA-graph batch and the persistent kernel at a fixed iteration count, each system
    against the oracle: history <= 1e-8 and X_m <= 1e-10 relative."""
    torch = need_gpu()
    import oracle.blcoc_oracle as O
    from paper_1601_05362_gb300 import blcoc
    from gpu_common import rel
    allp = P.helmholtz2d_batch(64)
    big = sorted(range(64), key=lambda i: -allp[i].n)[:3]
    small = sorted(range(64), key=lambda i: allp[i].n)[:2]
    pick = [allp[i] for i in big + small if allp[i].p <= 16]
    m = 10
    hs = [blcoc.Handle.from_csr(pr.A) for pr in pick]
    Bs = [to_dev(torch, pr.B) for pr in pick]
    Xs = [torch.zeros_like(B) for B in Bs]
    st, _, _ = blcoc.solve_batched(hs, Bs, Xs, tol=0.0, maxit=m, autotune=False, persistent=persistent)
    assert st == blcoc.BLCOC_NOT_CONVERGED
    assert max(pr.extra["side"] for pr in pick) >= 500
    for pr, h, X in zip(pick, hs, Xs):
        ref = O.bl_cocr_rq(pr.A.to_scipy(), pr.B, tol=0.0, maxit=m)
        info = h.info()
        assert info["iters"] == m
        assert np.max(np.abs(info["hist"] - np.array(ref.hist)) / np.array(ref.hist)) < 1e-8, pr.name
        assert rel(X.cpu().numpy(), ref.X) < 1e-10, pr.name
        h.close()


@pytest.mark.parametrize("conditional", [0, 1])
def test_batched_graph_runs_the_qr_fallback_like_separate_solves(conditional):
    """Tiny systems near finite termination lose rank to the single-pass Cholesky QR's
    resolution (one of these 40 does at iteration 6); blcoc_solve then completes the QR as
    shifted CholQR3 and converges.  The graph form runs the same fallback per handle, so
    every system equals its separate solve bit for bit, with the same status."""
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    tiny = P.helmholtz2d_batch(40, seed=11, side_range=(6, 14), k_range=(2.0, 5.0))

    def run(batched):
        hs = [blcoc.Handle.from_csr(pr.A) for pr in tiny]
        for h in hs:
            h.set_option("graph_conditional", conditional)
        Bs = [to_dev(torch, pr.B) for pr in tiny]
        Xs = [torch.zeros_like(B) for B in Bs]
        if batched:
            st, _, _ = blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=30, autotune=False)
            sts = None
        else:
            sts = [h.solve(B, X, tol=1e-10, maxit=30) for h, B, X in zip(hs, Bs, Xs)]
            st = max(sts)
        out = [(X.cpu().numpy(), h.info()) for X, h in zip(Xs, hs)]
        for h in hs:
            h.close()
        return st, sts, out

    st_g, _, graph = run(True)
    st_s, sts, sep = run(False)
    assert st_g == st_s
    for (Xg, ig), (Xs_, is_) in zip(graph, sep):
        assert ig["iters"] == is_["iters"]
        assert np.array_equal(Xg, Xs_) and np.array_equal(ig["hist"], is_["hist"])


@pytest.mark.parametrize("method", ["cocr_rq", "cocg_rq"])
def test_fallback_inside_the_graph_matches_direct_launches(method):
    """In the iterations' CUDA graph (option graph_conditional) the shifted-CholQR3 fallback
    is a conditional node that the Cholesky stage enables only when needed; launched
    directly its kernels run every iteration and return at once.  Both give the same bits, iteration count and number of
    fallbacks, and (bl_cocr_rq) at least one of these tiny systems does fall back."""
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    tiny = P.helmholtz2d_batch(40, seed=11, side_range=(6, 14), k_range=(2.0, 5.0))
    fell = 0
    for pr in tiny:
        out = []
        for graph in (1, 0):
            h = blcoc.Handle.from_csr(pr.A)
            h.set_option("graph", graph)
            h.set_option("graph_conditional", graph)
            B = to_dev(torch, pr.B)
            X = torch.zeros_like(B)
            st = h.solve(B, X, method=method, tol=1e-10, maxit=30, check=False)
            out.append((st, X.cpu().numpy(), h.info()["iters"], h.stat("qr_fallbacks")))
            h.close()
        (s1, X1, i1, f1), (s0, X0, i0, f0) = out
        assert (s1, i1, f1) == (s0, i0, f0)
        assert np.array_equal(X1, X0)
        fell += f1 > 0
    if method == "cocr_rq":
        assert fell >= 1
