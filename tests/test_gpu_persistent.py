"""Persistent batched solves (blcoc_solve_batched_persistent): every system's iterations in
one kernel launch whose CTAs take the stages' work items from a ring queue.

* parity: a batch of uneven systems (ragged n, p from 1 to 16) run for a fixed number of
  iterations matches the CPU oracle system by system (history <= 1e-8 relative for
  m <= 20, X <= 1e-10 relative), for both rq methods;
* a repeated batch is bitwise identical (fixed reduction order);
* a converged batch equals separate blcoc_solve calls bit for bit (each system's row
  passes run as the virtual grid of its single solve), under every autotuned shape;
* a wait for work that can never be satisfied (test hook: no first item is published)
  gives up after its time limit and the call returns BLCOC_ERR_TIMEOUT, after which the
  same handles solve normally.
"""
import numpy as np
import pytest

import oracle.blcoc_oracle as O
from paper_1601_05362_gb300 import problems as P
from gpu_common import need_gpu, to_dev, rel

pytestmark = pytest.mark.gpu

HIST_TOL = 1e-8
X_TOL = 1e-10
SIZES = [(700, 1), (1531, 3), (2304, 4), (999, 8), (3001, 13), (1777, 16), (64, 2)]


def _systems(seed0=0):
    out = []
    for i, (n, p) in enumerate(SIZES):
        A = P.random_complex_symmetric(n, 8, seed=400 + seed0 + i, diag=3.0 + 0.6j, scale=0.25)
        Bh = P.complex_normal(n, p, 500 + seed0 + i)
        out.append((A, Bh))
    return out


@pytest.mark.parametrize("method", ["cocg_rq", "cocr_rq"])
def test_persistent_fixed_iterations_match_oracle(method):
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    systems = _systems()
    m = 12
    f = O.bl_cocg_rq if method == "cocg_rq" else O.bl_cocr_rq
    refs = [f(A.to_scipy(), Bh, tol=0.0, maxit=m) for A, Bh in systems]
    hs = [blcoc.Handle.from_csr(A) for A, _ in systems]
    Bs = [to_dev(torch, Bh) for _, Bh in systems]
    Xs = [torch.zeros_like(B) for B in Bs]
    st, ms, msg = blcoc.solve_batched(hs, Bs, Xs, method=method, tol=0.0, maxit=m, autotune=False, persistent=True)
    assert st == blcoc.BLCOC_NOT_CONVERGED, msg
    for ref, X, h in zip(refs, Xs, hs):
        info = h.info()
        assert info["iters"] == m
        assert np.max(np.abs(info["hist"] - np.array(ref.hist)) / np.array(ref.hist)) < HIST_TOL
        assert rel(X.cpu().numpy(), ref.X) < X_TOL
    for h in hs:
        h.close()


def test_persistent_repeat_is_bitwise_identical():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    systems = _systems(20)
    hs = [blcoc.Handle.from_csr(A) for A, _ in systems]
    Bs = [to_dev(torch, Bh) for _, Bh in systems]
    runs = []
    for _ in range(2):
        Xs = [torch.zeros_like(B) for B in Bs]
        st, ms, msg = blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=400, autotune=False, persistent=True)
        assert st == blcoc.BLCOC_OK, msg
        runs.append(([X.cpu().numpy() for X in Xs], [h.info() for h in hs]))
    for X0, X1 in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(X0, X1)
    for i0, i1 in zip(runs[0][1], runs[1][1]):
        assert i0["iters"] == i1["iters"]
        assert np.array_equal(i0["hist"], i1["hist"])
    for h in hs:
        h.close()


@pytest.mark.parametrize("method", ["cocg_rq", "cocr_rq"])
@pytest.mark.parametrize("autotune", [False, True])
def test_persistent_batch_equals_separate_solves_bitwise(method, autotune):
    """Every system's row passes run as the virtual grid of its own single solve, so the
    reduction order is the same and the batch must reproduce separate blcoc_solve calls bit
    for bit, under every launch shape the autotuner tries."""
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    probs = P.helmholtz2d_batch(10, seed=5, side_range=(20, 72), k_range=(3.0, 9.0))
    hs = [blcoc.Handle.from_csr(pr.A) for pr in probs]
    Bs = [to_dev(torch, pr.B) for pr in probs]
    ref = []
    for h, B in zip(hs, Bs):
        X = torch.zeros_like(B)
        assert h.solve(B, X, method=method, tol=1e-10, maxit=5000) == 0
        ref.append((X.cpu().numpy(), h.info()))
    # autotuning: successive calls time the candidate grid sizes, then keep the fastest
    for call in range(4 if autotune else 1):
        Xs = [torch.zeros_like(B) for B in Bs]
        st, ms, msg = blcoc.solve_batched(hs, Bs, Xs, method=method, tol=1e-10, maxit=5000, autotune=autotune,
                                          persistent=True)
        assert st == blcoc.BLCOC_OK, msg
        assert msg.startswith("persistent kernel"), msg
        assert ms > 0
        assert hs[0].stat("persistent_graph") in (0, 1)
        for (Xr, ir), X, h in zip(ref, Xs, hs):
            info = h.info()
            assert info["iters"] == ir["iters"]
            assert np.array_equal(info["hist"], ir["hist"])
            assert np.array_equal(X.cpu().numpy(), Xr)
            assert info["relres_true"] == ir["relres_true"]
    if autotune:
        assert msg.endswith("autotuned"), msg
    for h in hs:
        h.close()


def test_persistent_barrier_time_limit_returns_timeout():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    systems = _systems(40)[:3]
    hs = [blcoc.Handle.from_csr(A) for A, _ in systems]
    Bs = [to_dev(torch, Bh) for _, Bh in systems]
    Xs = [torch.zeros_like(B) for B in Bs]
    hs[0].set_option("persistent_timeout_ms", 50)
    hs[0].set_option("persistent_stall", 1)
    with pytest.raises(blcoc.BlcocError) as e:
        blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=200, autotune=False, persistent=True)
    assert e.value.status == blcoc.BLCOC_ERR_TIMEOUT
    hs[0].set_option("persistent_stall", 0)
    Xs = [torch.zeros_like(B) for B in Bs]
    st, _, msg = blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=400, autotune=False, persistent=True)
    assert st == blcoc.BLCOC_OK, msg
    for h in hs:
        assert h.info()["relres_true"] <= 1e-9
        h.close()


def test_persistent_rejects_wide_blocks():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    A = P.random_complex_symmetric(300, 6, seed=1, diag=3.0 + 0.6j, scale=0.25)
    h = blcoc.Handle.from_csr(A)
    B = to_dev(torch, P.complex_normal(300, 17, 2))
    X = torch.zeros_like(B)
    with pytest.raises(blcoc.BlcocError):
        blcoc.solve_batched([h], [B], [X], persistent=True)
    h.close()


def test_persistent_edge_cases_match_graph_form_bitwise():
    """A zero right-hand side (stopped at setup), a system that reaches maxit, a one-system
    batch, and 40 tiny systems (the ticket ring wraps around many times): every system
    equals the graph-branch form and a separate solve bit for bit, with the same status."""
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    specs = [(900, 3, "zero"), (1200, 4, "ok"), (700, 2, "ok")]
    systems = []
    for i, (n, p, kind) in enumerate(specs):
        A = P.random_complex_symmetric(n, 8, seed=600 + i, diag=3.0 + 0.6j, scale=0.25)
        Bh = P.complex_normal(n, p, 700 + i) * (0.0 if kind == "zero" else 1.0)
        systems.append((A, Bh))
    hard = P.helmholtz2d_batch(1, seed=9, side_range=(60, 60), k_range=(20.0, 20.0))[0]
    systems.append((hard.A, hard.B))                      # needs far more than 30 iterations
    tiny = P.helmholtz2d_batch(40, seed=11, side_range=(6, 14), k_range=(2.0, 5.0))
    systems += [(pr.A, pr.B) for pr in tiny]
    maxit = 30

    def run(form):
        hs = [blcoc.Handle.from_csr(A) for A, _ in systems]
        for h in hs:   # the persistent kernel has no shifted-CholQR3 fallback: compare without it
            h.set_option("qr_fallback", 0)
        Bs = [to_dev(torch, Bh) for _, Bh in systems]
        Xs = [torch.zeros_like(B) for B in Bs]
        if form == "separate":
            sts = [h.solve(B, X, tol=1e-10, maxit=maxit) for h, B, X in zip(hs, Bs, Xs)]
            st = max(sts)
        else:
            st, _, _ = blcoc.solve_batched(hs, Bs, Xs, tol=1e-10, maxit=maxit, autotune=False,
                                           persistent=(form == "persistent"))
        out = [(X.cpu().numpy(), h.info()) for X, h in zip(Xs, hs)]
        for h in hs:
            h.close()
        return st, out

    st_p, pers = run("persistent")
    st_g, graph = run("graph")
    _, sep = run("separate")
    assert st_p == st_g == blcoc.BLCOC_NOT_CONVERGED          # the Helmholtz system hits maxit
    assert not pers[0][0].any() and pers[0][1]["iters"] == 0   # B = 0: X = 0 at once
    assert pers[3][1]["iters"] == maxit
    for (Xp, ip), (Xg, ig), (Xs_, is_) in zip(pers, graph, sep):
        assert ip["iters"] == ig["iters"] == is_["iters"]
        assert np.array_equal(Xp, Xg) and np.array_equal(Xp, Xs_)
        assert np.array_equal(ip["hist"], ig["hist"]) and np.array_equal(ip["hist"], is_["hist"])


def test_persistent_single_system_equals_solve():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    pr = P.helmholtz2d_n1024_p4("cocr_rq")
    h = blcoc.Handle.from_csr(pr.A)
    B = to_dev(torch, pr.B)
    X1 = torch.zeros_like(B)
    assert h.solve(B, X1, tol=1e-10, maxit=500) == blcoc.BLCOC_OK
    i1 = h.info()
    X2 = torch.zeros_like(B)
    st, _, msg = blcoc.solve_batched([h], [B], [X2], tol=1e-10, maxit=500, autotune=False, persistent=True)
    assert st == blcoc.BLCOC_OK, msg
    assert np.array_equal(X1.cpu().numpy(), X2.cpu().numpy())
    assert h.info()["iters"] == i1["iters"]
    h.close()
