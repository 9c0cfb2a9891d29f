"""The allocation-free residual norm (blcoc_residual_norm_noalloc).

Callers that cannot allocate device memory (their allocator or memory pool is held, or
they run inside another library's allocation-free section) use this entry point: it
takes raw device CSR arrays instead of a handle and keeps its scratch in a static device
array.  The test calls it through the C ABI twice in a row and checks it against the
handle-based blcoc_residual_norm and against ||B - A X||_F formed on the host with
numpy/scipy, within the tolerance the residual-norm test uses, and checks that the calls
leave the device's free memory unchanged.  It lives in its own file so that pytest
collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1601_05362_gb300 import problems as P
from gpu_common import need_gpu, to_dev

pytestmark = pytest.mark.gpu

RTOL = 1e-13   # as in test_gpu_parity.test_residual_norm


@pytest.mark.parametrize("shape", [("2d", 45, 3), ("2d", 45, 16), ("3d", 64, 16)])
def test_noalloc_residual_norm_matches_handle_version(shape):
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    lib = blcoc.load_library()
    kind, N, p = shape
    A = P.helmholtz_2d(N, 5.0, 0.05) if kind == "2d" else P.helmholtz_3d_absorbing(N, 20.0)
    B = to_dev(torch, P.complex_normal(A.n, p, 11))
    X = to_dev(torch, P.complex_normal(A.n, p, 12))
    with blcoc.Handle.from_csr(A) as h:
        ref = h.residual_norm(B, X)
    Bh, Xh = B.cpu().numpy(), X.cpu().numpy()
    ref_host = float(np.linalg.norm(Bh - A.to_scipy() @ Xh))
    rp, ci, va = to_dev(torch, A.row_ptr), to_dev(torch, A.col_idx), to_dev(torch, A.vals)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    def call():
        return lib.blcoc_residual_norm_noalloc(A.n, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), B.data_ptr(),
                                               X.data_ptr(), p, out.data_ptr(), stream)

    # a first call may load the library's kernel module (lazy module loading), which
    # takes device memory once per process; the calls after it must take none
    assert call() == blcoc.BLCOC_OK, lib.blcoc_last_error(None)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    values = []
    for _ in range(2):
        out.fill_(-1.0)
        st = call()
        assert st == blcoc.BLCOC_OK, lib.blcoc_last_error(None)
        torch.cuda.synchronize()
        values.append(float(out.item()))
    assert torch.cuda.mem_get_info()[0] == free_before   # no device memory taken by the calls
    for v in values:
        assert abs(v - ref) <= RTOL * ref, (v, ref)
        assert abs(v - ref_host) <= RTOL * ref_host, (v, ref_host)
    assert values[0] == values[1]          # fixed-order reduction: the same bits every call


def test_noalloc_rejects_out_of_range_sizes():
    torch = need_gpu()
    from paper_1601_05362_gb300 import blcoc
    lib = blcoc.load_library()
    A = P.helmholtz_2d(10, 3.0, 0.05)
    rp, ci, va = to_dev(torch, A.row_ptr), to_dev(torch, A.col_idx), to_dev(torch, A.vals)
    B = to_dev(torch, P.complex_normal(A.n, 4, 1))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n, p in ((A.n, 33), (A.n, 0), (0, 4), (1 << 31, 4)):
        st = lib.blcoc_residual_norm_noalloc(n, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), B.data_ptr(),
                                             B.data_ptr(), p, out.data_ptr(), 0)
        assert st == blcoc.BLCOC_ERR_INVALID_ARG
        assert lib.blcoc_last_error(None).decode().startswith("blcoc_residual_norm_noalloc")
