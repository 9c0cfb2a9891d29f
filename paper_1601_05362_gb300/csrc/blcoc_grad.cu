// Gradient support of the differentiable solve: the sampled outer product
//   dA_ij = - sum_k Lambda_ik conj(X_jk)   for every stored entry (i, j) of A,
// the derivative of a real loss through X = A^{-1} B with respect to the values of A
// (conjugate-Wirtinger convention), where Lambda = A^{-H} G is the adjoint solution.
#include <cuda_runtime.h>

#include "blcoc_common.cuh"

namespace blcoc {

// One warp per row i: the row's Lambda_i (p values) is read once per lane pair, lanes
// take the row's stored entries; lane l of a group handles entry j = beg + l.
__global__ void __launch_bounds__(256) k_sampled_grad(int64_t n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                      const double2* __restrict__ Lam, const double2* __restrict__ X,
                                                      int p, double2* __restrict__ out) {
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp_id; i < n; i += nwarps) {
    const int beg = rp[i], end = rp[i + 1];
    const double2* li = Lam + i * p;
    for (int e = beg + lane; e < end; e += 32) {
      const int64_t j = ci[e];
      const double2* xj = X + j * p;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < p; ++k) {
        const double2 l = __ldg(li + k), x = __ldg(xj + k);
        // acc += l * conj(x)
        acc.x = fma(l.x, x.x, acc.x);
        acc.x = fma(l.y, x.y, acc.x);
        acc.y = fma(l.y, x.x, acc.y);
        acc.y = fma(-l.x, x.y, acc.y);
      }
      out[e] = make_double2(-acc.x, -acc.y);
    }
  }
}

void launch_sampled_grad(int64_t n, const int* rp, const int* ci, const double2* Lam, const double2* X, int p,
                         double2* out, int num_sms, cudaStream_t s) {
  const int64_t warps = n < (int64_t)num_sms * 64 ? n : (int64_t)num_sms * 64;
  const int blocks = (int)((warps * 32 + 255) / 256);
  k_sampled_grad<<<blocks, 256, 0, s>>>(n, rp, ci, Lam, X, p, out);
}

}  // namespace blcoc
