// One-CTA kernels of the p x p stages (bodies in blcoc_small_dev.cuh), the deterministic
// cross-CTA Gram reduction, and the CSR checks of blcoc_create.
#include "blcoc_small_dev.cuh"
#include "blcoc_small.h"

namespace blcoc {

// ------------------------------------------------------------------------ cross-CTA reduce
// stage1[s][c] = sum of partials[q][c] over q in slice s, in a fixed order: warp g of the
// CTA sums q = q0 + g, q0 + g + 4, ... in turn, and the four warp sums are combined as
// (a0 + a1) + (a2 + a3).  Each thread thus issues about nparts / 64 independent loads.
__global__ void __launch_bounds__(128) k_reduce_stage1(const double* __restrict__ partials, int nparts, int ncomp,
                                                       double* __restrict__ stage1, const Ctrl* ctrl, int fb_only) {
  if (ctrl != nullptr && ctrl->done) return;
  if (fb_only && ctrl != nullptr && ctrl->qr_fb == 0) return;
  __shared__ double part[4][32];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const int s = blockIdx.y;
  const int q0 = (int)((int64_t)s * nparts / RED_SPLIT), q1 = (int)((int64_t)(s + 1) * nparts / RED_SPLIT);
  double a = 0.0;
  if (c < ncomp)
    for (int q = q0 + g; q < q1; q += 4) a += partials[(int64_t)q * ncomp + c];
  part[g][lane] = a;
  __syncthreads();
  if (g == 0 && c < ncomp) stage1[(int64_t)s * ncomp + c] = (part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane]);
}

#define SMALL_PROLOGUE                                                  \
  extern __shared__ __align__(16) unsigned char small_raw[];            \
  SmallShared& S = *reinterpret_cast<SmallShared*>(small_raw);

__global__ void k_small_setup(int p, int method, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl,
                              int inner, int plain, uint2* oz, int qr2) {
  SMALL_PROLOGUE
  d_small_setup(S, p, method, stage1, ncomp, mats, ctrl, inner, plain, oz, qr2);
}

__global__ void k_small_cocr_H0(int p, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl) {
  SMALL_PROLOGUE
  d_small_cocr_H0(S, p, stage1, ncomp, mats, ctrl);
}

// CTA 0: the alpha' step; CTA 1 (cocr launches two): the elimination of H_m for the beta' step.
__global__ void k_small_alpha(int p, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl, double* hist,
                              int plain, uint2* oz) {
  SMALL_PROLOGUE
  if (blockIdx.x == 1) d_small_hfactor(S, p, mats, ctrl);
  else d_small_alpha(S, p, stage1, ncomp, mats, ctrl, hist, plain, oz);
}

// COND: cond is the handle of the conditional graph node that holds this iteration's
// shifted-CholQR3 fallback passes, set to run them only when the fallback has started.  A
// separate instantiation, because Nsight Compute leaves out of its profile every kernel
// that contains the device-side graph call, whether or not it runs.
template <bool COND>
__global__ void k_small_chol(int p, int method, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl,
                             int plain, uint2* oz, int qr2, unsigned long long cond) {
  SMALL_PROLOGUE
  d_small_chol(S, p, method, stage1, ncomp, mats, ctrl, plain, oz, qr2);
  if constexpr (COND) {
    if (threadIdx.x == 0)
      cudaGraphSetConditional((cudaGraphConditionalHandle)cond, BLCOC_LD(&ctrl->qr_fb) != 0 ? 1u : 0u);
  }
}

__global__ void k_small_chol2(int p, int method, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl,
                              int setup, uint2* oz) {
  SMALL_PROLOGUE
  d_small_chol2(S, p, method, stage1, ncomp, mats, ctrl, setup, oz);
}

// One CTA per group of columns of beta' (gridDim.x groups).
__global__ void k_small_chol_fb(int p, int method, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl,
                                int setup, uint2* oz) {
  SMALL_PROLOGUE
  d_small_chol_fb(S, p, method, stage1, ncomp, mats, ctrl, setup, oz);
}

__global__ void k_small_cocr_beta(int p, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl, uint2* oz) {
  SMALL_PROLOGUE
  const int per = (p + gridDim.x - 1) / gridDim.x;
  const int j0 = blockIdx.x * per, j1 = j0 + per < p ? j0 + per : p;
  if (j0 < j1) d_small_cocr_beta(S, p, stage1, ncomp, mats, ctrl, oz, j0, j1);
}

__global__ void k_small_trr(int p, const double* stage1, int ncomp, Ctrl* ctrl) {
  SMALL_PROLOGUE
  d_small_trr(S, p, stage1, ncomp, ctrl);
}

// ------------------------------------------------------------------------ CSR checks
// flags[0]: structure errors, flags[1]: symmetry errors.
__global__ void k_validate_structure(int64_t n, int64_t nnz, const int* rp, const int* ci, int* flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = rp[i], e = rp[i + 1];
  if (i == 0 && b != 0) atomicAdd(&flags[0], 1);
  if (i == n - 1 && e != nnz) atomicAdd(&flags[0], 1);
  if (b < 0 || e < b || e > nnz) {
    atomicAdd(&flags[0], 1);
    return;
  }
  for (int64_t j = b; j < e; ++j) {
    const int c = ci[j];
    if (c < 0 || c >= n || (j > b && c <= ci[j - 1])) {
      atomicAdd(&flags[0], 1);
      return;
    }
  }
}

// Requires a structurally valid matrix (checked first).
__global__ void k_validate_symmetry(int64_t n, const int* rp, const int* ci, const double2* va, double rtol,
                                    int* flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = rp[i]; j < rp[i + 1]; ++j) {
    const int c = ci[j];
    int lo = rp[c], hi = rp[c + 1] - 1, pos = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int cm = ci[mid];
      if (cm == (int)i) { pos = mid; break; }
      if (cm < (int)i) lo = mid + 1;
      else hi = mid - 1;
    }
    if (pos < 0) {
      atomicAdd(&flags[1], 1);
      return;
    }
    const double2 x = va[j], y = va[pos];
    const double d = hypot(x.x - y.x, x.y - y.y);
    const double s = fmax(hypot(x.x, x.y), hypot(y.x, y.y));
    if (!(d <= rtol * s)) {
      atomicAdd(&flags[1], 1);
      return;
    }
  }
}

// ------------------------------------------------------------------------ host launchers
static size_t small_smem() { return sizeof(SmallShared); }

static void set_small_attrs() {
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  const int s = (int)small_smem();
  cudaFuncSetAttribute(k_small_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_small_cocr_H0, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_small_alpha, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_small_chol<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_small_chol<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_small_chol2, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_small_chol_fb, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_small_cocr_beta, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_small_trr, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  done[dev] = true;
}

void prepare_small_kernels() { set_small_attrs(); }

void launch_reduce(const double2* partials, int nparts, int ne, double* stage1, const Ctrl* ctrl, cudaStream_t s,
                   bool fb_only) {
  const int ncomp = 2 * ne;
  dim3 grid((ncomp + 31) / 32, RED_SPLIT);
  k_reduce_stage1<<<grid, 128, 0, s>>>(reinterpret_cast<const double*>(partials), nparts, ncomp, stage1, ctrl,
                                       fb_only ? 1 : 0);
}

void launch_small(SmallKind kind, int p, int method, const double* stage1, int ne, double2* mats, Ctrl* ctrl,
                  double* hist, cudaStream_t s, uint2* oz, unsigned long long cond) {
  const size_t sm = small_smem();
  const int ncomp = 2 * ne;
  // method: 0 cocg / 1 cocr, +16 plain form, +32 CholQR2
  const int m = method & 15, plain = (method >> 4) & 1, qr2 = (method >> 5) & 1;
  switch (kind) {
    case SK_SETUP:
      k_small_setup<<<1, SMALL_THREADS, sm, s>>>(p, m, stage1, ncomp, mats, ctrl, 0, plain, oz, qr2);
      break;
    case SK_SETUP_INNER:
      k_small_setup<<<1, SMALL_THREADS, sm, s>>>(p, m, stage1, ncomp, mats, ctrl, 1, plain, oz, qr2);
      break;
    case SK_CHOL2: k_small_chol2<<<1, SMALL_THREADS, sm, s>>>(p, m, stage1, ncomp, mats, ctrl, 0, oz); break;
    case SK_CHOL2_SETUP: k_small_chol2<<<1, SMALL_THREADS, sm, s>>>(p, m, stage1, ncomp, mats, ctrl, 1, oz); break;
    case SK_CHOL_FB: k_small_chol_fb<<<1, SMALL_THREADS, sm, s>>>(p, m, stage1, ncomp, mats, ctrl, 0, oz); break;
    case SK_CHOL_FB_SETUP: k_small_chol_fb<<<1, SMALL_THREADS, sm, s>>>(p, m, stage1, ncomp, mats, ctrl, 1, oz); break;
    case SK_COCR_H0: k_small_cocr_H0<<<1, SMALL_THREADS, sm, s>>>(p, stage1, ncomp, mats, ctrl); break;
    case SK_ALPHA:
      k_small_alpha<<<m == 1 ? 2 : 1, SMALL_THREADS, sm, s>>>(p, stage1, ncomp, mats, ctrl, hist, plain, oz);
      break;
    case SK_CHOL:
      if (cond != 0) k_small_chol<true><<<1, SMALL_THREADS, sm, s>>>(p, m, stage1, ncomp, mats, ctrl, plain, oz, qr2, cond);
      else k_small_chol<false><<<1, SMALL_THREADS, sm, s>>>(p, m, stage1, ncomp, mats, ctrl, plain, oz, qr2, 0);
      break;
    case SK_COCR_BETA:   // a CTA per column; one CTA where the exact-slice form is emitted
      k_small_cocr_beta<<<oz != nullptr ? 1 : p, SMALL_THREADS, sm, s>>>(p, stage1, ncomp, mats, ctrl, oz);
      break;
    case SK_TRR: k_small_trr<<<1, SMALL_THREADS, sm, s>>>(p, stage1, ncomp, ctrl); break;
  }
}

void launch_validate(int64_t n, int64_t nnz, const int* rp, const int* ci, const double2* va, int* flags, int which,
                     cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (which == 0) k_validate_structure<<<blocks, threads, 0, s>>>(n, nnz, rp, ci, flags);
  else k_validate_symmetry<<<blocks, threads, 0, s>>>(n, rp, ci, va, 1e-12, flags);
}

}  // namespace blcoc
