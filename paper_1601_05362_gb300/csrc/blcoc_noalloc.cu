// blcoc_residual_norm_noalloc: ||B - A X||_F without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool or allocator
// is locked by its owner, hooks that must not grow the process's device footprint, and
// code that runs inside another library's allocation-free section.  This entry point
// serves them.  It takes the CSR arrays and the blocks as caller-owned device pointers
// (no handle, because creating a handle allocates) and keeps its only scratch - one
// partial sum pair per CTA - in the file-scope device array below.
//
// The array is BLCOC_NOALLOC_MAX_CTAS * 2 doubles (16 KB).  Every GPU that loads the
// library holds it until the process exits.  The grid of the row pass is capped at
// BLCOC_NOALLOC_MAX_CTAS CTAs, so any n works; each call overwrites exactly the slots it
// later reads, so nothing has to be cleared between calls, but all calls share the one
// array: two calls whose kernels overlap on the GPU (different streams, or different host
// threads) race on it.
//
// The paper has no counterpart of this entry point; the arithmetic is the true residual of
// Sec. 3, as computed by the norm-only residual pass of the solver.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/blcoc.h"
#include "blcoc_common.cuh"

namespace blcoc {

constexpr int NOALLOC_MAX_CTAS = BLCOC_NOALLOC_MAX_CTAS;

static __device__ __align__(256) double g_noalloc_partials[2 * NOALLOC_MAX_CTAS];

// Norm-only residual pass (variant of the solver's residual kernel): lanes = columns of
// a row, PP/32 rows per instruction; each CTA writes (sum |R|^2, sum |B|^2) to its slot.
template <int PP>
__global__ void __launch_bounds__(NWARP * 32)
    k_resid_norm_noalloc(int64_t n, const int* __restrict__ rp, const int* __restrict__ ci,
                         const double2* __restrict__ va, const double2* __restrict__ B,
                         const double2* __restrict__ X, int p, double* partials) {
  constexpr int LPR = PP < 32 ? PP : 32, RPI = 32 / LPR;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LPR, k = lane - sub * LPR;
  double sr = 0.0, sb = 0.0;
  const int64_t nchunks = (n + CHUNK - 1) / CHUNK;
  for (int64_t c = (int64_t)blockIdx.x * NWARP + warp; c < nchunks; c += (int64_t)gridDim.x * NWARP) {
    for (int rr = 0; rr < CHUNK; rr += RPI) {
      const int64_t row = c * CHUNK + rr + sub;
      if (row < n && k < p) {
        double2 acc = B[row * p + k];
        sb = fma(acc.x, acc.x, sb);
        sb = fma(acc.y, acc.y, sb);
        for (int j = rp[row]; j < rp[row + 1]; ++j) cmsub(acc, va[j], X[(int64_t)ci[j] * p + k]);
        sr = fma(acc.x, acc.x, sr);
        sr = fma(acc.y, acc.y, sr);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  __shared__ double red[2 * NWARP];
  if (lane == 0) {
    red[2 * warp] = sr;
    red[2 * warp + 1] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = red[0], b = red[1];
    for (int w = 1; w < NWARP; ++w) {
      a += red[2 * w];
      b += red[2 * w + 1];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// Fixed-order sum of the used slots; writes ||B - A X||_F to out[0].
__global__ void k_noalloc_finish(const double* partials, int nparts, double* out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += partials[2 * q];
  out[0] = sqrt(s);
}

namespace {
std::mutex g_setup_mutex;
double* g_scratch_addr[64] = {nullptr};   // device address of the array, per device
int g_num_sms[64] = {0};

template <int PP>
void launch_noalloc(int grid, int64_t n, const int* rp, const int* ci, const double2* va, const double2* B,
                    const double2* X, int p, double* scratch, cudaStream_t s) {
  k_resid_norm_noalloc<PP><<<grid, NWARP * 32, 0, s>>>(n, rp, ci, va, B, X, p, scratch);
}
}  // namespace

}  // namespace blcoc

using namespace blcoc;

extern "C" blcoc_status blcoc_residual_norm_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                                    const void* vals, const void* B, const void* X, int p,
                                                    double* norm_out, void* cuda_stream) {
  if (n < 1 || n >= ((int64_t)1 << 31)) {
    set_global_error("blcoc_residual_norm_noalloc: n must satisfy 1 <= n < 2^31");
    return BLCOC_ERR_INVALID_ARG;
  }
  if (p < 1 || p > BLCOC_MAX_P) {
    set_global_error("blcoc_residual_norm_noalloc: p must be in [1, BLCOC_MAX_P = 32]");
    return BLCOC_ERR_INVALID_ARG;
  }
  if (!row_ptr || !col_idx || !vals || !B || !X || !norm_out) {
    set_global_error("blcoc_residual_norm_noalloc: NULL pointer");
    return BLCOC_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BLCOC_ERR_CUDA;
  double* scratch = nullptr;
  int num_sms = 0;
  {
    // first call on a device: look up the device address of the static array
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr) {
        cudaGetLastError();
        set_global_error("blcoc_residual_norm_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return BLCOC_ERR_CUDA;
      }
      int sms = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return BLCOC_ERR_CUDA;
      g_scratch_addr[dev] = static_cast<double*>(ptr);
      g_num_sms[dev] = sms;
    }
    scratch = g_scratch_addr[dev];
    num_sms = g_num_sms[dev];
  }
  const int64_t nchunks = (n + CHUNK - 1) / CHUNK;
  int64_t grid = (nchunks + NWARP - 1) / NWARP;
  const int64_t cap = (int64_t)num_sms * 4 < NOALLOC_MAX_CTAS ? (int64_t)num_sms * 4 : NOALLOC_MAX_CTAS;
  if (grid > cap) grid = cap;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int* rp = row_ptr;
  const int* ci = col_idx;
  const double2* va = (const double2*)vals;
  const double2* b = (const double2*)B;
  const double2* x = (const double2*)X;
  const int g = (int)grid;
  if (p <= 1) launch_noalloc<1>(g, n, rp, ci, va, b, x, p, scratch, s);
  else if (p <= 2) launch_noalloc<2>(g, n, rp, ci, va, b, x, p, scratch, s);
  else if (p <= 4) launch_noalloc<4>(g, n, rp, ci, va, b, x, p, scratch, s);
  else if (p <= 8) launch_noalloc<8>(g, n, rp, ci, va, b, x, p, scratch, s);
  else if (p <= 16) launch_noalloc<16>(g, n, rp, ci, va, b, x, p, scratch, s);
  else launch_noalloc<32>(g, n, rp, ci, va, b, x, p, scratch, s);
  k_noalloc_finish<<<1, 32, 0, s>>>(scratch, g, norm_out);
  return cudaGetLastError() == cudaSuccess ? BLCOC_OK : BLCOC_ERR_CUDA;
}
