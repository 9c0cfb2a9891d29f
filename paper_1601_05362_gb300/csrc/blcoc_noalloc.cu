// blcoc_residual_norm_noalloc: ||B - A X||_F without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool or allocator
// is locked by its owner, hooks that must not grow the process's device footprint, and
// code that runs inside another library's allocation-free section.  This entry point
// serves them.  It takes the CSR arrays and the blocks as caller-owned device pointers
// (no handle, because creating a handle allocates) and keeps its only scratch - one
// partial sum per CTA - in the file-scope device array below.
//
// The array is BLCOC_NOALLOC_MAX_CTAS doubles (8 KB).  Every GPU that loads the library
// holds it until the process exits.  The grid of the row pass is capped at
// BLCOC_NOALLOC_MAX_CTAS CTAs, so any n works; each call overwrites exactly the slots it
// later reads, so nothing has to be cleared between calls, but all calls share the one
// array: two calls whose kernels overlap on the GPU (different streams, or different host
// threads) race on it.
//
// The paper has no counterpart of this entry point; the arithmetic is the true residual of
// Sec. 3, as computed by the norm-only residual pass of the solver.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/blcoc.h"
#include "blcoc_common.cuh"

namespace blcoc {

constexpr int NOALLOC_MAX_CTAS = BLCOC_NOALLOC_MAX_CTAS;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_CTAS];

// Norm-only residual pass (variant of the solver's residual kernel): lanes = columns of
// a row, PP/32 rows per instruction; each CTA writes its sum |B - A X|^2 to its slot.
template <int PP>
__global__ void __launch_bounds__(NWARP * 32)
    k_resid_norm_noalloc(int64_t n, const int* __restrict__ rp, const int* __restrict__ ci,
                         const double2* __restrict__ va, const double2* __restrict__ B,
                         const double2* __restrict__ X, int p, double* partials) {
  constexpr int LPR = PP < 32 ? PP : 32, RPI = 32 / LPR;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LPR, k = lane - sub * LPR;
  double sr = 0.0;
  const int64_t nchunks = (n + CHUNK - 1) / CHUNK;
  for (int64_t c = (int64_t)blockIdx.x * NWARP + warp; c < nchunks; c += (int64_t)gridDim.x * NWARP) {
    for (int rr = 0; rr < CHUNK; rr += RPI) {
      const int64_t row = c * CHUNK + rr + sub;
      if (row < n && k < p) {
        double2 acc = B[row * p + k];
        for (int j = rp[row]; j < rp[row + 1]; ++j) cmsub(acc, va[j], X[(int64_t)ci[j] * p + k]);
        sr = fma(acc.x, acc.x, sr);
        sr = fma(acc.y, acc.y, sr);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) sr += __shfl_xor_sync(0xffffffffu, sr, o);
  __shared__ double red[NWARP];
  if (lane == 0) red[warp] = sr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = red[0];
    for (int w = 1; w < NWARP; ++w) a += red[w];
    partials[blockIdx.x] = a;
  }
}

// Fixed-order sum of the used slots; writes ||B - A X||_F to out[0].
__global__ void k_noalloc_finish(const double* partials, int nparts, double* out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += partials[q];
  out[0] = sqrt(s);
}

namespace {
std::mutex g_setup_mutex;
double* g_scratch_addr[64] = {nullptr};   // device address of the array, per device
int g_num_sms[64] = {0};

// Launches report their own status (cudaLaunchKernel returns it), so an error left
// behind by the caller's earlier work is neither returned nor cleared here.
template <int PP>
cudaError_t launch_noalloc(int grid, int64_t n, const int* rp, const int* ci, const double2* va, const double2* B,
                           const double2* X, int p, double* scratch, cudaStream_t s) {
  void* args[] = {&n, &rp, &ci, &va, &B, &X, &p, &scratch};
  return cudaLaunchKernel((const void*)&k_resid_norm_noalloc<PP>, dim3(grid), dim3(NWARP * 32), args, 0, s);
}

blcoc_status noalloc_cuda_error(const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "blcoc_residual_norm_noalloc: %s: %s", what, cudaGetErrorString(e));
  set_global_error(buf);
  return BLCOC_ERR_CUDA;
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
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_cuda_error("cudaGetDevice", e);
  if (dev < 0 || dev >= 64) {
    set_global_error("blcoc_residual_norm_noalloc: device index out of the supported range [0, 64)");
    return BLCOC_ERR_CUDA;
  }
  double* scratch = nullptr;
  int num_sms = 0;
  {
    // first call on a device: look up the device address of the static array
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
      if (e != cudaSuccess || !ptr) return noalloc_cuda_error("cudaGetSymbolAddress of the scratch array", e);
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return noalloc_cuda_error("cudaDeviceGetAttribute", e);
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
  int g = (int)grid;
  if (p <= 1) e = launch_noalloc<1>(g, n, rp, ci, va, b, x, p, scratch, s);
  else if (p <= 2) e = launch_noalloc<2>(g, n, rp, ci, va, b, x, p, scratch, s);
  else if (p <= 4) e = launch_noalloc<4>(g, n, rp, ci, va, b, x, p, scratch, s);
  else if (p <= 8) e = launch_noalloc<8>(g, n, rp, ci, va, b, x, p, scratch, s);
  else if (p <= 16) e = launch_noalloc<16>(g, n, rp, ci, va, b, x, p, scratch, s);
  else e = launch_noalloc<32>(g, n, rp, ci, va, b, x, p, scratch, s);
  if (e != cudaSuccess) return noalloc_cuda_error("row pass launch", e);
  const double* sc = scratch;
  void* fargs[] = {&sc, &g, &norm_out};
  e = cudaLaunchKernel((const void*)&k_noalloc_finish, dim3(1), dim3(32), fargs, 0, s);
  if (e != cudaSuccess) return noalloc_cuda_error("final sum launch", e);
  return BLCOC_OK;
}
