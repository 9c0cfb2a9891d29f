// Shared device-side definitions of libblcoc: control block, small-matrix slots,
// complex FP64 arithmetic, and the launch-table type the host code dispatches on.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace blcoc {

constexpr int PMAX = 32;        // largest block width (right-hand sides)
constexpr int CHUNK = 32;       // rows per warp chunk: lane i of a warp owns row i
constexpr int NWARP = 4;        // warps per CTA in the row-pass kernels (one per SMSP)
constexpr int RED_SPLIT = 16;   // first-stage slices of the cross-CTA Gram reduction
constexpr int SMALL_THREADS = 256;

// Loads of data that another CTA of the same launch may have written (blocks, factors,
// partial sums, the control block).  The translation unit of the persistent batched
// kernel defines BLCOC_COHERENT_LOADS before including this header: such loads then read
// L2 (ld.global.cg) and can never be served by the non-coherent read-only path or by a
// stale L1 line of an earlier phase.  Everywhere else they are plain loads.
#ifdef BLCOC_COHERENT_LOADS
#define BLCOC_LD(ptr) __ldcg(ptr)
#else
#define BLCOC_LD(ptr) (*(ptr))
#endif

// Device-resident control block of one solve.  Kernels of an iteration return at once
// when `done` is non-zero, so a batch of queued iterations past convergence is a no-op.
struct Ctrl {
  int done;       // 0 running, 1 converged, 2 iteration limit, 3 breakdown
  int iter;       // m: X holds X_m
  int maxit;
  int bd_code;    // breakdown site: 1 setup QR, 2 alpha solve, 3 QR, 4 beta solve, 5 non-finite xi
  int nhist;      // entries of the residual history written so far
  int hlu_ok;     // cocr: the LU factors of H_m in slots M_HLU (beside the alpha' step) are valid
  int qr_fb;      // shifted-CholQR3 fallback: re-orthogonalising passes still to run (0: none)
  int qr_fb_on;   // the fallback is enabled for this solve (rq methods, single-pass Cholesky QR)
  double tol;
  double nb;      // ||B||_F
  double relres;  // ||xi_iter||_F / ||B||_F
  double trr;     // ||B - A X||_F (after the final residual pass)
  double sumsq_b; // sum |B_ij|^2 (setup)
  double pad[2];
  double qr_shift; // fallback shift coefficient 11 (n p + p (p + 1)) u (times trace(W^H W))
  int fb_count;    // shifted-CholQR3 fallbacks started in this solve
};

// PassArgs::flag bit shared with the host: the row pass runs only while a shifted-CholQR3
// fallback is in progress (Ctrl::qr_fb > 0); the other bits are in blcoc_rowpass.cuh.
constexpr int F_FB = 32;
// PassArgs::flag bit: the residual pass also forms R^T R, the CholQR2 pass also Q1^T Q1.
constexpr int F_SYM2 = 2;

// p x p complex matrices live in one device array of slots, each PMAX*PMAX entries,
// row-major with row stride p (dense p x p in the first p*p entries).
enum MatSlot {
  M_XI = 0,      // xi_m
  M_TAU,         // tau_{m+1} (upper triangular, real positive diagonal)
  M_TINV,        // T = tau^{-1} of the current W (Q = W T)
  M_ALPHA,       // alpha'_m
  M_ALPHAXI,     // alpha'_m xi_m
  M_BETA,        // beta'_m
  M_H,           // cocr: H_m = Q_m^T V_m;  cocg: G_QQ = Q_m^T Q_m
  M_G1,          // spare
  // Three-product forms of the factors the FP64 row passes apply (T, alpha', alpha'xi,
  // beta'): entry (k, j) of M = Mr + i Mi is kept as Mr and (Mr + Mi, Mi - Mr), so that a
  // complex product y M costs three real products (Gauss): with s = y.re + y.im,
  //   re(y M) = s Mr - y.im (Mr + Mi),   im(y M) = s Mr + y.re (Mi - Mr).
  // Each form takes two slots: (Mr + Mi, Mi - Mr) pairs in the first, Mr in the first half
  // of the second; row stride p like the complex slots.
  M3_TINV = 8,
  M3_ALPHA = 10,
  M3_ALPHAXI = 12,
  M3_BETA = 14,
  M_HLU = 16,    // cocr: H_m after elimination with partial pivoting (multipliers below the
                 // diagonal, the pivot-scaled rows above), formed beside the alpha' step;
                 // slot 17: the pivots' reciprocals (entries 0..p-1) and rows (entries PMAX..)
  M_NSLOTS = 18
};

// Slot of the three-product form of a factor slot (-1: none kept).
__host__ __device__ constexpr int m3_slot(int slot) {
  return slot == M_TINV ? M3_TINV : slot == M_ALPHA ? M3_ALPHA : slot == M_ALPHAXI ? M3_ALPHAXI
                                                                   : slot == M_BETA ? M3_BETA : -1;
}

// Gram layouts in the partial buffers: "tri" = upper triangle a <= b, row-major
// (p(p+1)/2 entries); "full" = p*p row-major.
__host__ __device__ inline int tri_count(int p) { return p * (p + 1) / 2; }

// ----------------------------------------------------------------------------- complex
__device__ __forceinline__ double2 cz() { return make_double2(0.0, 0.0); }

// complex element type of a working precision: double -> double2, float -> float2
template <typename S> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };
template <typename C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
// conversions between the working precision and the FP64 factors / FP64 results
template <typename C> __device__ __forceinline__ C from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }

// acc += a * b  (4 DFMA)
__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
__device__ __forceinline__ void cmsub(double2& acc, double2 a, double2 b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cmac_conj(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// single-precision counterparts (complex64 working precision)
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmsub(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(-a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmac_conj(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// ----------------------------------------------------------------------------- launch table
struct CsrDev {
  int64_t n;
  int64_t nnz;
  const int* rp;
  const int* ci;
  const double2* va;
  const float2* vaf;   // complex64 copy of the values (mixed-precision inner solves)
};

struct PassArgs {
  CsrDev A;
  int p;
  double2* W;
  double2* S;
  double2* U;
  double2* V;         // cocr: V;  cocg: A S
  double2* Q;         // Q = W T of the current basis, written by the last pass of an iteration
  double2* X;
  const double2* B;
  const double2* mats;
  double2* partials;  // [grid][ne]
  const uint2* oz;    // exact-slice fragments of the p x p factors (tensor-core applies)
  int ne;             // partial entries per CTA
  Ctrl* ctrl;
  int flag;           // kernel-specific switch (first pass / apply T / norm only / cocg grams)
  int grid;
};

using LaunchFn = void (*)(const PassArgs&, cudaStream_t);

// Row-pass kernels for one compile-time block width PP (p <= PP).
struct KernelSet {
  LaunchFn resid;        // R = B - A X; grams R^H R (+ R^T R if flag&2); norms; flag&1: norm only
  LaunchFn spmm_gram;    // Y = A W; gram W^T Y; out = Y T (flag=1) or Y (flag=0)
  LaunchFn spmm_plain;   // Y = A W (no gram), for blcoc_spmm
  LaunchFn cocr_passA;   // W <- Q - U alpha'; gram W^H W
  LaunchFn cocr_passC;   // Q = W T (stored); X += S alpha'xi; S = Q + S beta'; U = V + U beta'; gram U^T U
  LaunchFn cocg_pass1;   // W <- Q - (AS) alpha'; X += S alpha'xi; grams W^H W, W^T W
  LaunchFn cocg_pass2;   // Q = W T (stored); S <- Q + S beta'
  LaunchFn axpy;         // X (FP64) += D (working precision), the refinement update
  LaunchFn qr2;          // CholQR2 second pass: W <- W T (stored); gram W^H W
  LaunchFn spmm_gram_s2; // spmm_gram with 2 / 4 lane groups splitting each row's nonzeros
  LaunchFn spmm_gram_s4; // (nullptr where the row bundle would be wider than a warp)
  int (*grid)(int64_t n, int kind, int num_sms);
  void (*prepare)();     // set the dynamic shared-memory limits (once per device)
};

// S = double: the FP64 path; S = float: complex64 working precision for the inner solves
// of the mixed-precision refinement (the residual pass stays FP64 and writes its R in
// complex64, the Grams are summed in FP64, the p x p stages are the FP64 kernels).
template <int PP, typename S = double> const KernelSet& kernel_set();
// FP64 path whose p x p applies run on the bf16 tensor cores by exact slicing (PP 8, 16)
template <int PP> const KernelSet& kernel_set_tc();

// Sets the message blcoc_last_error(NULL) returns (calling thread only).
void set_global_error(const char* msg);

}  // namespace blcoc
