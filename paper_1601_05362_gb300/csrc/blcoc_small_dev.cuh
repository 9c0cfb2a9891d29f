// Device code of the p x p stages of bl_cocg_rq / bl_cocr_rq (Algorithms 2-3, Sec. 2.2):
// every stage is a function of one CTA (any block size) on a SmallShared workspace.  The
// one-CTA kernels of blcoc_small.cu and the persistent batched kernel both call them.
//
// The p x p systems are complex symmetric, not Hermitian (their matrices are bilinear
// Grams Y^T Z), so they are solved by LU with partial pivoting (pivot = largest
// |re| + |im| in the column, ties to the lowest row).  The thin QR of the residual
// block is a Cholesky QR: tau^H tau = W^H W with tau upper triangular and a real
// positive diagonal, T = tau^{-1}.
#pragma once
#include "blcoc_common.cuh"
#include "blcoc_ozaki.cuh"

namespace blcoc {
namespace {

// Leading dimension of the p x p matrices in shared memory (the largest p a stage can
// take).  A translation unit that only runs p <= 16 defines BLCOC_SMALL_LD 16 first and
// gets a workspace a quarter the size.
#ifndef BLCOC_SMALL_LD
#define BLCOC_SMALL_LD PMAX
#endif
constexpr int LD = BLCOC_SMALL_LD;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ bool cfinite(double2 z) { return isfinite(z.x) && isfinite(z.y); }

// Second stage, inside the small kernels: gs[c] = sum_s stage1[s][c].
__device__ void sum_stage1(const double* stage1, int ncomp, double* gs) {
  static_assert(RED_SPLIT % 4 == 0, "stage-1 slices are summed four at a time");
  for (int c = threadIdx.x; c < ncomp; c += blockDim.x) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int s = 0; s < RED_SPLIT; ++s) a[s & 3] += BLCOC_LD(stage1 + (int64_t)s * ncomp + c);
    gs[c] = (a[0] + a[1]) + (a[2] + a[3]);
  }
  __syncthreads();
}

// 1/d for a positive double: the hardware's reciprocal estimate refined by two Newton
// steps r <- r (2 - d r), each of which squares the relative error (the estimate's ~2^-22
// becomes far below an ulp); d outside [1e-300, 1e300] takes a division.  Used where a
// division would sit on a long sequential chain (pivots of the p x p factorisations).
__device__ __forceinline__ double recip_pos(double d) {
  if (!(d > 1e-300 && d < 1e300)) return 1.0 / d;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

__device__ __forceinline__ void tri_decode(int e, int p, int& a, int& b) {
  int aa = 0, rem = e;
  while (rem >= p - aa) { rem -= p - aa; ++aa; }
  a = aa;
  b = aa + rem;
}

// Triangle (upper, row-major) -> full p x p; herm: M[b][a] = conj(M[a][b]).
__device__ void expand_tri(const double* gs, double2* M, int p, bool herm) {
  const int E = tri_count(p);
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    int a, b;
    tri_decode(e, p, a, b);
    const double2 v = make_double2(gs[2 * e], gs[2 * e + 1]);
    M[a * LD + b] = v;
    if (a != b) M[b * LD + a] = herm ? make_double2(v.x, -v.y) : v;
  }
  __syncthreads();
}

__device__ void gload(double2* s, const double2* g, int p) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) s[(e / p) * LD + e % p] = BLCOC_LD(g + e);
  __syncthreads();
}
__device__ void gstore(double2* __restrict__ g, const double2* s, int p) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) g[e] = s[(e / p) * LD + e % p];
  __syncthreads();
}

// C = op(A) op(B), op = transpose (no conjugation) when the flag is set; C must not alias.
// Every entry runs the full k range even where an operand is triangular: the zero half
// contributes exact zeros, and on GB300 an FP64 warp instruction costs the same with idle
// lanes, so a uniform loop is the faster one.  Even and odd k go to two accumulators.
__device__ void matmul(double2* C, const double2* A, bool tA, const double2* B, bool tB, int p) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    double2 acc0 = cz(), acc1 = cz();
    int k = 0;
    for (; k + 2 <= p; k += 2) {
      cmac(acc0, tA ? A[k * LD + i] : A[i * LD + k], tB ? B[j * LD + k] : B[k * LD + j]);
      cmac(acc1, tA ? A[(k + 1) * LD + i] : A[i * LD + k + 1], tB ? B[j * LD + k + 1] : B[(k + 1) * LD + j]);
    }
    if (k < p) cmac(acc0, tA ? A[k * LD + i] : A[i * LD + k], tB ? B[j * LD + k] : B[k * LD + j]);
    C[i * LD + j] = make_double2(acc0.x + acc1.x, acc0.y + acc1.y);
  }
  __syncthreads();
}

// Columns [j0, j1) of C = op(A) B (op = transpose without conjugation when tA): each entry
// is four partial sums over k = g, g + 4, ... (g = 0..3, one lane each, in turn) combined
// by an xor butterfly as (s0 + s1) + (s2 + s3) - the same value whatever range of columns
// a CTA takes, so one CTA per column and one CTA for all columns agree bit for bit.
__device__ void matmul_cols(double2* C, const double2* A, bool tA, const double2* B, int p, int j0, int j1) {
  const int nc = j1 - j0, items = p * nc * 4;
  for (int base = threadIdx.x & ~31; base < ((items + 31) & ~31); base += blockDim.x) {
    const int it = base + (threadIdx.x & 31);
    const int g = it & 3, ent = it >> 2;
    const int i = ent / nc, j = j0 + (ent - (ent / nc) * nc);
    double2 acc = cz();
    if (it < items)
      for (int k = g; k < p; k += 4) cmac(acc, tA ? A[k * LD + i] : A[i * LD + k], B[k * LD + j]);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
    if (it < items && g == 0) C[i * LD + j] = acc;
  }
  __syncthreads();
}

// ||M||_F in a fixed order that does not depend on the block size (the one-CTA kernels and
// the persistent kernel run these stages with different block sizes and must agree bit for
// bit): lane l of warp 0 sums entries l, l + 32, ... in turn, then a fixed butterfly.
__device__ double fro_norm(const double2* M, int p, double* red) {
  if (threadIdx.x < 32) {
    double acc = 0.0;
    for (int e = threadIdx.x; e < p * p; e += 32) {
      const double2 v = M[(e / p) * LD + e % p];
      acc += v.x * v.x + v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) red[32] = sqrt(acc);
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

// Right-looking Cholesky of a Hermitian G (upper triangle used, destroyed): tau^H tau = G.
// Per step warp 0 forms the pivot's inverse square root and row j of tau, then all threads
// update the trailing triangle: two barriers per step.
// Breakdown (returns false): a pivot that is not finite or not above 64 eps times G's
// original diagonal entry, i.e. column j of the block keeps less than about 1.2e-7 of its
// norm outside the span of the columns before it - below that a Cholesky QR cannot
// resolve the column (its error grows like cond^2 eps), and the block has lost rank to
// working accuracy.
__device__ bool chol_upper(double2* G, double2* tau, int p, double* sh) {
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) tau[e] = cz();
  __syncthreads();
  // warp 0: lane l keeps the original diagonal entry l (p <= 32); G's diagonal entry j is
  // first changed by step j - 1's update, after every lane read it here
  const double g0 = (threadIdx.x < 32 && (int)threadIdx.x < p) ? G[threadIdx.x * LD + threadIdx.x].x : 0.0;
  for (int j = 0; j < p; ++j) {
    if (threadIdx.x < 32) {
      const double d = G[j * LD + j].x;
      const double g0j = __shfl_sync(0xffffffffu, g0, j);
      const bool ok = d > 0x1p-46 * g0j && d > 0.0 && isfinite(d);
      if (ok) {
        const double ir = rsqrt(d);
        for (int i = j + 1 + threadIdx.x; i < p; i += 32) {
          const double2 g = G[j * LD + i];
          tau[j * LD + i] = make_double2(g.x * ir, g.y * ir);
        }
        if (threadIdx.x == 0) tau[j * LD + j] = make_double2(d * ir, 0.0);
      }
      if (threadIdx.x == 0) sh[0] = ok ? 1.0 : 0.0;
    }
    __syncthreads();
    if (sh[0] == 0.0) return false;
    const int m = p - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, l = j + 1 + e % m;
      if (l >= i) {
        const double2 ti = tau[j * LD + i], tl = tau[j * LD + l];
        double2 g = G[i * LD + l];
        // g -= conj(ti) * tl
        g.x -= ti.x * tl.x + ti.y * tl.y;
        g.y -= ti.x * tl.y - ti.y * tl.x;
        G[i * LD + l] = g;
      }
    }
    __syncthreads();
  }
  return true;
}

// T = tau^{-1} for upper-triangular tau with real positive diagonal, all columns at once by
// column-oriented back substitution: T starts as I; for k = p-1 .. 1 row k is final, and
// every entry (i < k, j >= k) subtracts tau_ik T_kj with T_kj = acc_kj / tau_kk formed on the
// fly (one barrier per k); the rows are scaled by 1 / tau_ii at the end.
__device__ void tri_inv_upper(const double2* tau, double2* T, int p, double* dinv) {
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
    const int i = e / LD, j = e - i * LD;
    T[e] = make_double2((i == j && i < p) ? 1.0 : 0.0, 0.0);
  }
  for (int i = threadIdx.x; i < p; i += blockDim.x) dinv[i] = recip_pos(tau[i * LD + i].x);
  __syncthreads();
  for (int k = p - 1; k > 0; --k) {
    const int w = p - k;
    const double dk = dinv[k];
    for (int e = threadIdx.x; e < k * w; e += blockDim.x) {
      const int i = e / w, j = k + (e - i * w);
      const double2 a = T[k * LD + j];
      cmsub(T[i * LD + j], tau[i * LD + k], make_double2(a.x * dk, a.y * dk));
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e - i * p;
    if (j >= i) {
      const double d = dinv[i];
      const double2 t = T[i * LD + j];
      T[i * LD + j] = make_double2(t.x * d, t.y * d);
    }
  }
  __syncthreads();
}

// Pivot key of a complex entry for the warp argmax: the high 32 bits of max(|re|, |im|)
// (for non-negative doubles the bit pattern orders like the value), whose 5 lowest bits
// are replaced by 31 - row, so that one 32-bit warp max picks the largest magnitude and,
// among magnitudes equal in their leading 15 mantissa bits, the lowest row.
__device__ __forceinline__ unsigned piv_key(double2 z, int row) {
  const unsigned hx = (unsigned)((unsigned long long)__double_as_longlong(z.x) >> 32) & 0x7FFFFFFFu;
  const unsigned hy = (unsigned)((unsigned long long)__double_as_longlong(z.y) >> 32) & 0x7FFFFFFFu;
  return ((hx > hy ? hx : hy) & ~31u) | (unsigned)(31 - row);
}

// 1/z = conj(z) / |z|^2 for a pivot.
__device__ __forceinline__ double2 crecip_piv(double2 z) {
  const double r = recip_pos(fma(z.x, z.x, z.y * z.y));
  return make_double2(z.x * r, -z.y * r);
}

// Solve M Z = R in place (R <- Z), Gaussian elimination with partial pivoting; M is
// destroyed.  Pivot: the largest max(|re|, |im|) in the column (piv_key).  Breakdown: a
// pivot that is not finite or not above 64 eps times the largest max(|re|, |im|) of M
// (M is singular to working accuracy).  Step k: warp 0 finds the pivot row
// while each of its lanes forms the reciprocal of its own candidate, then swaps rows k
// and piv (columns >= k of M, all of R) and scales the new row k by the pivot's reciprocal
// in one pass, a column per lane; all threads then subtract M_ik x row k from every row
// below.  Two barriers per step; the eliminated system has a unit upper triangle, so the
// back substitution is one multiply-subtract per entry and step.  p <= 32.
// piv / pinv (shared memory, optional): the pivot row and the pivot's reciprocal of each
// step, for lu_replay.
__device__ bool lu_solve(double2* M, double2* R, int p, int nrhs, double* sh, int* ish, int* piv = nullptr,
                         double2* pinvs = nullptr) {
  const int lane = threadIdx.x & 31;
  // breakdown threshold as a pivot key: the key of M's largest entry with its exponent
  // lowered by 46 (64 eps = 2^-46); every warp-0 lane computes it
  unsigned thr = 0u;
  if (threadIdx.x < 32) {
    unsigned mx = 0u;
    for (int e = lane; e < p * p; e += 32) mx = max(mx, piv_key(M[(e / p) * LD + e % p], 31) & ~31u);
    mx = __reduce_max_sync(0xffffffffu, mx);
    thr = ((mx >> 20) & 0x7FFu) > 46u ? mx - (46u << 20) : 0u;
  }
  for (int k = 0; k < p; ++k) {
    if (threadIdx.x < 32) {
      const bool cand = lane >= k && lane < p;
      const double2 z = cand ? M[lane * LD + k] : cz();
      const unsigned key = cand ? piv_key(z, lane) : 0u;
      const double2 zr = crecip_piv(cand ? z : make_double2(1.0, 0.0));
      const unsigned best = __reduce_max_sync(0xffffffffu, key);
      const int bi = 31 - (int)(best & 31u);
      const bool ok = (best & ~31u) > thr && ((best >> 20) & 0x7FFu) != 0x7FFu && bi >= k && bi < p;
      double2 pinv;
      pinv.x = __shfl_sync(0xffffffffu, zr.x, bi & 31);
      pinv.y = __shfl_sync(0xffffffffu, zr.y, bi & 31);
      __syncwarp();   // every lane has read its candidate before rows k and piv change
      if (ok) {
        const int nm = p - k;
        for (int c = lane; c < nm + nrhs; c += 32) {
          double2* pk = c < nm ? M + k * LD + k + c : R + k * LD + (c - nm);
          double2* pb = c < nm ? M + bi * LD + k + c : R + bi * LD + (c - nm);
          const double2 a = *pb, b = *pk;
          const double2 sc = cmul(a, pinv);
          if (bi != k) *pb = b;
          *pk = c == 0 ? a : sc;   // column k keeps the pivot (not read again)
        }
      }
      if (lane == 0) {
        ish[1] = ok ? 1 : 0;
        if (piv != nullptr) {
          piv[k] = bi;
          pinvs[k] = pinv;
        }
      }
    }
    __syncthreads();
    if (!ish[1]) return false;
    const int m = p - k - 1, w = m + nrhs;
    for (int e = threadIdx.x; e < m * w; e += blockDim.x) {
      const int i = k + 1 + e / w, c = e % w;
      const double2 l = M[i * LD + k];
      if (c < m) cmsub(M[i * LD + k + 1 + c], l, M[k * LD + k + 1 + c]);
      else cmsub(R[i * LD + (c - m)], l, R[k * LD + (c - m)]);
    }
    __syncthreads();
  }
  // back substitution with the unit upper triangle: row k of R is final at step k
  for (int k = p - 1; k > 0; --k) {
    for (int e = threadIdx.x; e < k * nrhs; e += blockDim.x) {
      const int i = e / nrhs, c = e - i * nrhs;
      cmsub(R[i * LD + c], M[i * LD + k], R[k * LD + c]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < p * nrhs; e += blockDim.x)
    if (!cfinite(R[(e / nrhs) * LD + e % nrhs])) ish[1] = 0;
  __syncthreads();
  return ish[1] != 0;
}

// Columns [j0, j1) of R <- M^{-1} R from the elimination lu_solve recorded (F: M after
// lu_solve, piv / pinvs: its pivots): the same swaps, scalings and multiply-subtracts in the
// same order, so every column is bitwise what lu_solve would have made of it.
__device__ void lu_replay(const double2* F, const int* piv, const double2* pinvs, double2* R, int p, int j0, int j1) {
  const int nc = j1 - j0;
  for (int k = 0; k < p; ++k) {
    const int b = piv[k];
    for (int c = j0 + threadIdx.x; c < j1; c += blockDim.x) {
      const double2 a = R[b * LD + c];
      if (b != k) R[b * LD + c] = R[k * LD + c];
      R[k * LD + c] = cmul(a, pinvs[k]);
    }
    __syncthreads();
    const int m = p - k - 1;
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
      const int i = k + 1 + e / nc, c = j0 + e % nc;
      cmsub(R[i * LD + c], F[i * LD + k], R[k * LD + c]);
    }
    __syncthreads();
  }
  for (int k = p - 1; k > 0; --k) {
    for (int e = threadIdx.x; e < k * nc; e += blockDim.x) {
      const int i = e / nc, c = j0 + e % nc;
      cmsub(R[i * LD + c], F[i * LD + k], R[k * LD + c]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------ shared layout
struct SmallShared {
  double gs[2 * (2 * LD * (LD + 1) / 2 + 2)];
  double red[2 * PMAX + 8];
  double2 pinvs[LD];
  int piv[LD];
  int ish[4];
  int colexp[64];
  double2 m[6][LD * LD];
};

// Exact-slice fragments of a p x p factor (smem, stride LD) for the tensor-core applies.
__device__ void emit_oz(uint2* oz, int slot, const double2* M, int p, int* sh) {
  if (oz == nullptr) return;
  uint2* f = oz + slot * OZ_SLOT_U2;
  if (p <= 8) oz_emit_factor<8>(M, LD, p, f, oz_colexp_of(f), sh);
  else if (p <= 16) oz_emit_factor<16>(M, LD, p, f, oz_colexp_of(f), sh);
  else oz_emit_factor<32>(M, LD, p, f, oz_colexp_of(f), sh);
}

__device__ __forceinline__ double2* slot(double2* mats, int s) { return mats + s * PMAX * PMAX; }

// A factor the row passes apply, from shared memory to its slot together with its
// three-product form (the pairs (Mr + Mi, Mi - Mr) and Mr).
__device__ void gstore_fac(double2* mats, int sl, const double2* s, int p) {
  double2* g = slot(mats, sl);
  double2* sd = slot(mats, m3_slot(sl));
  double* r = reinterpret_cast<double*>(slot(mats, m3_slot(sl) + 1));
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const double2 v = s[(e / p) * LD + e % p];
    g[e] = v;
    sd[e] = make_double2(v.x + v.y, v.y - v.x);
    r[e] = v.x;
  }
  __syncthreads();
}

// Columns [j0, j1) of a p x p matrix from shared memory to its slot (and, for a factor the
// row passes apply, to its three-product form).
__device__ void gstore_cols(double2* mats, int sl, const double2* s, int p, int j0, int j1) {
  double2* g = slot(mats, sl);
  const int s3 = m3_slot(sl);
  const int nc = j1 - j0;
  for (int e = threadIdx.x; e < p * nc; e += blockDim.x) {
    const int i = e / nc, j = j0 + (e - (e / nc) * nc);
    const double2 v = s[i * LD + j];
    g[i * p + j] = v;
    if (s3 >= 0) {
      slot(mats, s3)[i * p + j] = make_double2(v.x + v.y, v.y - v.x);
      reinterpret_cast<double*>(slot(mats, s3 + 1))[i * p + j] = v.x;
    }
  }
  __syncthreads();
}

// Cholesky factor of the Hermitian Gram in S.gs (its triangle): tau^H tau = G, tau in
// S.m[1].  With the fallback on (ctrl->qr_fb_on), a factorisation that fails the pivot test
// is retried on G + s I with s = ctrl->qr_shift * trace(G) >= 11 (n p + p(p+1)) u ||W||_2^2,
// the shift of shifted CholQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa), which
// makes the factorisation succeed for any W of condition below about u^-1; the two
// Cholesky QR passes that complete it then run (ctrl->qr_fb = 2, stage d_small_chol_fb).
// Returns 0 (failed: breakdown), 1 (plain Cholesky QR) or 2 (shifted: fallback started).
__device__ int chol_gram(SmallShared& S, int p, Ctrl* ctrl) {
  expand_tri(S.gs, S.m[0], p, true);
  if (chol_upper(S.m[0], S.m[1], p, S.red)) return 1;
  if (!BLCOC_LD(&ctrl->qr_fb_on) || !(ctrl->qr_shift > 0.0)) return 0;
  expand_tri(S.gs, S.m[0], p, true);
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int j = 0; j < p; ++j) tr += S.m[0][j * LD + j].x;
    S.red[0] = ctrl->qr_shift * tr;
  }
  __syncthreads();
  const double sh = S.red[0];
  __syncthreads();
  for (int j = threadIdx.x; j < p; j += blockDim.x) S.m[0][j * LD + j].x += sh;
  __syncthreads();
  if (!chol_upper(S.m[0], S.m[1], p, S.red)) return 0;
  if (threadIdx.x == 0) {
    ctrl->qr_fb = 2;
    ctrl->fb_count += 1;
  }
  __syncthreads();
  return 2;
}

// Setup after the residual pass: ||B||_F, Q_0 xi_0 = R_0 (Cholesky QR), T_0 = xi_0^{-1};
// cocg: G_QQ = Q_0^T Q_0 = T^T (R^T R) T.
// inner = 1 (refinement step): the stopping test is relative to ||R_0||_F, the norm of
// this solve's right-hand side, which is the outer residual.
__device__ __noinline__ void d_small_setup(SmallShared& S, int p, int method, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl,
                              int inner, int plain, uint2* oz, int qr2 = 0) {
  if (BLCOC_LD(&ctrl->done)) return;
  sum_stage1(stage1, ncomp, S.gs);
  const int E = tri_count(p);
  const double sb = inner ? S.gs[2 * (2 * E) + 1] : S.gs[2 * (2 * E)];
  if (threadIdx.x == 0) {
    ctrl->sumsq_b = sb;
    ctrl->nb = sqrt(sb);
    ctrl->trr = sqrt(S.gs[2 * (2 * E) + 1]);
    ctrl->pad[0] = S.gs[2 * (2 * E)];   // sum |B|^2
  }
  if (!(sb > 0.0) || !isfinite(sb)) {
    if (threadIdx.x == 0) {
      ctrl->done = (sb == 0.0) ? 1 : 3;
      ctrl->bd_code = (sb == 0.0) ? 0 : 5;
    }
    return;
  }
  if (plain) {
    // plain block methods (Algorithm 1, derived block COCG): no orthonormalisation, so
    // tau = T = xi = I and the row passes reduce to the plain recurrences
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      const double2 v = (e / p == e % p) ? make_double2(1.0, 0.0) : cz();
      slot(mats, M_XI)[e] = v;
      slot(mats, M_TAU)[e] = v;
      slot(mats, M_TINV)[e] = v;
      slot(mats, M3_TINV)[e] = make_double2(v.x, -v.x);
      reinterpret_cast<double*>(slot(mats, M3_TINV + 1))[e] = v.x;
    }
    if (threadIdx.x == 0) ctrl->pad[1] = S.gs[2 * (2 * E) + 1];   // ||R_0||_F^2
    if (method == 0) {
      expand_tri(S.gs + 2 * E, S.m[3], p, false);
      gstore(slot(mats, M_H), S.m[3], p);                       // R_0^T R_0
    }
    return;
  }
  const int qr = chol_gram(S, p, ctrl);
  if (qr == 0) {
    if (threadIdx.x == 0) { ctrl->done = 3; ctrl->bd_code = 1; }
    return;
  }
  tri_inv_upper(S.m[1], S.m[2], p, S.red);
  gstore(slot(mats, M_XI), S.m[1], p);
  gstore_fac(mats, M_TINV, S.m[2], p);
  emit_oz(oz, OZ_T, S.m[2], p, S.colexp);
  if (method == 0) {
    expand_tri(S.gs + 2 * E, S.m[3], p, false);
    if (qr2 || qr == 2) return;   // G_QQ needs the final basis: the last second-factor stage forms it
    matmul(S.m[4], S.m[2], true, S.m[3], false, p);   // T^T G
    matmul(S.m[5], S.m[4], false, S.m[2], false, p);  // (T^T G) T
    gstore(slot(mats, M_H), S.m[5], p);
  }
}

// cocr setup after A Q_0: H_0 = Q_0^T V_0 = T^T (W^T A W) T.
__device__ __noinline__ void d_small_cocr_H0(SmallShared& S, int p, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl) {
  if (BLCOC_LD(&ctrl->done)) return;
  sum_stage1(stage1, ncomp, S.gs);
  expand_tri(S.gs, S.m[0], p, false);
  gload(S.m[1], slot(mats, M_TINV), p);
  matmul(S.m[2], S.m[1], true, S.m[0], false, p);
  matmul(S.m[3], S.m[2], false, S.m[1], false, p);
  gstore(slot(mats, M_H), S.m[3], p);
}

// Top of iteration m (Algorithms 2-3, the stopping test and the alpha' step): record
// ||xi_m||_F/||B||_F, stop if
// <= tol or m = maxit; else alpha'_m = G1^{-1} RHS with G1 = U^T U (cocr) or S^T A S
// (cocg) and RHS = Q^T V (cocr) or Q^T Q (cocg); also alpha'_m xi_m.
// plain: the stopping test uses ||R_m||_F (Algorithm 1) recorded by the previous stage.
__device__ __noinline__ void d_small_alpha(SmallShared& S, int p, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl, double* hist,
                              int plain, uint2* oz) {
  if (BLCOC_LD(&ctrl->done)) return;
  const int m = ctrl->iter;
  gload(S.m[0], slot(mats, M_XI), p);
  const double rel = (plain ? sqrt(ctrl->pad[1]) : fro_norm(S.m[0], p, S.red)) / ctrl->nb;
  if (threadIdx.x == 0) {
    hist[m] = rel;
    ctrl->relres = rel;
    ctrl->nhist = m + 1;
  }
  if (!isfinite(rel)) {
    if (threadIdx.x == 0) { ctrl->done = 3; ctrl->bd_code = 5; }
    return;
  }
  if (rel <= ctrl->tol) {
    if (threadIdx.x == 0) ctrl->done = 1;
    return;
  }
  if (m >= ctrl->maxit) {
    if (threadIdx.x == 0) ctrl->done = 2;
    return;
  }
  sum_stage1(stage1, ncomp, S.gs);
  expand_tri(S.gs, S.m[1], p, false);     // G1 (symmetric)
  gload(S.m[2], slot(mats, M_H), p);      // RHS
  if (!lu_solve(S.m[1], S.m[2], p, p, S.red, S.ish)) {
    if (threadIdx.x == 0) { ctrl->done = 3; ctrl->bd_code = 2; }
    return;
  }
  gstore_fac(mats, M_ALPHA, S.m[2], p);
  matmul(S.m[3], S.m[2], false, S.m[0], false, p);   // alpha' xi, xi upper triangular
  gstore_fac(mats, M_ALPHAXI, S.m[3], p);
  emit_oz(oz, OZ_ALPHA, S.m[2], p, S.colexp);
  emit_oz(oz, OZ_ALPHAXI, S.m[3], p, S.colexp);
  if (threadIdx.x == 0) ctrl->iter = m + 1;
}

// After W_{m+1} (Algorithms 2-3, the QR of the new residual block): Cholesky QR tau, T = tau^{-1},
// xi_{m+1} = tau xi_m.  cocg also does the beta' step: G_QQ+ = T^T (W^T W) T and
// beta' = G_QQ^{-1} tau^T G_QQ+.
// plain: no QR; record ||R_{m+1}||_F^2 (trace of the Hermitian Gram) and, for block COCG,
// beta = (R_m^T R_m)^{-1} R_{m+1}^T R_{m+1}.
__device__ __noinline__ void d_small_chol(SmallShared& S, int p, int method, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl,
                             int plain, uint2* oz, int qr2 = 0) {
  if (BLCOC_LD(&ctrl->done)) return;
  sum_stage1(stage1, ncomp, S.gs);
  if (plain) {
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0, e = 0; i < p; e += p - i, ++i) t += S.gs[2 * e];   // diagonal entries of the triangle
      ctrl->pad[1] = t;
    }
    if (method == 0) {
      const int E = tri_count(p);
      expand_tri(S.gs + 2 * E, S.m[0], p, false);      // R_{m+1}^T R_{m+1}
      gload(S.m[3], slot(mats, M_H), p);                // R_m^T R_m
      for (int e = threadIdx.x; e < p * p; e += blockDim.x) S.m[4][(e / p) * LD + e % p] = S.m[0][(e / p) * LD + e % p];
      __syncthreads();
      gstore(slot(mats, M_H), S.m[0], p);
      if (!lu_solve(S.m[3], S.m[4], p, p, S.red, S.ish)) {
        if (threadIdx.x == 0) { ctrl->done = 3; ctrl->bd_code = 4; }
        return;
      }
      gstore_fac(mats, M_BETA, S.m[4], p);
    }
    __syncthreads();
    return;
  }
  const int qr = chol_gram(S, p, ctrl);
  if (qr == 0) {
    if (threadIdx.x == 0) {
      ctrl->done = 3;
      ctrl->bd_code = 3;
      if (method == 1) ctrl->iter -= 1;   // cocr forms X_{m+1} only in the last pass
    }
    return;
  }
  tri_inv_upper(S.m[1], S.m[2], p, S.red);
  gload(S.m[3], slot(mats, M_XI), p);
  matmul(S.m[4], S.m[1], false, S.m[3], false, p);   // xi_{m+1} = tau xi_m
  gstore(slot(mats, M_XI), S.m[4], p);
  gstore(slot(mats, M_TAU), S.m[1], p);
  gstore_fac(mats, M_TINV, S.m[2], p);
  emit_oz(oz, OZ_T, S.m[2], p, S.colexp);
  if (method == 0) {
    const int E = tri_count(p);
    expand_tri(S.gs + 2 * E, S.m[0], p, false);       // W^T W
    if (qr2 || qr == 2) return;   // G_QQ+ and beta' need the final basis: the last second-factor stage forms them
    matmul(S.m[3], S.m[2], true, S.m[0], false, p);   // T^T (W^T W)
    matmul(S.m[0], S.m[3], false, S.m[2], false, p);  // G_QQ+ = T^T W^T W T
    matmul(S.m[4], S.m[1], true, S.m[0], false, p);   // tau^T G_QQ+
    gload(S.m[3], slot(mats, M_H), p);                // G_QQ (old)
    gstore(slot(mats, M_H), S.m[0], p);
    if (!lu_solve(S.m[3], S.m[4], p, p, S.red, S.ish)) {
      if (threadIdx.x == 0) { ctrl->done = 3; ctrl->bd_code = 4; }
      return;
    }
    gstore_fac(mats, M_BETA, S.m[4], p);
    emit_oz(oz, OZ_BETA, S.m[4], p, S.colexp);
  }
}

// CholQR2, second factor (after the pass W <- Q1 = W T1, Grams Q1^H Q1 and, for cocg,
// Q1^T Q1): tau2, T2 with tau2^H tau2 = Q1^H Q1; the QR factor becomes tau = tau2 tau1 and
// the passes that follow apply T2 to the stored Q1.  Iteration: xi_{m+1} <- tau2 xi_{m+1}
// (the first stage applied tau1).  Setup (setup = 1): xi_0 = tau.  cocg, on the last such
// stage (last = 1; the shifted-CholQR3 fallback has two): G_QQ (setup) or G_QQ+ and beta'
// (iteration) from T2^T (Q1^T Q1) T2.
__device__ __noinline__ void d_small_chol2(SmallShared& S, int p, int method, const double* stage1, int ncomp,
                                           double2* mats, Ctrl* ctrl, int setup, uint2* oz, int last = 1) {
  if (BLCOC_LD(&ctrl->done)) return;
  sum_stage1(stage1, ncomp, S.gs);
  expand_tri(S.gs, S.m[0], p, true);                   // Q1^H Q1
  if (!chol_upper(S.m[0], S.m[1], p, S.red)) {
    if (threadIdx.x == 0) {
      ctrl->done = 3;
      ctrl->bd_code = setup ? 1 : 3;
      if (!setup && method == 1) ctrl->iter -= 1;
    }
    return;
  }
  tri_inv_upper(S.m[1], S.m[2], p, S.red);            // T2
  gload(S.m[3], slot(mats, setup ? M_XI : M_TAU), p);  // tau1
  matmul(S.m[4], S.m[1], false, S.m[3], false, p);   // tau = tau2 tau1
  if (setup) {
    gstore(slot(mats, M_XI), S.m[4], p);
  } else {
    gstore(slot(mats, M_TAU), S.m[4], p);
    gload(S.m[5], slot(mats, M_XI), p);
    matmul(S.m[3], S.m[1], false, S.m[5], false, p);   // xi <- tau2 xi
    gstore(slot(mats, M_XI), S.m[3], p);
  }
  if (method == 0 && last) {
    // Q^T Q of the final basis Q = Q1 T2 from the pass's unconjugated Gram Q1^T Q1 (Q1 is
    // well conditioned, so no cond(W)^2 loss)
    expand_tri(S.gs + 2 * tri_count(p), S.m[3], p, false);
    matmul(S.m[5], S.m[2], true, S.m[3], false, p);
    matmul(S.m[0], S.m[5], false, S.m[2], false, p);  // T2^T (Q1^T Q1) T2
    if (setup) {
      gstore(slot(mats, M_H), S.m[0], p);                   // G_QQ
    } else {
      matmul(S.m[5], S.m[4], true, S.m[0], false, p); // tau^T G_QQ+
      gload(S.m[3], slot(mats, M_H), p);                    // G_QQ (old)
      gstore(slot(mats, M_H), S.m[0], p);
      if (!lu_solve(S.m[3], S.m[5], p, p, S.red, S.ish)) {
        if (threadIdx.x == 0) { ctrl->done = 3; ctrl->bd_code = 4; }
        return;
      }
      gstore_fac(mats, M_BETA, S.m[5], p);
      emit_oz(oz, OZ_BETA, S.m[5], p, S.colexp);
    }
  }
  gstore_fac(mats, M_TINV, S.m[2], p);
  emit_oz(oz, OZ_T, S.m[2], p, S.colexp);
}

// Shifted-CholQR3 fallback, one of its two Cholesky QR passes (after the row pass
// W <- W T_prev with Gram W^H W): the CholQR2 second-factor step (tau <- tau_k tau, xi
// updated, T_k stored for the passes that follow).  Runs only while ctrl->qr_fb > 0.  After
// the last pass the whole factor tau must keep its rank the way the oracle's Householder
// QR is judged: a diagonal entry below 1e-14 of the largest is a breakdown.
__device__ __noinline__ void d_small_chol_fb(SmallShared& S, int p, int method, const double* stage1, int ncomp,
                                             double2* mats, Ctrl* ctrl, int setup, uint2* oz) {
  const int fb = BLCOC_LD(&ctrl->qr_fb);
  if (BLCOC_LD(&ctrl->done) || fb == 0) return;
  d_small_chol2(S, p, method, stage1, ncomp, mats, ctrl, setup, oz, fb == 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int left = ctrl->qr_fb - 1;
    ctrl->qr_fb = left;
    if (left == 0 && !ctrl->done) {
      const double2* tau = slot(mats, setup ? M_XI : M_TAU);
      double dmax = 0.0, dmin = 1e308;
      for (int j = 0; j < p; ++j) {
        const double d = fabs(tau[j * p + j].x);
        dmax = fmax(dmax, d);
        dmin = fmin(dmin, d);
      }
      if (!(dmin > 1e-14 * dmax)) {
        ctrl->done = 3;
        ctrl->bd_code = setup ? 1 : 3;
        if (!setup && method == 1) ctrl->iter -= 1;
      }
    }
  }
}

// cocr, beside the alpha' step (Algorithm 3): the elimination of H_m = Q_m^T V_m (slot M_H,
// final here) for the beta' step that follows the next QR, so that the beta' step replays
// it instead of factorising on its critical path.  A singular H_m is recorded in the
// control block and reported by the beta' step as its breakdown, as a failed solve there
// would be.
__device__ __noinline__ void d_small_hfactor(SmallShared& S, int p, double2* mats, Ctrl* ctrl) {
  if (BLCOC_LD(&ctrl->done)) return;
  gload(S.m[1], slot(mats, M_H), p);
  const bool ok = lu_solve(S.m[1], nullptr, p, 0, S.red, S.ish, S.piv, S.pinvs);
  gstore(slot(mats, M_HLU), S.m[1], p);
  double2* aux = slot(mats, M_HLU + 1);
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    aux[k] = S.pinvs[k];
    aux[PMAX + k] = make_double2((double)S.piv[k], 0.0);
  }
  if (threadIdx.x == 0) ctrl->hlu_ok = ok ? 1 : 0;
}

// cocr after V_{m+1} (Algorithm 3, the beta' step), columns [j0, j1):
// H+ = T^T (W^T A W T) by matrix-vector products (matmul_cols), beta' = H_m^{-1} (tau^T H+)
// by replaying the elimination of H_m made beside the alpha' step.  A launch may split the
// columns over CTAs; only a launch whose CTA takes all columns emits the exact-slice form.
__device__ __noinline__ void d_small_cocr_beta(SmallShared& S, int p, const double* stage1, int ncomp, double2* mats,
                                               Ctrl* ctrl, uint2* oz, int j0, int j1) {
  if (BLCOC_LD(&ctrl->done)) return;
  if (!BLCOC_LD(&ctrl->hlu_ok)) {
    if (threadIdx.x == 0 && atomicCAS(&ctrl->done, 0, 3) == 0) {
      ctrl->bd_code = 4;
      ctrl->iter -= 1;
    }
    return;
  }
  sum_stage1(stage1, ncomp, S.gs);
  expand_tri(S.gs, S.m[0], p, false);                  // W^T A W
  gload(S.m[1], slot(mats, M_TINV), p);
  gload(S.m[4], slot(mats, M_TAU), p);
  gload(S.m[3], slot(mats, M_HLU), p);
  {
    const double2* aux = slot(mats, M_HLU + 1);
    for (int k = threadIdx.x; k < p; k += blockDim.x) {
      S.pinvs[k] = BLCOC_LD(aux + k);
      S.piv[k] = (int)BLCOC_LD(aux + PMAX + k).x;
    }
  }
  matmul_cols(S.m[2], S.m[0], false, S.m[1], p, j0, j1);   // (W^T A W) T
  matmul_cols(S.m[5], S.m[1], true, S.m[2], p, j0, j1);    // H+
  matmul_cols(S.m[2], S.m[4], true, S.m[5], p, j0, j1);    // tau^T H+
  lu_replay(S.m[3], S.piv, S.pinvs, S.m[2], p, j0, j1);    // beta'
  gstore_cols(mats, M_H, S.m[5], p, j0, j1);
  gstore_cols(mats, M_BETA, S.m[2], p, j0, j1);
  bool bad = false;
  for (int e = threadIdx.x; e < p * (j1 - j0); e += blockDim.x)
    if (!cfinite(S.m[2][(e / (j1 - j0)) * LD + j0 + e % (j1 - j0)])) bad = true;
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0 && atomicCAS(&ctrl->done, 0, 3) == 0) {
      ctrl->bd_code = 4;
      ctrl->iter -= 1;
    }
    return;
  }
  if (j0 == 0 && j1 == p) emit_oz(oz, OZ_BETA, S.m[2], p, S.colexp);
}

// Norm of the residual from a norm-only residual pass (Sec. 3, true residual).
__device__ __noinline__ void d_small_trr(SmallShared& S, int p, const double* stage1, int ncomp, Ctrl* ctrl) {
  sum_stage1(stage1, ncomp, S.gs);
  if (threadIdx.x == 0) {
    const int E = tri_count(p);
    ctrl->trr = sqrt(S.gs[2 * (2 * E) + 1]);
    ctrl->sumsq_b = S.gs[2 * (2 * E)];
  }
}

}  // namespace
}  // namespace blcoc
