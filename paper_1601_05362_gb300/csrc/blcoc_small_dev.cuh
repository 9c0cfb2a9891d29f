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
__device__ __forceinline__ double2 crecip(double2 z) {
  const double d = z.x * z.x + z.y * z.y;
  return make_double2(z.x / d, -z.y / d);
}
__device__ __forceinline__ double cabs1(double2 z) { return fabs(z.x) + fabs(z.y); }
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

// Reciprocal of a positive finite double by Newton's iteration r <- r (2 - d r) from a
// single-precision start (two steps: ~48 correct bits -> within 1 ulp).  Used where a
// division would sit on a long sequential chain (pivots of the p x p factorisations).
// d = m 2^e is split with integer operations so that the float start never leaves the
// float range; exponents near the ends of the double range fall back to a division.
__device__ __forceinline__ double recip_pos(double d) {
  const long long bits = __double_as_longlong(d);
  const int ex = (int)((bits >> 52) & 0x7FF) - 1023;
  if (ex < -1000 || ex > 1000) return 1.0 / d;
  const double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);  // [1, 2)
  double r = (double)__frcp_rn((float)m);
  double e = fma(-m, r, 1.0);
  r = fma(r, e, r);
  e = fma(-m, r, 1.0);
  r = fma(r, e, r);
  return r * __longlong_as_double((long long)(1023 - ex) << 52);   // exact scaling by 2^-ex
}
__device__ __forceinline__ double2 crecip_fast(double2 z) {
  const double d = fma(z.x, z.x, z.y * z.y);
  const double r = recip_pos(d);
  return make_double2(z.x * r, -z.y * r);
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
// SA / SB: structure of op(A) / op(B) - 0 full, 1 upper triangular, 2 lower triangular -
// whose zero half is skipped.  Even and odd k go to two accumulators as in the full
// product, and the skipped terms are exact zeros, so the result is the full product's.
template <int SA = 0, int SB = 0>
__device__ void matmul(double2* C, const double2* A, bool tA, const double2* B, bool tB, int p) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    int k0 = 0, k1 = p;
    if (SA == 1) k0 = max(k0, i);
    if (SA == 2) k1 = min(k1, i + 1);
    if (SB == 1) k1 = min(k1, j + 1);
    if (SB == 2) k0 = max(k0, j);
    double2 acc0 = cz(), acc1 = cz();
    int k = k0 & ~1;
    for (; k + 2 <= k1; k += 2) {
      cmac(acc0, tA ? A[k * LD + i] : A[i * LD + k], tB ? B[j * LD + k] : B[k * LD + j]);
      cmac(acc1, tA ? A[(k + 1) * LD + i] : A[i * LD + k + 1], tB ? B[j * LD + k + 1] : B[(k + 1) * LD + j]);
    }
    if (k < k1) cmac(acc0, tA ? A[k * LD + i] : A[i * LD + k], tB ? B[j * LD + k] : B[k * LD + j]);
    C[i * LD + j] = make_double2(acc0.x + acc1.x, acc0.y + acc1.y);
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
__device__ bool chol_upper(double2* G, double2* tau, int p, double* sh) {
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) tau[e] = cz();
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    if (threadIdx.x == 0) {
      const double d = G[j * LD + j].x;
      if (!(d > 0.0) || !isfinite(d)) {
        sh[0] = 0.0;
      } else {
        const double ir = rsqrt(d);
        tau[j * LD + j] = make_double2(d * ir, 0.0);
        sh[0] = ir;
      }
    }
    __syncthreads();
    const double inv = sh[0];
    if (inv == 0.0) return false;
    for (int i = j + 1 + threadIdx.x; i < p; i += blockDim.x) {
      const double2 g = G[j * LD + i];
      tau[j * LD + i] = make_double2(g.x * inv, g.y * inv);
    }
    __syncthreads();
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

// T = tau^{-1} for upper-triangular tau with real positive diagonal.
__device__ void tri_inv_upper(const double2* tau, double2* T, int p, double* dinv) {
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) T[e] = cz();
  for (int i = threadIdx.x; i < p; i += blockDim.x) dinv[i] = 1.0 / tau[i * LD + i].x;
  __syncthreads();
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    T[j * LD + j] = make_double2(dinv[j], 0.0);
    for (int i = j - 1; i >= 0; --i) {
      double2 s0 = cz(), s1 = cz();
      int k = i + 1;
      for (; k + 2 <= j + 1; k += 2) {
        cmac(s0, tau[i * LD + k], T[k * LD + j]);
        cmac(s1, tau[i * LD + k + 1], T[(k + 1) * LD + j]);
      }
      if (k <= j) cmac(s0, tau[i * LD + k], T[k * LD + j]);
      const double d = -dinv[i];
      T[i * LD + j] = make_double2((s0.x + s1.x) * d, (s0.y + s1.y) * d);
    }
  }
  __syncthreads();
}

// Solve M Z = R in place (R <- Z), LU with partial pivoting; M is destroyed.
// Pivot = largest |re| + |im| in the column (ties to the lowest row).  For non-negative
// doubles the IEEE bit pattern orders like the value, so the warp argmax compares 64-bit
// integers (NaN patterns sort above +inf and are then reported as a breakdown).
__device__ bool lu_solve(double2* M, double2* R, int p, int nrhs, double* sh, int* ish) {
  for (int k = 0; k < p; ++k) {
    if (threadIdx.x < 32) {
      unsigned long long best = 0ull;
      int bi = p;
      for (int i = k + threadIdx.x; i < p; i += 32) {
        const unsigned long long key = (unsigned long long)__double_as_longlong(cabs1(M[i * LD + k]));
        if (bi == p || key > best) {
          best = key;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi < p && (bi == p || ob > best || (ob == best && oi < bi))) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) {
        const double v = __longlong_as_double((long long)best);
        ish[0] = bi;
        ish[1] = (bi < p && v > 0.0 && isfinite(v)) ? 1 : 0;
        if (ish[1]) {   // reciprocal of the pivot, formed once for the whole CTA
          const double2 r = crecip_fast(M[bi * LD + k]);
          sh[2 * PMAX] = r.x;
          sh[2 * PMAX + 1] = r.y;
        }
      }
    }
    __syncthreads();
    if (!ish[1]) return false;
    const int piv = ish[0];
    if (piv != k) {
      for (int c = threadIdx.x; c < p + nrhs; c += blockDim.x) {
        if (c < p) {
          const double2 t = M[k * LD + c];
          M[k * LD + c] = M[piv * LD + c];
          M[piv * LD + c] = t;
        } else {
          const int cc = c - p;
          const double2 t = R[k * LD + cc];
          R[k * LD + cc] = R[piv * LD + cc];
          R[piv * LD + cc] = t;
        }
      }
      __syncthreads();
    }
    const double2 pinv = make_double2(sh[2 * PMAX], sh[2 * PMAX + 1]);
    for (int i = k + 1 + threadIdx.x; i < p; i += blockDim.x) M[i * LD + k] = cmul(M[i * LD + k], pinv);
    __syncthreads();
    const int m = p - k - 1, w = m + nrhs;
    for (int e = threadIdx.x; e < m * w; e += blockDim.x) {
      const int i = k + 1 + e / w, c = e % w;
      const double2 l = M[i * LD + k];
      if (c < m) cmsub(M[i * LD + k + 1 + c], l, M[k * LD + k + 1 + c]);
      else cmsub(R[i * LD + (c - m)], l, R[k * LD + (c - m)]);
    }
    __syncthreads();
  }
  // back substitution with the diagonal reciprocals formed once, in parallel
  double2* dinv = reinterpret_cast<double2*>(sh);
  for (int k = threadIdx.x; k < p; k += blockDim.x) dinv[k] = crecip(M[k * LD + k]);
  __syncthreads();
  for (int k = p - 1; k >= 0; --k) {
    for (int c = threadIdx.x; c < nrhs; c += blockDim.x) R[k * LD + c] = cmul(R[k * LD + c], dinv[k]);
    __syncthreads();
    for (int e = threadIdx.x; e < k * nrhs; e += blockDim.x) {
      const int i = e / nrhs, c = e % nrhs;
      cmsub(R[i * LD + c], M[i * LD + k], R[k * LD + c]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < p * nrhs; e += blockDim.x)
    if (!cfinite(R[(e / nrhs) * LD + e % nrhs])) ish[1] = 0;
  __syncthreads();
  return ish[1] != 0;
}

// ------------------------------------------------------------------------ shared layout
struct SmallShared {
  double gs[2 * (2 * LD * (LD + 1) / 2 + 2)];
  double red[2 * PMAX + 8];
  int ish[4];
  int colexp[64];
  double2 m[6][LD * LD];
};

// Exact-slice fragments of a p x p factor (smem, stride LD) for the tensor-core applies.
__device__ void emit_oz(uint2* oz, int slot, const double2* M, int p, int* sh) {
  if (oz == nullptr) return;
  uint2* f = oz + slot * OZ_SLOT_U2;
  if (p <= 8) oz_emit_factor<8>(M, LD, p, f, oz_colexp_of(f), sh);
  else oz_emit_factor<16>(M, LD, p, f, oz_colexp_of(f), sh);
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
  expand_tri(S.gs, S.m[0], p, true);
  if (!chol_upper(S.m[0], S.m[1], p, S.red)) {
    if (threadIdx.x == 0) { ctrl->done = 3; ctrl->bd_code = 1; }
    return;
  }
  tri_inv_upper(S.m[1], S.m[2], p, S.red);
  gstore(slot(mats, M_XI), S.m[1], p);
  gstore_fac(mats, M_TINV, S.m[2], p);
  emit_oz(oz, OZ_T, S.m[2], p, S.colexp);
  if (method == 0) {
    expand_tri(S.gs + 2 * E, S.m[3], p, false);
    if (qr2) {   // G_QQ needs the final factor: the second stage forms it from R^T R
      gstore(slot(mats, M_G1), S.m[3], p);
      return;
    }
    matmul<2, 0>(S.m[4], S.m[2], true, S.m[3], false, p);   // T^T G
    matmul<0, 1>(S.m[5], S.m[4], false, S.m[2], false, p);  // (T^T G) T
    gstore(slot(mats, M_H), S.m[5], p);
  }
}

// cocr setup after A Q_0: H_0 = Q_0^T V_0 = T^T (W^T A W) T.
__device__ __noinline__ void d_small_cocr_H0(SmallShared& S, int p, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl) {
  if (BLCOC_LD(&ctrl->done)) return;
  sum_stage1(stage1, ncomp, S.gs);
  expand_tri(S.gs, S.m[0], p, false);
  gload(S.m[1], slot(mats, M_TINV), p);
  matmul<2, 0>(S.m[2], S.m[1], true, S.m[0], false, p);
  matmul<0, 1>(S.m[3], S.m[2], false, S.m[1], false, p);
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
  matmul<0, 1>(S.m[3], S.m[2], false, S.m[0], false, p);   // alpha' xi, xi upper triangular
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
  expand_tri(S.gs, S.m[0], p, true);
  if (!chol_upper(S.m[0], S.m[1], p, S.red)) {
    if (threadIdx.x == 0) {
      ctrl->done = 3;
      ctrl->bd_code = 3;
      if (method == 1) ctrl->iter -= 1;   // cocr forms X_{m+1} only in the last pass
    }
    return;
  }
  tri_inv_upper(S.m[1], S.m[2], p, S.red);
  gload(S.m[3], slot(mats, M_XI), p);
  matmul<1, 1>(S.m[4], S.m[1], false, S.m[3], false, p);   // xi_{m+1} = tau xi_m
  gstore(slot(mats, M_XI), S.m[4], p);
  gstore(slot(mats, M_TAU), S.m[1], p);
  gstore_fac(mats, M_TINV, S.m[2], p);
  emit_oz(oz, OZ_T, S.m[2], p, S.colexp);
  if (method == 0) {
    const int E = tri_count(p);
    expand_tri(S.gs + 2 * E, S.m[0], p, false);       // W^T W
    if (qr2) {   // G_QQ+ and beta' need the final factor: the second stage forms them
      gstore(slot(mats, M_G1), S.m[0], p);
      return;
    }
    matmul<2, 0>(S.m[3], S.m[2], true, S.m[0], false, p);   // T^T (W^T W)
    matmul<0, 1>(S.m[0], S.m[3], false, S.m[2], false, p);  // G_QQ+ = T^T W^T W T
    matmul<2, 0>(S.m[4], S.m[1], true, S.m[0], false, p);   // tau^T G_QQ+
    gload(S.m[3], slot(mats, M_H), p);                // G_QQ (old)
    gstore(slot(mats, M_H), S.m[0], p);
    if (!lu_solve(S.m[3], S.m[4], p, p, S.red, S.ish)) {
      if (threadIdx.x == 0) { ctrl->done = 3; ctrl->bd_code = 4; }
      return;
    }
    gstore_fac(mats, M_BETA, S.m[4], p);
  }
}

// CholQR2, second factor (after the pass W <- Q1 = W T1, Gram Q1^H Q1): tau2, T2 with
// tau2^H tau2 = Q1^H Q1; the QR factor becomes tau = tau2 tau1 and the passes that follow
// apply T2 to the stored Q1.  Iteration: xi_{m+1} <- tau2 xi_{m+1} (the first stage applied
// tau1).  Setup (setup = 1): xi_0 = tau.  cocg also forms G_QQ (setup) or G_QQ+ and beta'
// (iteration) from W^T W with the whole factor T1 T2.
__device__ __noinline__ void d_small_chol2(SmallShared& S, int p, int method, const double* stage1, int ncomp,
                                           double2* mats, Ctrl* ctrl, int setup, uint2* oz) {
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
  matmul<1, 1>(S.m[4], S.m[1], false, S.m[3], false, p);   // tau = tau2 tau1
  if (setup) {
    gstore(slot(mats, M_XI), S.m[4], p);
  } else {
    gstore(slot(mats, M_TAU), S.m[4], p);
    gload(S.m[5], slot(mats, M_XI), p);
    matmul<1, 1>(S.m[3], S.m[1], false, S.m[5], false, p);   // xi <- tau2 xi
    gstore(slot(mats, M_XI), S.m[3], p);
  }
  if (method == 0) {
    gload(S.m[5], slot(mats, M_TINV), p);                   // T1
    matmul<1, 1>(S.m[3], S.m[5], false, S.m[2], false, p);   // T1 T2
    gload(S.m[0], slot(mats, M_G1), p);                     // W^T W (R^T R at setup)
    matmul<2, 0>(S.m[5], S.m[3], true, S.m[0], false, p);
    matmul<0, 1>(S.m[0], S.m[5], false, S.m[3], false, p);  // (T1 T2)^T G (T1 T2)
    if (setup) {
      gstore(slot(mats, M_H), S.m[0], p);                   // G_QQ
    } else {
      matmul<2, 0>(S.m[5], S.m[4], true, S.m[0], false, p); // tau^T G_QQ+
      gload(S.m[3], slot(mats, M_H), p);                    // G_QQ (old)
      gstore(slot(mats, M_H), S.m[0], p);
      if (!lu_solve(S.m[3], S.m[5], p, p, S.red, S.ish)) {
        if (threadIdx.x == 0) { ctrl->done = 3; ctrl->bd_code = 4; }
        return;
      }
      gstore_fac(mats, M_BETA, S.m[5], p);
    }
  }
  gstore_fac(mats, M_TINV, S.m[2], p);
  emit_oz(oz, OZ_T, S.m[2], p, S.colexp);
}

// cocr after V_{m+1} (Algorithm 3, the beta' step): H+ = T^T (W^T A W) T, beta' = H^{-1} tau^T H+.
__device__ __noinline__ void d_small_cocr_beta(SmallShared& S, int p, const double* stage1, int ncomp, double2* mats, Ctrl* ctrl, uint2* oz) {
  if (BLCOC_LD(&ctrl->done)) return;
  sum_stage1(stage1, ncomp, S.gs);
  expand_tri(S.gs, S.m[0], p, false);
  gload(S.m[1], slot(mats, M_TINV), p);
  matmul<2, 0>(S.m[2], S.m[1], true, S.m[0], false, p);
  matmul<0, 1>(S.m[3], S.m[2], false, S.m[1], false, p);   // H+
  gload(S.m[4], slot(mats, M_TAU), p);
  matmul<2, 0>(S.m[5], S.m[4], true, S.m[3], false, p);    // tau^T H+
  gload(S.m[0], slot(mats, M_H), p);
  gstore(slot(mats, M_H), S.m[3], p);
  if (!lu_solve(S.m[0], S.m[5], p, p, S.red, S.ish)) {
    if (threadIdx.x == 0) {
      ctrl->done = 3;
      ctrl->bd_code = 4;
      ctrl->iter -= 1;
    }
    return;
  }
  gstore_fac(mats, M_BETA, S.m[5], p);
  emit_oz(oz, OZ_BETA, S.m[5], p, S.colexp);
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
