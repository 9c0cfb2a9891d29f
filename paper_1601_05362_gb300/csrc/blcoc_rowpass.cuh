// Row-pass kernels of bl_cocg_rq / bl_cocr_rq (Algorithms 2-3, Sec. 2.2), templated on
// the block width PP (the solve's p satisfies p <= PP) and on the working precision S
// (double: the FP64 path; float: the complex64 inner solves of the mixed-precision form).
//
// Work decomposition.  On GB300 every FP64 operation of this path is issued by the FP64
// pipe (about 2 DFMA per clock per SM), which binds long before HBM does; the design
// therefore spends no FP64 operation it does not need:
//   * a warp owns chunks of 32 consecutive rows; the chunk's n x p slices are staged in
//     the warp's own shared-memory tiles, so warps never wait on each other;
//   * p x p right-multiplications (Y <- Y M) run with lane = row: all lanes walk the same
//     (k, j) sequence, so the upper-triangular tau^{-1} applies cost exactly p(p+1)/2
//     complex MACs per row and the p x p factor is a shared-memory broadcast;
//   * Gram products G = Y^T Z (or Y^H Z) over the chunk run with lane = Gram entry;
//     symmetric / Hermitian Grams compute only the upper triangle, and the remainder
//     entries are spread over row groups so every lane does the same work;
//   * per-CTA Gram partials are summed in a fixed order (first here, then by a
//     deterministic two-stage reduction), so results are bitwise reproducible.
// Tiles are [k][32 rows] with the row index XOR-swizzled by (k & 7): lane = row reads,
// lane = entry reads and the coalesced global <-> shared transposes are all free of
// shared-memory bank conflicts.
#pragma once

#include <type_traits>

#include "blcoc_common.cuh"
#include "blcoc_ozaki.cuh"

namespace blcoc {

template <int PP, typename S = double>
struct Geo {
  using C = typename Cx<S>::T;
  static constexpr int TILE = PP * CHUNK;                      // elements per staged block
  static constexpr int NTRI = (PP * (PP + 1) / 2 + 31) / 32;   // gram slots per lane, triangle
  static constexpr int JB = PP >= 8 ? 8 : PP;                  // output columns per apply sweep
  static constexpr bool MATS_SMEM = PP <= 16 || sizeof(S) == 4;  // p x p factors staged in smem
  static constexpr int LPR = PP < 32 ? PP : 32;                // lanes per row in the CSR gather
  static constexpr int RPI = 32 / LPR;                         // rows per gather instruction
};

__device__ __forceinline__ int tix(int k, int r) { return k * CHUNK + (r ^ (k & 7)); }

// Parts a staged p x p factor is kept in: FP64 one; complex64 two, hi = fl(M) and
// lo = fl(M - hi), so that a complex64 row pass applies the FP64 factor to about 2^-48
// relative accuracy instead of rounding it to 2^-24.  (Rounding the factors is not
// harmless: every row of the block then moves by the same relative error, which on
// indefinite problems destroys the bilinear orthogonality of Table 1 within a few dozen
// iterations.)
template <typename S>
constexpr int mat_parts() { return sizeof(S) == 4 ? 2 : 1; }

// Elements taken by nm staged p x p factors, rounded up to a 16-byte boundary so that the
// tiles (and the FP64 reduction area that reuses them) stay 16-byte aligned.
template <int PP, typename S>
constexpr int mats_off(int nm) {
  using C = typename Cx<S>::T;
  return Geo<PP, S>::MATS_SMEM
             ? (int)((((size_t)nm * mat_parts<S>() * PP * PP * sizeof(C) + 15) / 16 * 16) / sizeof(C))
             : 0;
}

// ---------------------------------------------------------------------------------- tiles
// Coalesced load of rows [r0, r0+32) (clipped to n) of a row-major n x p block into a
// swizzled tile; rows past n are zero.
template <int PP, typename C>
__device__ __forceinline__ void load_tile(C* t, const C* __restrict__ g, int64_t r0, int64_t n, int p, int lane) {
  const int rows = (int)min((int64_t)CHUNK, n - r0);
  const int total = CHUNK * p;
  const int valid = rows * p;
  const C* src = g + r0 * p;
  for (int e = lane; e < total; e += 32) {
    const int r = e / p, k = e - r * p;
    t[tix(k, r)] = (e < valid) ? BLCOC_LD(src + e) : czero<C>();
  }
}

template <int PP, typename C>
__device__ __forceinline__ void store_tile(C* __restrict__ g, const C* t, int64_t r0, int64_t n, int p, int lane) {
  const int rows = (int)min((int64_t)CHUNK, n - r0);
  const int valid = rows * p;
  C* dst = g + r0 * p;
  for (int e = lane; e < valid; e += 32) {
    const int r = e / p, k = e - r * p;
    dst[e] = t[tix(k, r)];
  }
}

// FP64 tile -> complex64 block (the residual pass of the mixed-precision form)
template <int PP>
__device__ __forceinline__ void store_tile_f32(float2* __restrict__ g, const double2* t, int64_t r0, int64_t n, int p,
                                               int lane) {
  const int rows = (int)min((int64_t)CHUNK, n - r0);
  const int valid = rows * p;
  float2* dst = g + r0 * p;
  for (int e = lane; e < valid; e += 32) {
    const int r = e / p, k = e - r * p;
    dst[e] = from_d2<float2>(t[tix(k, r)]);
  }
}

// A factor entry of the complex64 passes: hi + lo (see mat_parts).
struct f2pair {
  float2 hi, lo;
};
// acc += y (hi + lo), acc -= y (hi + lo): the small part first, then the large one.
__device__ __forceinline__ void cmac(float2& acc, float2 y, f2pair m) {
  cmac(acc, y, m.lo);
  cmac(acc, y, m.hi);
}
__device__ __forceinline__ void cmsub(float2& acc, float2 y, f2pair m) {
  cmsub(acc, y, m.lo);
  cmsub(acc, y, m.hi);
}

// Write FP64 factor entry v at index i of a staged factor whose parts are `stride`
// elements apart (one part for FP64, hi and lo for complex64).
__device__ __forceinline__ void put_fac(double2* s, int i, int, double2 v) { s[i] = v; }
__device__ __forceinline__ void put_fac(float2* s, int i, int stride, double2 v) {
  const float2 hi = make_float2((float)v.x, (float)v.y);
  s[i] = hi;
  s[stride + i] = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
}

// Stage a p x p FP64 factor (row stride p in global) as PP x PP in the working precision,
// zero padded (complex64: hi part, then lo part PP*PP elements further).
template <int PP, typename C>
__device__ __forceinline__ void load_mat(C* s, const double2* __restrict__ g, int p) {
  for (int e = threadIdx.x; e < PP * PP; e += blockDim.x) {
    const int k = e / PP, j = e - k * PP;
    put_fac(s, e, PP * PP, (k < p && j < p) ? BLCOC_LD(g + k * p + j) : cz());
  }
}

// Factor access: shared memory (stride PP) or, for FP64 at PP = 32, global memory
// through the read-only path (row stride p).  complex64: the hi + lo pair.
template <int PP, typename S>
struct Fac {
  using C = typename Cx<S>::T;
  const C* m;
  int ld;
  __device__ __forceinline__ auto operator()(int k, int j) const {
    if constexpr (sizeof(S) == 4) return f2pair{m[k * PP + j], m[PP * PP + k * PP + j]};
    else if constexpr (Geo<PP, S>::MATS_SMEM) return m[k * PP + j];
    else return __ldg(m + k * ld + j);
  }
};

template <int PP>
constexpr int tri_packed() { return PP * (PP + 1) / 2; }

// Upper-triangular factor packed row by row in shared memory (row k holds columns k..PP-1);
// only entries with j >= k are read.  complex64: the hi + lo pair.
template <int PP, typename S>
struct FacTri {
  using C = typename Cx<S>::T;
  const C* m;
  __device__ __forceinline__ auto operator()(int k, int j) const {
    const int i = k * PP - (k * (k - 1)) / 2 + (j - k);
    if constexpr (sizeof(S) == 4) return f2pair{m[i], m[tri_packed<PP>() + i]};
    else return m[i];
  }
};

// Stage the upper triangle of a p x p FP64 factor, packed (zero outside p; complex64: hi
// part, then lo part tri_packed elements further).
template <int PP, typename C>
__device__ __forceinline__ void load_mat_tri(C* s, const double2* __restrict__ g, int p) {
  for (int e = threadIdx.x; e < PP * PP; e += blockDim.x) {
    const int k = e / PP, j = e - k * PP;
    if (j >= k)
      put_fac(s, k * PP - (k * (k - 1)) / 2 + (j - k), tri_packed<PP>(), (k < p && j < p) ? BLCOC_LD(g + k * p + j) : cz());
  }
}

// Pass C's staged factors: T packed, alpha'xi and beta' full (elements of the working
// precision, rounded up to a 16-byte boundary).
template <int PP, typename S>
constexpr int passC_mats_elems() {
  using C = typename Cx<S>::T;
  return Geo<PP, S>::MATS_SMEM
             ? (int)((((size_t)(tri_packed<PP>() + 2 * PP * PP) * mat_parts<S>() * sizeof(C) + 15) / 16 * 16) /
                     sizeof(C))
             : 0;
}

// ---------------------------------------------------------------------------------- applies
// t <- t * T with T upper triangular (lane = row).  Columns are produced from the last
// block to the first, so a column slot is overwritten only after every later column
// that needs it has been formed.  Cost: exactly sum_j (j+1) complex MACs per row.
template <int PP, typename S, typename F>
__device__ __forceinline__ void tri_apply_inplace(typename Cx<S>::T* t, const F& T, int p, int lane) {
  using C = typename Cx<S>::T;
  constexpr int JB = Geo<PP, S>::JB;
  for (int j0 = ((p - 1) / JB) * JB; j0 >= 0; j0 -= JB) {
    C acc[JB];
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) acc[jj] = czero<C>();
    for (int k = 0; k < j0; ++k) {
      const C y = t[tix(k, lane)];
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) cmac(acc[jj], y, T(k, j0 + jj));
    }
#pragma unroll
    for (int kk = 0; kk < JB; ++kk) {
      if (j0 + kk < p) {
        const C y = t[tix(j0 + kk, lane)];
#pragma unroll
        for (int jj = kk; jj < JB; ++jj) cmac(acc[jj], y, T(j0 + kk, j0 + jj));
      }
    }
#pragma unroll
    for (int jj = 0; jj < JB; ++jj)
      if (j0 + jj < p) t[tix(j0 + jj, lane)] = acc[jj];
  }
}

// out <- base + in * M  (SUB: base - in * M), lane = row.  `out` may be `base`
// (each column of base is read only for the same column of out) but not `in`.
template <int PP, typename S, bool SUB>
__device__ __forceinline__ void apply_full(typename Cx<S>::T* out, const typename Cx<S>::T* base,
                                           const typename Cx<S>::T* in, const Fac<PP, S>& M, int p, int lane) {
  using C = typename Cx<S>::T;
  constexpr int JB = Geo<PP, S>::JB;
  for (int j0 = 0; j0 < p; j0 += JB) {
    C acc[JB];
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) acc[jj] = (j0 + jj < p) ? base[tix(j0 + jj, lane)] : czero<C>();
    for (int k = 0; k < p; ++k) {
      const C y = in[tix(k, lane)];
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) {
        if constexpr (SUB) cmsub(acc[jj], y, M(k, j0 + jj));
        else cmac(acc[jj], y, M(k, j0 + jj));
      }
    }
#pragma unroll
    for (int jj = 0; jj < JB; ++jj)
      if (j0 + jj < p) out[tix(j0 + jj, lane)] = acc[jj];
  }
}

// ------------------------------------------------------------------ three-product applies
// FP64 block widths from 8 up apply the p x p factors in three real products per complex
// MAC instead of four (Gauss's multiplication): for y = a + ib and M = c + id,
//   re(y M) = (a + b) c - b (c + d),   im(y M) = (a + b) c + a (d - c),
// with c, c + d and d - c formed once per factor (three-product slots, written by the p x p
// stages) and a + b once per row and k.  Per output the shared term (a + b) c is summed
// once and added to both parts at the end: 3 p^2 + 3 p FP64 operations per full apply and
// row instead of 4 p^2.  The error bound stays of the order of the four-product one,
// relative to |y| |M| (the terms are bounded by (|a| + |b|)(|c| + |d|) <= 2 |y| |M|).
template <int PP, typename S, bool OZ = false>
constexpr bool m3_apply() { return sizeof(S) == 8 && !OZ && PP >= 8; }
// FP64 passes at p = 32 keep one tile per warp: the second operand of each block update
// (and W in the SpMM's Gram) is read from global memory through L1 (lane = row; a 128-byte
// line serves 8 consecutive columns of a row) instead of a second 16 KB tile, so that two
// 4-warp CTAs fit an SM instead of one (two warps per SM sub-partition instead of one).
template <int PP, typename S, bool OZ>
constexpr bool one_tile() { return PP >= 32 && sizeof(S) == 8 && !OZ; }

// Tensor-core Grams (exact slices, per-warp FP64 sums in shared memory) are built for
// p <= 16; at p = 32 the tensor-core passes keep their Grams on the FP64 pipe (the sums
// of 64 x 64 real entries per warp would not fit beside the tiles).
template <int PP, bool OZ>
constexpr bool oz_gram() { return OZ && PP <= 16; }
// The tensor-core kernel set's SpMM has the T apply on the tensor cores, and up to p = 16
// the W^T Y Gram as well; at p = 32 it keeps one tile per warp (W for its FP64 Gram read
// from global memory), as the FP64 SpMM there does.

// The tensor-core passes A and C at p = 32 keep one tile per warp, as the FP64 ones do:
// the second operand of each block update is split into slice digits straight from global
// memory (through L1), so that two CTAs fit an SM.
template <int PP, bool OZ>
constexpr bool tc_one_tile() { return OZ && PP >= 32; }

// out = base (+/-) in * M on the tensor cores, M given by its exact-slice fragments.
template <int PP, bool SUB, bool BASE>
__device__ __forceinline__ void oz_apply_any(double2* out, const double2* base, const double2* in, const uint2* fz,
                                             int p, int lane) {
  if constexpr (PP >= 32)
    oz_apply_t<PP, SUB, BASE, false>(out, base, in, nullptr, 0, reinterpret_cast<const uint4*>(fz), oz_colexp_of(fz),
                                     p, lane);
  else oz_apply<PP, SUB, BASE>(out, base, in, fz, oz_colexp_of(fz), p, lane);
}
// The same with `in` read from global memory (in_g = the chunk's first row, `rows` of them
// inside n); p = 32 only.
template <int PP, bool SUB, bool BASE>
__device__ __forceinline__ void oz_apply_gin(double2* out, const double2* base, const double2* in_g, int rows,
                                             const uint2* fz, int p, int lane) {
  oz_apply_t<PP, SUB, BASE, true>(out, base, nullptr, in_g, rows, reinterpret_cast<const uint4*>(fz),
                                  oz_colexp_of(fz), p, lane);
}
template <int PP, typename S>
constexpr bool m3_gram() { return sizeof(S) == 8 && PP >= 8; }
// The CholQR2 pass (which also forms Q1^T Q1 for bl_cocg_rq): three-product Grams from a
// companion tile up to p = 16; at p = 32 two such accumulators would not fit in registers.
template <int PP, typename S>
constexpr bool qr2_m3() { return m3_gram<PP, S>() && PP <= 16; }

// Three-product form of a factor, read from its slots (row stride p) through the L1 path;
// every lane of a warp reads the same entry.
struct Fac3 {
  const double2* sd;   // (Mr + Mi, Mi - Mr)
  const double* r;     // Mr
  int ld;
  __device__ __forceinline__ Fac3(const double2* mats, int slot, int p)
      : sd(mats + m3_slot(slot) * PMAX * PMAX),
        r(reinterpret_cast<const double*>(mats + (m3_slot(slot) + 1) * PMAX * PMAX)),
        ld(p) {}
  __device__ __forceinline__ double re(int k, int j) const { return BLCOC_LD(r + k * ld + j); }
  __device__ __forceinline__ double2 sdif(int k, int j) const { return BLCOC_LD(sd + k * ld + j); }
};

// acc += y M(k, j) in three products; kk accumulates the shared term (a + b) c.
template <bool SUB>
__device__ __forceinline__ void mac3(double2& acc, double& kk, double2 y, double ys, double mr, double2 m) {
  if constexpr (SUB) {
    kk = fma(-ys, mr, kk);
    acc.x = fma(y.y, m.x, acc.x);
    acc.y = fma(-y.x, m.y, acc.y);
  } else {
    kk = fma(ys, mr, kk);
    acc.x = fma(-y.y, m.x, acc.x);
    acc.y = fma(y.x, m.y, acc.y);
  }
}

// out <- base + in * M (SUB: base - in * M), three products per MAC; aliasing as apply_full.
template <int PP, bool SUB>
__device__ __forceinline__ void apply_full3(double2* out, const double2* base, const double2* in, const Fac3& M,
                                            int p, int lane) {
  constexpr int JB = Geo<PP>::JB;
  for (int j0 = 0; j0 < p; j0 += JB) {
    double2 acc[JB];
    double kk[JB];
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) {
      acc[jj] = (j0 + jj < p) ? base[tix(j0 + jj, lane)] : cz();
      kk[jj] = 0.0;
    }
    for (int k = 0; k < p; ++k) {
      const double2 y = in[tix(k, lane)];
      const double ys = y.x + y.y;
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) mac3<SUB>(acc[jj], kk[jj], y, ys, M.re(k, j0 + jj), M.sdif(k, j0 + jj));
    }
#pragma unroll
    for (int jj = 0; jj < JB; ++jj)
      if (j0 + jj < p) out[tix(j0 + jj, lane)] = make_double2(acc[jj].x + kk[jj], acc[jj].y + kk[jj]);
  }
}

// out <- base + in * M (SUB: base - in * M), three products per MAC, with `in` read from
// global memory: in_g = the chunk's first row of a row-major n x p block, rows = the chunk's
// rows inside n (rows past it read as zero).  `out` may be `base`.
template <int PP, bool SUB>
__device__ __forceinline__ void apply_full3_g(double2* out, const double2* base, const double2* __restrict__ in_g,
                                              int rows, const Fac3& M, int p, int lane) {
  constexpr int JB = Geo<PP>::JB;
  const double2* row = in_g + (int64_t)lane * p;
  const bool live = lane < rows;
  for (int j0 = 0; j0 < p; j0 += JB) {
    double2 acc[JB];
    double kk[JB];
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) {
      acc[jj] = (j0 + jj < p) ? base[tix(j0 + jj, lane)] : cz();
      kk[jj] = 0.0;
    }
#pragma unroll 4
    for (int k = 0; k < p; ++k) {
      const double2 y = live ? __ldg(row + k) : cz();
      const double ys = y.x + y.y;
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) mac3<SUB>(acc[jj], kk[jj], y, ys, M.re(k, j0 + jj), M.sdif(k, j0 + jj));
    }
#pragma unroll
    for (int jj = 0; jj < JB; ++jj)
      if (j0 + jj < p) out[tix(j0 + jj, lane)] = make_double2(acc[jj].x + kk[jj], acc[jj].y + kk[jj]);
  }
}

// t <- t * T, T upper triangular, three products per MAC; column order as tri_apply_inplace.
template <int PP>
__device__ __forceinline__ void tri_apply3_inplace(double2* t, const Fac3& T, int p, int lane) {
  constexpr int JB = Geo<PP>::JB;
  for (int j0 = ((p - 1) / JB) * JB; j0 >= 0; j0 -= JB) {
    double2 acc[JB];
    double kk[JB];
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) {
      acc[jj] = cz();
      kk[jj] = 0.0;
    }
    for (int k = 0; k < j0; ++k) {
      const double2 y = t[tix(k, lane)];
      const double ys = y.x + y.y;
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) mac3<false>(acc[jj], kk[jj], y, ys, T.re(k, j0 + jj), T.sdif(k, j0 + jj));
    }
#pragma unroll
    for (int kq = 0; kq < JB; ++kq) {
      if (j0 + kq < p) {
        const double2 y = t[tix(j0 + kq, lane)];
        const double ys = y.x + y.y;
#pragma unroll
        for (int jj = kq; jj < JB; ++jj)
          mac3<false>(acc[jj], kk[jj], y, ys, T.re(j0 + kq, j0 + jj), T.sdif(j0 + kq, j0 + jj));
      }
    }
#pragma unroll
    for (int jj = 0; jj < JB; ++jj)
      if (j0 + jj < p) t[tix(j0 + jj, lane)] = make_double2(acc[jj].x + kk[jj], acc[jj].y + kk[jj]);
  }
}

// sd <- (re + im, im - re) of every element of the tile t (lane = row), for the
// three-product Grams of t with itself.
template <int PP>
__device__ __forceinline__ void sd_tile(double2* sd, const double2* t, int p, int lane) {
  for (int k = 0; k < p; ++k) {
    const double2 v = t[tix(k, lane)];
    sd[tix(k, lane)] = make_double2(v.x + v.y, v.y - v.x);
  }
}

// ---------------------------------------------------------------------------------- grams
enum GramKind { G_FULL = 0, G_SYM = 1, G_HERM = 2 };

// Double-float accumulator of a complex Gram entry (complex64 passes, unconjugated Grams).
struct DF2 {
  float2 hi, lo;
};
// hi + lo += a b with the product taken exactly (fma gives its rounding error) and the
// sum's rounding error kept (Knuth's two-sum); explicit _rn operations so the compiler
// neither contracts nor reorders them.
__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float a, float b) {
  const float pr = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -pr);
  const float s = __fadd_rn(hi, pr);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(pr, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, pe));
}
// d += y z (unconjugated), every real product exact and every sum compensated.
__device__ __forceinline__ void df_cmac(DF2& d, float2 y, float2 z) {
  df_add_prod(d.hi.x, d.lo.x, y.x, z.x);
  df_add_prod(d.hi.x, d.lo.x, -y.y, z.y);
  df_add_prod(d.hi.y, d.lo.y, y.x, z.y);
  df_add_prod(d.hi.y, d.lo.y, y.y, z.x);
}

template <int NS, typename S, bool M3 = false>
struct GramAcc {
  // Entries e = lane + 32 i (i < F) take all 32 rows of a chunk.  The Er = E mod 32
  // remainder entries, when Er divides 32, are spread over G = 32/Er row groups so that
  // every lane does the same number of MACs (a warp instruction costs the same with
  // idle lanes); the G partial sums are combined by shuffles at the end.
  // FP64: products accumulate directly in FP64.  complex64: each chunk's products
  // accumulate in FP32 and the chunk total is added to the FP64 accumulator.
  // M3 (FP64 self-Grams Y^T Y / Y^H Y): three products per MAC, as the applies, from the
  // tile and its (re + im, im - re) companion; kk holds the term shared by both parts.
  using C = typename Cx<S>::T;
  double2 acc[NS];
  double kk[M3 ? NS : 1];
  short a[NS], b[NS];
  int E, F, Er, G;
  __device__ __forceinline__ void init(int kind, int p, int lane) {
    E = (kind == G_FULL) ? p * p : tri_count(p);
    F = E / 32;
    Er = E - 32 * F;
    G = (Er > 0 && (32 % Er) == 0) ? 32 / Er : 1;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      acc[i] = cz();
      if constexpr (M3) kk[i] = 0.0;
      int e = lane + 32 * i;
      if (i == F && G > 1) e = 32 * F + lane % Er;
      int aa = 0, bb = 0;
      if (e < E) {
        if (kind == G_FULL) {
          aa = e / p;
          bb = e - aa * p;
        } else {
          int rem = e;
          while (rem >= p - aa) { rem -= p - aa; ++aa; }
          bb = aa + rem;
        }
      }
      a[i] = (short)aa;
      b[i] = (short)bb;
    }
  }
  // entry index held by this lane in slot i (E or more: none)
  __device__ __forceinline__ int entry(int i, int lane) const {
    if (i == F && G > 1) return 32 * F + lane % Er;
    return lane + 32 * i;
  }
  template <bool CONJ, typename A>
  __device__ __forceinline__ void mac(A& dst, int i, const C* Y, const C* Z, int r) const {
    const C y = Y[tix(a[i], r)];
    const C z = Z[tix(b[i], r)];
    if constexpr (std::is_same<A, DF2>::value) df_cmac(dst, y, z);
    else if constexpr (CONJ) cmac_conj(dst, y, z);
    else cmac(dst, y, z);
  }
  template <bool CONJ, typename A>
  __device__ __forceinline__ void add_rows(A* dst, const C* Y, const C* Z, int lane) const {
#pragma unroll 2
    for (int r = 0; r < CHUNK; ++r) {
#pragma unroll
      for (int i = 0; i < NS; ++i)
        if (i < F) mac<CONJ>(dst[i], i, Y, Z, r);
    }
    if (F < NS && Er > 0) {
      if (G > 1) {
        const int rows = CHUNK / G, r0 = (lane / Er) * rows;
        for (int r = r0; r < r0 + rows; ++r) {
#pragma unroll
          for (int i = 0; i < NS; ++i)
            if (i == F) mac<CONJ>(dst[i], i, Y, Z, r);
        }
      } else if (lane < Er) {
        for (int r = 0; r < CHUNK; ++r) {
#pragma unroll
          for (int i = 0; i < NS; ++i)
            if (i == F) mac<CONJ>(dst[i], i, Y, Z, r);
        }
      }
    }
  }
  // FP64, Y read from global memory (Yg = the chunk's first row, rows inside n), Z a tile.
  template <bool CONJ>
  __device__ __forceinline__ void mac_g(double2& dst, int i, const double2* __restrict__ Yg, int rows, int p,
                                        const double2* Z, int r) const {
    const double2 y = r < rows ? __ldg(Yg + (int64_t)r * p + a[i]) : cz();
    const double2 z = Z[tix(b[i], r)];
    if constexpr (CONJ) cmac_conj(dst, y, z);
    else cmac(dst, y, z);
  }
  template <bool CONJ>
  __device__ __forceinline__ void add_g(const double2* __restrict__ Yg, int rows, int p, const double2* Z, int lane) {
    static_assert(sizeof(S) == 8 && !M3, "FP64 four-product Gram");
#pragma unroll 2
    for (int r = 0; r < CHUNK; ++r) {
#pragma unroll
      for (int i = 0; i < NS; ++i)
        if (i < F) mac_g<CONJ>(acc[i], i, Yg, rows, p, Z, r);
    }
    if (F < NS && Er > 0) {
      if (G > 1) {
        const int rr = CHUNK / G, r0 = (lane / Er) * rr;
        for (int r = r0; r < r0 + rr; ++r) {
#pragma unroll
          for (int i = 0; i < NS; ++i)
            if (i == F) mac_g<CONJ>(acc[i], i, Yg, rows, p, Z, r);
        }
      } else if (lane < Er) {
        for (int r = 0; r < CHUNK; ++r) {
#pragma unroll
          for (int i = 0; i < NS; ++i)
            if (i == F) mac_g<CONJ>(acc[i], i, Yg, rows, p, Z, r);
        }
      }
    }
  }
  // acc[e] += sum_r op(Y[r][a_e]) Z[r][b_e] over the 32 rows of a chunk.
  // complex64, unconjugated (the coefficient Grams of Table 1): every product of two
  // complex64 entries is exact and the chunk sum is double-float, so the Gram is about as
  // accurate as an FP64 sum of the stored values.  These bilinear forms cancel heavily
  // (|Y^T Z| can be far below sum |y||z|); summed in plain FP32 their error stops the
  // iteration on indefinite problems.  The Hermitian Gram of the Cholesky QR keeps the
  // FP32 chunk sums (its terms do not cancel).
  template <bool CONJ>
  __device__ __forceinline__ void add(const C* Y, const C* Z, int lane) {
    if constexpr (sizeof(S) == 8) {
      add_rows<CONJ>(acc, Y, Z, lane);
    } else if constexpr (!CONJ) {
      DF2 part[NS];
#pragma unroll
      for (int i = 0; i < NS; ++i) part[i] = DF2{czero<C>(), czero<C>()};
      add_rows<false>(part, Y, Z, lane);
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        acc[i].x += (double)part[i].hi.x + (double)part[i].lo.x;
        acc[i].y += (double)part[i].hi.y + (double)part[i].lo.y;
      }
    } else {
      C part[NS];
#pragma unroll
      for (int i = 0; i < NS; ++i) part[i] = czero<C>();
      add_rows<CONJ>(part, Y, Z, lane);
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        acc[i].x += (double)part[i].x;
        acc[i].y += (double)part[i].y;
      }
    }
  }
  // Three-product self-Gram, entry (a, b) over row r, y = Y[a], z = Y[b], (s, d) their
  // companions:  SYM  y z      = (kk + acc.x, kk + acc.y), kk += z.re s_y, acc += (-y.im s_z, y.re d_z);
  //              HERM conj(y) z: kk -= z.re d_y, acc += (y.im s_z, y.re d_z).
  // On the diagonal of the Hermitian Gram kk and acc.y take opposite roundings of the same
  // products, so its imaginary part is exactly zero.
  template <bool HERM>
  __device__ __forceinline__ void mac3g(int i, const double2* Y, const double2* SD, int r) {
    const double2 y = Y[tix(a[i], r)];
    const double2 sy = SD[tix(a[i], r)];
    const double zx = Y[tix(b[i], r)].x;
    const double2 sz = SD[tix(b[i], r)];
    if constexpr (HERM) {
      kk[i] = fma(-zx, sy.y, kk[i]);
      acc[i].x = fma(y.y, sz.x, acc[i].x);
    } else {
      kk[i] = fma(zx, sy.x, kk[i]);
      acc[i].x = fma(-y.y, sz.x, acc[i].x);
    }
    acc[i].y = fma(y.x, sz.y, acc[i].y);
  }
  template <bool HERM>
  __device__ __forceinline__ void add3(const double2* Y, const double2* SD, int lane) {
    static_assert(M3, "three-product Gram");
#pragma unroll 2
    for (int r = 0; r < CHUNK; ++r) {
#pragma unroll
      for (int i = 0; i < NS; ++i)
        if (i < F) mac3g<HERM>(i, Y, SD, r);
    }
    if (F < NS && Er > 0) {
      if (G > 1) {
        const int rows = CHUNK / G, r0 = (lane / Er) * rows;
        for (int r = r0; r < r0 + rows; ++r) {
#pragma unroll
          for (int i = 0; i < NS; ++i)
            if (i == F) mac3g<HERM>(i, Y, SD, r);
        }
      } else if (lane < Er) {
        for (int r = 0; r < CHUNK; ++r) {
#pragma unroll
          for (int i = 0; i < NS; ++i)
            if (i == F) mac3g<HERM>(i, Y, SD, r);
        }
      }
    }
  }
  // combine the row-group partial sums of the remainder slot (fixed butterfly order)
  __device__ __forceinline__ void fold() {
    if constexpr (M3) {
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        acc[i].x += kk[i];
        acc[i].y += kk[i];
      }
    }
    if (F < NS && G > 1) {
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        if (i == F) {
          for (int o = Er; o < 32; o <<= 1) {
            acc[i].x += __shfl_xor_sync(0xffffffffu, acc[i].x, o);
            acc[i].y += __shfl_xor_sync(0xffffffffu, acc[i].y, o);
          }
        }
      }
    }
  }
};

// Sum the warps' accumulators of one Gram in a fixed order and write the CTA partial.
// `red` is shared scratch of at least NWARP*E double2; caller syncs before reuse.
template <int NS, typename S, bool M3>
__device__ __forceinline__ void cta_write_gram(GramAcc<NS, S, M3>& g, double2* red, double2* __restrict__ out, int warp,
                                               int lane) {
  g.fold();
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int e = g.entry(i, lane);
    const bool owner = !(i == g.F && g.G > 1) || lane < g.Er;
    if (e < g.E && owner) red[warp * g.E + e] = g.acc[i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < g.E; e += blockDim.x) {
    double2 s = red[e];
    for (int w = 1; w < NWARP; ++w) {
      s.x += red[w * g.E + e].x;
      s.y += red[w * g.E + e].y;
    }
    out[e] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------- gather
// Y[r][k] = sum_j a_{row,j} X[j][k] (lanes = columns, PP/32 rows per instruction), written
// to a swizzled tile.  RESID: Y = B - A X, also accumulating |B|^2 and |Y|^2 per lane.
// Row bundle: LPR = p lanes (one per column) per row, 32 / LPR rows per instruction.  SPL > 1
// (not with RESID): SPL lane groups split each row's nonzeros (interleaved), and the SPL
// partial sums are combined by an xor butterfly in a fixed order.
template <int PP, typename C, bool RESID, int SPL = 1>
__device__ __forceinline__ void gather_rows(C* Yt, const CsrDev& A, const C* __restrict__ va, const C* __restrict__ Xg,
                                            const C* __restrict__ Bg, int64_t r0, int p, int lane, double& sb,
                                            double& sr) {
  constexpr int LPR = Geo<PP>::LPR, LW = LPR * SPL, RPI = 32 / LW;
  static_assert(LW <= 32 && (SPL == 1 || !RESID), "row bundle wider than a warp");
  const int sub = lane / LW, rem = lane - sub * LW, part = rem / LPR, k = rem - part * LPR;
  for (int rr = 0; rr < CHUNK; rr += RPI) {
    const int r = rr + sub;
    const int64_t row = r0 + r;
    C acc = czero<C>();
    if (row < A.n && k < p) {
      if constexpr (RESID) {
        acc = BLCOC_LD(Bg + row * p + k);
        sb = fma((double)acc.x, (double)acc.x, sb);
        sb = fma((double)acc.y, (double)acc.y, sb);
      }
      const int beg = A.rp[row], end = A.rp[row + 1];
      for (int j = beg + part; j < end; j += SPL) {
        const int c = __ldg(A.ci + j);
        const C av = __ldg(va + j);
        const C x = BLCOC_LD(Xg + (int64_t)c * p + k);
        if constexpr (RESID) cmsub(acc, av, x);
        else cmac(acc, av, x);
      }
      if constexpr (RESID) {
        sr = fma((double)acc.x, (double)acc.x, sr);
        sr = fma((double)acc.y, (double)acc.y, sr);
      }
    }
    if constexpr (SPL > 1) {
#pragma unroll
      for (int o = LPR; o < LW; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (part == 0) Yt[tix(k, r)] = acc;
    } else {
      Yt[tix(k, r)] = acc;
    }
  }
}

__device__ __forceinline__ double warp_sum_fixed(double v) {
  // fixed butterfly order: deterministic
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------- kernels
// PassArgs::flag bits
constexpr int F_FIRST = 1;      // setup variant of a pass / norm-only residual / apply T
// F_SYM2 (blcoc_common.cuh): residual pass also R^T R; CholQR2 pass also Q1^T Q1
constexpr int F_UEXPL = 4;      // explicit-U variant: SpMM gram Y^T Y; pass C without the U update
constexpr int F_FORCE = 16;     // run even when the control block says the solve is done

#define BLCOC_PROLOGUE(CT)                                          \
  if (!(a.flag & F_FORCE) && BLCOC_LD(&a.ctrl->done)) return;       \
  if ((a.flag & F_FB) && BLCOC_LD(&a.ctrl->qr_fb) == 0) return;     \
  extern __shared__ __align__(16) unsigned char smem_raw[];         \
  CT* smem = reinterpret_cast<CT*>(smem_raw);                       \
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;       \
  const int64_t n = a.A.n;                                          \
  const int p = a.p;                                                \
  const int64_t nchunks = (n + CHUNK - 1) / CHUNK;                  \
  const int64_t cstride = (int64_t)vgrid * NWARP;

template <typename C>
__device__ __forceinline__ C* blk(double2* p) { return reinterpret_cast<C*>(p); }
template <typename S>
__device__ __forceinline__ const typename Cx<S>::T* vals_of(const CsrDev& A) {
  if constexpr (sizeof(S) == 8) return A.va;
  else return A.vaf;
}

// R = B - A X in FP64 (Sec. 3 residual, the setup of Algorithms 2-3); R is written in
// the working precision S.  flag&1: norms only; flag&2: also R^T R (cocg).
// Partials: [R^H R tri][R^T R tri][sum|B|^2, sum|R|^2]
template <int PP, typename S>
__device__ __forceinline__ void d_resid(const PassArgs& a, const int vblk, const int vgrid) {
  BLCOC_PROLOGUE(double2)
  using G = Geo<PP>;
  const bool norm_only = a.flag & F_FIRST, sym2 = a.flag & F_SYM2;
  double2* tR = smem + warp * G::TILE;
  double2* red = smem;
  GramAcc<G::NTRI, double> gh, gs;
  gh.init(G_HERM, p, lane);
  gs.init(G_SYM, p, lane);
  double sb = 0.0, sr = 0.0;
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    gather_rows<PP, double2, true>(tR, a.A, a.A.va, a.X, a.B, r0, p, lane, sb, sr);
    if (!norm_only) {
      __syncwarp();
      gh.template add<true>(tR, tR, lane);
      if (sym2) gs.template add<false>(tR, tR, lane);
      if constexpr (sizeof(S) == 8) store_tile<PP>(a.W, tR, r0, n, p, lane);
      else store_tile_f32<PP>(blk<float2>(a.W), tR, r0, n, p, lane);
    }
    __syncwarp();
  }
  sb = warp_sum_fixed(sb);
  sr = warp_sum_fixed(sr);
  __syncthreads();
  double2* out = a.partials + (int64_t)vblk * a.ne;
  const int E = tri_count(p);
  if (!norm_only) {
    cta_write_gram(gh, red, out, warp, lane);
    if (sym2) cta_write_gram(gs, red, out + E, warp, lane);
  }
  if (lane == 0) red[warp] = make_double2(sb, sr);
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = red[0];
    for (int w = 1; w < NWARP; ++w) { s.x += red[w].x; s.y += red[w].y; }
    out[2 * E] = s;
  }
}
template <int PP, typename S>
__global__ void __launch_bounds__(NWARP * 32) k_resid(const PassArgs a) {
  d_resid<PP, S>(a, blockIdx.x, gridDim.x);
}

// Y = A W over the chunk, W = the block in a.W; gram W^T Y (symmetric since A = A^T);
// out = Y T (flag=1, cocr: V = A Q = (A W) tau^{-1}) or out = Y (flag=0, cocg: a.W = S,
// out = A S).  flag&F_UEXPL: gram Y^T Y instead (explicit U = A S and U^T U).
// Partials: [W^T Y or Y^T Y tri].
template <int PP, typename S, bool OZ = false, int SPL = 1>
__device__ __forceinline__ void d_spmm_gram(const PassArgs& a, const int vblk, const int vgrid) {
  using C = typename Cx<S>::T;
  BLCOC_PROLOGUE(C)
  using G = Geo<PP, S>;
  constexpr bool M3A = m3_apply<PP, S, OZ>();
  // W for the Gram read from global memory: the FP64 SpMM at p = 32 and every tensor-core
  // SpMM (at p <= 16 its W^T Y slices are cut from global memory, so that the tile and the
  // per-warp Gram sums allow 3 CTAs per SM instead of 2)
  constexpr bool OT = one_tile<PP, S, OZ>() || OZ;
  C* T_s = smem;
  C* tiles = smem + ((M3A || OZ) ? 0 : mats_off<PP, S>(1));   // the tensor-core apply reads slices
  C* tY = tiles + warp * (OT ? 1 : 2) * G::TILE;
  C* tW = tY + G::TILE;
  const bool applyT = a.flag & 1;
  if constexpr (G::MATS_SMEM && !M3A && !OZ) {
    load_mat<PP>(T_s, a.mats + M_TINV * PMAX * PMAX, p);
    __syncthreads();
  }
  Fac<PP, S> T{G::MATS_SMEM ? T_s : reinterpret_cast<const C*>(a.mats + M_TINV * PMAX * PMAX), p};
  GramAcc<G::NTRI, S> g;
  g.init(G_SYM, p, lane);
  constexpr bool OZG = oz_gram<PP, OZ>();
  double* zsums = reinterpret_cast<double*>(tiles + NWARP * (OT ? 1 : 2) * G::TILE);   // tensor-core Gram sums
  if constexpr (OZG) {
    for (int i = lane; i < OzGramGeo<PP>::ACC; i += 32) zsums[warp * OzGramGeo<PP>::ACC + i] = 0.0;
  }
  double dummy0 = 0.0, dummy1 = 0.0;
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    gather_rows<PP, C, false, SPL>(tY, a.A, vals_of<S>(a.A), blk<C>(a.W), nullptr, r0, p, lane, dummy0, dummy1);
    if (!OT && !(a.flag & F_UEXPL)) load_tile<PP>(tW, blk<C>(a.W), r0, n, p, lane);   // Y^T Y needs no W
    __syncwarp();
    if constexpr (OZG) {
      if (a.flag & F_UEXPL)
        oz_gram_add<PP, true>(zsums + warp * OzGramGeo<PP>::ACC, tY, tY, p, lane);
      else
        oz_gram_add<PP, false, true>(zsums + warp * OzGramGeo<PP>::ACC, nullptr, tY, p, lane, a.W + r0 * p,
                                     (int)min((int64_t)CHUNK, n - r0));
    } else if constexpr (OT) {
      if (a.flag & F_UEXPL) g.template add<false>(tY, tY, lane);
      else g.template add_g<false>(a.W + r0 * p, (int)min((int64_t)CHUNK, n - r0), p, tY, lane);
    } else {
      g.template add<false>((a.flag & F_UEXPL) ? tY : tW, tY, lane);
    }
    __syncwarp();   // every lane has read Y for the Gram before the in-place apply
    if (applyT) {
      if constexpr (OZ) {
        oz_apply_any<PP, false, false>(tY, nullptr, tY, a.oz + OZ_T * OZ_SLOT_U2, p, lane);
      } else if constexpr (M3A) {
        tri_apply3_inplace<PP>(tY, Fac3(a.mats, M_TINV, p), p, lane);
      } else {
        tri_apply_inplace<PP, S>(tY, T, p, lane);
      }
      __syncwarp();
    }
    store_tile<PP>(blk<C>(a.V), tY, r0, n, p, lane);
    __syncwarp();
  }
  __syncthreads();
  if constexpr (OZG) oz_gram_write<PP, false>(zsums, a.partials + (int64_t)vblk * a.ne, p, NWARP);
  else cta_write_gram(g, reinterpret_cast<double2*>(tiles), a.partials + (int64_t)vblk * a.ne, warp, lane);
}
// Two tiles per warp allow at most 3 CTAs per SM (1 at PP = 32), so registers up to that
// bound cost no occupancy.
template <int PP, typename S, bool OZ = false, int SPL = 1>
__global__ void __launch_bounds__(NWARP * 32, PP >= 32 ? ((one_tile<PP, S, OZ>() || tc_one_tile<PP, OZ>()) ? 2 : 1) : 3)
    k_spmm_gram(const PassArgs a) {
  d_spmm_gram<PP, S, OZ, SPL>(a, blockIdx.x, gridDim.x);
}

// Y = A W, nothing else (blcoc_spmm).
template <int PP, typename S>
__device__ __forceinline__ void d_spmm_plain(const PassArgs& a, const int vblk, const int vgrid) {
  using C = typename Cx<S>::T;
  BLCOC_PROLOGUE(C)
  using G = Geo<PP, S>;
  C* tY = smem + warp * G::TILE;
  double d0 = 0.0, d1 = 0.0;
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    gather_rows<PP, C, false>(tY, a.A, vals_of<S>(a.A), blk<C>(a.W), nullptr, r0, p, lane, d0, d1);
    __syncwarp();
    store_tile<PP>(blk<C>(a.V), tY, r0, n, p, lane);
    __syncwarp();
  }
}
template <int PP, typename S>
__global__ void __launch_bounds__(NWARP * 32) k_spmm_plain(const PassArgs a) {
  d_spmm_plain<PP, S>(a, blockIdx.x, gridDim.x);
}

// bl_cocr_rq pass A (Algorithm 3, the new residual block before its QR): W_{m+1} = Q_m - U_m alpha'_m
// (Q_m stored by the previous pass C); gram W^H W for the Cholesky QR.
template <int PP, typename S, bool OZ = false>
__device__ __forceinline__ void d_cocr_passA(const PassArgs& a, const int vblk, const int vgrid) {
  using C = typename Cx<S>::T;
  BLCOC_PROLOGUE(C)
  using G = Geo<PP, S>;
  constexpr bool M3A = m3_apply<PP, S, OZ>();
  constexpr bool OZG = oz_gram<PP, OZ>();
  constexpr bool OT = one_tile<PP, S, OZ>();   // U read from global memory, four-product Gram
  constexpr bool OTZ = tc_one_tile<PP, OZ>();  // the same for the p = 32 tensor-core pass
  // W^H W: three products where the applies take them and two tiles are kept; the p <= 16
  // tensor-core pass forms it on the tensor cores
  constexpr bool M3G = ((M3A && !OT) || (OZ && !OZG)) && !OTZ;
  C* mA = smem;
  C* tiles = smem + (M3A ? 0 : mats_off<PP, S>(1));
  C* tW = tiles + warp * ((OT || OTZ) ? 1 : 2) * G::TILE;
  C* tU = tW + G::TILE;
  if constexpr (G::MATS_SMEM && !M3A) {
    load_mat<PP>(mA, a.mats + M_ALPHA * PMAX * PMAX, p);
    __syncthreads();
  }
  Fac<PP, S> AL{G::MATS_SMEM ? mA : reinterpret_cast<const C*>(a.mats + M_ALPHA * PMAX * PMAX), p};
  GramAcc<G::NTRI, S, M3G> g;
  g.init(G_HERM, p, lane);
  double* zsums = reinterpret_cast<double*>(tiles + NWARP * 2 * G::TILE);   // tensor-core Gram sums
  if constexpr (OZG) {
    for (int i = lane; i < OzGramGeo<PP>::ACC; i += 32) zsums[warp * OzGramGeo<PP>::ACC + i] = 0.0;
  }
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    load_tile<PP>(tW, blk<C>(a.Q), r0, n, p, lane);
    if constexpr (!OT && !OTZ) load_tile<PP>(tU, blk<C>(a.U), r0, n, p, lane);
    __syncwarp();
    if constexpr (OTZ) {
      oz_apply_gin<PP, true, true>(tW, tW, a.U + r0 * p, (int)min((int64_t)CHUNK, n - r0),
                                   a.oz + OZ_ALPHA * OZ_SLOT_U2, p, lane);   // W_{m+1} = Q_m - U_m alpha'
    } else if constexpr (OT) {
      apply_full3_g<PP, true>(tW, tW, a.U + r0 * p, (int)min((int64_t)CHUNK, n - r0), Fac3(a.mats, M_ALPHA, p), p,
                              lane);                                       // W_{m+1} = Q_m - U_m alpha'
    } else if constexpr (OZ) {
      oz_apply_any<PP, true, true>(tW, tW, tU, a.oz + OZ_ALPHA * OZ_SLOT_U2, p, lane);
      if constexpr (M3G) {
        __syncwarp();
        sd_tile<PP>(tU, tW, p, lane);                                         // U_m is no longer needed
      }
    } else if constexpr (M3A) {
      apply_full3<PP, true>(tW, tW, tU, Fac3(a.mats, M_ALPHA, p), p, lane);   // W_{m+1} = Q_m - U_m alpha'
      sd_tile<PP>(tU, tW, p, lane);                                           // U_m is no longer needed
    } else {
      apply_full<PP, S, true>(tW, tW, tU, AL, p, lane);    // W_{m+1} = Q_m - U_m alpha'
    }
    __syncwarp();
    if constexpr (OZG) oz_gram_add<PP, true>(zsums + warp * OzGramGeo<PP>::ACC, tW, tW, p, lane);
    else if constexpr (M3G) g.template add3<true>(tW, tU, lane);
    else g.template add<true>(tW, tW, lane);
    store_tile<PP>(blk<C>(a.W), tW, r0, n, p, lane);
    __syncwarp();
  }
  __syncthreads();
  if constexpr (OZG) oz_gram_write<PP, true>(zsums, a.partials + (int64_t)vblk * a.ne, p, NWARP);
  else cta_write_gram(g, reinterpret_cast<double2*>(tiles), a.partials + (int64_t)vblk * a.ne, warp, lane);
}
// FP64: two tiles per warp allow at most 3 CTAs per SM (1 at PP = 32), so registers up to
// that bound cost no occupancy.  The tensor-core variant keeps the compiler's own choice.
template <int PP, typename S, bool OZ = false>
__global__ void __launch_bounds__(NWARP * 32, PP >= 32 ? (one_tile<PP, S, OZ>() ? 2 : 1) : 3) k_cocr_passA(const PassArgs a) {
  d_cocr_passA<PP, S, OZ>(a, blockIdx.x, gridDim.x);
}
template <int PP>
__global__ void __launch_bounds__(NWARP * 32) k_cocr_passA_tc(const PassArgs a) {
  d_cocr_passA<PP, double, true>(a, blockIdx.x, gridDim.x);
}

// bl_cocr_rq pass C (Algorithm 3, the X, S and U updates) with Q_{m+1} = W_{m+1} T_{m+1} (stored
// for the next pass A):
//   X_{m+1} = X_m + S_m (alpha'_m xi_m);  S_{m+1} = Q_{m+1} + S_m beta'_m;
//   U_{m+1} = V_{m+1} + U_m beta'_m;  gram U^T U (next alpha').
// flag=1 (setup): S_0 = Q_0, U_0 = V_0, X untouched.  flag&F_UEXPL: no U update
// and no gram (U_{m+1} = A S_{m+1} is formed by the SpMM that follows).
template <int PP, typename S, bool OZ = false>
__device__ __forceinline__ void d_cocr_passC(const PassArgs& a, const int vblk, const int vgrid) {
  using C = typename Cx<S>::T;
  BLCOC_PROLOGUE(C)
  using G = Geo<PP, S>;
  const bool first = a.flag & 1;
  const bool uexpl = a.flag & F_UEXPL;
  constexpr bool M3A = m3_apply<PP, S, OZ>();
  constexpr bool OT = one_tile<PP, S, OZ>();   // S and U read from global memory
  constexpr bool OTZ = tc_one_tile<PP, OZ>();  // the same for the p = 32 tensor-core pass
  constexpr bool M3G = m3_gram<PP, S>() && !OT && !OTZ;
  // staged factors (four-product forms): T packed (upper triangle), alpha'xi, beta'
  C* mT = smem;
  C* mAX = smem + tri_packed<PP>() * mat_parts<S>();
  C* mB = mAX + PP * PP * mat_parts<S>();
  C* tiles = smem + (M3A ? 0 : passC_mats_elems<PP, S>());
  // two tiles per warp: Q is stored as soon as it is formed and read back (from L2, by the
  // same threads) for the S update, so X, S and Q never need three tiles at once
  C* b0 = tiles + warp * ((OT || OTZ) ? 1 : 2) * G::TILE;
  C* b1 = b0 + G::TILE;
  if constexpr (G::MATS_SMEM && !M3A) {
    load_mat_tri<PP>(mT, a.mats + M_TINV * PMAX * PMAX, p);
    load_mat<PP>(mAX, a.mats + M_ALPHAXI * PMAX * PMAX, p);
    load_mat<PP>(mB, a.mats + M_BETA * PMAX * PMAX, p);
    __syncthreads();
  }
  Fac<PP, S> AX{G::MATS_SMEM ? mAX : reinterpret_cast<const C*>(a.mats + M_ALPHAXI * PMAX * PMAX), p};
  Fac<PP, S> BE{G::MATS_SMEM ? mB : reinterpret_cast<const C*>(a.mats + M_BETA * PMAX * PMAX), p};
  GramAcc<G::NTRI, S, M3G> g;
  g.init(G_SYM, p, lane);
  if constexpr (OT || OTZ) {
    // one tile per warp (p = 32): the same updates, S_m and U_m streamed from global memory
    // (FP64 three-product applies, or the tensor-core applies splitting them from there)
    for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
      const int64_t r0 = c * CHUNK;
      const int rows = (int)min((int64_t)CHUNK, n - r0);
      load_tile<PP>(b0, a.W, r0, n, p, lane);
      __syncwarp();
      if constexpr (OTZ) oz_apply_any<PP, false, false>(b0, nullptr, b0, a.oz + OZ_T * OZ_SLOT_U2, p, lane);
      else tri_apply3_inplace<PP>(b0, Fac3(a.mats, M_TINV, p), p, lane);   // Q_{m+1}
      __syncwarp();
      store_tile<PP>(a.Q, b0, r0, n, p, lane);
      if (!first) {
        __syncwarp();
        load_tile<PP>(b0, a.X, r0, n, p, lane);
        __syncwarp();
        if constexpr (OTZ)
          oz_apply_gin<PP, false, true>(b0, b0, a.S + r0 * p, rows, a.oz + OZ_ALPHAXI * OZ_SLOT_U2, p, lane);
        else
          apply_full3_g<PP, false>(b0, b0, a.S + r0 * p, rows, Fac3(a.mats, M_ALPHAXI, p), p, lane);   // X_{m+1}
        __syncwarp();
        store_tile<PP>(a.X, b0, r0, n, p, lane);
        __syncwarp();
        load_tile<PP>(b0, a.Q, r0, n, p, lane);   // Q_{m+1}, just stored
        __syncwarp();
        if constexpr (OTZ)
          oz_apply_gin<PP, false, true>(b0, b0, a.S + r0 * p, rows, a.oz + OZ_BETA * OZ_SLOT_U2, p, lane);
        else
          apply_full3_g<PP, false>(b0, b0, a.S + r0 * p, rows, Fac3(a.mats, M_BETA, p), p, lane);   // S_{m+1}
      }
      __syncwarp();
      store_tile<PP>(a.S, b0, r0, n, p, lane);       // (setup: S_0 = Q_0)
      __syncwarp();
      if (uexpl) continue;
      load_tile<PP>(b0, a.V, r0, n, p, lane);
      __syncwarp();
      if (!first) {
        if constexpr (OTZ)
          oz_apply_gin<PP, false, true>(b0, b0, a.U + r0 * p, rows, a.oz + OZ_BETA * OZ_SLOT_U2, p, lane);
        else
          apply_full3_g<PP, false>(b0, b0, a.U + r0 * p, rows, Fac3(a.mats, M_BETA, p), p, lane);   // U_{m+1}
        __syncwarp();
      }
      g.template add<false>(b0, b0, lane);
      store_tile<PP>(a.U, b0, r0, n, p, lane);
      __syncwarp();
    }
    if (uexpl) return;
    __syncthreads();
    cta_write_gram(g, reinterpret_cast<double2*>(tiles), a.partials + (int64_t)vblk * a.ne, warp, lane);
    return;
  }
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    load_tile<PP>(b0, blk<C>(a.W), r0, n, p, lane);
    __syncwarp();
    if constexpr (OZ) {
      oz_apply_any<PP, false, false>(b0, nullptr, b0, a.oz + OZ_T * OZ_SLOT_U2, p, lane);
    } else if constexpr (M3A) {
      tri_apply3_inplace<PP>(b0, Fac3(a.mats, M_TINV, p), p, lane);       // Q_{m+1}
    } else if constexpr (G::MATS_SMEM) {
      tri_apply_inplace<PP, S>(b0, FacTri<PP, S>{mT}, p, lane);     // Q_{m+1}
    } else {
      tri_apply_inplace<PP, S>(b0, Fac<PP, S>{reinterpret_cast<const C*>(a.mats + M_TINV * PMAX * PMAX), p}, p,
                               lane);
    }
    __syncwarp();
    store_tile<PP>(blk<C>(a.Q), b0, r0, n, p, lane);
    if (!first) {
      __syncwarp();
      load_tile<PP>(b0, blk<C>(a.X), r0, n, p, lane);
      load_tile<PP>(b1, blk<C>(a.S), r0, n, p, lane);
      __syncwarp();
      if constexpr (OZ) {
        oz_apply_any<PP, false, true>(b0, b0, b1, a.oz + OZ_ALPHAXI * OZ_SLOT_U2, p, lane);
      } else if constexpr (M3A) {
        apply_full3<PP, false>(b0, b0, b1, Fac3(a.mats, M_ALPHAXI, p), p, lane);   // X_{m+1}
      } else {
        apply_full<PP, S, false>(b0, b0, b1, AX, p, lane);  // X_{m+1}
      }
      __syncwarp();
      store_tile<PP>(blk<C>(a.X), b0, r0, n, p, lane);
      __syncwarp();
      load_tile<PP>(b0, blk<C>(a.Q), r0, n, p, lane);      // Q_{m+1}, just stored
      __syncwarp();
      if constexpr (OZ) {
        oz_apply_any<PP, false, true>(b0, b0, b1, a.oz + OZ_BETA * OZ_SLOT_U2, p, lane);
      } else if constexpr (M3A) {
        apply_full3<PP, false>(b0, b0, b1, Fac3(a.mats, M_BETA, p), p, lane);      // S_{m+1} = Q + S beta'
      } else {
        apply_full<PP, S, false>(b0, b0, b1, BE, p, lane);  // S_{m+1} = Q + S beta'
      }
      __syncwarp();
    }
    store_tile<PP>(blk<C>(a.S), b0, r0, n, p, lane);       // (setup: S_0 = Q_0)
    __syncwarp();
    if (uexpl) continue;
    load_tile<PP>(b0, blk<C>(a.V), r0, n, p, lane);
    if (!first) load_tile<PP>(b1, blk<C>(a.U), r0, n, p, lane);
    __syncwarp();
    if (!first) {
      if constexpr (OZ) {
        oz_apply_any<PP, false, true>(b0, b0, b1, a.oz + OZ_BETA * OZ_SLOT_U2, p, lane);
      } else if constexpr (M3A) {
        apply_full3<PP, false>(b0, b0, b1, Fac3(a.mats, M_BETA, p), p, lane);      // U_{m+1} = V + U beta'
      } else {
        apply_full<PP, S, false>(b0, b0, b1, BE, p, lane);  // U_{m+1} = V + U beta'
      }
      __syncwarp();
    }
    if constexpr (M3G) {
      sd_tile<PP>(b1, b0, p, lane);   // U_m is no longer needed
      __syncwarp();
      g.template add3<false>(b0, b1, lane);
    } else {
      g.template add<false>(b0, b0, lane);
    }
    store_tile<PP>(blk<C>(a.U), b0, r0, n, p, lane);
    __syncwarp();
  }
  if (uexpl) return;
  __syncthreads();
  cta_write_gram(g, reinterpret_cast<double2*>(tiles), a.partials + (int64_t)vblk * a.ne, warp, lane);
}
// Registers bounded to what 3 CTAs per SM allow (2 for the one-tile pass at p = 32), which
// the shared memory also allows; left free the compiler takes about 220 at p = 16.
template <int PP, typename S, bool OZ = false>
__global__ void __launch_bounds__(NWARP * 32, one_tile<PP, S, OZ>() ? 2 : 3) k_cocr_passC(const PassArgs a) {
  d_cocr_passC<PP, S, OZ>(a, blockIdx.x, gridDim.x);
}
// The tensor-core pass C: up to p = 16 its shared memory allows 3 CTAs per SM, and so does
// this bound on its registers (otherwise about 238, 2 per SM); at p = 32 (one tile per
// warp) two.
template <int PP>
__global__ void __launch_bounds__(NWARP * 32, PP >= 32 ? 2 : 3) k_cocr_passC_tc(const PassArgs a) {
  d_cocr_passC<PP, double, true>(a, blockIdx.x, gridDim.x);
}

// bl_cocg_rq pass 1 (Algorithm 2, the X update and the new residual block), Q_m stored by
// the previous pass 2:
//   W_{m+1} = Q_m - (A S_m) alpha'_m;  X_{m+1} = X_m + S_m (alpha'_m xi_m);
//   grams W^H W (QR) and W^T W (Q^T Q of the beta' step).  Partials: [W^H W tri][W^T W tri].
template <int PP, typename S>
__device__ __forceinline__ void d_cocg_pass1(const PassArgs& a, const int vblk, const int vgrid) {
  using C = typename Cx<S>::T;
  BLCOC_PROLOGUE(C)
  using G = Geo<PP, S>;
  constexpr bool M3A = m3_apply<PP, S>();
  constexpr bool M3G = m3_gram<PP, S>() && PP <= 16;   // two Grams of 17 slots at PP = 32: no room
  C* mAX = smem;
  C* mA = smem + PP * PP * mat_parts<S>();
  C* tiles = smem + (M3A ? 0 : mats_off<PP, S>(2));
  C* b0 = tiles + warp * 3 * G::TILE;
  C* b1 = b0 + G::TILE;
  C* b2 = b1 + G::TILE;
  if constexpr (G::MATS_SMEM && !M3A) {
    load_mat<PP>(mAX, a.mats + M_ALPHAXI * PMAX * PMAX, p);
    load_mat<PP>(mA, a.mats + M_ALPHA * PMAX * PMAX, p);
    __syncthreads();
  }
  Fac<PP, S> AX{G::MATS_SMEM ? mAX : reinterpret_cast<const C*>(a.mats + M_ALPHAXI * PMAX * PMAX), p};
  Fac<PP, S> AL{G::MATS_SMEM ? mA : reinterpret_cast<const C*>(a.mats + M_ALPHA * PMAX * PMAX), p};
  GramAcc<G::NTRI, S, M3G> gh, gs;
  gh.init(G_HERM, p, lane);
  gs.init(G_SYM, p, lane);
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    load_tile<PP>(b0, blk<C>(a.Q), r0, n, p, lane);
    load_tile<PP>(b1, blk<C>(a.V), r0, n, p, lane);
    __syncwarp();
    if constexpr (M3A) apply_full3<PP, true>(b0, b0, b1, Fac3(a.mats, M_ALPHA, p), p, lane);
    else apply_full<PP, S, true>(b0, b0, b1, AL, p, lane);     // W_{m+1} = Q_m - A S_m alpha'
    __syncwarp();
    load_tile<PP>(b1, blk<C>(a.S), r0, n, p, lane);
    load_tile<PP>(b2, blk<C>(a.X), r0, n, p, lane);
    __syncwarp();
    if constexpr (M3A) apply_full3<PP, false>(b2, b2, b1, Fac3(a.mats, M_ALPHAXI, p), p, lane);
    else apply_full<PP, S, false>(b2, b2, b1, AX, p, lane);    // X_{m+1}
    if constexpr (M3G) {
      sd_tile<PP>(b1, b0, p, lane);   // S_m is no longer needed (each lane rewrites its own row)
      __syncwarp();
      gh.template add3<true>(b0, b1, lane);
      gs.template add3<false>(b0, b1, lane);
    } else {
      gh.template add<true>(b0, b0, lane);
      gs.template add<false>(b0, b0, lane);
    }
    __syncwarp();
    store_tile<PP>(blk<C>(a.X), b2, r0, n, p, lane);
    store_tile<PP>(blk<C>(a.W), b0, r0, n, p, lane);
    __syncwarp();
  }
  __syncthreads();
  double2* out = a.partials + (int64_t)vblk * a.ne;
  cta_write_gram(gh, reinterpret_cast<double2*>(tiles), out, warp, lane);
  cta_write_gram(gs, reinterpret_cast<double2*>(tiles), out + tri_count(p), warp, lane);
}
template <int PP, typename S>
__global__ void __launch_bounds__(NWARP * 32) k_cocg_pass1(const PassArgs a) {
  d_cocg_pass1<PP, S>(a, blockIdx.x, gridDim.x);
}

// bl_cocg_rq pass 1 with the p x p updates on the tensor cores (option fp64_tc): the same
// results as d_cocg_pass1, in two tiles per warp (the Grams are taken from W before X is
// updated, so the slice digits of p = 32 fit beside the tiles).  The self-Grams W^H W and
// W^T W run in three real products from W and its companion tile up to p = 16, in four at
// p = 32 (two three-product accumulators would not fit in registers there).
template <int PP>
__device__ __forceinline__ void d_cocg_pass1_tc(const PassArgs& a, const int vblk, const int vgrid) {
  using C = double2;
  BLCOC_PROLOGUE(C)
  using G = Geo<PP, double>;
  constexpr bool M3G = PP <= 16;
  C* tiles = smem;   // no staged factors: the applies read slice fragments
  C* b0 = tiles + warp * 2 * G::TILE;
  C* b1 = b0 + G::TILE;
  GramAcc<G::NTRI, double, M3G> gh, gs;
  gh.init(G_HERM, p, lane);
  gs.init(G_SYM, p, lane);
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    load_tile<PP>(b0, a.Q, r0, n, p, lane);
    load_tile<PP>(b1, a.V, r0, n, p, lane);
    __syncwarp();
    oz_apply_any<PP, true, true>(b0, b0, b1, a.oz + OZ_ALPHA * OZ_SLOT_U2, p, lane);   // W = Q - A S alpha'
    __syncwarp();
    if constexpr (M3G) {
      sd_tile<PP>(b1, b0, p, lane);   // A S_m is no longer needed
      __syncwarp();
      gh.template add3<true>(b0, b1, lane);
      gs.template add3<false>(b0, b1, lane);
    } else {
      gh.template add<true>(b0, b0, lane);
      gs.template add<false>(b0, b0, lane);
    }
    store_tile<PP>(a.W, b0, r0, n, p, lane);
    __syncwarp();
    load_tile<PP>(b0, a.X, r0, n, p, lane);
    load_tile<PP>(b1, a.S, r0, n, p, lane);
    __syncwarp();
    oz_apply_any<PP, false, true>(b0, b0, b1, a.oz + OZ_ALPHAXI * OZ_SLOT_U2, p, lane);   // X_{m+1}
    __syncwarp();
    store_tile<PP>(a.X, b0, r0, n, p, lane);
    __syncwarp();
  }
  __syncthreads();
  double2* out = a.partials + (int64_t)vblk * a.ne;
  cta_write_gram(gh, reinterpret_cast<double2*>(tiles), out, warp, lane);
  cta_write_gram(gs, reinterpret_cast<double2*>(tiles), out + tri_count(p), warp, lane);
}
template <int PP>
__global__ void __launch_bounds__(NWARP * 32, PP >= 32 ? 1 : 2) k_cocg_pass1_tc(const PassArgs a) {
  d_cocg_pass1_tc<PP>(a, blockIdx.x, gridDim.x);
}

// bl_cocg_rq pass 2 on the tensor cores: Q_{m+1} = W_{m+1} T_{m+1} (stored), S_{m+1} =
// Q_{m+1} + S_m beta'_m (setup, flag 1: S_0 = Q_0).
template <int PP>
__device__ __forceinline__ void d_cocg_pass2_tc(const PassArgs& a, const int vblk, const int vgrid) {
  using C = double2;
  BLCOC_PROLOGUE(C)
  using G = Geo<PP, double>;
  const bool first = a.flag & 1;
  C* tiles = smem;
  C* b0 = tiles + warp * 2 * G::TILE;
  C* b1 = b0 + G::TILE;
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    load_tile<PP>(b0, a.W, r0, n, p, lane);
    if (!first) load_tile<PP>(b1, a.S, r0, n, p, lane);
    __syncwarp();
    oz_apply_any<PP, false, false>(b0, nullptr, b0, a.oz + OZ_T * OZ_SLOT_U2, p, lane);   // Q_{m+1}
    __syncwarp();
    store_tile<PP>(a.Q, b0, r0, n, p, lane);
    if (!first) {
      __syncwarp();
      oz_apply_any<PP, false, true>(b0, b0, b1, a.oz + OZ_BETA * OZ_SLOT_U2, p, lane);   // S_{m+1}
    }
    __syncwarp();
    store_tile<PP>(a.S, b0, r0, n, p, lane);
    __syncwarp();
  }
}
template <int PP>
__global__ void __launch_bounds__(NWARP * 32) k_cocg_pass2_tc(const PassArgs a) {
  d_cocg_pass2_tc<PP>(a, blockIdx.x, gridDim.x);
}

// bl_cocg_rq pass 2 (Algorithm 2, the S update): Q_{m+1} = W_{m+1} T_{m+1} (stored for the next
// pass 1), S_{m+1} = Q_{m+1} + S_m beta'_m.  flag=1 (setup): S_0 = Q_0 = W_0 T_0.
template <int PP, typename S>
__device__ __forceinline__ void d_cocg_pass2(const PassArgs& a, const int vblk, const int vgrid) {
  using C = typename Cx<S>::T;
  BLCOC_PROLOGUE(C)
  using G = Geo<PP, S>;
  const bool first = a.flag & 1;
  constexpr bool M3A = m3_apply<PP, S>();
  C* mT = smem;
  C* mB = smem + PP * PP * mat_parts<S>();
  C* tiles = smem + (M3A ? 0 : mats_off<PP, S>(2));
  C* b0 = tiles + warp * 2 * G::TILE;
  C* b1 = b0 + G::TILE;
  if constexpr (G::MATS_SMEM && !M3A) {
    load_mat<PP>(mT, a.mats + M_TINV * PMAX * PMAX, p);
    load_mat<PP>(mB, a.mats + M_BETA * PMAX * PMAX, p);
    __syncthreads();
  }
  Fac<PP, S> T{G::MATS_SMEM ? mT : reinterpret_cast<const C*>(a.mats + M_TINV * PMAX * PMAX), p};
  Fac<PP, S> BE{G::MATS_SMEM ? mB : reinterpret_cast<const C*>(a.mats + M_BETA * PMAX * PMAX), p};
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    load_tile<PP>(b0, blk<C>(a.W), r0, n, p, lane);
    if (!first) load_tile<PP>(b1, blk<C>(a.S), r0, n, p, lane);
    __syncwarp();
    if constexpr (M3A) tri_apply3_inplace<PP>(b0, Fac3(a.mats, M_TINV, p), p, lane);
    else tri_apply_inplace<PP, S>(b0, T, p, lane);            // Q_{m+1}
    __syncwarp();
    store_tile<PP>(blk<C>(a.Q), b0, r0, n, p, lane);
    __syncwarp();
    if (!first) {
      if constexpr (M3A) apply_full3<PP, false>(b0, b0, b1, Fac3(a.mats, M_BETA, p), p, lane);
      else apply_full<PP, S, false>(b0, b0, b1, BE, p, lane);
    }
    __syncwarp();
    store_tile<PP>(blk<C>(a.S), b0, r0, n, p, lane);
    __syncwarp();
  }
}
template <int PP, typename S>
__global__ void __launch_bounds__(NWARP * 32) k_cocg_pass2(const PassArgs a) {
  d_cocg_pass2<PP, S>(a, blockIdx.x, gridDim.x);
}

// CholQR2, second pass (the thin QR of Sec. 2.2 with one re-orthogonalisation): the
// first Cholesky factor's T1 is applied to W in place (W <- Q1 = W T1, stored) and the
// Gram Q1^H Q1 is formed for the second factor.  flag & F_SYM2 (bl_cocg_rq): also the
// unconjugated Q1^T Q1, from which the stage after it forms Q^T Q of the final basis (a
// well-conditioned block, unlike the W the first factor came from).  The shifted-CholQR3
// fallback runs this pass twice.  Partials: [Q1^H Q1 tri] (+ [Q1^T Q1 tri]).
template <int PP, typename S>
__device__ __forceinline__ void d_qr2(const PassArgs& a, const int vblk, const int vgrid) {
  using C = typename Cx<S>::T;
  BLCOC_PROLOGUE(C)
  using G = Geo<PP, S>;
  constexpr bool M3A = m3_apply<PP, S>();
  constexpr bool M3G = qr2_m3<PP, S>();
  const bool sym2 = a.flag & F_SYM2;
  C* mT = smem;
  C* tiles = smem + (M3A ? 0 : mats_off<PP, S>(1));
  C* tW = tiles + warp * (M3G ? 2 : 1) * G::TILE;
  C* tSD = tW + G::TILE;   // (re + im, im - re) companion of W for the three-product Gram
  if constexpr (G::MATS_SMEM && !M3A) {
    load_mat<PP>(mT, a.mats + M_TINV * PMAX * PMAX, p);
    __syncthreads();
  }
  Fac<PP, S> T{G::MATS_SMEM ? mT : reinterpret_cast<const C*>(a.mats + M_TINV * PMAX * PMAX), p};
  GramAcc<G::NTRI, S, M3G> g;
  g.init(G_HERM, p, lane);
  constexpr bool M3S = M3G;
  GramAcc<G::NTRI, S, M3S> gs;
  gs.init(G_SYM, p, lane);
  for (int64_t c = (int64_t)vblk * NWARP + warp; c < nchunks; c += cstride) {
    const int64_t r0 = c * CHUNK;
    load_tile<PP>(tW, blk<C>(a.W), r0, n, p, lane);
    __syncwarp();
    if constexpr (M3A) tri_apply3_inplace<PP>(tW, Fac3(a.mats, M_TINV, p), p, lane);
    else tri_apply_inplace<PP, S>(tW, T, p, lane);
    if constexpr (M3G) sd_tile<PP>(tSD, tW, p, lane);
    __syncwarp();
    if constexpr (M3G) g.template add3<true>(tW, tSD, lane);
    else g.template add<true>(tW, tW, lane);
    if (sym2) {
      if constexpr (M3S) gs.template add3<false>(tW, tSD, lane);
      else gs.template add<false>(tW, tW, lane);
    }
    store_tile<PP>(blk<C>(a.W), tW, r0, n, p, lane);
    __syncwarp();
  }
  __syncthreads();
  double2* out = a.partials + (int64_t)vblk * a.ne;
  cta_write_gram(g, reinterpret_cast<double2*>(tiles), out, warp, lane);
  if (sym2) cta_write_gram(gs, reinterpret_cast<double2*>(tiles), out + tri_count(p), warp, lane);
}
template <int PP, typename S>
__global__ void __launch_bounds__(NWARP * 32) k_qr2(const PassArgs a) {
  d_qr2<PP, S>(a, blockIdx.x, gridDim.x);
}

// Refinement update of the mixed-precision form: X (FP64) += D (working precision, held
// in a.V), elementwise over the n x p block.
template <int PP, typename S>
__global__ void __launch_bounds__(256) k_axpy(const PassArgs a) {
  using C = typename Cx<S>::T;
  const int64_t total = a.A.n * a.p;
  const C* D = blk<C>(a.V);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const C d = D[e];
    double2 x = a.X[e];
    x.x += (double)d.x;
    x.y += (double)d.y;
    a.X[e] = x;
  }
}

#undef BLCOC_PROLOGUE

// ---------------------------------------------------------------------------------- launch
enum PassKind { K_RESID = 0, K_SPMM_GRAM, K_SPMM_PLAIN, K_COCR_A, K_COCR_C, K_COCG_1, K_COCG_2, K_AXPY, K_QR2, K_NKIND };

// OZ: the tensor-core variant, whose pass A and SpMM also keep every warp's running Gram
// sums (OzGramGeo<PP>::ACC doubles) after the tiles.
template <int PP, typename S, bool OZ = false>
constexpr size_t pass_smem(int kind) {
  using G = Geo<PP, S>;
  const size_t esz = sizeof(typename Cx<S>::T);
  const size_t tile = (size_t)G::TILE * esz;
  const int nmats[K_NKIND] = {0, 1, 0, 1, 3, 2, 2, 0, 1};
  const int ntiles[K_NKIND] = {1, 2, 1, 2, 2, 3, 2, 0, 1};
  if (kind == K_RESID) return (size_t)NWARP * PP * CHUNK * sizeof(double2);   // FP64 residual tile
  // three-product applies read their factors from global memory (L1); the CholQR2 pass
  // then keeps a second tile for the companion of its three-product Gram
  const bool oz_kind = OZ && (kind == K_SPMM_GRAM || kind == K_COCR_A || kind == K_COCR_C || kind == K_COCG_1 ||
                              kind == K_COCG_2);
  const bool oz_cocg = OZ && (kind == K_COCG_1 || kind == K_COCG_2);
  // no staged factors: three-product applies, the bl_cocg_rq tensor-core passes and the
  // tensor-core SpMM (their applies read slice fragments)
  const bool m3 = (m3_apply<PP, S>() && !oz_kind) || oz_cocg || (OZ && kind == K_SPMM_GRAM);
  const bool ot = ((one_tile<PP, S, OZ>() || tc_one_tile<PP, OZ>()) &&
                   (kind == K_SPMM_GRAM || kind == K_COCR_A || kind == K_COCR_C)) ||
                  (OZ && kind == K_SPMM_GRAM);
  const int nt = (kind == K_QR2 && qr2_m3<PP, S>()) ? 2 : ((oz_cocg ? 2 : ntiles[kind]) / (ot ? 2 : 1));
  const size_t mats =
      m3 ? 0 : (size_t)(kind == K_COCR_C ? passC_mats_elems<PP, S>() : mats_off<PP, S>(nmats[kind])) * esz;
  size_t s = mats + (size_t)NWARP * nt * tile;
  // the CTA-level Gram reduction reuses the tile area: NWARP * E double2 (two Grams at most
  // are written one after the other, so one E-sized area suffices)
  const size_t red = (size_t)NWARP * tri_count(PP) * sizeof(double2);
  const bool has_gram =
      kind == K_SPMM_GRAM || kind == K_COCR_A || kind == K_COCR_C || kind == K_COCG_1 || kind == K_QR2;
  if (has_gram && s < mats + red) s = mats + red;
  if (oz_gram<PP, OZ>() && (kind == K_COCR_A || kind == K_SPMM_GRAM))
    s += (size_t)NWARP * OzGramGeo<PP>::ACC * sizeof(double);
  return s;
}

// The pass kernel of one kind (OZ: the tensor-core variant where one exists).
template <int PP, typename S, bool OZ>
const void* pass_kernel(int kind) {
  switch (kind) {
    case K_RESID: return (const void*)k_resid<PP, S>;
    case K_SPMM_GRAM: return (const void*)k_spmm_gram<PP, S, OZ>;
    case K_SPMM_PLAIN: return (const void*)k_spmm_plain<PP, S>;
    case K_COCR_A:
      if constexpr (OZ) return (const void*)k_cocr_passA_tc<PP>;
      else return (const void*)k_cocr_passA<PP, S>;
    case K_COCR_C:
      if constexpr (OZ) return (const void*)k_cocr_passC_tc<PP>;
      else return (const void*)k_cocr_passC<PP, S>;
    case K_COCG_1:
      if constexpr (OZ) return (const void*)k_cocg_pass1_tc<PP>;
      else return (const void*)k_cocg_pass1<PP, S>;
    case K_COCG_2:
      if constexpr (OZ) return (const void*)k_cocg_pass2_tc<PP>;
      else return (const void*)k_cocg_pass2<PP, S>;
    case K_QR2: return (const void*)k_qr2<PP, S>;
    default: return nullptr;
  }
}

// One wave of CTAs: SMs x the CTAs per SM the kernel's registers AND shared memory allow
// (occupancy of that exact kernel, cached per device; at most 4), or fewer when the rows
// need fewer.  Call after the kernel set's prepare() (shared-memory limits).
template <int PP, typename S, bool OZ>
int pass_grid(int64_t n, int kind, int num_sms) {
  if (kind == K_AXPY) return num_sms * 4;
  static int cache[64][K_NKIND] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = (dev >= 0 && dev < 64) ? cache[dev][kind] : 0;
  if (per_sm == 0) {
    const size_t smem = pass_smem<PP, S, OZ>(kind);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_kernel<PP, S, OZ>(kind), NWARP * 32, smem) ==
            cudaSuccess &&
        per_sm > 0) {
      per_sm = per_sm > 4 ? 4 : per_sm;
      if (dev >= 0 && dev < 64) cache[dev][kind] = per_sm;
    } else {   // shared-memory limit not raised yet: shared memory alone decides, uncached
      cudaGetLastError();
      per_sm = (int)((227u * 1024u) / (smem + 1024u));
      per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    }
  }
  const int64_t nchunks = (n + CHUNK - 1) / CHUNK;
  int64_t want = (nchunks + NWARP - 1) / NWARP;
  int64_t g = (int64_t)num_sms * per_sm;
  if (want < g) g = want;
  return (int)(g < 1 ? 1 : g);
}

template <int PP, typename S, int KIND, void (*K)(const PassArgs), bool OZ = false>
void launch_pass(const PassArgs& a, cudaStream_t s) {
  if constexpr (KIND == K_AXPY) K<<<a.grid, 256, 0, s>>>(a);
  else K<<<a.grid, NWARP * 32, pass_smem<PP, S, OZ>(KIND), s>>>(a);
}

// The SpMM with SPL lane groups per row, where the bundle fits a warp.
template <int PP, typename S, bool OZ, int SPL>
constexpr LaunchFn spmm_split_fn() {
  if constexpr (Geo<PP>::LPR * SPL <= 32) return &launch_pass<PP, S, K_SPMM_GRAM, k_spmm_gram<PP, S, OZ, SPL>, OZ>;
  else return nullptr;
}
template <int PP, typename S, bool OZ, int SPL>
void set_spmm_split_smem() {
  if constexpr (Geo<PP>::LPR * SPL <= 32)
    cudaFuncSetAttribute(k_spmm_gram<PP, S, OZ, SPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pass_smem<PP, S, OZ>(K_SPMM_GRAM));
}

template <int PP, typename S>
void prepare_pass_kernels() {
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaFuncSetAttribute(k_resid<PP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem<PP, S>(K_RESID));
  cudaFuncSetAttribute(k_spmm_gram<PP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, S>(K_SPMM_GRAM));
  cudaFuncSetAttribute(k_spmm_plain<PP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, S>(K_SPMM_PLAIN));
  cudaFuncSetAttribute(k_cocr_passA<PP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, S>(K_COCR_A));
  cudaFuncSetAttribute(k_cocr_passC<PP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, S>(K_COCR_C));
  cudaFuncSetAttribute(k_cocg_pass1<PP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, S>(K_COCG_1));
  cudaFuncSetAttribute(k_cocg_pass2<PP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, S>(K_COCG_2));
  cudaFuncSetAttribute(k_qr2<PP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem<PP, S>(K_QR2));
  set_spmm_split_smem<PP, S, false, 2>();
  set_spmm_split_smem<PP, S, false, 4>();
  done[dev] = true;
}

template <int PP, typename S>
const KernelSet& kernel_set() {
  static const KernelSet ks = {
      &launch_pass<PP, S, K_RESID, k_resid<PP, S>>,
      &launch_pass<PP, S, K_SPMM_GRAM, k_spmm_gram<PP, S>>,
      &launch_pass<PP, S, K_SPMM_PLAIN, k_spmm_plain<PP, S>>,
      &launch_pass<PP, S, K_COCR_A, k_cocr_passA<PP, S>>,
      &launch_pass<PP, S, K_COCR_C, k_cocr_passC<PP, S>>,
      &launch_pass<PP, S, K_COCG_1, k_cocg_pass1<PP, S>>,
      &launch_pass<PP, S, K_COCG_2, k_cocg_pass2<PP, S>>,
      &launch_pass<PP, S, K_AXPY, k_axpy<PP, S>>,
      &launch_pass<PP, S, K_QR2, k_qr2<PP, S>>,
      spmm_split_fn<PP, S, false, 2>(),
      spmm_split_fn<PP, S, false, 4>(),
      &pass_grid<PP, S, false>,
      &prepare_pass_kernels<PP, S>,
  };
  return ks;
}

template <int PP>
void prepare_pass_kernels_tc() {
  prepare_pass_kernels<PP, double>();
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaFuncSetAttribute(k_spmm_gram<PP, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, double, true>(K_SPMM_GRAM));
  cudaFuncSetAttribute(k_cocr_passA_tc<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, double, true>(K_COCR_A));
  cudaFuncSetAttribute(k_cocr_passC_tc<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, double, true>(K_COCR_C));
  cudaFuncSetAttribute(k_cocg_pass1_tc<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, double, true>(K_COCG_1));
  cudaFuncSetAttribute(k_cocg_pass2_tc<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<PP, double, true>(K_COCG_2));
  set_spmm_split_smem<PP, double, true, 2>();
  set_spmm_split_smem<PP, double, true, 4>();
  done[dev] = true;
}

// Launch-grid rule of the tensor-core set.
template <int PP>
int pass_grid_tc(int64_t n, int kind, int num_sms) {
  return pass_grid<PP, double, true>(n, kind, num_sms);
}

template <int PP>
const KernelSet& kernel_set_tc() {
  static const KernelSet ks = {
      &launch_pass<PP, double, K_RESID, k_resid<PP, double>>,
      &launch_pass<PP, double, K_SPMM_GRAM, k_spmm_gram<PP, double, true>, true>,
      &launch_pass<PP, double, K_SPMM_PLAIN, k_spmm_plain<PP, double>>,
      &launch_pass<PP, double, K_COCR_A, k_cocr_passA_tc<PP>, true>,
      &launch_pass<PP, double, K_COCR_C, k_cocr_passC_tc<PP>, true>,
      &launch_pass<PP, double, K_COCG_1, k_cocg_pass1_tc<PP>, true>,
      &launch_pass<PP, double, K_COCG_2, k_cocg_pass2_tc<PP>, true>,
      &launch_pass<PP, double, K_AXPY, k_axpy<PP, double>>,
      &launch_pass<PP, double, K_QR2, k_qr2<PP, double>>,
      spmm_split_fn<PP, double, true, 2>(),
      spmm_split_fn<PP, double, true, 4>(),
      &pass_grid_tc<PP>,
      &prepare_pass_kernels_tc<PP>,
  };
  return ks;
}

}  // namespace blcoc
