// FP64-accurate products Y (32 rows x p) = X (32 x p) * M (p x p), complex, on the bf16
// tensor cores (warp-level mma.sync), by exact integer slicing (the scheme of Ozaki,
// Ogita, Oishi and Rump: split both operands into slices whose pairwise products are
// exact in the accumulator, multiply slice by slice, add the exact partial products).
//
// Complex as real: Y' = [Yr | Yi] = [Xr | Xi] * [[Mr, Mi], [-Mi, Mr]] with K = N = 2p.
// Slicing: every row of X' is scaled by 2^e (e: above its largest magnitude) and every
// column of M' by 2^f; each value becomes a 56-bit fixed-point magnitude cut into eight
// 7-bit digits (sign kept), digit s weighted 2^(e - 7 s).  A digit (<= 127) is exact in
// bf16, a digit product (< 2^14) is exact in fp32, and a level L = s + t sums at most 8
// slice pairs over K <= 64 terms: 8 * 64 * 127^2 < 2^23, still exact in the fp32
// accumulator.  Levels
// 2..10 are kept (43 slice products); the dropped levels and the 56-bit cut contribute
// about 2^-54 of |X'| |M'|, the size of FP64's own rounding in a K-term dot product.
// Recombination: the nine exact level sums are combined as two 64-bit integers and turned
// into a double with two conversions and two FMAs, added to the base value.
//
// The p x p stage kernels write each factor already split (`oz_emit_factor`); the row
// passes split X' in registers: 16 rows at a time as the A operand up to p = 16
// (`oz_apply`), and at p = 32, where eight slices of four k16 steps of 16 rows would not
// fit, transposed (Y'^T = M'^T X'^T) with 8 rows at a time as the B operand (`oz_apply_t`).
#pragma once

#include "blcoc_common.cuh"

namespace blcoc {

// per-factor slot in the handle's slice buffer: fragments of the largest supported width
// (p <= 32: 8 slices x 4 k16 steps x 8 n8 tiles x 32 lanes) followed by the 2p column
// exponents
constexpr int OZ_FRAG_MAX = 8 * 4 * 8 * 32;         // uint2 units (64 KB)
constexpr int OZ_SLOT_U2 = OZ_FRAG_MAX + 32;        // + 64 ints of column exponents
enum OzSlot { OZ_T = 0, OZ_ALPHA, OZ_ALPHAXI, OZ_BETA, OZ_NSLOTS };
__host__ __device__ inline const int* oz_colexp_of(const uint2* slot) {
  return reinterpret_cast<const int*>(slot + OZ_FRAG_MAX);
}
__host__ __device__ inline int* oz_colexp_of(uint2* slot) { return reinterpret_cast<int*>(slot + OZ_FRAG_MAX); }

constexpr int OZ_NSL = 8;    // digits per value
constexpr int OZ_DB = 7;     // bits per digit
constexpr int OZ_LMAX = 10;  // highest level kept (s + t)
constexpr int OZ_NLEV = OZ_LMAX - 1;   // levels 2..10

template <int PP>
struct OzGeo {
  static constexpr int NR = 2 * PP;        // real width
  static constexpr int KS = NR / 16;       // k16 steps
  static constexpr int NT = NR / 8;        // n8 tiles
  static constexpr int FRAG = OZ_NSL * KS * NT * 32;   // uint2 per factor
};

// biased exponent field of |x| (0 for zero and subnormals, 2047 for inf/nan)
__device__ __forceinline__ int oz_bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// 56-bit fixed-point magnitude of x relative to a row/column whose largest biased
// exponent is eb (|x| < 2^(eb - 1022)): F = |x| 2^(56 - (eb - 1022)), truncated.
__device__ __forceinline__ unsigned long long oz_fixed(double x, int eb) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ev = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & 0x000FFFFFFFFFFFFFull;
  int e = ev;
  if (ev == 0) e = 1;                      // subnormal: no implicit bit
  else m |= 0x0010000000000000ull;         // implicit bit
  const int sh = max(eb, 1) - e;           // >= 0 (subnormals count as exponent 1)
  if (m == 0 || sh >= 59) return 0ull;
  return (m << 3) >> sh;
}

// bf16 bit pattern of the signed digit (sign bit | magnitude d <= 127), exact:
// float(d) through the 2^23 magic constant, top half of the float.
__device__ __forceinline__ unsigned oz_bf16(unsigned d, unsigned sign) {
  const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;
  return (__float_as_uint(f) >> 16) | (sign << 15);
}

// Real entry (k, j) of M' = [[Mr, Mi], [-Mi, Mr]] for a p x p complex M (row stride ld),
// zero outside p in either half.
template <int PP>
__device__ __forceinline__ double oz_mbig(const double2* M, int ld, int p, int k, int j) {
  const int kk = k % PP, jj = j % PP;
  if (kk >= p || jj >= p) return 0.0;
  const double2 v = M[kk * ld + jj];
  const bool kim = k >= PP, jim = j >= PP;
  if (!kim && !jim) return v.x;
  if (!kim && jim) return v.y;
  if (kim && !jim) return -v.y;
  return v.x;
}

// Split a p x p factor into OZ_NSL bf16 slices.  Up to p = 16, in the B-fragment order of
// mma.m16n8k16 (row.col): frag[((t*KS + ks)*NT + nt)*32 + lane] = {rows 16ks+2q, +1 ; rows
// +8, +9} of column 8nt + g, g = lane/4, q = lane%4.  At p = 32, where the row passes
// multiply transposed (Y'^T = M'^T X'^T, oz_apply_t), in the A-fragment order of M'^T:
// frag4[((t*KS + ks)*MT + mt)*32 + lane] = the four registers {A[m0][k0], A[m0][k0+1]},
// {A[m1][k0], A[m1][k0+1]}, {A[m0][k0+8], A[m0][k0+9]}, {A[m1][k0+8], A[m1][k0+9]} with
// A[m][k] = M'[k][m], m0 = 16mt + g, m1 = m0 + 8, k0 = 16ks + 2q.  colexp[j]: largest
// biased exponent in column j of M'.  All threads of the CTA call this; it synchronises
// internally.
template <int PP>
__device__ void oz_emit_factor(const double2* M, int ld, int p, uint2* __restrict__ frag, int* __restrict__ colexp,
                               int* sh_colexp) {
  using G = OzGeo<PP>;
  for (int j = threadIdx.x; j < G::NR; j += blockDim.x) {
    int eb = 0;
    for (int k = 0; k < G::NR; ++k) eb = max(eb, oz_bexp(oz_mbig<PP>(M, ld, p, k, j)));
    sh_colexp[j] = eb;
    colexp[j] = eb;
  }
  __syncthreads();
  if constexpr (PP >= 32) {
    constexpr int MT = G::NR / 16;
    uint4* frag4 = reinterpret_cast<uint4*>(frag);
    for (int w = threadIdx.x; w < G::KS * MT * 32; w += blockDim.x) {
      const int lane = w & 31, mt = (w >> 5) % MT, ks = (w >> 5) / MT;
      const int g = lane >> 2, q = lane & 3;
      const int m0 = 16 * mt + g, m1 = m0 + 8, k0 = 16 * ks + 2 * q;
      const int km[8] = {k0, k0 + 1, k0, k0 + 1, k0 + 8, k0 + 9, k0 + 8, k0 + 9};
      const int mm[8] = {m0, m0, m1, m1, m0, m0, m1, m1};
      unsigned long long F[8];
      unsigned sg[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const double v = oz_mbig<PP>(M, ld, p, km[r], mm[r]);
        F[r] = oz_fixed(v, sh_colexp[mm[r]]);
        sg[r] = (__double_as_longlong(v) < 0) ? 1u : 0u;
      }
#pragma unroll
      for (int t = 1; t <= OZ_NSL; ++t) {
        const int shft = 56 - OZ_DB * t;
        unsigned h[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) h[r] = oz_bf16((unsigned)((F[r] >> shft) & 127ull), sg[r]);
        frag4[((t - 1) * G::KS + ks) * MT * 32 + mt * 32 + lane] =
            make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
      }
    }
    __syncthreads();
    return;
  }
  for (int w = threadIdx.x; w < G::KS * G::NT * 32; w += blockDim.x) {
    const int lane = w & 31, nt = (w >> 5) % G::NT, ks = (w >> 5) / G::NT;
    const int g = lane >> 2, q = lane & 3, j = 8 * nt + g;
    const int eb = sh_colexp[j];
    unsigned long long F[4];
    unsigned sg[4];
    const int rows[4] = {16 * ks + 2 * q, 16 * ks + 2 * q + 1, 16 * ks + 2 * q + 8, 16 * ks + 2 * q + 9};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const double v = oz_mbig<PP>(M, ld, p, rows[r], j);
      F[r] = oz_fixed(v, eb);
      sg[r] = (__double_as_longlong(v) < 0) ? 1u : 0u;
    }
#pragma unroll
    for (int t = 1; t <= OZ_NSL; ++t) {
      const int shft = 56 - OZ_DB * t;
      unsigned h[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) h[r] = oz_bf16((unsigned)((F[r] >> shft) & 127ull), sg[r]);
      frag[((t - 1) * G::KS + ks) * G::NT * 32 + nt * 32 + lane] = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void oz_mma(float (&c)[4], const unsigned (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// Exact integer value of a level sum.  K: the longest dot product behind it.  A level sums
// at most 8 slice pairs, so |sum| <= 8 K 127^2; below 2^22 (K <= 32) it is read through the
// 1.5 2^23 constant on the FP32 and integer pipes, above that by a conversion.
template <int K>
__device__ __forceinline__ int oz_level_int(float f) {
  if constexpr (8 * K * 127 * 127 < (1 << 22)) return __float_as_int(f + 12582912.0f) - 0x4B400000;
  else return __float2int_rn(f);
}

// One output from its nine exact level sums: value = sum_L acc_L 2^(E - 7L), E = e_r + f_c
// (the row and column scalings).  W = value 2^(53 - E) is formed as a 64-bit integer:
// levels 2..7 exactly (|W| < 2^62.02), levels 8..10 summed in FP32 and rounded to an
// integer (error below one unit of W, 2^(E - 53), against the 2^(E - 56) truncation of
// every one of the K operand pairs).  One conversion to double, then the scaling by 2^(E - 53)
// as an add to the exponent field: a single operation on the FP64 pipe instead of five.
template <int K>
__device__ __forceinline__ double oz_value(const float (&acc)[OZ_NLEV][4], int o, int E) {
  static_assert(OZ_NLEV == 9 && OZ_DB == 7, "the integer frame below is laid out for levels 2..10 of 7-bit digits");
  const int a = oz_level_int<K>(acc[0][o]) * 128 + oz_level_int<K>(acc[1][o]);   // levels 2, 3: weight 2^32
  const int b = oz_level_int<K>(acc[2][o]) * 128 + oz_level_int<K>(acc[3][o]);   // levels 4, 5: 2^18
  const int c = oz_level_int<K>(acc[4][o]) * 128 + oz_level_int<K>(acc[5][o]);   // levels 6, 7: 2^4
  // levels 8..10 (weights 2^-3, 2^-10, 2^-17): |t| < 2^23.02, t / 8 rounded to an integer
  const float t = fmaf(acc[8][o], 0x1p-14f, fmaf(acc[7][o], 0x1p-7f, acc[6][o]));
  const int d = __float_as_int(fmaf(t, 0.125f, 12582912.0f)) - 0x4B400000;
  const long long w = (long long)a * 4294967296ll + (long long)b * 262144ll + (long long)c * 16ll + d;
  double v = (double)w;
  const int s = E - 53;
  if (s >= -1022 && s <= 960) {   // |v| in [1, 2^63] when w != 0: the scaled value stays normal
    if (w != 0) v = __hiloint2double(__double2hiint(v) + (int)((unsigned)s << 20), __double2loint(v));
  } else {
    v = ldexp(v, s);
  }
  return v;
}

// Recombination of the four outputs one lane holds for n-tile nt of an m-tile
// ((ra, 8nt+2q), (ra, 8nt+2q+1), (rb, 8nt+2q), (rb, 8nt+2q+1)) from their nine exact level
// sums, and their write to `out` (added to / subtracted from `base`).
template <int PP, bool SUB, bool BASE>
__device__ __forceinline__ void oz_store_outputs(double2* out, const double2* base, const float (&acc)[OZ_NLEV][4],
                                                 const int* __restrict__ colexp, int ra, int rb, int eba, int ebb,
                                                 int nt, int q, int p) {
  auto tx = [](int k, int r) { return k * 32 + (r ^ (k & 7)); };
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int row = (o < 2) ? ra : rb;
    const int col = 8 * nt + 2 * q + (o & 1);
    const int ebr = (o < 2) ? eba : ebb;
    const int ebc = __ldg(colexp + col);
    // e = eb - 1022 for the row and the column
    double v = oz_value<2 * PP>(acc, o, (max(ebr, 1) - 1022) + (max(ebc, 1) - 1022));
    if (ebr == 2047 || ebc == 2047) v = __longlong_as_double(0x7FF8000000000000ll);   // propagate inf/nan
    const int kc = col % PP;
    if (kc < p) {
      double2 cur = BASE ? base[tx(kc, row)] : make_double2(0.0, 0.0);
      double& dst = (col >= PP) ? cur.y : cur.x;
      dst = SUB ? dst - v : dst + v;
      // the real and imaginary halves of one complex output are written by different
      // lanes (n-tiles nt and nt + NT/2): write only this lane's half
      if (col >= PP) out[tx(kc, row)].y = cur.y;
      else out[tx(kc, row)].x = cur.x;
    }
  }
}

// out = base (+/-) in * M for the warp's 32-row chunk (swizzled [k][32] tiles of double2,
// columns >= p of `in` are ignored).  `out` may alias `base` or, without a base, `in`.
// frag / colexp: the factor as written by oz_emit_factor (global memory).
template <int PP, bool SUB, bool BASE>
__device__ __forceinline__ void oz_apply(double2* out, const double2* base, const double2* in,
                                         const uint2* __restrict__ frag, const int* __restrict__ colexp, int p,
                                         int lane) {
  using G = OzGeo<PP>;
  static_assert(PP == 8 || PP == 16, "exact-slice products are built for p <= 16");
  auto tx = [](int k, int r) { return k * 32 + (r ^ (k & 7)); };
  // row exponents (lane = row)
  int eb_row = 0;
  for (int k = 0; k < p; ++k) {
    const double2 v = in[tx(k, lane)];
    eb_row = max(eb_row, max(oz_bexp(v.x), oz_bexp(v.y)));
  }
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int ra = 16 * mt + g, rb = ra + 8;
    const int eba = __shfl_sync(0xffffffffu, eb_row, ra), ebb = __shfl_sync(0xffffffffu, eb_row, rb);
    // A fragments of all slices: a[t][ks][4]
    unsigned A[OZ_NSL][G::KS][4];
#pragma unroll
    for (int ks = 0; ks < G::KS; ++ks) {
      // real columns 16ks + {2q, 2q+1, 2q+8, 2q+9}; rows ra, rb
      unsigned long long F[8];
      unsigned sg[8];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = 16 * ks + 2 * q + (c & 1) + 8 * (c >> 1);
        const int kc = col % PP;
        const bool im = col >= PP;
        double va = 0.0, vb = 0.0;
        if (kc < p) {
          const double2 xa = in[tx(kc, ra)], xb = in[tx(kc, rb)];
          va = im ? xa.y : xa.x;
          vb = im ? xb.y : xb.x;
        }
        F[2 * c] = oz_fixed(va, eba);
        sg[2 * c] = (__double_as_longlong(va) < 0) ? 1u : 0u;
        F[2 * c + 1] = oz_fixed(vb, ebb);
        sg[2 * c + 1] = (__double_as_longlong(vb) < 0) ? 1u : 0u;
      }
#pragma unroll
      for (int t = 0; t < OZ_NSL; ++t) {
        const int shft = 56 - OZ_DB * (t + 1);
        unsigned h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) h[e] = oz_bf16((unsigned)((F[e] >> shft) & 127ull), sg[e]);
        // a0,a1: (ra, 2q,2q+1)  a2,a3: (rb, 2q,2q+1)  a4,a5: (ra, 2q+8,+9)  a6,a7: (rb, 2q+8,+9)
        A[t][ks][0] = h[0] | (h[2] << 16);
        A[t][ks][1] = h[1] | (h[3] << 16);
        A[t][ks][2] = h[4] | (h[6] << 16);
        A[t][ks][3] = h[5] | (h[7] << 16);
      }
    }
#pragma unroll 1
    for (int nt = 0; nt < G::NT; ++nt) {
      uint2 Bf[OZ_NSL][G::KS];
#pragma unroll
      for (int t = 0; t < OZ_NSL; ++t)
#pragma unroll
        for (int ks = 0; ks < G::KS; ++ks) Bf[t][ks] = __ldg(frag + (t * G::KS + ks) * G::NT * 32 + nt * 32 + lane);
      float acc[OZ_NLEV][4];
#pragma unroll
      for (int l = 0; l < OZ_NLEV; ++l) acc[l][0] = acc[l][1] = acc[l][2] = acc[l][3] = 0.f;
#pragma unroll
      for (int s = 1; s <= OZ_NSL; ++s) {
#pragma unroll
        for (int t = 1; t <= OZ_NSL; ++t) {
          if (s + t > OZ_LMAX) continue;
#pragma unroll
          for (int ks = 0; ks < G::KS; ++ks) oz_mma(acc[s + t - 2], A[s - 1][ks], Bf[t - 1][ks]);
        }
      }
      oz_store_outputs<PP, SUB, BASE>(out, base, acc, colexp, ra, rb, eba, ebb, nt, q, p);
    }
  }
}

// out = base (+/-) in * M for the warp's 32-row chunk at p = 32, computed transposed,
// Y'^T = M'^T X'^T, one 8-row group at a time: the group's rows are the B operand
// (k16 x n8), so a lane holds the digits of its row g's real columns 16 ks + {2q, 2q+1,
// 2q+8, 2q+9} for all four k-steps in registers (8 slices x 4 k-steps x 2 registers), and
// the factor's slices are the A operand, read per use from its fragment buffer (A-fragment
// order of M'^T, oz_emit_factor).  Same slicing, same levels, same exactness as oz_apply.
// GIN: `in` is read from global memory (in_g = the chunk's first row of a row-major n x p
// block, `rows` of them inside n, the rest zero) instead of a swizzled tile.  `out` may
// alias `base` or `in` (a group's rows are all read before any of them is written).
template <int PP, bool SUB, bool BASE, bool GIN>
__device__ __forceinline__ void oz_apply_t(double2* out, const double2* base, const double2* in,
                                           const double2* __restrict__ in_g, int rows,
                                           const uint4* __restrict__ frag, const int* __restrict__ colexp, int p,
                                           int lane) {
  using G = OzGeo<PP>;
  static_assert(PP == 32, "the transposed exact-slice product is laid out for p = 32");
  constexpr int MT = G::NR / 16;   // m16 tiles of output real columns
  auto tx = [](int k, int r) { return k * 32 + (r ^ (k & 7)); };
  const int g = lane >> 2, q = lane & 3;
#pragma unroll 1
  for (int grp = 0; grp < CHUNK / 8; ++grp) {
    const int row = 8 * grp + g;
    // this lane's complex entries of its row: kc = 2q + {0, 1, 8, 9, 16, 17, 24, 25}
    double2 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int kc = 2 * q + (j & 1) + 8 * (j >> 1);
      double2 x = make_double2(0.0, 0.0);
      if (kc < p) {
        if constexpr (GIN) {
          if (row < rows) x = __ldg(in_g + (int64_t)row * p + kc);
        } else {
          x = in[tx(kc, row)];
        }
      }
      v[j] = x;
    }
    // the row's exponent: its 64 real entries are spread over the four lanes of group g
    int eb = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) eb = max(eb, max(oz_bexp(v[j].x), oz_bexp(v[j].y)));
    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 1));
    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 2));
    // B fragments: k-step ks holds real columns 16 ks + {2q, 2q+1, 2q+8, 2q+9}: the real
    // parts of v[0..3] (ks = 0) and v[4..7] (ks = 1), their imaginary parts (ks = 2, 3)
    unsigned Bd[OZ_NSL][G::KS][2];
#pragma unroll
    for (int ks = 0; ks < G::KS; ++ks) {
      unsigned long long F[4];
      unsigned sg[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double2 x = v[(ks & 1) * 4 + c];
        const double val = (ks >= 2) ? x.y : x.x;
        F[c] = oz_fixed(val, eb);
        sg[c] = (__double_as_longlong(val) < 0) ? 1u : 0u;
      }
#pragma unroll
      for (int t = 0; t < OZ_NSL; ++t) {
        const int shft = 56 - OZ_DB * (t + 1);
        unsigned h[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) h[c] = oz_bf16((unsigned)((F[c] >> shft) & 127ull), sg[c]);
        Bd[t][ks][0] = h[0] | (h[1] << 16);
        Bd[t][ks][1] = h[2] | (h[3] << 16);
      }
    }
    // output rows 2q and 2q + 1 of the group: their exponents sit with lanes 8q and 8q + 4
    const int ebn0 = __shfl_sync(0xffffffffu, eb, 8 * q), ebn1 = __shfl_sync(0xffffffffu, eb, 8 * q + 4);
    __syncwarp();   // every lane has read the group's rows before any is written
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
      float acc[OZ_NLEV][4];
#pragma unroll
      for (int l = 0; l < OZ_NLEV; ++l) acc[l][0] = acc[l][1] = acc[l][2] = acc[l][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < G::KS; ++ks) {
#pragma unroll
        for (int t = 1; t <= OZ_NSL; ++t) {
          const uint4 a4 = __ldg(frag + ((t - 1) * G::KS + ks) * MT * 32 + mt * 32 + lane);
          const unsigned A[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
          for (int s2 = 1; s2 <= OZ_NSL; ++s2) {
            if (s2 + t > OZ_LMAX) continue;
            oz_mma(acc[s2 + t - 2], A, make_uint2(Bd[s2 - 1][ks][0], Bd[s2 - 1][ks][1]));
          }
        }
      }
      // C fragment: (m0, 2q), (m0, 2q+1), (m0+8, 2q), (m0+8, 2q+1), m0 = 16 mt + g
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const int m = 16 * mt + g + 8 * (o >> 1);
        const int r = 8 * grp + 2 * q + (o & 1);
        const int ebr = (o & 1) ? ebn1 : ebn0;
        const int ebc = __ldg(colexp + m);
        double vv = oz_value<2 * PP>(acc, o, (max(ebr, 1) - 1022) + (max(ebc, 1) - 1022));
        if (ebr == 2047 || ebc == 2047) vv = __longlong_as_double(0x7FF8000000000000ll);   // propagate inf/nan
        const int kc = m % PP;
        if (kc < p) {
          double2 cur = BASE ? base[tx(kc, r)] : make_double2(0.0, 0.0);
          double& dst = (m >= PP) ? cur.y : cur.x;
          dst = SUB ? dst - vv : dst + vv;
          // the real and imaginary halves of one complex output come from m-tiles mt and
          // mt + MT/2: write only this half
          if (m >= PP) out[tx(kc, r)].y = cur.y;
          else out[tx(kc, r)].x = cur.x;
        }
      }
    }
    __syncwarp();   // the group's writes land before the next group's reads (in-place use)
  }
}

// ------------------------------------------------------------------------------ Grams
// FP64-accurate Gram of one warp's 32-row chunk on the tensor cores: P = Y'^T Z' with
// Y' = [Yr | Yi], Z' = [Zr | Zi] (32 x 2p real), K = the 32 rows.  Every column of Y' and of
// Z' is scaled by a power of two above its largest magnitude in the chunk and cut into
// eight 7-bit digits, as in oz_apply; a level sums at most 8 slice pairs over K = 32 terms
// (< 2^22, exact in fp32).  Each chunk's P is recombined to doubles (C-fragment order of
// mma.m16n8k16) and added to the warp's running FP64 sums, which live in shared memory
// between chunks.  The complex Gram follows from the four real blocks of P:
//   Y^T Z = (P11 - P22) + i (P12 + P21),   Y^H Z = (P11 + P22) + i (P12 - P21).
template <int PP>
struct OzGramGeo {
  static constexpr int NR = 2 * PP;        // real columns
  static constexpr int MT = NR / 16;       // m16 tiles (rows of P)
  static constexpr int NT = NR / 8;        // n8 tiles (columns of P)
  static constexpr int NTILE = MT * NT;
  static constexpr int ACC = NTILE * 4 * 32;   // doubles of one warp's running sums
};

// largest biased exponent of real column m (< 2PP) of [Tr | Ti] over the chunk's 32 rows;
// lane m returns it (other lanes 0)
template <int PP>
__device__ __forceinline__ int oz_tile_colexp(const double2* T, int p, int lane) {
  int eb = 0;
  const int kc = lane % PP;
  if (lane < 2 * PP && kc < p) {
    const bool im = lane >= PP;
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const double2 v = T[kc * 32 + (r ^ (kc & 7))];
      eb = max(eb, oz_bexp(im ? v.y : v.x));
    }
  }
  return eb;
}

// real entry (row r, real column m) of [Tr | Ti], zero for columns >= p
template <int PP>
__device__ __forceinline__ double oz_tile_val(const double2* T, int p, int r, int m) {
  const int kc = m % PP;
  if (kc >= p) return 0.0;
  const double2 v = T[kc * 32 + (r ^ (kc & 7))];
  return m >= PP ? v.y : v.x;
}

// exact level sums of a Gram entry (K = the chunk's 32 rows) -> double, e = eb - 1022
__device__ __forceinline__ double oz_recombine(const float (&acc)[OZ_NLEV][4], int o, int ebr, int ebc) {
  if (ebr == 2047 || ebc == 2047) return __longlong_as_double(0x7FF8000000000000ll);   // propagate inf/nan
  return oz_value<32>(acc, o, (max(ebr, 1) - 1022) + (max(ebc, 1) - 1022));
}

// largest biased exponent of real column m (< 2PP) of [Yr | Yi] over the chunk's rows, Y
// read from global memory (Yg = the chunk's first row of a row-major n x p block, `rows`
// of them inside n); lane m returns it (other lanes 0)
template <int PP>
__device__ __forceinline__ int oz_global_colexp(const double2* __restrict__ Yg, int rows, int p, int lane) {
  int eb = 0;
  const int kc = lane % PP;
  if (lane < 2 * PP && kc < p) {
    const bool im = lane >= PP;
    for (int r = 0; r < rows; ++r) {
      const double2 v = __ldg(Yg + (int64_t)r * p + kc);
      eb = max(eb, oz_bexp(im ? v.y : v.x));
    }
  }
  return eb;
}

// sums[tile][o][lane] += P of this chunk (Y, Z: swizzled [k][32] tiles; SAME: Z is Y).
// YG: Y is read from global memory instead (Yg, `rows` rows inside n, the rest zero).
template <int PP, bool SAME, bool YG = false>
__device__ __forceinline__ void oz_gram_add(double* sums, const double2* Y, const double2* Z, int p, int lane,
                                            const double2* __restrict__ Yg = nullptr, int rows = 0) {
  using G = OzGramGeo<PP>;
  static_assert(PP == 8 || PP == 16, "exact-slice Grams are built for p <= 16");
  static_assert(!(SAME && YG), "a self-Gram reads its one operand from the tile");
  // entry (r, m) of Y' = [Yr | Yi]
  auto yval = [&](int r, int m) -> double {
    if constexpr (YG) {
      const int kc = m % PP;
      if (kc >= p || r >= rows) return 0.0;
      const double2 v = __ldg(Yg + (int64_t)r * p + kc);
      return m >= PP ? v.y : v.x;
    } else {
      return oz_tile_val<PP>(Y, p, r, m);
    }
  };
  int ey;
  if constexpr (YG) ey = oz_global_colexp<PP>(Yg, rows, p, lane);
  else ey = oz_tile_colexp<PP>(Y, p, lane);
  const int ez = SAME ? ey : oz_tile_colexp<PP>(Z, p, lane);
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int mt = 0; mt < G::MT; ++mt) {
    const int ma = 16 * mt + g, mb = ma + 8;
    const int eba = __shfl_sync(0xffffffffu, ey, ma), ebb = __shfl_sync(0xffffffffu, ey, mb);
    // A = Y'^T: rows m (columns of Y'), columns k (rows of the chunk)
    unsigned A[OZ_NSL][2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      unsigned long long F[8];
      unsigned sg[8];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int r = 16 * ks + 2 * q + (c & 1) + 8 * (c >> 1);
        const double va = yval(r, ma), vb = yval(r, mb);
        F[2 * c] = oz_fixed(va, eba);
        sg[2 * c] = (__double_as_longlong(va) < 0) ? 1u : 0u;
        F[2 * c + 1] = oz_fixed(vb, ebb);
        sg[2 * c + 1] = (__double_as_longlong(vb) < 0) ? 1u : 0u;
      }
#pragma unroll
      for (int t = 0; t < OZ_NSL; ++t) {
        const int shft = 56 - OZ_DB * (t + 1);
        unsigned h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) h[e] = oz_bf16((unsigned)((F[e] >> shft) & 127ull), sg[e]);
        A[t][ks][0] = h[0] | (h[2] << 16);
        A[t][ks][1] = h[1] | (h[3] << 16);
        A[t][ks][2] = h[4] | (h[6] << 16);
        A[t][ks][3] = h[5] | (h[7] << 16);
      }
    }
#pragma unroll 1
    for (int nt = 0; nt < G::NT; ++nt) {
      // B = Z': rows k (rows of the chunk), column n = 8 nt + g
      const int n = 8 * nt + g;
      const int ebn = __shfl_sync(0xffffffffu, ez, n);
      uint2 Bf[OZ_NSL][2];
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        unsigned long long F[4];
        unsigned sg[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int r = 16 * ks + 2 * q + (c & 1) + 8 * (c >> 1);
          const double v = oz_tile_val<PP>(Z, p, r, n);
          F[c] = oz_fixed(v, ebn);
          sg[c] = (__double_as_longlong(v) < 0) ? 1u : 0u;
        }
#pragma unroll
        for (int t = 0; t < OZ_NSL; ++t) {
          const int shft = 56 - OZ_DB * (t + 1);
          unsigned h[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) h[c] = oz_bf16((unsigned)((F[c] >> shft) & 127ull), sg[c]);
          Bf[t][ks] = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
        }
      }
      float acc[OZ_NLEV][4];
#pragma unroll
      for (int l = 0; l < OZ_NLEV; ++l) acc[l][0] = acc[l][1] = acc[l][2] = acc[l][3] = 0.f;
#pragma unroll
      for (int s = 1; s <= OZ_NSL; ++s) {
#pragma unroll
        for (int t = 1; t <= OZ_NSL; ++t) {
          if (s + t > OZ_LMAX) continue;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) oz_mma(acc[s + t - 2], A[s - 1][ks], Bf[t - 1][ks]);
        }
      }
      // outputs (ma, 8nt+2q), (ma, 8nt+2q+1), (mb, 8nt+2q), (mb, 8nt+2q+1)
      const int ec0 = __shfl_sync(0xffffffffu, ez, 8 * nt + 2 * q), ec1 = __shfl_sync(0xffffffffu, ez, 8 * nt + 2 * q + 1);
      double* dst = sums + ((mt * G::NT + nt) * 4) * 32 + lane;
#pragma unroll
      for (int o = 0; o < 4; ++o) dst[o * 32] += oz_recombine(acc, o, o < 2 ? eba : ebb, (o & 1) ? ec1 : ec0);
    }
  }
}

// P[m][n] of one warp's sums (C-fragment order)
template <int PP>
__device__ __forceinline__ double oz_gram_at(const double* sums, int m, int n) {
  using G = OzGramGeo<PP>;
  const int mt = m >> 4, mr = m & 15, nt = n >> 3, nc = n & 7;
  const int o = (mr >> 3) * 2 + (nc & 1), lane = (mr & 7) * 4 + (nc >> 1);
  return sums[((mt * G::NT + nt) * 4 + o) * 32 + lane];
}

// The CTA's triangle (a <= b, row-major) of Y^H Z (HERM) or Y^T Z from every warp's sums,
// summed over the warps in order; all threads call it after a CTA barrier.
template <int PP, bool HERM>
__device__ __forceinline__ void oz_gram_write(const double* sums_all, double2* __restrict__ out, int p, int nwarp) {
  using G = OzGramGeo<PP>;
  const int E = p * (p + 1) / 2;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    int a = 0, rem = e;
    while (rem >= p - a) {
      rem -= p - a;
      ++a;
    }
    const int b = a + rem;
    double re = 0.0, im = 0.0;
    for (int w = 0; w < nwarp; ++w) {
      const double* S = sums_all + w * G::ACC;
      const double p11 = oz_gram_at<PP>(S, a, b), p22 = oz_gram_at<PP>(S, PP + a, PP + b);
      const double p12 = oz_gram_at<PP>(S, a, PP + b), p21 = oz_gram_at<PP>(S, PP + a, b);
      re += HERM ? p11 + p22 : p11 - p22;
      im += HERM ? p12 - p21 : p12 + p21;
    }
    out[e] = make_double2(re, im);
  }
}

}  // namespace blcoc
