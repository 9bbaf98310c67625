// Fixed-point number format of the Krylov and Chebyshev kernels (sm_103a):
// int64 (re, im) mantissas with one exponent per vector, exact integer
// neighbour sums, products of a scalar mantissa with a stored value by the
// high half of a 64 x 64 product, exact 128-bit reductions; and the stage
// operator applies in that format (XXZ chain, DIA, CSR).  See kernels_fx.cu for
// the number format's bounds and rounding.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "cfet_internal.h"
#include "scalar_bounds.cuh"

namespace cfet {

// ------------------------------------------------------------------ fixed-point helpers
constexpr int kFxBits = 57;  // stored |M| < 2^57
// Per-thread exact 128-bit sums of products (< 2^115 each, at most 4096 per
// thread) are shifted right by kRedShift before the CTA and grid reductions,
// so that up to 2^17 threads cannot overflow 127 bits; the dropped bits are
// below 2^-68 of any non-zero sum of squares.
constexpr int kRedShift = 24;

// The scalar bookkeeping below uses integer operations on the bit patterns of
// positive normal doubles (the FP64 units run at 1/64 rate).
__device__ __forceinline__ int fx_ilog2(double v) {  // floor(log2 v), v > 0 normal
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff) - 1023;
}
// floor(log2(v (1 + eps))) for a tiny eps > 0: values within 2^-40 below a power
// of two count as that power (a safety margin for bounds computed in FP64).
__device__ __forceinline__ int fx_ilog2_up(double v) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  return ((b & 0xFFFFFFFFFFFFFLL) >= 0xFFFFFFFFFF000LL) ? e + 1 : e;
}
// Exponent E with bound < 2^(bits + E); a zero, negative, tiny (< 2^-963)
// or huge bound gives a very small E.  (Range checks on the bit pattern.)
__device__ __forceinline__ int fx_exp_for(double bound, int bits) {
  const long long b = __double_as_longlong(bound);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (b <= 0 || ex < 1023 - 963 || ex > 1023 + 963) return -960;
  return fx_ilog2_up(bound) - (bits - 1);
}
// Left shift that brings a value of magnitude <= a (a >= 1) to < 2^62.
__device__ __forceinline__ int fx_norm_shift(double a) {
  if (__double_as_longlong(a) < 0x3FF0000000000000LL) return 0;  // a < 1 (or negative)
  const int p = 61 - fx_ilog2_up(a);
  return p < 0 ? 0 : (p > 61 ? 61 : p);
}
// x * 2^e exactly, by exponent arithmetic when the result stays normal.
__device__ __forceinline__ double fx_scale2(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0 || ex + e <= 0 || ex + e >= 2047) return ldexp(x, e);
  return __longlong_as_double(b + ((long long)e << 52));
}

// Exact decomposition v = m * 2^e with |m| in [2^61, 2^62) (m = 0 for 0).
struct Mant {
  long long m;
  int e;
};
__device__ __forceinline__ Mant fx_mant(double v) {
  Mant r;
  const long long b = __double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) { r.m = 0; r.e = 0; return r; }  // zero (subnormals treated as zero)
  const long long frac = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  r.m = frac << 9;
  r.e = ex - 1075 - 9;
  if (b < 0) r.m = -r.m;
  return r;
}

// h * 2^-s rounded (half up); s is uniform across the warp.
__device__ __forceinline__ long long fx_rshr(long long h, int s) {
  if (s <= 0) return s <= -62 ? 0LL : (h << (-s));
  if (s >= 63) return 0LL;
  return (h + (1LL << (s - 1))) >> s;
}
// round(m * x * 2^-(64 + s)); |m|, |x| < 2^62.
// High 64 bits of m * x from three 32x32 partial products (the dropped low
// partial product changes the result by at most 2 units).
__device__ __forceinline__ long long fx_mulhi(long long m, long long x) {
  const int mh = (int)(m >> 32), xh = (int)(x >> 32);
  const unsigned ml = (unsigned)m, xl = (unsigned)x;
  // 32 x 32 -> 64-bit partial products; |mid| < 2^63 for |m|, |x| < 2^62
  const long long mid = (long long)mh * (long long)xl + (long long)xh * (long long)ml;
  return (long long)mh * (long long)xh + (mid >> 32);
}
__device__ __forceinline__ long long fx_mul(long long m, long long x, int s) {
  return fx_rshr(fx_mulhi(m, x), s);
}
// Scalar mantissa with the product shift folded in: fx_mulhi(fx_fold(m, s), x)
// ~= fx_mul(m, x, s).  For s <= 9 the fold is exact (the mantissa of a double
// uses 53 of its 62 bits); for larger s the term is at most 2^-s of the result
// bound and the dropped bits stay below 2^-62 of it.  s < 0 does not occur for
// non-zero terms (the result bound covers every term); it is clamped.
__device__ __forceinline__ long long fx_fold(long long m, int s) {
  if (s <= 0) return m;
  if (s >= 63) return 0;
  return (m + (1LL << (s - 1))) >> s;
}
// p * 2^-sh as int64 (truncated); callers guarantee the result fits.
__device__ __forceinline__ long long fx_shr128(__int128 p, int sh) {
  if (sh >= 127) return p < 0 ? -1LL : 0LL;
  if (sh >= 0) return (long long)(p >> sh);
  if (sh <= -63) return 0LL;
  return (long long)(p << (-sh));
}
__device__ __forceinline__ long long fx_absmax(long long a, long long b) {
  const long long x = a < 0 ? -a : a, y = b < 0 ? -b : b;
  return x > y ? x : y;
}

// ------------------------------------------------------------------ exact reductions
// Sum over a warp of (lo, hi) 128-bit values and max of an int64 (lane 0 result).
__device__ __forceinline__ void fx_warp_reduce(unsigned long long& lo, long long& hi, long long& mx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo2 = __shfl_down_sync(0xffffffffu, lo, o);
    const long long hi2 = __shfl_down_sync(0xffffffffu, hi, o);
    const long long mx2 = __shfl_down_sync(0xffffffffu, mx, o);
    const unsigned long long s = lo + lo2;
    hi = hi + hi2 + (s < lo ? 1 : 0);
    lo = s;
    mx = mx > mx2 ? mx : mx2;
  }
}
// (hi 2^64 + lo) 2^kRedShift rounded to the nearest double, by integer operations.
__device__ __forceinline__ double fx_i128_to_double(unsigned long long lo, long long hi) {
  return sb_i128_to_double(lo, hi, kRedShift);
}


// ------------------------------------------------------------------ apply constants
struct FxConstA {
  // spin
  long long m_cz, m_hop, m_x, m_p;
  int s_d, s_diag, s_hop, s_x, s_p, s_nu;
  int pk, ph, px, pp;
  int use_prev;
  int Eu;
  // dia: per operator P_o = shr128(sum VAL q, sh_pre[o]); term = fx_mul(m_op[o], P_o, s_op[o])
  long long m_op[1 + kMaxDrives];
  int sh_pre[1 + kMaxDrives];
  int s_op[1 + kMaxDrives];
};

// ------------------------------------------------------------------ applies
__device__ __forceinline__ longlong2 fx_apply_spin(const longlong2* q, const longlong2* qm, int x,
                                                   const OpSpinFx& op, const FxConstA& c, const long long* mb) {
  const int N = op.N, L = op.lo_bits;
  const long long dz = __ldg(op.DZ_lo + (x & ((1 << L) - 1))) + __ldg(op.DZ_hi + (x >> (L - 1)));
  // D = c0 s_k dz(x) 2^-s_diag (m_cz carries both shifts), then D * q_k[x]
  const long long Dp = fx_mulhi(c.m_cz, dz << 1) << 3;
  const longlong2 v = q[x];
  long long ur = fx_mulhi(Dp, v.x << c.pk);
  long long ui = fx_mulhi(Dp, v.y << c.pk);
  long long hr = 0, hi = 0;
  const unsigned anti = ((unsigned)x ^ ((unsigned)x >> 1)) & ((1u << (N - 1)) - 1u);
#pragma unroll 4
  for (int i = 0; i < N - 1; ++i) {  // antiparallel bonds only (predicated)
    if ((anti >> i) & 1u) {
      const longlong2 w = q[x ^ (3 << i)];
      hr += w.x;
      hi += w.y;
    }
  }
  ur += fx_mulhi(c.m_hop, hr << c.ph);
  ui += fx_mulhi(c.m_hop, hi << c.ph);
  if (op.uniform) {
    long long xr = 0, xi = 0;
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const longlong2 w = q[x ^ (1 << i)];
      xr += w.x;
      xi += w.y;
    }
    ur += fx_mulhi(c.m_x, xr << c.px);
    ui += fx_mulhi(c.m_x, xi << c.px);
  } else {
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const longlong2 w = q[x ^ (1 << i)];
      ur += fx_mulhi(mb[i], w.x << c.pk);
      ui += fx_mulhi(mb[i], w.y << c.pk);
    }
  }
  if (c.use_prev) {
    const longlong2 w = qm[x];
    ur += fx_mulhi(c.m_p, w.x << c.pp);
    ui += fx_mulhi(c.m_p, w.y << c.pp);
  }
  return make_longlong2(ur, ui);
}

// Two elements x and x2 per call: the neighbour loads of both are issued in
// the same loop iterations (twice the independent requests per warp).
__device__ __forceinline__ void fx_apply_spin2(const longlong2* q, const longlong2* qm, int x, int x2,
                                               const OpSpinFx& op, const FxConstA& c, const long long* mb,
                                               longlong2& r1, longlong2& r2) {
  const int N = op.N, L = op.lo_bits;
  const long long dz1 = __ldg(op.DZ_lo + (x & ((1 << L) - 1))) + __ldg(op.DZ_hi + (x >> (L - 1)));
  const long long dz2 = __ldg(op.DZ_lo + (x2 & ((1 << L) - 1))) + __ldg(op.DZ_hi + (x2 >> (L - 1)));
  const long long Dp1 = fx_mulhi(c.m_cz, dz1 << 1) << 3;
  const long long Dp2 = fx_mulhi(c.m_cz, dz2 << 1) << 3;
  const longlong2 v1 = q[x], v2 = q[x2];
  long long ur1 = fx_mulhi(Dp1, v1.x << c.pk), ui1 = fx_mulhi(Dp1, v1.y << c.pk);
  long long ur2 = fx_mulhi(Dp2, v2.x << c.pk), ui2 = fx_mulhi(Dp2, v2.y << c.pk);
  long long hr1 = 0, hi1 = 0, hr2 = 0, hi2 = 0;
  const unsigned mask = (1u << (N - 1)) - 1u;
  const unsigned anti1 = ((unsigned)x ^ ((unsigned)x >> 1)) & mask;
  const unsigned anti2 = ((unsigned)x2 ^ ((unsigned)x2 >> 1)) & mask;
#pragma unroll 4
  for (int i = 0; i < N - 1; ++i) {
    if ((anti1 >> i) & 1u) {
      const longlong2 w = q[x ^ (3 << i)];
      hr1 += w.x;
      hi1 += w.y;
    }
    if ((anti2 >> i) & 1u) {
      const longlong2 w = q[x2 ^ (3 << i)];
      hr2 += w.x;
      hi2 += w.y;
    }
  }
  ur1 += fx_mulhi(c.m_hop, hr1 << c.ph);
  ui1 += fx_mulhi(c.m_hop, hi1 << c.ph);
  ur2 += fx_mulhi(c.m_hop, hr2 << c.ph);
  ui2 += fx_mulhi(c.m_hop, hi2 << c.ph);
  if (op.uniform) {
    long long xr1 = 0, xi1 = 0, xr2 = 0, xi2 = 0;
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const longlong2 w1 = q[x ^ (1 << i)];
      const longlong2 w2 = q[x2 ^ (1 << i)];
      xr1 += w1.x;
      xi1 += w1.y;
      xr2 += w2.x;
      xi2 += w2.y;
    }
    ur1 += fx_mulhi(c.m_x, xr1 << c.px);
    ui1 += fx_mulhi(c.m_x, xi1 << c.px);
    ur2 += fx_mulhi(c.m_x, xr2 << c.px);
    ui2 += fx_mulhi(c.m_x, xi2 << c.px);
  } else {
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const longlong2 w1 = q[x ^ (1 << i)];
      const longlong2 w2 = q[x2 ^ (1 << i)];
      ur1 += fx_mulhi(mb[i], w1.x << c.pk);
      ui1 += fx_mulhi(mb[i], w1.y << c.pk);
      ur2 += fx_mulhi(mb[i], w2.x << c.pk);
      ui2 += fx_mulhi(mb[i], w2.y << c.pk);
    }
  }
  if (c.use_prev) {
    const longlong2 w1 = qm[x], w2 = qm[x2];
    ur1 += fx_mulhi(c.m_p, w1.x << c.pp);
    ui1 += fx_mulhi(c.m_p, w1.y << c.pp);
    ur2 += fx_mulhi(c.m_p, w2.x << c.pp);
    ui2 += fx_mulhi(c.m_p, w2.y << c.pp);
  }
  r1 = make_longlong2(ur1, ui1);
  r2 = make_longlong2(ur2, ui2);
}

__device__ __forceinline__ longlong2 fx_apply_dia(const longlong2* q, const longlong2* qm, int r, int dim,
                                                  const OpDiaFx& op, const FxConstA& c) {
  long long ur = 0, ui = 0;
  for (int o = 0; o < op.nops; ++o) {
    __int128 ar = 0, ai = 0;
    const int d0 = op.dfirst[o], d1 = d0 + op.dcount[o];
    for (int d = d0; d < d1; ++d) {
      const long long cidx = (long long)r + __ldg(op.off + d);
      if (cidx >= 0 && cidx < dim) {
        const long long a = __ldg(op.VAL + (size_t)d * dim + r);
        const longlong2 w = q[cidx];
        ar += (__int128)a * w.x;
        ai += (__int128)a * w.y;
      }
    }
    ur += fx_mulhi(c.m_op[o], fx_shr128(ar, c.sh_pre[o]));
    ui += fx_mulhi(c.m_op[o], fx_shr128(ai, c.sh_pre[o]));
  }
  if (c.use_prev) {
    const longlong2 w = qm[r];
    ur += fx_mulhi(c.m_p, w.x << c.pp);
    ui += fx_mulhi(c.m_p, w.y << c.pp);
  }
  return make_longlong2(ur, ui);
}

// CSR: per operator the exact 128-bit sums of VAL * q over the row's entries
// (complex values: re = sum VR w.x - VI w.y, im = sum VR w.y + VI w.x; the row
// sums of |VR| + |VI| stay below 2^62 and |q| < 2^57, so no sum overflows),
// then one rounded product with the operator's scalar mantissa as for DIA.
__device__ __forceinline__ longlong2 fx_apply_csr(const longlong2* q, const longlong2* qm, int r, int dim,
                                                  const OpCsrFx& op, const FxConstA& c) {
  long long ur = 0, ui = 0;
  for (int o = 0; o < op.nops; ++o) {
    const int* rp = op.rp + (size_t)o * (dim + 1);
    const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
    __int128 ar = 0, ai = 0;
    if (op.VI) {
      for (int e = e0; e < e1; ++e) {
        const long long a = __ldg(op.VR + e), b = __ldg(op.VI + e);
        const longlong2 w = q[__ldg(op.col + e)];
        ar += (__int128)a * w.x - (__int128)b * w.y;
        ai += (__int128)a * w.y + (__int128)b * w.x;
      }
    } else {
      for (int e = e0; e < e1; ++e) {
        const long long a = __ldg(op.VR + e);
        const longlong2 w = q[__ldg(op.col + e)];
        ar += (__int128)a * w.x;
        ai += (__int128)a * w.y;
      }
    }
    ur += fx_mulhi(c.m_op[o], fx_shr128(ar, c.sh_pre[o]));
    ui += fx_mulhi(c.m_op[o], fx_shr128(ai, c.sh_pre[o]));
  }
  if (c.use_prev) {
    const longlong2 w = qm[r];
    ur += fx_mulhi(c.m_p, w.x << c.pp);
    ui += fx_mulhi(c.m_p, w.y << c.pp);
  }
  return make_longlong2(ur, ui);
}

// The two stored-matrix families behind one name (DIA, CSR).
__device__ __forceinline__ longlong2 fx_apply_sparse(const longlong2* q, const longlong2* qm, int r, int dim,
                                                     const OpDiaFx& op, const FxConstA& c) {
  return fx_apply_dia(q, qm, r, dim, op, c);
}
__device__ __forceinline__ longlong2 fx_apply_sparse(const longlong2* q, const longlong2* qm, int r, int dim,
                                                     const OpCsrFx& op, const FxConstA& c) {
  return fx_apply_csr(q, qm, r, dim, op, c);
}

}  // namespace cfet
