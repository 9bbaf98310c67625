// Scalar work of the control warp without FP64 instructions where an exact
// FP64 result is not needed.
//
// On this GPU one dependent FP64 instruction costs 64 cycles (a conversion,
// a minimum, a reciprocal or a square root several times that), while FP32 and
// integer instructions cost a few.  The helpers below take decisions that the
// FP64 form would take, from bit-pattern arithmetic on doubles and FP32
// arithmetic with explicit error margins: a helper either returns the FP64
// decision for certain or says that it cannot, and the caller then evaluates
// the FP64 form.  Everything here also compiles for the host, where
// cfet_selftest_i128_to_double, cfet_selftest_ll_to_double_up and
// cfet_selftest_krylov_bounds expose it to tests against exact arithmetic.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

namespace cfet {

__host__ __device__ __forceinline__ long long sb_bits(double v) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(v);
#else
  long long b;
  memcpy(&b, &v, sizeof b);
  return b;
#endif
}
__host__ __device__ __forceinline__ double sb_double(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  memcpy(&v, &b, sizeof v);
  return v;
#endif
}
__host__ __device__ __forceinline__ float sb_float(unsigned b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float v;
  memcpy(&v, &b, sizeof v);
  return v;
#endif
}
__host__ __device__ __forceinline__ unsigned sb_fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ int sb_clz64(unsigned long long v) {  // v != 0
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}
__host__ __device__ __forceinline__ float sb_log2f(float x) {  // x in [1/64, 64]: absolute error below 2^-20
#ifdef __CUDA_ARCH__
  return __log2f(x);
#else
  return std::log2(x);
#endif
}
__host__ __device__ __forceinline__ float sb_expf(float x) {  // x in [0, 1]: relative error below 2^-20
#ifdef __CUDA_ARCH__
  return __expf(x);
#else
  return std::exp(x);
#endif
}

// ------------------------------------------------------------------ conversions
// (hi 2^64 + lo) 2^shift, the two's-complement 128-bit integer scaled by a
// power of two, rounded to the nearest double (ties to even) by integer
// operations; |result| stays far inside the double range for |shift| < 800.
__host__ __device__ __forceinline__ double sb_i128_to_double(unsigned long long lo, long long hi, int shift) {
  const bool neg = hi < 0;
  unsigned long long l = lo, h = (unsigned long long)hi;
  if (neg) {  // two's-complement negation (-2^127 stays 2^127 as an unsigned magnitude)
    l = ~l + 1ULL;
    h = ~h + (l == 0 ? 1ULL : 0ULL);
  }
  if (h == 0 && l == 0) return 0.0;
  const int lz = h ? sb_clz64(h) : 64 + sb_clz64(l);
  if (lz >= 64) {
    h = l << (lz - 64);
    l = 0;
  } else if (lz > 0) {
    h = (h << lz) | (l >> (64 - lz));
    l <<= lz;
  }
  // leading one at bit 63 of h: 53 mantissa bits, 11 guard bits, the rest sticky
  unsigned long long m = h >> 11;
  const unsigned long long g = h & 0x7FFULL;
  if (g > 0x400ULL || (g == 0x400ULL && (l != 0 || (m & 1ULL)))) ++m;
  int e = 127 - lz + shift;
  if (m >> 53) {
    m >>= 1;
    ++e;
  }
  return sb_double(((unsigned long long)(e + 1023) << 52) | (m & 0xFFFFFFFFFFFFFULL) | (neg ? (1ULL << 63) : 0ULL));
}

// Non-negative int64 as a double not below it (rounded up), by integer operations.
__host__ __device__ __forceinline__ double sb_ll_to_double_up(long long v) {
  if (v <= 0) return 0.0;
  const unsigned long long u = (unsigned long long)v;
  const int e = 63 - sb_clz64(u);  // leading one at bit e
  if (e <= 52) return sb_double(((unsigned long long)(e + 1023) << 52) | ((u << (52 - e)) & 0xFFFFFFFFFFFFFULL));
  const int sh = e - 52;
  unsigned long long m = u >> sh;
  int ee = e;
  if (u & ((1ULL << sh) - 1ULL)) {
    ++m;
    if (m >> 53) {
      m >>= 1;
      ++ee;
    }
  }
  return sb_double(((unsigned long long)(ee + 1023) << 52) | (m & 0xFFFFFFFFFFFFFULL));
}

// Exact float -> double by integer operations (subnormal floats through the
// conversion instruction).
__host__ __device__ __forceinline__ double sb_f2d(float f) {
  const unsigned u = sb_fbits(f);
  const unsigned ef = (u >> 23) & 0xFFu;
  if (ef == 0) return (double)f;
  const unsigned long long e = ef == 0xFFu ? 0x7FFULL : (unsigned long long)(ef - 127 + 1023);
  return sb_double(((unsigned long long)(u >> 31) << 63) | (e << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29));
}
// Inf or NaN.
__host__ __device__ __forceinline__ int sb_nonfinite(double v) {
  return (((unsigned long long)sb_bits(v) >> 52) & 0x7FFULL) == 0x7FFULL;
}

// |v| as a float not above |v| (mantissa truncated: relative error below
// 2^-23); subnormal and tiny magnitudes give 0, huge ones (and Inf, NaN) 3.4e38.
__host__ __device__ __forceinline__ float sb_abs_down(double v) {
  const unsigned long long b = (unsigned long long)sb_bits(v) & 0x7FFFFFFFFFFFFFFFULL;
  const int ef = (int)(b >> 52) - 1023 + 127;
  if (ef <= 0) return 0.f;
  if (ef >= 255) return 3.4e38f;
  return sb_float(((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7FFFFFULL));
}
// |v| as a float not below |v| (relative error below 2^-22); non-finite v gives +inf.
__host__ __device__ __forceinline__ float sb_abs_up(double v) {
  const unsigned long long b = (unsigned long long)sb_bits(v) & 0x7FFFFFFFFFFFFFFFULL;
  if (b == 0) return 0.f;
  const int ef = (int)(b >> 52) - 1023 + 127;
  if (ef <= 0) return 1.17549435e-38f;  // 2^-126 >= |v|
  if (ef >= 255) return sb_float(0x7F800000u);
  const unsigned f = ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7FFFFFULL);
  return sb_float((b & 0x1FFFFFFFULL) ? f + 1u : f);
}
// Signed float within 2^-23 |v| of v (truncated toward zero); |v| beyond the
// float range gives +-3.4e38.
__host__ __device__ __forceinline__ float sb_trunc(double v) {
  const float a = sb_abs_down(v);
  return sb_bits(v) < 0 ? -a : a;  // sign bit (no FP64 comparison)
}
// log2 |v| for normal v with 2^-100 < |v| < 2^100, absolute error below 2^-17
// (mantissa truncated to 23 bits, the FP32 logarithm, one FP32 sum); NaN
// otherwise, which fails every comparison of the callers.
__host__ __device__ __forceinline__ float sb_log2_abs(double v) {
  const unsigned long long b = (unsigned long long)sb_bits(v) & 0x7FFFFFFFFFFFFFFFULL;
  const int e = (int)(b >> 52) - 1023;
  if (e < -100 || e > 100) return sb_float(0x7FC00000u);
  const float m = sb_float(0x3F800000u | (unsigned)((b >> 29) & 0x7FFFFFULL));
  return (float)e + sb_log2f(m);
}

// ------------------------------------------------------------------ Krylov estimate: certain decisions
// The a-posteriori estimate of Sec. 8.1 rejects Krylov dimension k when
// err = scale |y_{k-1}| > thr, y = exp(-i ts T_k) e_0, T_k the Lanczos
// tridiagonal (diagonal a_0..a_{k-1}, couplings b_0..b_{k-2} > 0).  For any
// real shift sigma the Taylor series of exp(-i ts (T_k - sigma)) gives row
// k-1 no term before n = k-1, and that term has modulus
//   lead = |ts|^{k-1} b_0 ... b_{k-2} / (k-1)!.
// Every later term is a sum over walks of n steps from row 0 to row k-1: each
// level is crossed upward once more than downward (one factor b_j per level),
// the extra up/down pairs contribute at most B^2 each (B = max b_j) and the
// stays at most D = max |a_r - sigma|.  Counting the walks without the
// boundary constraints bounds the sum of the moduli of all terms by
//   lead sum_{w,s} |ts|^{2w+s} B^{2w} D^s (k-1)! / ((k-1+w)! w! s!)
//     <= lead exp(g),  g = |ts| D + (|ts| B)^2 / k,
// hence lead (2 - e^g) <= |y_{k-1}| <= lead e^g.
// The accumulator collects the logarithms and extrema entry by entry (one
// lane, as the Lanczos recurrence produces them, or lanes merged like a
// reduction); sb_lead_decide takes the decision.
struct LeadAcc {
  float slog;  // sum over j < k-1 of log2 b_j - log2 (j + 1)
  float sabs;  // sum of the moduli of those terms (rounding margin of slog)
  float bmax;  // max b_j (truncated)
  float amin, amax, amag;  // min, max, max modulus of the truncated a_r
  int bad;     // a coupling that is not a positive normal double, or a non-finite a_r
};
__host__ __device__ __forceinline__ void sb_lead_init(LeadAcc& s) {
  s.slog = 0.f;
  s.sabs = 0.f;
  s.bmax = 0.f;
  s.amin = 3.4e38f;
  s.amax = -3.4e38f;
  s.amag = 0.f;
  s.bad = 0;
}
// Diagonal entry a_r (any row) and coupling b_j (j < k - 1) of T_k.
__host__ __device__ __forceinline__ void sb_lead_diag(LeadAcc& s, double ar) {
  if ((((unsigned long long)sb_bits(ar) >> 52) & 0x7FFULL) > 1023 + 100) s.bad = 1;  // |a_r| >= 2^101, Inf, NaN
  const float at = sb_trunc(ar);
  s.amin = at < s.amin ? at : s.amin;
  s.amax = at > s.amax ? at : s.amax;
  const float am = at < 0.f ? -at : at;
  s.amag = am > s.amag ? am : s.amag;
}
__host__ __device__ __forceinline__ void sb_lead_coupling(LeadAcc& s, int j, double bj) {
  const float lb = sb_log2_abs(bj);
  if (((unsigned long long)sb_bits(bj) >> 63) || !(lb == lb)) s.bad = 1;  // negative, zero, tiny, huge
  const float t = lb - sb_log2f((float)(j + 1));
  s.slog += t;
  s.sabs += t < 0.f ? -t : t;
  const float bt = sb_abs_down(bj);
  s.bmax = bt > s.bmax ? bt : s.bmax;
}
__host__ __device__ __forceinline__ void sb_lead_row(LeadAcc& s, int r, int k, const double* a, const double* b) {
  sb_lead_diag(s, a[r]);
  if (r < k - 1) sb_lead_coupling(s, r, b[r]);
}
__host__ __device__ __forceinline__ void sb_lead_merge(LeadAcc& s, const LeadAcc& o) {
  s.slog += o.slog;
  s.sabs += o.sabs;
  s.bmax = o.bmax > s.bmax ? o.bmax : s.bmax;
  s.amin = o.amin < s.amin ? o.amin : s.amin;
  s.amax = o.amax > s.amax ? o.amax : s.amax;
  s.amag = o.amag > s.amag ? o.amag : s.amag;
  s.bad |= o.bad;
}
// Certified bounds of log2 |y_{k-1}| (every rounding of the FP32 evaluation
// taken off): the lower bound lead (2 - e^g), or -1e30 when g > 0.6 leaves it
// void; the upper bound lead e^g, or 1e30.  Both void for k < 2 or a bad entry.
__host__ __device__ __forceinline__ void sb_lead_log2_bounds(const LeadAcc& s, int k, double ts, float& lo, float& hi) {
  lo = -1e30f;
  hi = 1e30f;
  if (s.bad || k < 2) return;
  const float xl = sb_log2_abs(ts), x = sb_abs_up(ts) * (1.0f + 0x1p-20f);
  if (!(xl == xl)) return;
  // sigma = the midpoint of the truncated diagonal: |a_r - sigma| <= D
  const float D = 0.5f * (s.amax - s.amin) * (1.0f + 0x1p-20f) + 0x1p-20f * s.amag;
  const float B = s.bmax * (1.0f + 0x1p-20f);
  const float g = (x * D + (x * B) * (x * B) / (float)k) * (1.0f + 0x1p-18f);
  if (!(g <= 64.0f)) return;
  // error of the sums: 2^-17 per logarithm (log2 |ts| counted k - 1 times,
  // k - 1 couplings, k - 1 integers, f), 2^-24 of the partial sums' moduli per
  // FP32 operation (at most 2k of them)
  const float margin = 0x1p-17f * (float)(3 * k + 1) +
                       0x1p-23f * (float)k * (s.sabs + (float)(k - 1) * (xl < 0.f ? -xl : xl) + 4.0f + g);
  const float lead = (float)(k - 1) * xl + s.slog;
  hi = lead + g * 1.4426951f * (1.0f + 0x1p-18f) + margin;  // log2 e^g
  if (g <= 0.6f) {
    const float f = 2.0f - sb_expf(g) * (1.0f + 0x1p-18f);  // in [0.17, 1]
    lo = lead + sb_log2f(f) - margin;
  }
}
// The estimate's decision err = beta0 beta_k |y_{k-1}| <= thr, with room for
// the FP64 evaluation's own error (relative 2^-20, absolute 1e-16 in |y|):
// 0 = rejected for certain, 1 = accepted for certain (the FP64 evaluation is
// then still needed for y itself), -1 = undecided.
__host__ __device__ __forceinline__ int sb_lead_decide(const LeadAcc& s, int k, double ts, double beta0, double betak,
                                                      double thr) {
  float lo, hi;
  sb_lead_log2_bounds(s, k, ts, lo, hi);
  // log2 (thr / scale) with 2^-17 per logarithm
  const float r = sb_log2_abs(thr) - sb_log2_abs(beta0) - sb_log2_abs(betak);
  if (!(r == r)) return -1;
  // rejected: |y| >= 2^-49, so 1e-16 is at most 5.7 % of it: log2 (1 - 0.057) > -0.09
  if (lo >= -49.0f && lo - 0.09f - 0x1p-19f - 0x1p-15f > r) return 0;
  // accepted: |y| (1 + 2^-19) + 1e-16 <= 2 max(|y| (1 + 2^-19), 2^-53)
  const float m = hi + 0x1p-18f > -53.0f ? hi + 0x1p-18f : -53.0f;
  if (m + 1.0f + 0x1p-15f < r) return 1;
  return -1;
}

// ------------------------------------------------------------------ Gershgorin gate
// The estimate is consulted only when |ts| w <= 2k (Sec. 8.1), w the
// Gershgorin width of T_k: max_r (a_r + rad_r) - min_r (a_r - rad_r),
// rad_r = b_{r-1} + b_r (absent couplings count 0).  FP32 form from the
// truncated entries: |w - w32| <= 2^-20 (max |a_r| + 2 max b_j) + 2^-22 |w32|.
struct GershAcc {
  float lo, hi, amag, bmag;
};
__host__ __device__ __forceinline__ void sb_gersh_init(GershAcc& s) {
  s.lo = 3.4e38f;
  s.hi = -3.4e38f;
  s.amag = 0.f;
  s.bmag = 0.f;
}
// Row with diagonal a and couplings bl (left) and br (right), 0 where absent.
__host__ __device__ __forceinline__ void sb_gersh_add(GershAcc& s, double a, double bld, double brd) {
  const float at = sb_trunc(a);
  const float bl = sb_abs_down(bld), br = sb_abs_down(brd);
  const float rad = bl + br;
  s.lo = at - rad < s.lo ? at - rad : s.lo;
  s.hi = at + rad > s.hi ? at + rad : s.hi;
  const float am = at < 0.f ? -at : at;
  s.amag = am > s.amag ? am : s.amag;
  const float bm = bl > br ? bl : br;
  s.bmag = bm > s.bmag ? bm : s.bmag;
}
__host__ __device__ __forceinline__ void sb_gersh_row(GershAcc& s, int r, int k, const double* a, const double* b) {
  sb_gersh_add(s, a[r], r > 0 ? b[r - 1] : 0.0, r < k - 1 ? b[r] : 0.0);
}
__host__ __device__ __forceinline__ void sb_gersh_merge(GershAcc& s, const GershAcc& o) {
  s.lo = o.lo < s.lo ? o.lo : s.lo;
  s.hi = o.hi > s.hi ? o.hi : s.hi;
  s.amag = o.amag > s.amag ? o.amag : s.amag;
  s.bmag = o.bmag > s.bmag ? o.bmag : s.bmag;
}
// 1: |ts| w <= 2k for certain; 0: |ts| w > 2k for certain; -1: undecided (the
// caller evaluates the FP64 form).  Non-finite entries give -1.
__host__ __device__ __forceinline__ int sb_gersh_gate(const GershAcc& s, int k, double ts) {
  const float w = s.hi - s.lo;
  const float err = 0x1p-20f * (s.amag + 2.0f * s.bmag) + 0x1p-22f * (w < 0.f ? -w : w);
  if (!(w == w) || !(err < 1e37f)) return -1;
  const float t = sb_abs_down(ts), tu = t * (1.0f + 0x1p-20f);
  const float kk = 2.0f * (float)k;
  if (tu * (w + err) * (1.0f + 0x1p-20f) <= kk * (1.0f - 0x1p-20f)) return 1;
  const float wl = w - err;
  if (wl > 0.f && t * wl * (1.0f - 0x1p-20f) > kk * (1.0f + 0x1p-20f)) return 0;
  return -1;
}

// ------------------------------------------------------------------ breakdown test
// Lanczos breakdown: beta <= 1e-13 (|alpha| + beta_prev + 1).  1: no
// breakdown for certain; -1: undecided.
__host__ __device__ __forceinline__ int sb_no_breakdown(double beta, double alpha, double beta_prev) {
  const float rhs = 1e-13f * (sb_abs_up(alpha) + sb_abs_up(beta_prev) + 1.0f) * (1.0f + 0x1p-16f);
  return sb_abs_down(beta) > rhs ? 1 : -1;
}

}  // namespace cfet
