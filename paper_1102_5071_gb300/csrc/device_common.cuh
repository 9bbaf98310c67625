// Device helpers shared by the FP64 and fixed-point persistent kernels:
// bounded grid barrier, CTA/grid reductions, and the small tridiagonal
// exponential exp(-i tau T_k) e_1 with the Gershgorin spread of T_k.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "cfet_internal.h"
#include "scalar_bounds.cuh"

namespace cfet {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ long long global_timer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t) : : "memory");
  return t;
}

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// SM cycle counter, ordered with respect to surrounding memory operations.
static __device__ __forceinline__ long long sm_clock() {
  long long t;
  asm volatile("mov.u64 %0, %%clock64;" : "=l"(t) : : "memory");
  return t;
}
// Bounded grid barrier executed by one warp of each CTA (lane 0 arrives and
// spins; `spin` accumulates its SM cycles).  Returns false in every lane when
// the wait limit expired or another CTA reported an error.
static __device__ bool warp_grid_barrier(unsigned* bar, unsigned& gen, int* status, long long timeout_ns, long long& spin) {
  const int lane = threadIdx.x & 31;
  int ok = 1;
  if (gridDim.x > 1 && lane == 0) {
    const long long c0 = sm_clock();
    const unsigned target = gen + 1;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], target);
    } else {
      const long long t0 = global_timer_ns();
      unsigned spins = 0;
      while (ld_volatile_u32(&bar[1]) != target) {
        if ((++spins & 63u) == 0u) {
          if (ld_volatile_i32(status) != 0) { ok = 0; break; }
          if (global_timer_ns() - t0 > timeout_ns) {
            atomicCAS(status, 0, (int)CFET_ETIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
    spin += sm_clock() - c0;
  }
  gen += 1;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return ok != 0;
}

// ------------------------------------------------------------------ tagged exchange
// Grid-wide exchange of small per-CTA records, executed by one warp of each
// CTA; it is the grid barrier of the kernels with a control warp.  A record is
// W 32-bit payload words, each published as one 64-bit word
// (tag << 32 | payload), so that a reader sees a payload together with its tag
// (aligned 64-bit stores are single-copy atomic); readers wait until the words
// of every CTA carry `tag`.  No atomics and no last-arriver step: one store and
// one round of loads per exchange.  Records of up to 8 words are stored
// contiguously (word w of CTA i at rec[i S + w], S = W rounded up to 8 for
// 5..8 words, so that no record straddles two 64-byte halves of a line);
// wider ones word-major (rec[w G + i]), so that a warp's load of one word of
// 32 consecutive CTAs touches two 128-byte lines: a 16-word exchange of 152
// CTAs took 11.1 us contiguous and 4.0 us word-major, while the 4- and 6-word
// records of the Krylov kernels were 3-10 % faster contiguous (measured both
// ways); a 6-word exchange took 6.2 us at stride 6 and 4.5 us at stride 8.
// Lane l reads the records of CTAs l, l + 32, ..., l + 32 (kExchMaxPerLane - 1)
// in that order and passes each to acc.add(); acc.reset() starts every polling
// round.  `fence` orders the CTA's earlier global stores before its record
// (writer) and the records before the CTA's later loads (reader); it is needed
// when other CTAs will read vectors written before the exchange.  Returns false
// in every lane when the wait limit expired (CFET_ETIMEOUT recorded) or another
// CTA reported an error.  A slot of W words per CTA needs S G words.
constexpr int kExchMaxPerLane = 8;  // grids of at most 256 CTAs

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

template <int W, class Acc>
static __device__ bool ctl_exchange(unsigned long long* rec, const unsigned (&mine)[W], unsigned tag, bool fence,
                                    int* status, long long timeout_ns, long long& spin, Acc& acc) {
  constexpr bool kWordMajor = W > 8;
  constexpr int kStride = (W > 4 && W <= 8) ? 8 : W;  // contiguous records: words per CTA
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x;
  if (G == 1) {  // a single CTA: its own record is the total; nothing to publish or wait for
    acc.reset();  // (as below: lane 0 holds record 0, the caller combines the lanes)
    if (lane == 0) acc.add(mine);
    return true;
  }
  const long long c0 = sm_clock();
  if (lane == 0) {
    if (fence) __threadfence();
#pragma unroll
    for (int w = 0; w < W; ++w)
      st_relaxed_u64(kWordMajor ? rec + (size_t)w * G + blockIdx.x : rec + (size_t)blockIdx.x * kStride + w,
                     ((unsigned long long)tag << 32) | mine[w]);
  }
  __syncwarp();
  int ok = 1;
  const long long t0 = global_timer_ns();
  unsigned rounds = 0;
  while (true) {
    acc.reset();
    int ready = 1;
#pragma unroll
    for (int j = 0; j < kExchMaxPerLane; ++j) {
      const int i = lane + 32 * j;
      if (i < G) {
        unsigned v[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const unsigned long long x =
              ld_relaxed_u64(kWordMajor ? rec + (size_t)w * G + i : rec + (size_t)i * kStride + w);
          v[w] = (unsigned)x;
          ready &= (unsigned)(x >> 32) == tag;
        }
        acc.add(v);
      }
    }
    if (__all_sync(0xffffffffu, ready)) break;
    if ((++rounds & 15u) == 0u) {
      int bad = 0;
      if (lane == 0) {
        if (ld_volatile_i32(status) != 0) {
          bad = 1;
        } else if (global_timer_ns() - t0 > timeout_ns) {
          atomicCAS(status, 0, (int)CFET_ETIMEOUT);
          bad = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, bad, 0)) {
        ok = 0;
        break;
      }
    }
  }
  if (fence) __threadfence();
  if (lane == 0) spin += sm_clock() - c0;
  return ok != 0;
}

// Bounded grid-wide barrier (arrival counter + generation).  Returns false in
// every thread of the CTA when the wait limit expired or another CTA reported
// an error; the first CTA to time out records CFET_ETIMEOUT.
static __device__ bool grid_barrier(unsigned* bar, unsigned& gen, int* status, long long timeout_ns, int* s_ok) {
  __syncthreads();
  if (gridDim.x == 1) {
    gen += 1;
    return true;
  }
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = gen + 1;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], target);
    } else {
      const long long t0 = global_timer_ns();
      unsigned spins = 0;
      while (ld_volatile_u32(&bar[1]) != target) {
        if ((++spins & 63u) == 0u) {
          if (ld_volatile_i32(status) != 0) { ok = 0; break; }
          if (global_timer_ns() - t0 > timeout_ns) {
            atomicCAS(status, 0, (int)CFET_ETIMEOUT);
            ok = 0;
            break;
          }
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  gen += 1;
  __syncthreads();
  return *s_ok != 0;
}

// Sum over the CTA of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
  }
  return s;
}

// Deterministic sum of the per-CTA partials (same order in every CTA);
// executed by warp 0, result returned to all lanes of warp 0.
__device__ __forceinline__ double sum_partials(const double* part) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < (int)gridDim.x; i += 32) s += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Maximum over the CTA of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) s = fmax(s, red[i]);
  }
  return s;
}

// Maximum of the per-CTA partials (warp 0, result in all lanes of warp 0).
__device__ __forceinline__ double max_partials(const double* part) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < (int)gridDim.x; i += 32) s = fmax(s, part[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  return s;
}

// ------------------------------------------------------------------ FP64 spin apply
// Spin family:  (c0 H0 + sum_k c_k V_k) v at index x, everything pre-scaled.
//   diag   cz * dz(x) v[x],             dz(x) = J Delta sum s_i s_{i+1} + sum h_i s_i
//   hop    cxx * sum_{antiparallel bonds i} v[x ^ (3 << i)]     (cxx = 2 J c0)
//   field  sum_i b_i v[x ^ (1 << i)]                             (b_i = sum_k c_k a_{k,i})
struct SpinScaled {
  double cz, cxx;
};

static __device__ __forceinline__ double2 apply_spin_at(const double2* q, int x, const OpSpin& op, const SpinScaled& sc,
                                                 const double* bsite) {
  const int N = op.N, L = op.lo_bits;
  const double dz = __ldg(op.dz_lo + (x & ((1 << L) - 1))) + __ldg(op.dz_hi + (x >> (L - 1)));
  const double2 v = q[x];
  const double cd = sc.cz * dz;
  double2 acc = make_double2(cd * v.x, cd * v.y);
  double hx = 0.0, hy = 0.0;
  unsigned anti = ((unsigned)x ^ ((unsigned)x >> 1)) & ((1u << (N - 1)) - 1u);
  while (anti) {
    const int i = __ffs(anti) - 1;
    anti &= anti - 1u;
    const double2 w = q[x ^ (3 << i)];
    hx += w.x;
    hy += w.y;
  }
  acc.x = fma(sc.cxx, hx, acc.x);
  acc.y = fma(sc.cxx, hy, acc.y);
  for (int i = 0; i < N; ++i) {
    const double2 w = q[x ^ (1 << i)];
    acc.x = fma(bsite[i], w.x, acc.x);
    acc.y = fma(bsite[i], w.y, acc.y);
  }
  return acc;
}

// ------------------------------------------------------------------ small problem
// y = exp(-i ts T) e_1 for the k x k real symmetric tridiagonal T (diagonal
// a[0..k-1], off-diagonal b[0..k-2]); executed by one warp, rows r = lane and
// lane + 32.  Method: spectral shift by the Gershgorin centre sigma, S equal
// substeps with x = |ts| rho / S <= 1 (rho the Gershgorin radius), each a
// Taylor series of n(x) terms, n(x) the smallest count in {10, 12, 15,
// kSmallTaylorTerms} with x^(n+1) / (n+1)! below 1e-17 for the x range;
// exp(-i ts T) = e^{-i ts sigma} exp(-i ts (T - sigma)).
// For a = |ts| rho > kChebyshevFrom the Taylor substeps would cost about 18 a
// matrix-vector products; the Chebyshev expansion (Jacobi-Anger)
//   e^{-i s a x} = J_0(a) + 2 sum_{n>=1} (-i s)^n J_n(a) T_n(x),  x in [-1, 1],
// needs about a + 12 a^(1/3) + 24 terms.  It is summed with Clenshaw's
// backward recurrence on X = (T - sigma) / rho, fused with Miller's backward
// recurrence J_{n-1} = (2n/a) J_n - J_{n+1} for the Bessel values from a tiny
// start, normalised at the end by J_0 + 2 sum_k J_2k = 1 (the sum is linear in
// the coefficients, so one scale fixes both).
// The FP64 units of this GPU issue one warp instruction per many cycles, so
// the per-term work is kept to one multiply and two FMAs per row and part:
// the shifted diagonal and both couplings of a row stay in registers and the
// term factors hstep / n come from a table of reciprocals.
constexpr double kChebyshevFrom = 8.0;

__constant__ double kInvN[kSmallTaylorTerms + 1] = {
    0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10,
    1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18};

static __device__ void small_expm_e1(int k, const double* a, const double* b, double ts, double* yr, double* yi,
                                     double* tr, double* ti) {
  const int lane = threadIdx.x & 31;
  // Spectral interval of T_k from FP32 Gershgorin bounds of the truncated
  // entries, widened by their error: the shift and the number of terms only
  // need bounds.  Without a shift (|ts| max |lambda| <= 1/2) the phase
  // e^{-i ts sig} and its sincos drop out.
  GershAcc g;
  sb_gersh_init(g);
  int bad = 0;
  for (int r = lane; r < k; r += 32) {
    sb_gersh_row(g, r, k, a, b);
    bad |= sb_nonfinite(a[r]) | (r < k - 1 ? sb_nonfinite(b[r]) : 0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    GershAcc t;
    t.lo = __shfl_xor_sync(0xffffffffu, g.lo, o);
    t.hi = __shfl_xor_sync(0xffffffffu, g.hi, o);
    t.amag = __shfl_xor_sync(0xffffffffu, g.amag, o);
    t.bmag = __shfl_xor_sync(0xffffffffu, g.bmag, o);
    sb_gersh_merge(g, t);
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  const float werr = 0x1p-19f * (g.amag + 2.0f * g.bmag) + 0x1p-21f * (fabsf(g.lo) + fabsf(g.hi));
  const float lo32 = g.lo - werr, hi32 = g.hi + werr, mag = fmaxf(fabsf(lo32), fabsf(hi32));
  const float tsa = sb_abs_up(ts) * (1.0f + 0x1p-20f);
  const bool noshift = tsa * mag <= 0.5f;
  // half-width about sig (sig rounded to a float: 2^-24 mag more)
  const float rho32 = noshift ? mag : (0.5f * (hi32 - lo32) * (1.0f + 0x1p-20f) + 0x1p-23f * mag);
  const double sig = noshift ? 0.0 : sb_f2d(0.5f * (lo32 + hi32));
  const float sr32 = tsa * rho32 * (1.0f + 0x1p-20f);
  // number of Taylor substeps, bounded: non-finite entries give S = 1 (the
  // result is then non-finite and rejected by the caller), a huge spread 65536
  int S = 1;
  if (!bad) S = sr32 < 65536.0f ? (int)ceilf(sr32) : 65536;
  if (S < 1) S = 1;
  const double hstep = S == 1 ? ts : ts / S;
  const float x = bad ? 1.0f : sr32 / (float)S;
  const int nterms = x > 0.5f ? kSmallTaylorTerms : (x > 0.25f ? 15 : (x > 0.1f ? 12 : 10));
  // rows owned by this lane: shifted diagonal and couplings in registers
  const int r0 = lane, r1 = lane + 32;
  const bool on0 = r0 < k, on1 = r1 < k;
  const double d0 = on0 ? a[r0] - sig : 0.0, d1 = on1 ? a[r1] - sig : 0.0;
  const double bl0 = (on0 && r0 > 0) ? b[r0 - 1] : 0.0, br0 = (on0 && r0 < k - 1) ? b[r0] : 0.0;
  const double bl1 = on1 ? b[r1 - 1] : 0.0, br1 = (on1 && r1 < k - 1) ? b[r1] : 0.0;
  if (!bad && !noshift && sr32 > (float)kChebyshevFrom && sr32 < 4096.0f) {
    const double rho = sb_f2d(rho32), sr = fabs(ts) * rho;
    const double a_ = sr, inv_a = 1.0 / a_, inv_rho = 1.0 / rho;
    const bool neg = ts < 0.0;  // (-i s)^n with s = sign(ts)
    const double x0 = d0 * inv_rho, xl0 = bl0 * inv_rho, xr0 = br0 * inv_rho;
    const double x1 = d1 * inv_rho, xl1 = bl1 * inv_rho, xr1 = br1 * inv_rho;
    const int nstart = (int)ceil(a_ + 12.0 * cbrt(a_) + 24.0);
    double jn1 = 0.0, jn = 1e-200, norm = 0.0;  // J_{n+1}, J_n (unscaled)
    // Clenshaw state b_{n+1}, b_{n+2} (real and imaginary parts) of each row
    double pr0 = 0, qr0 = 0, pi0 = 0, qi0 = 0, pr1 = 0, qr1 = 0, pi1 = 0, qi1 = 0;
    for (int n = nstart; n >= 1; --n) {
      // coefficient 2 (-i s)^n J_n: the phase (-i)^m, m = n or -n mod 4
      const int m = neg ? ((4 - (n & 3)) & 3) : (n & 3);
      const double c = 2.0 * jn;
      const double cre = m == 0 ? c : (m == 2 ? -c : 0.0);
      const double cim = m == 1 ? -c : (m == 3 ? c : 0.0);
      if (on0) { tr[r0] = pr0; ti[r0] = pi0; }
      if (on1) { tr[r1] = pr1; ti[r1] = pi1; }
      __syncwarp();
      double nr0 = 0, ni0 = 0, nr1 = 0, ni1 = 0;
      if (on0) {
        const double lr = r0 > 0 ? tr[r0 - 1] : 0.0, li = r0 > 0 ? ti[r0 - 1] : 0.0;
        const double rr = r0 < k - 1 ? tr[r0 + 1] : 0.0, ri = r0 < k - 1 ? ti[r0 + 1] : 0.0;
        nr0 = 2.0 * fma(xr0, rr, fma(xl0, lr, x0 * pr0)) - qr0 + (r0 == 0 ? cre : 0.0);
        ni0 = 2.0 * fma(xr0, ri, fma(xl0, li, x0 * pi0)) - qi0 + (r0 == 0 ? cim : 0.0);
      }
      if (on1) {
        const double lr = tr[r1 - 1], li = ti[r1 - 1];
        const double rr = r1 < k - 1 ? tr[r1 + 1] : 0.0, ri = r1 < k - 1 ? ti[r1 + 1] : 0.0;
        nr1 = 2.0 * fma(xr1, rr, fma(xl1, lr, x1 * pr1)) - qr1;
        ni1 = 2.0 * fma(xr1, ri, fma(xl1, li, x1 * pi1)) - qi1;
      }
      __syncwarp();
      qr0 = pr0; qi0 = pi0; pr0 = nr0; pi0 = ni0;
      qr1 = pr1; qi1 = pi1; pr1 = nr1; pi1 = ni1;
      // Miller step and the normalisation sum J_0 + 2 sum_k J_2k
      if ((n & 1) == 0) norm += 2.0 * jn;
      const double jm = 2.0 * n * inv_a * jn - jn1;
      jn1 = jn;
      jn = jm;
    }
    norm += jn;  // J_0
    // S = J_0 e_1 + X b_1 - b_2
    if (on0) { tr[r0] = pr0; ti[r0] = pi0; }
    if (on1) { tr[r1] = pr1; ti[r1] = pi1; }
    __syncwarp();
    double sr0 = 0, si0 = 0, sr1 = 0, si1 = 0;
    if (on0) {
      const double lr = r0 > 0 ? tr[r0 - 1] : 0.0, li = r0 > 0 ? ti[r0 - 1] : 0.0;
      const double rr = r0 < k - 1 ? tr[r0 + 1] : 0.0, ri = r0 < k - 1 ? ti[r0 + 1] : 0.0;
      sr0 = fma(xr0, rr, fma(xl0, lr, x0 * pr0)) - qr0 + (r0 == 0 ? jn : 0.0);
      si0 = fma(xr0, ri, fma(xl0, li, x0 * pi0)) - qi0;
    }
    if (on1) {
      const double lr = tr[r1 - 1], li = ti[r1 - 1];
      const double rr = r1 < k - 1 ? tr[r1 + 1] : 0.0, ri = r1 < k - 1 ? ti[r1 + 1] : 0.0;
      sr1 = fma(xr1, rr, fma(xl1, lr, x1 * pr1)) - qr1;
      si1 = fma(xr1, ri, fma(xl1, li, x1 * pi1)) - qi1;
    }
    __syncwarp();
    const double inv_norm = 1.0 / norm;
    double sn, cs;
    sincos(ts * sig, &sn, &cs);
    // y = e^{-i ts sig} S / norm, e^{-i ts sig} = cs - i sn
    if (on0) { yr[r0] = (sr0 * cs + si0 * sn) * inv_norm; yi[r0] = (si0 * cs - sr0 * sn) * inv_norm; }
    if (on1) { yr[r1] = (sr1 * cs + si1 * sn) * inv_norm; yi[r1] = (si1 * cs - sr1 * sn) * inv_norm; }
    __syncwarp();
    return;
  }
  if (k <= 16) {
    // Rows on half-warps: lane l holds the real (l < 16) or the imaginary part
    // (l >= 16) of row l & 15, neighbours by shuffles within each half.  The
    // same expressions as the two-rows-per-lane form below (bit-identical
    // results) with half the FP64 instructions per term.
    const int r = lane & 15;
    const bool imag = lane >= 16, on = r < k;
    const double d = on ? a[r] - sig : 0.0;
    const double bl = (on && r > 0) ? b[r - 1] : 0.0, br = (on && r < k - 1) ? b[r] : 0.0;
    double acc = (r == 0 && !imag) ? 1.0 : 0.0;  // current y
    for (int sidx = 0; sidx < S; ++sidx) {
      double t = acc;
      for (int n = 1; n <= nterms; ++n) {
        const double c = hstep * kInvN[n];
        const double tl = __shfl_up_sync(0xffffffffu, t, 1, 16);    // row r - 1 (own value at r = 0: bl = 0)
        const double tn = __shfl_down_sync(0xffffffffu, t, 1, 16);  // row r + 1 (own value at r = 15: br = 0)
        const double z = fma(br, tn, fma(bl, tl, d * t));
        const double zo = __shfl_xor_sync(0xffffffffu, z, 16);       // the other part of the same row
        t = imag ? -c * zo : c * zo;                                 // (-i c) z
        acc += t;
      }
    }
    if (noshift) {
      if (on) (imag ? yi : yr)[r] = acc;
      __syncwarp();
      return;
    }
    double sn, cs;
    sincos(ts * sig, &sn, &cs);
    const double ao = __shfl_xor_sync(0xffffffffu, acc, 16);
    // multiply by e^{-i ts sig} = cs - i sn
    if (on) {
      if (imag) yi[r] = acc * cs - ao * sn;
      else yr[r] = acc * cs + ao * sn;
    }
    __syncwarp();
    return;
  }
  double ar0 = (r0 == 0) ? 1.0 : 0.0, ai0 = 0.0, ar1 = 0.0, ai1 = 0.0;  // current y
  for (int sidx = 0; sidx < S; ++sidx) {
    double t_r0 = ar0, t_i0 = ai0, t_r1 = ar1, t_i1 = ai1;
    if (on0) { tr[r0] = t_r0; ti[r0] = t_i0; }
    if (on1) { tr[r1] = t_r1; ti[r1] = t_i1; }
    __syncwarp();
    for (int n = 1; n <= nterms; ++n) {
      const double c = hstep * kInvN[n];
      double zr0 = 0, zi0 = 0, zr1 = 0, zi1 = 0;
      if (on0) {
        const double lr = r0 > 0 ? tr[r0 - 1] : 0.0, li = r0 > 0 ? ti[r0 - 1] : 0.0;
        const double rr = r0 < k - 1 ? tr[r0 + 1] : 0.0, ri = r0 < k - 1 ? ti[r0 + 1] : 0.0;
        zr0 = fma(br0, rr, fma(bl0, lr, d0 * t_r0));
        zi0 = fma(br0, ri, fma(bl0, li, d0 * t_i0));
      }
      if (on1) {
        const double lr = tr[r1 - 1], li = ti[r1 - 1];
        const double rr = r1 < k - 1 ? tr[r1 + 1] : 0.0, ri = r1 < k - 1 ? ti[r1 + 1] : 0.0;
        zr1 = fma(br1, rr, fma(bl1, lr, d1 * t_r1));
        zi1 = fma(br1, ri, fma(bl1, li, d1 * t_i1));
      }
      __syncwarp();
      // t <- (-i c) z
      t_r0 = c * zi0; t_i0 = -c * zr0;
      t_r1 = c * zi1; t_i1 = -c * zr1;
      ar0 += t_r0; ai0 += t_i0; ar1 += t_r1; ai1 += t_i1;
      if (on0) { tr[r0] = t_r0; ti[r0] = t_i0; }
      if (on1) { tr[r1] = t_r1; ti[r1] = t_i1; }
      __syncwarp();
    }
  }
  double sn = 0.0, cs = 1.0;
  if (!noshift) sincos(ts * sig, &sn, &cs);
  // multiply by e^{-i ts sig} = cs - i sn
  if (on0) { yr[r0] = ar0 * cs + ai0 * sn; yi[r0] = ai0 * cs - ar0 * sn; }
  if (on1) { yr[r1] = ar1 * cs + ai1 * sn; yi[r1] = ai1 * cs - ar1 * sn; }
  __syncwarp();
}

__constant__ float kInvNf[kSmallTaylorTerms + 1] = {
    0.f, 1.f, 1.f / 2, 1.f / 3, 1.f / 4, 1.f / 5, 1.f / 6, 1.f / 7, 1.f / 8, 1.f / 9, 1.f / 10,
    1.f / 11, 1.f / 12, 1.f / 13, 1.f / 14, 1.f / 15, 1.f / 16, 1.f / 17, 1.f / 18};

// FP32 screen of the Krylov error estimate err = scale |y_k|, y =
// exp(-i ts T_k) e_1 (whole warp; k <= 16 rows on half-warps as in
// small_expm_e1; only one Taylor step, |ts| rho <= 1).  The shifted Taylor
// series is summed in FP32 together with the same recurrence on magnitudes,
// m_n = |c_n| |T - sig| m_{n-1}, m_0 = e_1, which bounds every rounding error
// of the FP32 terms (each term's component is off by at most about 4 n 2^-24
// of m_n; 2^-15 per unit of sum_n m_n covers 18 terms with a margin of 8).
// True only when err exceeds thr even after that bound is taken off: the FP64
// evaluation (same series, same number of terms) would then reject k too, so
// the FP64 small exponential can be skipped.  Warp-uniform result.
static __device__ bool small_expm_rejects32(int k, const double* a, const double* b, double ts, double scale,
                                            double thr) {
  if (k < 1 || k > 16 || !(thr >= 0.0)) return false;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int r = lane & 15;
  const bool imag = lane >= 16, on = r < k;
  const double ad = on ? a[r] : 0.0;
  const float bl = (on && r > 0) ? (float)b[r - 1] : 0.f, br = (on && r < k - 1) ? (float)b[r] : 0.f;
  const float rad = fabsf(bl) + fabsf(br);
  float lo = on ? (float)ad - rad : 3e38f, hi = on ? (float)ad + rad : -3e38f;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {  // both halves hold the same rows
    lo = fminf(lo, __shfl_xor_sync(full, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(full, hi, o));
  }
  const float sig = 0.5f * (lo + hi), rho = 0.5f * (hi - lo);
  const float x = fabsf((float)ts) * rho * 1.001f;  // (the FP64 path's substep count is ceil(|ts| rho))
  if (!(x <= 1.0f)) return false;
  const int nterms = x > 0.5f ? kSmallTaylorTerms : (x > 0.25f ? 15 : (x > 0.1f ? 12 : 10));
  const float d = on ? (float)(ad - (double)sig) : 0.f, ad_ = fabsf(d), abl = fabsf(bl), abr = fabsf(br);
  const float tsf = (float)ts;
  float t = (r == 0 && !imag) ? 1.f : 0.f, acc = t, m = t, msum = 0.f;
  for (int n = 1; n <= nterms; ++n) {
    const float c = tsf * kInvNf[n];
    const float tl = __shfl_up_sync(full, t, 1, 16), tn = __shfl_down_sync(full, t, 1, 16);
    const float ml = __shfl_up_sync(full, m, 1, 16), mn = __shfl_down_sync(full, m, 1, 16);
    const float z = fmaf(br, tn, fmaf(bl, tl, d * t));
    const float w = fmaf(abr, mn, fmaf(abl, ml, ad_ * m));
    const float zo = __shfl_xor_sync(full, z, 16), wo = __shfl_xor_sync(full, w, 16);
    t = imag ? -c * zo : c * zo;
    m = fabsf(c) * wo;
    acc += t;
    msum += m;
  }
  // row k - 1: real part on lane k - 1, imaginary part on lane k + 15
  const float yre = __shfl_sync(full, acc, k - 1), yim = __shfl_sync(full, acc, k + 15);
  const float bnd = __shfl_sync(full, msum, k - 1) + __shfl_sync(full, msum, k + 15);
  const double yk = (double)hypotf(yre, yim);
  // (1e-16: the FP64 path may truncate its series after a different number of
  // terms; every such tail is below 1e-17 for |ts| rho <= 1)
  const double lower = yk * (1.0 - 0x1p-20) - 0x1p-15 * (double)bnd - 1e-16;
  return scale * lower > thr;
}

// Gershgorin width of T (max of a_r + radius minus min of a_r - radius), an
// upper bound of its eigenvalue spread; warp-uniform result.
static __device__ double gersh_width(int k, const double* a, const double* b) {
  const int lane = threadIdx.x & 31;
  double lo = 1e300, hi = -1e300;
  for (int r = lane; r < k; r += 32) {
    const double rad = (r > 0 ? fabs(b[r - 1]) : 0.0) + (r < k - 1 ? fabs(b[r]) : 0.0);
    lo = fmin(lo, a[r] - rad);
    hi = fmax(hi, a[r] + rad);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  return hi - lo;
}

// |ts| gersh_width(k, a, b) <= 2k (the gate of the Krylov estimate), decided
// in FP32 (sb_gersh_gate) unless that cannot be certain; whole warp,
// warp-uniform result.
static __device__ bool gersh_gate(int k, const double* a, const double* b, double ts) {
  const int lane = threadIdx.x & 31;
  GershAcc s;
  sb_gersh_init(s);
  for (int r = lane; r < k; r += 32) sb_gersh_row(s, r, k, a, b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    GershAcc t;
    t.lo = __shfl_xor_sync(0xffffffffu, s.lo, o);
    t.hi = __shfl_xor_sync(0xffffffffu, s.hi, o);
    t.amag = __shfl_xor_sync(0xffffffffu, s.amag, o);
    t.bmag = __shfl_xor_sync(0xffffffffu, s.bmag, o);
    sb_gersh_merge(s, t);
  }
  const int g = sb_gersh_gate(s, k, ts);
  if (g >= 0) return g == 1;
  return fabs(ts) * gersh_width(k, a, b) <= 2.0 * k;
}

// Certain rejection of Krylov dimension k by the estimate
// scale |y_{k-1}| > thr from the leading Taylor term (sb_lead_decide), rows
// on lanes; whole warp, warp-uniform result.
static __device__ bool krylov_lead_rejects(int k, const double* a, const double* b, double ts, double scale,
                                           double thr) {
  const int lane = threadIdx.x & 31;
  LeadAcc s;
  sb_lead_init(s);
  for (int r = lane; r < k; r += 32) sb_lead_row(s, r, k, a, b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    LeadAcc t;
    t.slog = __shfl_xor_sync(0xffffffffu, s.slog, o);
    t.sabs = __shfl_xor_sync(0xffffffffu, s.sabs, o);
    t.bmax = __shfl_xor_sync(0xffffffffu, s.bmax, o);
    t.amin = __shfl_xor_sync(0xffffffffu, s.amin, o);
    t.amax = __shfl_xor_sync(0xffffffffu, s.amax, o);
    t.amag = __shfl_xor_sync(0xffffffffu, s.amag, o);
    t.bad = __shfl_xor_sync(0xffffffffu, s.bad, o);
    sb_lead_merge(s, t);
  }
  return sb_lead_decide(s, k, ts, scale, 1.0, thr) == 0;
}

// Running FP32 bounds of T_it for the control warps that keep them in shared
// memory (members lead, gfull, alpha[1..], beta[1..]): one lane adds row
// it - 1 (a = alpha[it], left coupling beta[it - 1]) and completes row it - 2,
// and returns the FP32 gate decision for the step ts (sb_gersh_gate).
template <class Sm>
__device__ int krylov_bounds_update(Sm& S, int it, double ts) {
  if (it == 1) {
    sb_lead_init(S.lead);
    sb_gersh_init(S.gfull);
  } else {
    sb_lead_coupling(S.lead, it - 2, S.beta[it - 1]);
    sb_gersh_add(S.gfull, S.alpha[it - 1], it > 2 ? S.beta[it - 2] : 0.0, S.beta[it - 1]);
  }
  sb_lead_diag(S.lead, S.alpha[it]);
  GershAcc g = S.gfull;
  sb_gersh_add(g, S.alpha[it], it > 1 ? S.beta[it - 1] : 0.0, 0.0);
  return sb_gersh_gate(g, it, ts);
}
// The estimate's certain decision (sb_lead_decide) from running bounds,
// evaluated by lane 0 and returned to the whole warp.
__device__ __forceinline__ int krylov_lead_decide(const LeadAcc& lead, int k, double ts, double beta0, double betak,
                                                  double thr) {
  int d = -1;
  if ((threadIdx.x & 31) == 0) d = sb_lead_decide(lead, k, ts, beta0, betak, thr);
  return __shfl_sync(0xffffffffu, d, 0);
}

}  // namespace cfet
