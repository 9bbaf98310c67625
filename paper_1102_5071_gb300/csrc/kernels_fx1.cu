// One-pass fixed-point persistent Lanczos kernel (sm_103a).
//
// Same method, decisions and number format as k_propagate_fx (kernels_fx.cu):
// the stage exponential exp(-i tau H_j) psi of a CFET step (Alvermann &
// Fehske, arXiv:1102.5071, Sec. 4 Eq. (Ucf), Sec. 7 Eq. (OmGLeg)) by the
// Lanczos / Krylov method of Sec. 8.1.  The iteration is reorganised so that
// each Lanczos iteration is one pass over the vectors and one grid-wide
// exchange instead of two of each.  Pass P(k) applies the operator to the
// stored u_k = H q_k - beta_{k-1} q_{k-1} (not to q_{k+1}), using
//     q_{k+1} = (u_k - alpha_k q_k) / beta_k                     (stored as w)
//     u_{k+1} = H q_{k+1} - beta_k q_k
//             = (H u_k - alpha_k u_k - alpha_k beta_{k-1} q_{k-1}) / beta_k - beta_k q_k,
// and accumulates the exact 128-bit sums <w, u_{k+1}>, ||u_{k+1}||^2 and
// ||w||^2.  After the exchange alpha_{k+1} = <q_{k+1}, u_{k+1}> and
//     beta_{k+1}^2 = (||u||^2 ||w||^2 - <w, u>^2) / ||w||^2
// follow, the Gram numerator in exact 256-bit integer arithmetic, so that the
// cancellation of ||u||^2 - alpha^2 costs no accuracy.  The exponent of every
// stored vector comes from a rigorous bound as in the two-pass kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cfet_internal.h"
#include "device_common.cuh"
#include "fx_common.cuh"

namespace cfet {
namespace fx1 {

// ------------------------------------------------------------------ shared state
struct SmemFx {
  // per-warp partials of the workers
  unsigned long long wlo[32];
  long long whi[32];
  long long wmx[32];
  // per-warp partials of a pass: three 128-bit sums and two maxima
  unsigned long long plo[3][32];
  long long phi[3][32];
  long long pmx[2][32];
  // u buffers (parity of the Krylov index): exponent and max stored |M|
  int Eub[2];
  double Aub[2];
  // pass constants beyond the apply: -alpha/beta u_k, -beta s_k q_k
  long long m_self, m_qk;
  int pq;
  // Lanczos scalars (FP64) and vector metadata
  double alpha[kMaxKrylov + 2];
  double beta[kMaxKrylov + 2];
  double scale[kMaxKrylov + 3];  // 1 / ||q_i||, real units
  double A[kMaxKrylov + 3];      // max stored |M| of q_i
  int E[kMaxKrylov + 3];         // exponent of q_i
  double yr[kMaxKrylov], yi[kMaxKrylov];
  double tr[kMaxKrylov], ti[kMaxKrylov];
  // reconstruction constants
  long long crm[kMaxKrylov], cim[kMaxKrylov];
  int csr[kMaxKrylov], csi[kMaxKrylov], cp[kMaxKrylov];
  // stage data
  double scal[1 + kMaxDrives];
  double bsite_raw[kMaxSites];
  double bsum_raw, bmax_raw;  // sum and max over sites of |bsite_raw|
  int eb;                     // exponent of the per-site table mb
  long long mb[kMaxSites];
  FxConstA ca;
  // phase B constants
  long long m_a;
  int s_a, sh_u, pk_b;
  int Eu, Ew, Epsi;
  // control flags
  int abort_flag;     // leave the kernel
  int stop_prev;      // the deferred check accepted the previous iteration
  int accept_now;     // accepted at the current iteration
  int pend;           // a check of the current iteration is deferred
  int y_ready;        // yr/yi hold exp(-i ts T_k) e_1 for the accepted (k, ts)
  int acc_h;
  int final_rec;
  double err_now, err_prev;
  double beta0;
};

// ------------------------------------------------------------------ control-warp helpers
// Exact accumulation of exchanged CTA records: 128-bit sum (words 0-3) and
// int64 max (words 4-5).
struct FxAcc {
  unsigned long long lo;
  long long hi, m;
  __device__ void reset() { lo = 0; hi = 0; m = 0; }
  __device__ void add(const unsigned (&v)[6]) {
    const unsigned long long l2 = ((unsigned long long)v[1] << 32) | v[0];
    const long long h2 = (long long)(((unsigned long long)v[3] << 32) | v[2]);
    const long long m2 = (long long)(((unsigned long long)v[5] << 32) | v[4]);
    const unsigned long long t = lo + l2;
    hi = hi + h2 + (t < lo ? 1 : 0);
    lo = t;
    m = m > m2 ? m : m2;
  }
};

// Control warp: combine the workers' per-warp partials into this CTA's record,
// exchange records with every CTA (the grid barrier), and return the exact
// global sum (as FP64) and the global max to all lanes.
__device__ bool fx_ctl_reduce(SmemFx& S, int NW, unsigned long long* part, unsigned tag, bool fence, int* status,
                              long long timeout_ns, double& sum, long long& mxi, long long& spin) {
  const int lane = threadIdx.x & 31;
  unsigned long long lo = 0;
  long long hi = 0, m = 0;
  if (lane < NW) { lo = S.wlo[lane]; hi = S.whi[lane]; m = S.wmx[lane]; }
  fx_warp_reduce(lo, hi, m);
  lo = __shfl_sync(0xffffffffu, lo, 0);
  hi = __shfl_sync(0xffffffffu, hi, 0);
  m = __shfl_sync(0xffffffffu, m, 0);
  const unsigned mine[6] = {(unsigned)lo, (unsigned)(lo >> 32), (unsigned)hi,
                            (unsigned)((unsigned long long)hi >> 32), (unsigned)m,
                            (unsigned)((unsigned long long)m >> 32)};
  FxAcc acc;
  if (!ctl_exchange<6>(part, mine, tag, fence, status, timeout_ns, spin, acc)) return false;
  lo = acc.lo;
  hi = acc.hi;
  m = acc.m;
  fx_warp_reduce(lo, hi, m);
  lo = __shfl_sync(0xffffffffu, lo, 0);
  hi = __shfl_sync(0xffffffffu, hi, 0);
  m = __shfl_sync(0xffffffffu, m, 0);
  sum = fx_i128_to_double(lo, hi);
  mxi = m;
  return true;
}

// Worker warps: per-warp reduction of (int128 sum, int64 max) into shared memory.
__device__ __forceinline__ void fx_worker_partial(SmemFx& S, __int128 acc, long long mx) {
  acc >>= kRedShift;
  unsigned long long lo = (unsigned long long)acc;
  long long hi = (long long)(acc >> 64);
  fx_warp_reduce(lo, hi, mx);
  if ((threadIdx.x & 31) == 0) {
    const int w = threadIdx.x >> 5;
    S.wlo[w] = lo;
    S.whi[w] = hi;
    S.wmx[w] = mx;
  }
}

// Scalar part of the phase-A constants (one lane).
template <int FAMILY, class Op>
__device__ void fx_const_a_scalars(SmemFx& S, const Op& op, int it) {
  FxConstA& c = S.ca;
  const double sk = S.scale[it];
  const int Ek = S.E[it];
  const double Ak = S.A[it];
  const double Akr = fx_scale2(Ak, Ek);
  const double bp = it > 1 ? S.beta[it - 1] * S.scale[it - 1] : 0.0;
  const double Apr = it > 1 ? fx_scale2(S.A[it - 1], S.E[it - 1]) : 0.0;
  c.pk = fx_norm_shift(Ak);
  double B = fabs(bp) * Apr;
  if constexpr (FAMILY == kFamilySpin) {
    const double cz = S.scal[0] * sk;
    const double ch = cz * op.J2;
    // sum and max of |b_i s_k| from the per-stage sums of |b_i|
    const double bsum = fabs(sk) * S.bsum_raw, bmax = fabs(sk) * S.bmax_raw;
    B += (fabs(cz) * op.maxdz + fabs(ch) * (op.N - 1) + bsum) * Akr;
    const int Eu = fx_exp_for(B, kFxBits);
    const Mant mcz = fx_mant(cz);
    const int ED = fx_exp_for(fabs(cz) * op.maxdz, 59);
    c.m_cz = mcz.m;
    c.s_d = ED - mcz.e - (op.E_dz - 1) - 64;
    c.s_diag = Eu - (ED - 3) - (Ek - c.pk) - 64;
    c.m_cz = fx_fold(mcz.m, c.s_d + c.s_diag);
    const Mant mh = fx_mant(ch);
    c.ph = fx_norm_shift((op.N > 1 ? op.N - 1 : 1) * Ak);
    c.m_hop = mh.m;
    c.s_hop = Eu - mh.e - (Ek - c.ph) - 64;
    c.m_hop = fx_fold(c.m_hop, c.s_hop);
    if (op.uniform) {
      const Mant mx = fx_mant(S.bsite_raw[0] * sk);
      c.px = fx_norm_shift(op.N * Ak);
      c.m_x = mx.m;
      c.s_x = Eu - mx.e - (Ek - c.px) - 64;
      c.m_x = fx_fold(c.m_x, c.s_x);
    } else {
      const int eb = fx_exp_for(bmax, 62);
      c.s_nu = Eu - eb - (Ek - c.pk) - 64;
      S.eb = eb;
    }
    c.Eu = Eu;
  } else {
    for (int o = 0; o < op.nops; ++o) B += fabs(S.scal[o] * sk) * op.maxrow[o] * Akr;
    const int Eu = fx_exp_for(B, kFxBits);
    c.Eu = Eu;
    for (int o = 0; o < op.nops; ++o) {
      const int Epre = fx_exp_for(op.maxrow[o] * Akr, 62);  // |P_o| < 2^62
      c.sh_pre[o] = Epre - op.E_op[o] - Ek;
      const Mant m = fx_mant(S.scal[o] * sk);
      c.m_op[o] = m.m;
      c.s_op[o] = Eu - m.e - Epre - 64;
      c.m_op[o] = fx_fold(c.m_op[o], c.s_op[o]);
    }
  }
  const Mant mp = fx_mant(-bp);
  c.pp = it > 1 ? fx_norm_shift(S.A[it - 1]) : 0;
  c.m_p = mp.m;
  c.s_p = c.Eu - mp.e - (it > 1 ? S.E[it - 1] - c.pp : 0) - 64;
  c.m_p = fx_fold(c.m_p, c.s_p);
  c.use_prev = it > 1;
  S.Eu = c.Eu;
}

// Phase-A constants (called by the whole control warp: lane 0 computes the
// scalars, the per-site table is split over the lanes): result exponent of
// u = s_k H q_k - beta_{k-1} s_{k-1} q_{k-1} from the bound of every term,
// normalising shifts and product shifts.
template <int FAMILY, class Op>
__device__ void fx_const_a(SmemFx& S, const Op& op, int it) {
  const int lane = threadIdx.x & 31;
  FxConstA& c = S.ca;
  if (lane == 0) fx_const_a_scalars<FAMILY>(S, op, it);
  __syncwarp();
  if constexpr (FAMILY == kFamilySpin) {
    if (!op.uniform) {
      const double sk = S.scale[it];
      for (int i = lane; i < op.N; i += 32)
        S.mb[i] = fx_fold(__double2ll_rn(fx_scale2(S.bsite_raw[i] * sk, -S.eb)), c.s_nu);
    }
  }
}

// Error estimate of iteration k (control warp): err = beta0 beta_k |y_k| with
// y = exp(-i ts T_k) e_1 left in S.yr/S.yi.
__device__ double fx_estimate(SmemFx& S, int k, double ts) {
  small_expm_e1(k, S.alpha + 1, S.beta + 1, ts, S.yr, S.yi, S.tr, S.ti);
  return S.beta0 * S.beta[k] * hypot(S.yr[k - 1], S.yi[k - 1]);
}

// ------------------------------------------------------------------ one-pass helpers
// Worker warps: per-warp reduction of three int128 sums and two int64 maxima.
__device__ __forceinline__ void f1_worker_partial(SmemFx& S, __int128 s1, __int128 s2, __int128 s3, long long m1,
                                                  long long m2) {
  const __int128 in[3] = {s1 >> kRedShift, s2 >> kRedShift, s3 >> kRedShift};
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    unsigned long long lo = (unsigned long long)in[j];
    long long hi = (long long)(in[j] >> 64);
    long long mx = j == 0 ? m1 : m2;
    fx_warp_reduce(lo, hi, mx);
    if (lane == 0) {
      S.plo[j][w] = lo;
      S.phi[j][w] = hi;
      if (j < 2) S.pmx[j][w] = mx;
    }
  }
}

struct F1Sums {
  unsigned long long lo[3];
  long long hi[3];
  long long m[2];
};

// Exchange accumulator: three 128-bit sums (words 4j .. 4j+3) and two maxima
// (words 12-13, 14-15).
struct F1Acc {
  F1Sums s;
  __device__ void reset() {
    for (int j = 0; j < 3; ++j) { s.lo[j] = 0; s.hi[j] = 0; }
    s.m[0] = 0;
    s.m[1] = 0;
  }
  __device__ void add(const unsigned (&v)[16]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const unsigned long long l2 = ((unsigned long long)v[4 * j + 1] << 32) | v[4 * j];
      const long long h2 = (long long)(((unsigned long long)v[4 * j + 3] << 32) | v[4 * j + 2]);
      const unsigned long long t = s.lo[j] + l2;
      s.hi[j] = s.hi[j] + h2 + (t < s.lo[j] ? 1 : 0);
      s.lo[j] = t;
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const long long m2 = (long long)(((unsigned long long)v[13 + 2 * j] << 32) | v[12 + 2 * j]);
      s.m[j] = s.m[j] > m2 ? s.m[j] : m2;
    }
  }
};

__device__ __forceinline__ void f1_warp_reduce(F1Sums& r) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    long long dummy = 0;
    fx_warp_reduce(r.lo[j], r.hi[j], dummy);
    r.lo[j] = __shfl_sync(0xffffffffu, r.lo[j], 0);
    r.hi[j] = __shfl_sync(0xffffffffu, r.hi[j], 0);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r.m[j] = max(r.m[j], __shfl_xor_sync(0xffffffffu, r.m[j], o));
  }
}

// Control warp: this CTA's record from the workers' partials, the exchange
// (16-word records, word-major), and the grid totals in every lane.
__device__ bool f1_ctl_reduce(SmemFx& S, int NW, unsigned long long* part, unsigned tag, bool fence, int* status,
                              long long timeout_ns, F1Sums& out, long long& spin) {
  const int lane = threadIdx.x & 31;
  F1Sums c;
  for (int j = 0; j < 3; ++j) {
    c.lo[j] = lane < NW ? S.plo[j][lane] : 0;
    c.hi[j] = lane < NW ? S.phi[j][lane] : 0;
  }
  for (int j = 0; j < 2; ++j) c.m[j] = lane < NW ? S.pmx[j][lane] : 0;
  f1_warp_reduce(c);
  unsigned mine[16];
  for (int j = 0; j < 3; ++j) {
    mine[4 * j] = (unsigned)c.lo[j];
    mine[4 * j + 1] = (unsigned)(c.lo[j] >> 32);
    mine[4 * j + 2] = (unsigned)c.hi[j];
    mine[4 * j + 3] = (unsigned)((unsigned long long)c.hi[j] >> 32);
  }
  for (int j = 0; j < 2; ++j) {
    mine[12 + 2 * j] = (unsigned)c.m[j];
    mine[13 + 2 * j] = (unsigned)((unsigned long long)c.m[j] >> 32);
  }
  F1Acc acc;
  if (!ctl_exchange<16>(part, mine, tag, fence, status, timeout_ns, spin, acc)) return false;
  out = acc.s;
  f1_warp_reduce(out);
  return true;
}

// (hi * 2^64 + lo) as a double (no kRedShift factor)
__device__ __forceinline__ double f1_i128_to_double(unsigned long long lo, long long hi) {
  return fma(__ll2double_rn(hi), 18446744073709551616.0, __ull2double_rn(lo));
}

// a * b for unsigned 128-bit a, b: 256-bit result (hi, lo)
__device__ __forceinline__ void f1_mul128(unsigned __int128 a, unsigned __int128 b, unsigned __int128& hi,
                                         unsigned __int128& lo) {
  const unsigned long long a0 = (unsigned long long)a, a1 = (unsigned long long)(a >> 64);
  const unsigned long long b0 = (unsigned long long)b, b1 = (unsigned long long)(b >> 64);
  const unsigned __int128 p00 = (unsigned __int128)a0 * b0, p01 = (unsigned __int128)a0 * b1;
  const unsigned __int128 p10 = (unsigned __int128)a1 * b0, p11 = (unsigned __int128)a1 * b1;
  const unsigned __int128 mid = (p00 >> 64) + (unsigned long long)p01 + (unsigned long long)p10;
  lo = (mid << 64) | (unsigned long long)p00;
  hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
}

// Gram numerator T2 T3 - T1^2 (T1 = <w,u>, T2 = ||u||^2, T3 = ||w||^2, exact
// reduced sums) in 256-bit integers, as a double; clamped at 0.
__device__ double f1_gram(const F1Sums& r) {
  const __int128 t1 = ((__int128)r.hi[0] << 64) | r.lo[0];
  const unsigned __int128 t2 = ((unsigned __int128)(unsigned long long)r.hi[1] << 64) | r.lo[1];
  const unsigned __int128 t3 = ((unsigned __int128)(unsigned long long)r.hi[2] << 64) | r.lo[2];
  const unsigned __int128 a1 = t1 < 0 ? (unsigned __int128)(-t1) : (unsigned __int128)t1;
  unsigned __int128 ph, pl, qh, ql;
  f1_mul128(t2, t3, ph, pl);
  f1_mul128(a1, a1, qh, ql);
  if (ph < qh || (ph == qh && pl < ql)) return 0.0;
  const unsigned __int128 dl = pl - ql;
  const unsigned __int128 dh = ph - qh - (pl < ql ? 1 : 0);
  const double two64 = 18446744073709551616.0;
  const double h = fma(__ull2double_rn((unsigned long long)(dh >> 64)), two64, __ull2double_rn((unsigned long long)dh));
  const double l = fma(__ull2double_rn((unsigned long long)(dl >> 64)), two64, __ull2double_rn((unsigned long long)dl));
  return fma(h, two64 * two64, l);
}

// Constants of pass P(k) (control warp; scalars on lane 0, per-site table over
// the lanes).  mode 0 (k = 0): u_1 = s_1 H q_1.  mode 1: apply to u_k with the
// scale 1/beta_k, the previous-vector term -alpha_k beta_{k-1} s_{k-1} / beta_k
// q_{k-1}, the terms -alpha_k/beta_k u_k and -beta_k s_k q_k, and
// w = u_k - alpha_k s_k q_k.  Every result exponent from the bound of its terms.
template <int FAMILY, class Op>
__device__ void f1_const(SmemFx& S, const Op& op, int k, int mode) {
  const int lane = threadIdx.x & 31;
  FxConstA& c = S.ca;
  double sk = 0.0;
  if (lane == 0) {
    double Ak, bp = 0.0, Apr = 0.0, cself = 0.0, cq = 0.0, Aq = 0.0, a = 0.0;
    int Ek, Epr = 0, Eq = 0;
    if (mode == 0) {
      sk = S.scale[1];
      Ek = S.E[1];
      Ak = S.A[1];
    } else {
      a = S.alpha[k];
      const double b = S.beta[k];
      sk = 1.0 / b;
      Ek = S.Eub[k & 1];
      Ak = S.Aub[k & 1];
      if (k >= 2) {
        bp = a * S.beta[k - 1] * S.scale[k - 1] / b;
        Apr = S.A[k - 1];
        Epr = S.E[k - 1];
      }
      cself = -a / b;
      cq = -b * S.scale[k];
      Aq = S.A[k];
      Eq = S.E[k];
    }
    const double Akr = fx_scale2(Ak, Ek);
    const double Aprr = k >= 2 && mode == 1 ? fx_scale2(Apr, Epr) : 0.0;
    const double Aqr = mode == 1 ? fx_scale2(Aq, Eq) : 0.0;
    c.pk = fx_norm_shift(Ak);
    double B = fabs(bp) * Aprr + fabs(cself) * Akr + fabs(cq) * Aqr;
    if constexpr (FAMILY == kFamilySpin) {
      const double cz = S.scal[0] * sk;
      const double ch = cz * op.J2;
      const double bsum = fabs(sk) * S.bsum_raw, bmax = fabs(sk) * S.bmax_raw;
      B += (fabs(cz) * op.maxdz + fabs(ch) * (op.N - 1) + bsum) * Akr;
      const int Eu = fx_exp_for(B, kFxBits);
      const Mant mcz = fx_mant(cz);
      const int ED = fx_exp_for(fabs(cz) * op.maxdz, 59);
      c.m_cz = mcz.m;
      c.s_d = ED - mcz.e - (op.E_dz - 1) - 64;
      c.s_diag = Eu - (ED - 3) - (Ek - c.pk) - 64;
      c.m_cz = fx_fold(mcz.m, c.s_d + c.s_diag);
      const Mant mh = fx_mant(ch);
      c.ph = fx_norm_shift((op.N > 1 ? op.N - 1 : 1) * Ak);
      c.s_hop = Eu - mh.e - (Ek - c.ph) - 64;
      c.m_hop = fx_fold(mh.m, c.s_hop);
      if (op.uniform) {
        const Mant mx = fx_mant(S.bsite_raw[0] * sk);
        c.px = fx_norm_shift(op.N * Ak);
        c.s_x = Eu - mx.e - (Ek - c.px) - 64;
        c.m_x = fx_fold(mx.m, c.s_x);
      } else {
        const int eb = fx_exp_for(bmax, 62);
        c.s_nu = Eu - eb - (Ek - c.pk) - 64;
        S.eb = eb;
      }
      c.Eu = Eu;
    } else {
      const double Akr2 = Akr;
      for (int o = 0; o < op.nops; ++o) B += fabs(S.scal[o] * sk) * op.maxrow[o] * Akr2;
      const int Eu = fx_exp_for(B, kFxBits);
      c.Eu = Eu;
      for (int o = 0; o < op.nops; ++o) {
        const int Epre = fx_exp_for(op.maxrow[o] * Akr2, 62);  // |P_o| < 2^62
        c.sh_pre[o] = Epre - op.E_op[o] - Ek;
        const Mant m = fx_mant(S.scal[o] * sk);
        c.m_op[o] = m.m;
        c.s_op[o] = Eu - m.e - Epre - 64;
        c.m_op[o] = fx_fold(c.m_op[o], c.s_op[o]);
      }
    }
    const int Eu = c.Eu;
    const Mant mp = fx_mant(-bp);
    c.pp = (mode == 1 && k >= 2) ? fx_norm_shift(Apr) : 0;
    c.m_p = mp.m;
    c.s_p = Eu - mp.e - ((mode == 1 && k >= 2) ? Epr - c.pp : 0) - 64;
    c.m_p = fx_fold(c.m_p, c.s_p);
    c.use_prev = mode == 1 && k >= 2;
    S.pq = fx_norm_shift(Aq);
    const Mant ms = fx_mant(cself), mq = fx_mant(cq);
    S.m_self = ms.m == 0 ? 0 : fx_fold(ms.m, Eu - ms.e - (Ek - c.pk) - 64);
    S.m_qk = mq.m == 0 ? 0 : fx_fold(mq.m, Eu - mq.e - (Eq - S.pq) - 64);
    if (mode == 1) {  // w = u_k - alpha_k s_k q_k
      const double am = a * S.scale[k];
      const double Bw = Akr + fabs(am) * Aqr;
      const int Ew = fx_exp_for(Bw, kFxBits);
      const Mant ma = fx_mant(-am);
      S.Ew = Ew;
      S.sh_u = Ew - Ek;
      S.m_a = ma.m == 0 ? 0 : fx_fold(ma.m, Ew - ma.e - (Eq - S.pq) - 64);
    }
  }
  __syncwarp();
  if constexpr (FAMILY == kFamilySpin) {
    if (!op.uniform) {
      sk = __shfl_sync(0xffffffffu, sk, 0);
      for (int i = lane; i < op.N; i += 32)
        S.mb[i] = fx_fold(__double2ll_rn(fx_scale2(S.bsite_raw[i] * sk, -S.eb)), c.s_nu);
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------------ the kernel
template <int FAMILY, class Op>
__global__ void __launch_bounds__(CFET_CTL_MAX_THREADS, 1) k_propagate_fx1(PropParams p, Op op) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemFx& S = *reinterpret_cast<SmemFx*>(smem_raw);
  const int tid = threadIdx.x;
  const int NW = (int)(blockDim.x >> 5) - 1;   // worker warps
  const bool ctl = (tid >> 5) == NW;            // control warp
  const int lane = tid & 31;
  const bool lead = ctl && lane == 0;
  const int dim = p.dim;
  const int G = gridDim.x;
  // each CTA walks one contiguous chunk of the vectors, so that the
  // neighbours of low-bit flips (and short band offsets) are found in L1
  const int chunk = (dim + G - 1) / G;
  const int wstep = NW * 32;
  const int wx0 = blockIdx.x * chunk + tid;  // workers only
  const int wxe = min(dim, (blockIdx.x + 1) * chunk);
  const int ncoef = 1 + p.nV;
  // record exchange: three slots (phase A, phase B, reconstruction) of six
  // tagged words per CTA; two uses of one slot are always separated by an
  // exchange on another slot; tags continue across launches
  const unsigned tag0 = (unsigned)ld_volatile_i32((const int*)&p.st->tag_base);
  unsigned gen = 0;
  // slots: part0 / part1 alternate for the 16-word pass records (word-major),
  // partA / partB (conversion) and partR (reconstruction) hold 6-word records
  unsigned long long* part0 = reinterpret_cast<unsigned long long*>(p.partials);
  unsigned long long* part1 = part0 + 16 * G;
  unsigned long long* partA = part0 + 32 * G;
  unsigned long long* partB = part0 + 40 * G;
  unsigned long long* partR = part0 + 48 * G;
  DevStatus* st = p.st;
  const bool glead = (blockIdx.x == 0) && lead;
  // trace (see cfet_stats.phase_ns): worker loop times by thread 0, control
  // own-time and barrier waits by the control lane 0, in SM clock cycles
  long long tacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long twe = 0;  // thread 0: end of its last worker loop
  const bool fixed_k = p.tol <= 0.0;
  const bool forced = p.f_nsub != nullptr;

  long long fpos = st->forced_pos;
  long long rpos = st->rec_pos;
  long long n_app = 0, n_sub = 0;
  int max_k = 0;
  double max_err = 0.0;

  auto Q = [&](int i) -> longlong2* { return p.qbasis + (size_t)(i - 1) * dim; };
  // u_k of the pass structure: two buffers after the m_max + 1 basis vectors
  auto U = [&](int k) -> longlong2* { return p.qbasis + (size_t)(p.m_max + 1 + (k & 1)) * dim; };

  // ---------------- psi (complex128) -> q_1
  // pass 1: max |component| (as ordered bit patterns of |v|) and NaN/Inf detection
  {
    if (!ctl) {
      long long mx = 0;
      for (int x = wx0; x < wxe; x += wstep) {
        const double2 v = p.psi[x];
        const long long a = __double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFLL;
        const long long b = __double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFLL;
        mx = max(mx, max(a, b));
      }
      fx_worker_partial(S, 0, mx);
    }
    __syncthreads();
    if (ctl) {
      // the max bit pattern is reduced in the int64 max lane
      double sum;
      long long bits;
      if (!fx_ctl_reduce(S, NW, partA, tag0 + (++gen), false, &st->status, p.timeout_ns, sum, bits, tacc[5])) {
        if (lane == 0) S.abort_flag = 1;
      } else if (lane == 0) {
        S.abort_flag = 0;
        if (bits >= 0x7FF0000000000000LL) {
          atomicCAS(&st->status, 0, (int)CFET_ENAN);
          S.abort_flag = 1;
        } else {
          S.E[1] = fx_exp_for(__longlong_as_double(bits), kFxBits);
        }
      }
    }
    __syncthreads();
    if (S.abort_flag) return;
    // pass 2: convert and take ||q_1||^2, max |M|
    if (!ctl) {
      const double sc = fx_scale2(1.0, -S.E[1]);
      __int128 a2 = 0;
      long long mx = 0;
      for (int x = wx0; x < wxe; x += wstep) {
        const double2 v = p.psi[x];
        const longlong2 qv = make_longlong2(__double2ll_rn(v.x * sc), __double2ll_rn(v.y * sc));
        Q(1)[x] = qv;
        a2 += (__int128)qv.x * qv.x + (__int128)qv.y * qv.y;
        mx = max(mx, fx_absmax(qv.x, qv.y));
      }
      fx_worker_partial(S, a2, mx);
    }
    __syncthreads();
    if (ctl) {
      double sum;
      long long mxi;
      if (!fx_ctl_reduce(S, NW, partB, tag0 + (++gen), true, &st->status, p.timeout_ns, sum, mxi, tacc[5])) {
        if (lane == 0) S.abort_flag = 1;
      } else if (lane == 0) {
        S.beta0 = fx_scale2(sqrt(sum), S.E[1]);
        S.A[1] = __ll2double_ru(mxi);
      }
    }
    __syncthreads();
    if (S.abort_flag) return;
  }

  for (long long e = 0; e < p.nexp; ++e) {
    if (tid < ncoef) S.scal[tid] = p.scal[e * ncoef + tid];
    __syncthreads();
    if constexpr (FAMILY == kFamilySpin) {
      if (ctl) {  // per-site transverse fields of this stage (N <= 30 lanes)
        double bi = 0.0;
        if (lane < op.N) {
          for (int k = 0; k < p.nV; ++k) bi = fma(S.scal[1 + k], __ldg(op.xf + k * op.N + lane), bi);
          S.bsite_raw[lane] = bi;
        }
        double bs = fabs(bi), bm = fabs(bi);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          bs += __shfl_xor_sync(0xffffffffu, bs, o);
          bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
        }
        if (lane == 0) {
          S.bsum_raw = bs;
          S.bmax_raw = bm;
        }
      }
      __syncthreads();
    }
    const long long eg = p.exp_base + e;
    const bool last_exp = (e == p.nexp - 1);
    const int nforced = forced ? p.f_nsub[eg] : 0;
    double remaining = p.tau;
    int nsub_e = 0;
    while (true) {
      if (nsub_e >= p.max_substeps || (forced && nsub_e >= nforced)) {
        if (glead) atomicCAS(&st->status, 0, (int)CFET_EKRYLOV);
        return;
      }
      int kf = -1, hf = 0;
      if (forced) {
        kf = p.f_k[fpos];
        hf = p.f_h[fpos];
      }
      const double beta0 = S.beta0;
      int acc_k = 0, acc_h = 0;
      double acc_err = 0.0;
      if (beta0 != 0.0) {
        const int klimit = forced ? kf : p.m_max;
        if (lead) {
          S.scale[1] = 1.0 / beta0;
          S.pend = 0;
          S.stop_prev = 0;
          S.accept_now = 0;
          S.y_ready = 0;
        }
        if (ctl) {
          __syncwarp();
          f1_const<FAMILY>(S, op, 0, 0);
        }
        __syncthreads();
        // P(0): u_1 = s_1 H q_1 with the sums <q_1, u_1>, ||u_1||^2, ||q_1||^2
        int it = 0;
        int xslot = 0;
        for (;;) {
          // -------- pass P(it) on the workers; deferred estimate of it on the control warp
          const int pend = S.pend;
          if (!ctl) {
            const FxConstA& c = S.ca;
            const longlong2* uin = it == 0 ? Q(1) : U(it);      // apply input
            const longlong2* qk = it == 0 ? Q(1) : Q(it);       // q_it (own elements)
            const longlong2* qm = it >= 2 ? Q(it - 1) : qk;     // q_{it-1}
            longlong2* wout = Q(it + 1);                         // w = beta_it q_{it+1} (it >= 1)
            longlong2* uout = U(it + 1);
            const long long m_self = S.m_self, m_qk = S.m_qk, m_a = S.m_a;
            const int pq = S.pq, sh_u = S.sh_u, pk = c.pk;
            __int128 s1 = 0, s2 = 0, s3 = 0;
            long long my = 0, mw = 0;
            const long long tw0 = sm_clock();
            auto finish = [&](int x, longlong2 y) {
              longlong2 w;
              const longlong2 v = uin[x];
              if (it >= 1) {
                const longlong2 q = qk[x];
                y.x += fx_mulhi(m_self, v.x << pk) + fx_mulhi(m_qk, q.x << pq);
                y.y += fx_mulhi(m_self, v.y << pk) + fx_mulhi(m_qk, q.y << pq);
                w.x = fx_rshr(v.x, sh_u) + fx_mulhi(m_a, q.x << pq);
                w.y = fx_rshr(v.y, sh_u) + fx_mulhi(m_a, q.y << pq);
                wout[x] = w;
              } else {
                w = v;
              }
              uout[x] = y;
              s1 += (__int128)w.x * y.x + (__int128)w.y * y.y;
              s2 += (__int128)y.x * y.x + (__int128)y.y * y.y;
              s3 += (__int128)w.x * w.x + (__int128)w.y * w.y;
              my = max(my, fx_absmax(y.x, y.y));
              mw = max(mw, fx_absmax(w.x, w.y));
            };
            for (int x = wx0; x < wxe; x += wstep) {
              longlong2 hv;
              if constexpr (FAMILY == kFamilySpin) hv = fx_apply_spin(uin, qm, x, op, c, S.mb);
              else hv = fx_apply_dia(uin, qm, x, dim, op, c);
              finish(x, hv);
            }
            f1_worker_partial(S, s1, s2, s3, my, mw);
            if (tid == 0) {
              twe = sm_clock();
              tacc[0] += twe - tw0;
            }
          } else if (pend) {
            const long long te0 = sm_clock();
            const double err = fx_estimate(S, it, remaining);
            if (lane == 0) {
              S.err_prev = err;
              S.stop_prev = err <= p.tol * remaining / p.tau;
              S.y_ready = S.stop_prev;
              tacc[6] += sm_clock() - te0;
            }
            __syncwarp();
          }
          __syncthreads();
          if (ctl) {
            const long long tc0 = sm_clock(), sp0 = tacc[5];
            F1Sums r;
            if (!f1_ctl_reduce(S, NW, xslot ? part1 : part0, tag0 + (++gen), true, &st->status, p.timeout_ns, r,
                               tacc[5])) {
              if (lane == 0) S.abort_flag = 1;
            } else if (!S.stop_prev) {
              const int k = it + 1;  // the Krylov dimension decided now
              const int Ey = S.ca.Eu;
              const int Ewk = it == 0 ? S.E[1] : S.Ew;
              if (lane == 0) {
                // q_k = w (for k = 1 it is q_1 itself): exponent, max, 1 / ||q_k||
                const double n3 = f1_i128_to_double(r.lo[2], r.hi[2]);  // ||w||^2 / 2^kRedShift, mantissa units
                if (it >= 1) {
                  S.E[k] = Ewk;
                  S.A[k] = __ll2double_ru(r.m[1]);
                  S.scale[k] = n3 > 0.0 ? fx_scale2(rsqrt(n3 * (double)(1 << kRedShift)), -Ewk) : 0.0;
                }
                S.Eub[k & 1] = Ey;
                S.Aub[k & 1] = __ll2double_ru(r.m[0]);
                // alpha_k = s_k <q_k, u_k>;  beta_k^2 = ||u_k||^2 - <q_k,u_k>^2 / ||q_k||^2 (exact Gram numerator)
                const double n1 = f1_i128_to_double(r.lo[0], r.hi[0]);
                S.alpha[k] = fx_scale2(n1 * (double)(1 << kRedShift), Ewk + Ey) * S.scale[k];
                const double g = f1_gram(r);  // (T2 T3 - T1^2) as a double (>= 0)
                const double b2 = n3 > 0.0 ? g / n3 * (double)(1 << kRedShift) : 0.0;
                S.beta[k] = fx_scale2(sqrt(b2), Ey);
                if (__ll2double_ru(r.m[0]) >= 1.152921504606846976e18 ||
                    __ll2double_ru(r.m[1]) >= 1.152921504606846976e18) {  // 2^60: range exceeded (not expected)
                  atomicCAS(&st->status, 0, (int)CFET_ENAN);
                  S.abort_flag = 1;
                }
              }
              __syncwarp();
              const double b = S.beta[k];
              const double prev_b = k > 1 ? S.beta[k - 1] : 0.0;
              const bool breakdown = b <= 1e-13 * (fabs(S.alpha[k]) + prev_b + 1.0);
              int acc_flag = 0, pend_next = 0;
              double err = 0.0;
              if (forced) {
                acc_flag = (k == kf);
              } else if (fixed_k) {
                acc_flag = (k == p.m_max) || breakdown;
              } else if (breakdown) {
                acc_flag = 1;
              } else if (k >= p.m_min &&
                         fabs(remaining) * gersh_width(k, S.alpha + 1, S.beta + 1) <= 2.0 * k) {
                if (k < klimit) {
                  pend_next = 1;  // estimate runs during the next pass
                } else {
                  err = fx_estimate(S, k, remaining);
                  acc_flag = err <= p.tol * remaining / p.tau;
                }
              }
              if (lane == 0) {
                S.accept_now = acc_flag;
                S.pend = pend_next;
                S.err_now = err;
                S.y_ready = acc_flag && !forced && !fixed_k && !breakdown;
              }
              __syncwarp();
              if (!acc_flag && k < klimit && !S.abort_flag) f1_const<FAMILY>(S, op, k, 1);
            }
            if (lane == 0) tacc[3] += sm_clock() - tc0 - (tacc[5] - sp0);
          }
          xslot ^= 1;
          __syncthreads();
          if (tid == 0) tacc[7] += sm_clock() - twe;
          if (S.abort_flag) return;
          if (S.stop_prev) {  // the deferred estimate accepted dimension it
            acc_err = S.err_prev;
            break;
          }
          it += 1;
          if (S.accept_now) {
            acc_err = S.err_now;
            break;
          }
          if (it >= klimit) break;
        }
        acc_k = it;
        const bool accepted = S.accept_now || S.stop_prev;
        acc_h = 0;
        if (forced) {
          acc_h = hf;
        } else if (!accepted) {
          // halve the substep on the same basis until the estimate meets the
          // proportional tolerance (control warp)
          if (ctl) {
            int hh = 0;
            double err = 0.0;
            const double width = gersh_width(it, S.alpha + 1, S.beta + 1);
            for (int h = 1; h <= 40; ++h) {
              const double ts = fx_scale2(remaining, -h);
              if (!(fabs(ts) * width <= 2.0 * it)) continue;
              err = fx_estimate(S, it, ts);
              if (err <= p.tol * ts / p.tau) { hh = h; break; }
            }
            if (lane == 0) { S.acc_h = hh; S.err_now = err; S.y_ready = hh > 0; }
          }
          __syncthreads();
          acc_h = S.acc_h;
          acc_err = S.err_now;
          if (acc_h == 0) {
            if (glead) atomicCAS(&st->status, 0, (int)CFET_EKRYLOV);
            return;
          }
        }
        n_app += acc_k;
      }
      const double ts = fx_scale2(remaining, -acc_h);
      const bool final_rec = last_exp && acc_h == 0;
      if (acc_k > 0) {
        // -------- reconstruct q_1 <- beta0 sum_i y_i s_i q_i
        if (ctl) {
          const long long tr0 = sm_clock();
          if (!S.y_ready) small_expm_e1(acc_k, S.alpha + 1, S.beta + 1, ts, S.yr, S.yi, S.tr, S.ti);
          __syncwarp();
          double bnd = 0.0;
          for (int i = lane; i < acc_k; i += 32) {
            const double f = beta0 * S.scale[i + 1];
            const double cr = f * S.yr[i], ci = f * S.yi[i];
            S.yr[i] = cr;
            S.yi[i] = ci;
            bnd += (fabs(cr) + fabs(ci)) * fx_scale2(S.A[i + 1], S.E[i + 1]);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) bnd += __shfl_xor_sync(0xffffffffu, bnd, o);
          const int Ep = fx_exp_for(bnd, kFxBits);
          for (int i = lane; i < acc_k; i += 32) {
            const Mant mr = fx_mant(S.yr[i]), mi = fx_mant(S.yi[i]);
            const int pi = fx_norm_shift(S.A[i + 1]);
            S.crm[i] = mr.m;
            S.cim[i] = mi.m;
            S.cp[i] = pi;
            S.csr[i] = Ep - mr.e - (S.E[i + 1] - pi) - 64;
            S.csi[i] = Ep - mi.e - (S.E[i + 1] - pi) - 64;
            S.crm[i] = fx_fold(mr.m, S.csr[i]);
            S.cim[i] = fx_fold(mi.m, S.csi[i]);
          }
          if (lane == 0) {
            S.Epsi = Ep;
            tacc[6] += sm_clock() - tr0;
          }
        }
        __syncthreads();
        if (!ctl) {
          const double outscale = fx_scale2(1.0, S.Epsi);
          __int128 a2 = 0;
          long long mx = 0;
          const long long tw0 = sm_clock();
          for (int x = wx0; x < wxe; x += wstep) {
            long long re = 0, im = 0;
            for (int i = 0; i < acc_k; ++i) {
              const longlong2 v = Q(i + 1)[x];
              const int pi = S.cp[i];
              const long long cr = S.crm[i], ci = S.cim[i];
              const long long vr = v.x << pi, vi = v.y << pi;
              // (cr + i ci)(vr + i vi) with three products; the sums (< 2^63)
              // are halved to stay in fx_mulhi's operand range
              const long long p1 = fx_mulhi(cr, vr), p2 = fx_mulhi(ci, vi);
              const long long p3 = fx_mulhi((cr + ci) >> 1, (vr + vi) >> 1) << 2;
              re += p1 - p2;
              im += p3 - p1 - p2;
            }
            Q(1)[x] = make_longlong2(re, im);
            if (final_rec) p.psi[x] = make_double2(__ll2double_rn(re) * outscale, __ll2double_rn(im) * outscale);
            a2 += (__int128)re * re + (__int128)im * im;
            mx = max(mx, fx_absmax(re, im));
          }
          fx_worker_partial(S, a2, mx);
          if (tid == 0) {
              twe = sm_clock();
              tacc[4] += twe - tw0;
            }
        }
        __syncthreads();
        if (ctl) {
          double sum;
          long long mxi;
          if (!fx_ctl_reduce(S, NW, partR, tag0 + (++gen), true, &st->status, p.timeout_ns, sum, mxi, tacc[5])) {
            if (lane == 0) S.abort_flag = 1;
          } else if (lane == 0) {
            S.beta0 = fx_scale2(sqrt(sum), S.Epsi);
            S.E[1] = S.Epsi;
            S.A[1] = __ll2double_ru(mxi);
          }
        }
        __syncthreads();
        if (tid == 0) tacc[7] += sm_clock() - twe;
        if (S.abort_flag) return;
      }
      if (glead && p.r_k != nullptr) {
        if (rpos < p.r_cap) {
          p.r_k[rpos] = acc_k;
          p.r_h[rpos] = acc_h;
        } else {
          st->rec_overflow = 1;
        }
      }
      rpos += 1;
      if (forced) fpos += 1;
      n_sub += 1;
      nsub_e += 1;
      if (acc_k > max_k) max_k = acc_k;
      if (acc_err > max_err) max_err = acc_err;
      if (acc_h == 0) break;
      remaining -= ts;
    }
    if (glead && p.r_nsub != nullptr) p.r_nsub[eg] = nsub_e;
  }
  if (glead) {
    st->tag_base = tag0 + gen;
    st->forced_pos = fpos;
    st->rec_pos = rpos;
    st->n_exp += p.nexp;
    st->n_sub += n_sub;
    st->n_app += n_app;
    if (max_k > st->max_k) st->max_k = max_k;
    if (max_err > st->max_err) st->max_err = max_err;
  }
  if (tid == 0 || lead) {  // every CTA: mean and max of its phase times
    // thread 0 holds the worker slots 0, 2, 4, 7; the control lane 1, 3, 5, 6
    const int mine[2][4] = {{0, 2, 4, 7}, {1, 3, 5, 6}};
    for (int j = 0; j < 4; ++j) {
      const int i = mine[tid == 0 ? 0 : 1][j];
      atomicAdd((unsigned long long*)&st->phase_ns[i], (unsigned long long)(tacc[i] / G));
      atomicMax(&st->phase_max_ns[i], tacc[i]);
    }
  }
}

}  // namespace fx1

// ------------------------------------------------------------------ launchers
template <int FAMILY, class Op>
static int launch_prop_fx1(const PropParams& p, const Op& op, int grid, int block, void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = sizeof(fx1::SmemFx);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, fx1::k_propagate_fx1<FAMILY, Op>, p, op);
}

int launch_propagate_spin_fx1(const PropParams& p, const OpSpinFx& op, int grid, int block, void* stream) {
  return launch_prop_fx1<kFamilySpin>(p, op, grid, block, stream);
}
int launch_propagate_dia_fx1(const PropParams& p, const OpDiaFx& op, int grid, int block, void* stream) {
  return launch_prop_fx1<kFamilyDia>(p, op, grid, block, stream);
}

int max_coresident_blocks_fx1(int family, int block) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(fx1::k_propagate_fx1<kFamilySpin, OpSpinFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(fx1::k_propagate_fx1<kFamilyDia, OpDiaFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaError_t e;
  if (family == kFamilySpin)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fx1::k_propagate_fx1<kFamilySpin, OpSpinFx>, block,
                                                      sizeof(fx1::SmemFx));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fx1::k_propagate_fx1<kFamilyDia, OpDiaFx>, block,
                                                      sizeof(fx1::SmemFx));
  if (e != cudaSuccess) return -1;
  return per * nsm;
}

}  // namespace cfet
