// Chebyshev stage exponentials in the fixed-point format (sm_103a).
//
// Sec. 8.1 names the Chebyshev technique as the alternative to the Krylov
// method for exp(-i tau H_j) psi.  With [b - a, b + a] bounding the spectrum
// of H_j (host: Gershgorin intervals combined by Weyl's inequality) and
// Htilde = (H_j - b) / a,
//
//     exp(-i tau H_j) psi = exp(-i tau b) sum_{k=0}^{K} r_k (-i)^k v_k,
//     v_0 = psi,  v_1 = Htilde psi,  v_{k+1} = 2 Htilde v_k - v_{k-1},
//     r_k = (2 - delta_k0) J_k(tau a)                       (Jacobi-Anger),
//
// K and r_k come from the host (the Bessel tail bound).  No reductions are
// needed: one persistent launch runs all stage exponentials of a chunk of
// steps, one fused pass per term (apply with neighbour gathers of v_k, the
// recurrence, the accumulation of sum_k r_k (-i)^k v_k) followed by one
// grid-wide record exchange (the barrier).  The last term of an exponential
// writes exp(-i tau b) * sum as the next v_0.
//
// Number format: the fixed-point format of kernels_fx.cu (int64 (re, im)
// mantissas, exact integer neighbour sums, one rounding per scalar product)
// with ONE exponent E for every v_k of the launch.  In exact arithmetic
// ||v_k||_2 <= ||psi||_2 (|T_k| <= 1 on [-1, 1] contains the spectrum of
// Htilde), so every component stays below ||psi||_2 < 2^(52 + E) when E is
// taken from 32 ||psi||_2 < 2^(57 + E); the sum is kept at its own exponent
// E + ea from the bound sum_k |r_k| ||psi||_2.  Products are rounded once to
// the unit of the result, as in the Krylov kernel.
//
// CTA layout: every warp does element work; warp 0 also runs the exchange.
// Each CTA walks one contiguous chunk of the vectors (low-bit neighbours in L1).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cfet_internal.h"
#include "device_common.cuh"
#include "fx_common.cuh"

namespace cfet {

// Threads per CTA (launch bound).
#ifndef CFET_CHEB_THREADS
#define CFET_CHEB_THREADS 768
#endif
constexpr int kChebThreads = CFET_CHEB_THREADS;

struct SmemCheb {
  // constants of the current term
  FxConstA c;
  long long mb[kMaxSites];        // per-site field table (site-dependent fields)
  long long m_s;                  // shift term -g b v
  long long m_r, m_r0;            // r_k (-i)^k y and r_0 v_0 into the sum
  int py, p0;                     // normalising shifts of y and v_0 in those products
  int sa;                         // right shift of the stored sum before this term's addition
  int E_acc;                      // exponent of the sum after this term
  int E_out;                      // exponent of this term's output
  long long m_cs, m_sn;           // conversion of the sum to v_0: cos(tau b), -sin(tau b)
  int L_rot;
  // per exponential
  double scal[1 + kMaxDrives];
  double bsite[kMaxSites];
  double bsum, bmax;
  // per exponential and kind of term (0: first, Htilde; 1: later, 2 Htilde):
  // mantissas of the scalars and the coefficient sum of the output bound
  struct TermScalars {
    double csum;                 // B = A_prev + csum * A_k (real units)
    Mant mcz, mh, mx, ms;        // c0 g, c0 g 2J, b_0 g (uniform fields), -g b
    int ED, eb;                  // exponent of the diagonal bound; of the per-site table
    Mant mop[1 + kMaxDrives];    // DIA: scal[o] g
    long long mbraw[kMaxSites];  // per-site table before the product shift
  } ts[2];
  // vectors: exponent and measured max |mantissa| of the three slots
  int Ev[3];
  long long Av[3];
  long long accmax;               // measured max |mantissa| of the sum
  // reductions
  unsigned long long wmy[32], wma[32];
  double wsum[32];
  long long t_const, t_pass;      // trace (SM cycles): term constants (warp 0), element passes (thread 0)
  int abort_flag;
};

// Exchange accumulators.
struct ChebSumMax {  // FP64 sum + max (the initial pass)
  double s;
  unsigned long long m;
  __device__ void reset() { s = 0.0; m = 0; }
  __device__ void add(const unsigned (&v)[4]) {
    s += __longlong_as_double((long long)(((unsigned long long)v[1] << 32) | v[0]));
    const unsigned long long x = ((unsigned long long)v[3] << 32) | v[2];
    m = x > m ? x : m;
  }
};
struct ChebMax2 {    // two maxima
  unsigned long long a, b;
  __device__ void reset() { a = 0; b = 0; }
  __device__ void add(const unsigned (&v)[4]) {
    const unsigned long long x = ((unsigned long long)v[1] << 32) | v[0];
    const unsigned long long y = ((unsigned long long)v[3] << 32) | v[2];
    a = x > a ? x : a;
    b = y > b ? y : b;
  }
};

// Per-exponential part of the term constants (warp 0: lane 0 for the scalars,
// the lanes for the per-site table) for the term kind `slot` with
// y = g H_j v - g b v - use_prev v_prev.
template <int FAMILY, class Op>
__device__ void cheb_exp_scalars(SmemCheb& S, int slot, const Op& op, double g, double gb) {
  const int lane = threadIdx.x & 31;
  SmemCheb::TermScalars& T = S.ts[slot];
  if (lane == 0) {
    T.ms = fx_mant(-gb);
    double cs = fabs(gb);
    if constexpr (FAMILY == kFamilySpin) {
      const double cz = S.scal[0] * g;
      const double ch = cz * op.J2;
      cs += fabs(cz) * op.maxdz + fabs(ch) * (op.N - 1) + fabs(g) * S.bsum;
      T.mcz = fx_mant(cz);
      T.ED = fx_exp_for(fabs(cz) * op.maxdz, 59);
      T.mh = fx_mant(ch);
      if (op.uniform) T.mx = fx_mant(S.bsite[0] * g);
      else T.eb = fx_exp_for(fabs(g) * S.bmax, 62);
    } else {
      for (int o = 0; o < op.nops; ++o) {
        cs += fabs(S.scal[o] * g) * op.maxrow[o];
        T.mop[o] = fx_mant(S.scal[o] * g);
      }
    }
    T.csum = cs;
  }
  if constexpr (FAMILY == kFamilySpin) {
    if (!op.uniform) {
      __syncwarp();
      const int eb = T.eb;
      for (int i = lane; i < op.N; i += 32) T.mbraw[i] = __double2ll_rn(fx_scale2(S.bsite[i] * g, -eb));
    }
  }
  __syncwarp();
}

// Constants of the term  y = g H_j v - g b v - use_prev * v_prev  (warp 0):
// v has measured max |mantissa| Ak at exponent Ek, v_prev Apr at Epr; y gets
// the exponent of the rigorous bound B of its terms (returned in real units),
// as in the Krylov kernel (kernels_fx.cu).  Uses the per-exponential scalars
// of cheb_exp_scalars; only shifts and folds depend on the term.
template <int FAMILY, class Op>
__device__ double cheb_term_const(SmemCheb& S, int slot, const Op& op, int use_prev, long long Ak, int Ek,
                                  long long Apr, int Epr) {
  const int lane = threadIdx.x & 31;
  FxConstA& c = S.c;
  const SmemCheb::TermScalars& T = S.ts[slot];
  double B = 0.0;
  if (lane == 0) {
    const double A = (double)Ak;
    const double Akr = fx_scale2(A, Ek);
    c.pk = fx_norm_shift(A);
    B = (use_prev ? fx_scale2((double)Apr, Epr) : 0.0) + T.csum * Akr;
    const int Eu = fx_exp_for(B, kFxBits);
    c.Eu = Eu;
    if constexpr (FAMILY == kFamilySpin) {
      c.s_d = T.ED - T.mcz.e - (op.E_dz - 1) - 64;
      c.s_diag = Eu - (T.ED - 3) - (Ek - c.pk) - 64;
      c.m_cz = fx_fold(T.mcz.m, c.s_d + c.s_diag);
      c.ph = fx_norm_shift((op.N > 1 ? op.N - 1 : 1) * A);
      c.s_hop = Eu - T.mh.e - (Ek - c.ph) - 64;
      c.m_hop = fx_fold(T.mh.m, c.s_hop);
      if (op.uniform) {
        c.px = fx_norm_shift(op.N * A);
        c.s_x = Eu - T.mx.e - (Ek - c.px) - 64;
        c.m_x = fx_fold(T.mx.m, c.s_x);
      } else {
        c.s_nu = Eu - T.eb - (Ek - c.pk) - 64;
      }
    } else {
      for (int o = 0; o < op.nops; ++o) {
        const int Epre = fx_exp_for(op.maxrow[o] * Akr, 62);  // |P_o| < 2^62
        c.sh_pre[o] = Epre - op.E_op[o] - Ek;
        c.s_op[o] = Eu - T.mop[o].e - Epre - 64;
        c.m_op[o] = fx_fold(T.mop[o].m, c.s_op[o]);
      }
    }
    // -v_prev: mantissa of -1 is -2^61 at exponent -61
    c.pp = use_prev ? fx_norm_shift((double)Apr) : 0;
    c.s_p = Eu + 61 - (Epr - c.pp) - 64;
    c.m_p = use_prev ? fx_fold(-(1LL << 61), c.s_p) : 0;
    c.use_prev = use_prev;
    S.m_s = T.ms.m == 0 ? 0 : fx_fold(T.ms.m, Eu - T.ms.e - (Ek - c.pk) - 64);
  }
  if constexpr (FAMILY == kFamilySpin) {
    if (!op.uniform) {
      __syncwarp();
      const int s_nu = c.s_nu;
      for (int i = lane; i < op.N; i += 32) S.mb[i] = fx_fold(T.mbraw[i], s_nu);
    }
  }
  __syncwarp();
  return __shfl_sync(0xffffffffu, B, 0);
}

// fx_mulhi(fold(mant(r)), x << p) = r * x * 2^(Ex - Eout) for x at exponent Ex
// (|x| normalised by p), result at exponent Eout.
__device__ __forceinline__ long long cheb_coef(double r, int Eout, int Ex, int p) {
  const Mant m = fx_mant(r);
  if (m.m == 0) return 0;
  return fx_fold(m.m, Eout - m.e - (Ex - p) - 64);
}

// (-i)^k (yr + i yi)
__device__ __forceinline__ void cheb_rot(int k, long long yr, long long yi, long long& zr, long long& zi) {
  switch (k & 3) {
    case 0: zr = yr; zi = yi; break;
    case 1: zr = yi; zi = -yr; break;
    case 2: zr = -yr; zi = -yi; break;
    default: zr = -yi; zi = yr; break;
  }
}

template <int FAMILY, class Op>
__device__ __forceinline__ longlong2 cheb_apply1(const longlong2* cur, const longlong2* prev, int x, int dim,
                                                 const Op& op, const FxConstA& c, const long long* mb, long long m_s) {
  longlong2 y;
  if constexpr (FAMILY == kFamilySpin) y = fx_apply_spin(cur, prev, x, op, c, mb);
  else y = fx_apply_sparse(cur, prev, x, dim, op, c);
  if (m_s != 0) {
    const longlong2 v = cur[x];
    y.x += fx_mulhi(m_s, v.x << c.pk);
    y.y += fx_mulhi(m_s, v.y << c.pk);
  }
  return y;
}

// One term over this thread's elements: y = apply (APPLY), the sum updated
// (FIRST: r_0 v_0 + r_1 (-i) y; else shifted old sum + r_k (-i)^k y) and
// either stored with y (not LAST) or converted to the next v_0 (LAST; written
// to dst, or in place for the phase-only case, and to psi at the end).
template <int FAMILY, bool FIRST, bool LAST, bool APPLY, class Op>
__device__ __forceinline__ void cheb_pass(const SmemCheb& S, const Op& op, const PropParams& p, int k,
                                          const longlong2* cur, const longlong2* prev, longlong2* dst,
                                          longlong2* acc, const longlong2* v0, int wx0, int wxe, int wstep,
                                          bool last_exp, long long& my, long long& ma) {
  const int dim = p.dim;
  // the sum and the outputs of one element, given its y
  auto elem = [&](int x, const longlong2 y) {
    long long ar, ai;
    if (FIRST) {
      const longlong2 v = v0[x];
      ar = fx_mulhi(S.m_r0, v.x << S.p0);
      ai = fx_mulhi(S.m_r0, v.y << S.p0);
    } else {
      const longlong2 a = acc[x];
      ar = fx_rshr(a.x, S.sa);
      ai = fx_rshr(a.y, S.sa);
    }
    if (APPLY) {
      long long zr, zi;
      cheb_rot(k, y.x, y.y, zr, zi);
      ar += fx_mulhi(S.m_r, zr << S.py);
      ai += fx_mulhi(S.m_r, zi << S.py);
    }
    if (!LAST) {
      dst[x] = y;
      acc[x] = make_longlong2(ar, ai);
      my = max(my, fx_absmax(y.x, y.y));
      ma = max(ma, fx_absmax(ar, ai));
    } else {
      const int L = S.L_rot;
      const long long nr = (fx_mulhi(S.m_cs, ar << 4) - fx_mulhi(S.m_sn, ai << 4)) << L;
      const long long ni = (fx_mulhi(S.m_sn, ar << 4) + fx_mulhi(S.m_cs, ai << 4)) << L;
      dst[x] = make_longlong2(nr, ni);
      my = max(my, fx_absmax(nr, ni));
      if (last_exp) {
        const double osc = fx_scale2(1.0, S.E_out);
        p.psi[x] = make_double2(__ll2double_rn(nr) * osc, __ll2double_rn(ni) * osc);
      }
    }
  };
  int x = wx0;
  for (; x < wxe; x += wstep) {
    longlong2 y = make_longlong2(0, 0);
    if (APPLY) y = cheb_apply1<FAMILY>(cur, prev, x, dim, op, S.c, S.mb, S.m_s);
    elem(x, y);
  }
}

template <int FAMILY, class Op>
__global__ void __launch_bounds__(kChebThreads, 1) k_cheb_fx(PropParams p, Op op) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemCheb& S = *reinterpret_cast<SmemCheb*>(smem_raw);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int NW = blockDim.x >> 5;
  const int dim = p.dim;
  const int G = gridDim.x;
  const int chunk = (dim + G - 1) / G;
  const int wstep = blockDim.x;
  const int wx0 = blockIdx.x * chunk + tid;
  const int wxe = min(dim, (blockIdx.x + 1) * chunk);
  const int ncoef = 1 + p.nV;
  const unsigned tag0 = (unsigned)ld_volatile_i32((const int*)&p.st->tag_base);
  unsigned gen = 0;
  int slot = 0;  // exchange slot, alternating: two uses of a slot are separated by the other
  unsigned long long* rec = reinterpret_cast<unsigned long long*>(p.partials);
  DevStatus* st = p.st;
  const bool glead = blockIdx.x == 0 && tid == 0;
  long long t_loop = 0, t_wait = 0;
  longlong2* V[3] = {p.qbasis, p.qbasis + dim, p.qbasis + 2 * (size_t)dim};
  int sA = 0, sB = 1;
  const int sC = 2;  // the sum

  // CTA maxima of |y| and |sum| -> grid maxima (exchange by warp 0); false on abort
  auto exchange_max = [&](long long my, long long ma, bool fence, unsigned long long& gy,
                          unsigned long long& ga) -> bool {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      my = max(my, __shfl_xor_sync(0xffffffffu, my, o));
      ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    }
    if (lane == 0) {
      S.wmy[warp] = (unsigned long long)my;
      S.wma[warp] = (unsigned long long)ma;
    }
    __syncthreads();
    if (warp == 0) {
      unsigned long long cy = lane < NW ? S.wmy[lane] : 0, ca = lane < NW ? S.wma[lane] : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        cy = max(cy, __shfl_xor_sync(0xffffffffu, cy, o));
        ca = max(ca, __shfl_xor_sync(0xffffffffu, ca, o));
      }
      const unsigned mine[4] = {(unsigned)cy, (unsigned)(cy >> 32), (unsigned)ca, (unsigned)(ca >> 32)};
      ChebMax2 acc;
      const bool ok = ctl_exchange<4>(rec + (size_t)slot * 4 * G, mine, tag0 + (++gen), fence, &st->status,
                                      p.timeout_ns, t_wait, acc);
      unsigned long long ty = acc.a, ta = acc.b;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ty = max(ty, __shfl_xor_sync(0xffffffffu, ty, o));
        ta = max(ta, __shfl_xor_sync(0xffffffffu, ta, o));
      }
      gy = ty;
      ga = ta;
      if (lane == 0 && !ok) S.abort_flag = 1;
    } else {
      ++gen;
    }
    slot ^= 1;
    return true;
  };

  // ---------------- psi: NaN check and max |psi| -> E_0; convert to v_0
  {
    if (tid == 0) {
      S.abort_flag = 0;
      S.t_const = 0;
      S.t_pass = 0;
    }
    unsigned long long mx = 0;
    for (int x = wx0; x < wxe; x += wstep) {
      const double2 v = p.psi[x];
      const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFULL;
      const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFULL;
      mx = max(mx, max(a, b));
    }
    unsigned long long gm = 0, unused = 0;
    exchange_max((long long)mx, 0, false, gm, unused);
    if (warp == 0 && lane == 0 && !S.abort_flag) {
      if (gm >= 0x7FF0000000000000ULL) {
        atomicCAS(&st->status, 0, (int)CFET_ENAN);
        S.abort_flag = 1;
      } else {
        S.Ev[sA] = fx_exp_for(__longlong_as_double((long long)gm), kFxBits);
      }
    }
    __syncthreads();
    if (S.abort_flag) return;
    const double sc = fx_scale2(1.0, -S.Ev[sA]);
    long long my = 0;
    for (int x = wx0; x < wxe; x += wstep) {
      const double2 v = p.psi[x];
      const longlong2 q = make_longlong2(__double2ll_rn(v.x * sc), __double2ll_rn(v.y * sc));
      V[sA][x] = q;
      my = max(my, fx_absmax(q.x, q.y));
    }
    unsigned long long gy = 0;
    exchange_max(my, 0, true, gy, unused);
    if (warp == 0 && lane == 0) S.Av[sA] = (long long)gy;
    __syncthreads();
    if (S.abort_flag) return;
  }

  long long n_app = 0;
  int max_k = 0;
  double max_tail = 0.0;
  for (long long e = 0; e < p.nexp; ++e) {
    const long long eg = p.exp_base + e;
    const double* R = p.cheb + eg * kChebRec;
    const int K = (int)R[2];
    const double* rk = p.cheb_coef + (long long)R[3];
    const bool last_exp = e == p.nexp - 1;
    if (tid < ncoef) S.scal[tid] = p.scal[e * ncoef + tid];
    __syncthreads();
    if constexpr (FAMILY == kFamilySpin) {
      if (warp == 0) {  // per-site transverse fields of this stage
        double bi = 0.0;
        if (lane < op.N) {
          for (int k = 0; k < p.nV; ++k) bi = fma(S.scal[1 + k], __ldg(op.xf + k * op.N + lane), bi);
          S.bsite[lane] = bi;
        }
        double bs = fabs(bi), bm = fabs(bi);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          bs += __shfl_xor_sync(0xffffffffu, bs, o);
          bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
        }
        if (lane == 0) {
          S.bsum = bs;
          S.bmax = bm;
        }
        __syncwarp();
      }
    }
    if (warp == 0 && K >= 1) {
      cheb_exp_scalars<FAMILY>(S, 0, op, R[0], R[1]);
      if (K >= 2) cheb_exp_scalars<FAMILY>(S, 1, op, 2.0 * R[0], 2.0 * R[1]);
    }
    const long long t0 = sm_clock();
    for (int k = (K == 0 ? 0 : 1); k <= K; ++k) {
      const bool last = k == K;
      const bool first = k <= 1;
      // v_{k-1} is in (k-1 even ? sA : sB), v_{k-2} in the other; y = v_k goes to v_{k-2}'s slot
      const int scur = ((k - 1) & 1) ? sB : sA;
      const int sdst = ((k - 1) & 1) ? sA : sB;
      // ---- constants of this term (warp 0)
      if (warp == 0) {
        const long long tc0 = sm_clock();
        double By = 0.0;  // bound of |y| (real units)
        if (k >= 1)
          By = cheb_term_const<FAMILY>(S, first ? 0 : 1, op, first ? 0 : 1, S.Av[scur], S.Ev[scur],
                                       first ? 0 : S.Av[sdst], first ? 0 : S.Ev[sdst]);
        if (lane == 0) {
          const int Ey = S.c.Eu;
          S.py = fx_norm_shift(k >= 1 ? fx_scale2(By, -Ey) : 0.0);
          // the sum: old part (measured) plus this term's bound
          double Bacc;
          int Eacc;
          if (first) {
            const double A0r = fx_scale2((double)S.Av[sA], S.Ev[sA]);
            Bacc = fabs(rk[0]) * A0r + (k >= 1 ? fabs(rk[1]) * By : 0.0);
            Eacc = fx_exp_for(Bacc, kFxBits);
            S.sa = 0;
            S.p0 = fx_norm_shift((double)S.Av[sA]);
            S.m_r0 = cheb_coef(rk[0], Eacc, S.Ev[sA], S.p0);
          } else {
            Bacc = fx_scale2((double)S.accmax, S.E_acc) + fabs(rk[k]) * By;
            Eacc = max(S.E_acc, fx_exp_for(Bacc, kFxBits));
            S.sa = Eacc - S.E_acc;
          }
          S.m_r = k >= 1 ? cheb_coef(rk[k], Eacc, Ey, S.py) : 0;
          S.E_acc = Eacc;
          if (last) {
            // v_0 of the next exponential: (cos - i sin) sum, |component| <= sqrt(2) Bacc
            const int E0 = fx_exp_for(1.4142135623730951 * Bacc * (1.0 + 1e-12), kFxBits);
            S.E_out = E0;
            const Mant mc = fx_mant(R[5]), ms = fx_mant(R[6]);
            // fx_mulhi(m, sum << 4) << L = value at E0
            const int sc_ = mc.m ? E0 - mc.e - (Eacc - 4) - 64 : 1 << 20;
            const int ss_ = ms.m ? E0 - ms.e - (Eacc - 4) - 64 : 1 << 20;
            int L = 0;
            if (-sc_ > L) L = -sc_;
            if (-ss_ > L) L = -ss_;
            S.L_rot = L;
            S.m_cs = mc.m ? fx_fold(mc.m, sc_ + L) : 0;
            S.m_sn = ms.m ? fx_fold(ms.m, ss_ + L) : 0;
          } else {
            S.E_out = Ey;
          }
          S.t_const += sm_clock() - tc0;
        }
      }
      __syncthreads();
      const long long tp0 = sm_clock();
      long long my = 0, ma = 0;
      {
        const longlong2* cur = V[scur];
        longlong2* dst = V[sdst];
        const longlong2* prev = k >= 2 ? dst : cur;
        if (k == 0)
          cheb_pass<FAMILY, true, true, false>(S, op, p, 0, V[sA], V[sA], V[sA], V[sC], V[sA], wx0, wxe, wstep,
                                               last_exp, my, ma);
        else if (first && last)
          cheb_pass<FAMILY, true, true, true>(S, op, p, k, cur, prev, dst, V[sC], V[sA], wx0, wxe, wstep, last_exp,
                                              my, ma);
        else if (first)
          cheb_pass<FAMILY, true, false, true>(S, op, p, k, cur, prev, dst, V[sC], V[sA], wx0, wxe, wstep, last_exp,
                                               my, ma);
        else if (last)
          cheb_pass<FAMILY, false, true, true>(S, op, p, k, cur, prev, dst, V[sC], V[sA], wx0, wxe, wstep, last_exp,
                                               my, ma);
        else
          cheb_pass<FAMILY, false, false, true>(S, op, p, k, cur, prev, dst, V[sC], V[sA], wx0, wxe, wstep,
                                                last_exp, my, ma);
      }
      if (tid == 0) S.t_pass += sm_clock() - tp0;
      if (last && last_exp) break;
      unsigned long long gy = 0, ga = 0;
      exchange_max(my, ma, true, gy, ga);
      if (warp == 0 && lane == 0) {
        const int sw = (k == 0) ? sA : sdst;
        S.Ev[sw] = S.E_out;
        S.Av[sw] = (long long)gy;
        S.accmax = (long long)ga;
        if (gy >= (1ULL << 60)) {  // fixed-point range exceeded (not expected)
          atomicCAS(&st->status, 0, (int)CFET_ENAN);
          S.abort_flag = 1;
        }
      }
      __syncthreads();
      if (S.abort_flag) return;
    }
    if (tid == 0) t_loop += sm_clock() - t0;
    // the new v_0 is where the last term wrote
    if (K >= 1 && (K - 1) % 2 == 0) {
      const int t = sA;
      sA = sB;
      sB = t;
    }
    n_app += K;
    max_k = K > max_k ? K : max_k;
    max_tail = R[7] > max_tail ? R[7] : max_tail;
  }
  if (glead) {
    st->tag_base = tag0 + gen;
    st->n_exp += p.nexp;
    st->n_sub += p.nexp;
    st->n_app += n_app;
    if (max_k > st->max_k) st->max_k = max_k;
    if (max_tail > st->max_err) st->max_err = max_tail;
  }
  if (tid == 0) {  // trace: [0] term loops, [1] term constants, [2] element passes, [5] exchange waits
    const long long v[4] = {t_loop, S.t_const, S.t_pass, t_wait};
    const int slot_of[4] = {0, 1, 2, 5};
    for (int j = 0; j < 4; ++j) {
      atomicAdd((unsigned long long*)&st->phase_ns[slot_of[j]], (unsigned long long)(v[j] / G));
      atomicMax(&st->phase_max_ns[slot_of[j]], v[j]);
    }
  }
}

// ------------------------------------------------------------------ launchers
template <int FAMILY, class Op>
static int launch_cheb(const PropParams& p, const Op& op, int grid, int block, void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = sizeof(SmemCheb);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_cheb_fx<FAMILY, Op>, p, op);
}

int launch_cheb_spin_fx(const PropParams& p, const OpSpinFx& op, int grid, int block, void* stream) {
  return launch_cheb<kFamilySpin>(p, op, grid, block, stream);
}
int launch_cheb_dia_fx(const PropParams& p, const OpDiaFx& op, int grid, int block, void* stream) {
  return launch_cheb<kFamilyDia>(p, op, grid, block, stream);
}
int launch_cheb_csr_fx(const PropParams& p, const OpCsrFx& op, int grid, int block, void* stream) {
  return launch_cheb<kFamilyCsr>(p, op, grid, block, stream);
}

int cheb_threads(int workers) { return workers < kChebThreads ? workers : kChebThreads; }

int max_coresident_blocks_cheb(int family, int block) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(k_cheb_fx<kFamilySpin, OpSpinFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_cheb_fx<kFamilyDia, OpDiaFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_cheb_fx<kFamilyCsr, OpCsrFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaError_t e;
  if (family == kFamilySpin)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cheb_fx<kFamilySpin, OpSpinFx>, block,
                                                      sizeof(SmemCheb));
  else if (family == kFamilyCsr)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cheb_fx<kFamilyCsr, OpCsrFx>, block,
                                                      sizeof(SmemCheb));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cheb_fx<kFamilyDia, OpDiaFx>, block,
                                                      sizeof(SmemCheb));
  if (e != cudaSuccess) return -1;
  return per * nsm;
}

}  // namespace cfet
