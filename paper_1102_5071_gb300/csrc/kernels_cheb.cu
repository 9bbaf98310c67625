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

constexpr int kChebThreads = 768;   // launch bound of the kernel
constexpr double kChebA = 4503599627370496.0;  // 2^52: bound of every stored |v_k| mantissa

struct SmemCheb {
  FxConstA c[2];                  // term 1 (Htilde, no v_{k-1}) and terms k >= 2 (2 Htilde, -v_{k-1})
  long long mb[2][kMaxSites];     // per-site field tables of both (non-uniform fields)
  long long m_s[2];               // shift terms -b/a v and -2b/a v
  double scal[1 + kMaxDrives];
  double bsite[kMaxSites];
  double bsum, bmax;
  // accumulation and rotation
  long long m_cs, m_sn;           // cos(tau b), -sin(tau b) at the conversion of the sum to v_0
  int ea, L_rot, K;
  int E;
  // reductions of the initial pass
  double wsum[32];
  unsigned long long wmax[32];
  int abort_flag;
};

// Exchange accumulators (records of 4, 2 or 1 words).
struct ChebSumMax {
  double s;
  unsigned long long m;
  __device__ void reset() { s = 0.0; m = 0; }
  __device__ void add(const unsigned (&v)[4]) {
    s += __longlong_as_double((long long)(((unsigned long long)v[1] << 32) | v[0]));
    const unsigned long long x = ((unsigned long long)v[3] << 32) | v[2];
    m = x > m ? x : m;
  }
};
struct ChebMax {
  unsigned long long m;
  __device__ void reset() { m = 0; }
  __device__ void add(const unsigned (&v)[2]) {
    const unsigned long long x = ((unsigned long long)v[1] << 32) | v[0];
    m = x > m ? x : m;
  }
};
struct ChebNone {
  __device__ void reset() {}
  __device__ void add(const unsigned (&)[1]) {}
};

// Fixed-point constants of  y = g H_j v - g b v - use_prev v_prev  with v,
// v_prev mantissas below 2^52 at exponent E and y at exponent E (scalar part on
// lane 0 of warp 0, per-site table over the lanes).  Returns false when the
// term bound does not fit the format at exponent E (not expected: the
// Gershgorin interval bounds every row).
template <int FAMILY, class Op>
__device__ bool cheb_const(SmemCheb& S, int slot, const Op& op, double g, double gb, int use_prev, int E) {
  const int lane = threadIdx.x & 31;
  FxConstA& c = S.c[slot];
  int ok = 1;
  if (lane == 0) {
    const double Ak = kChebA;
    const double Akr = fx_scale2(Ak, E);
    c.pk = fx_norm_shift(Ak);
    double B = (use_prev ? Akr : 0.0) + fabs(gb) * Akr;
    if constexpr (FAMILY == kFamilySpin) {
      const double cz = S.scal[0] * g;
      const double ch = cz * op.J2;
      B += (fabs(cz) * op.maxdz + fabs(ch) * (op.N - 1) + fabs(g) * S.bsum) * Akr;
    } else {
      for (int o = 0; o < op.nops; ++o) B += fabs(S.scal[o] * g) * op.maxrow[o] * Akr;
    }
    if (fx_exp_for(B, kFxBits) > E) ok = 0;
    const int Eu = E;
    if constexpr (FAMILY == kFamilySpin) {
      const double cz = S.scal[0] * g;
      const double ch = cz * op.J2;
      const Mant mcz = fx_mant(cz);
      const int ED = fx_exp_for(fabs(cz) * op.maxdz, 59);
      c.s_d = ED - mcz.e - (op.E_dz - 1) - 64;
      c.s_diag = Eu - (ED - 3) - (E - c.pk) - 64;
      c.m_cz = fx_fold(mcz.m, c.s_d + c.s_diag);
      const Mant mh = fx_mant(ch);
      c.ph = fx_norm_shift((op.N > 1 ? op.N - 1 : 1) * Ak);
      c.s_hop = Eu - mh.e - (E - c.ph) - 64;
      c.m_hop = fx_fold(mh.m, c.s_hop);
      if (op.uniform) {
        const Mant mx = fx_mant(S.bsite[0] * g);
        c.px = fx_norm_shift(op.N * Ak);
        c.s_x = Eu - mx.e - (E - c.px) - 64;
        c.m_x = fx_fold(mx.m, c.s_x);
      } else {
        const int eb = fx_exp_for(fabs(g) * S.bmax, 62);
        c.s_nu = Eu - eb - (E - c.pk) - 64;
        c.Eu = eb;  // carried to the lanes below
      }
    } else {
      for (int o = 0; o < op.nops; ++o) {
        const int Epre = fx_exp_for(op.maxrow[o] * Akr, 62);  // |P_o| < 2^62
        c.sh_pre[o] = Epre - op.E_op[o] - E;
        const Mant m = fx_mant(S.scal[o] * g);
        c.s_op[o] = Eu - m.e - Epre - 64;
        c.m_op[o] = fx_fold(m.m, c.s_op[o]);
      }
    }
    const Mant mp = fx_mant(-1.0);
    c.pp = c.pk;
    c.s_p = Eu - mp.e - (E - c.pp) - 64;
    c.m_p = fx_fold(mp.m, c.s_p);
    c.use_prev = use_prev;
    const Mant ms = fx_mant(-gb);
    S.m_s[slot] = ms.m == 0 ? 0 : fx_fold(ms.m, Eu - ms.e - (E - c.pk) - 64);
  }
  __syncwarp();
  if constexpr (FAMILY == kFamilySpin) {
    if (!op.uniform) {
      const int eb = c.Eu;
      for (int i = lane; i < op.N; i += 32)
        S.mb[slot][i] = fx_fold(__double2ll_rn(fx_scale2(S.bsite[i] * g, -eb)), c.s_nu);
    }
  }
  __syncwarp();
  c.Eu = E;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// acc-term constant: r * y (y mantissa < 2^52 at E) at exponent E + ea.
__device__ __forceinline__ long long cheb_rk(double r, int ea, int py) {
  const Mant m = fx_mant(r);
  if (m.m == 0) return 0;
  return fx_fold(m.m, ea - m.e - (-py) - 64);
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

// One element of a term: y = (apply) + shift; returns y.
template <int FAMILY, class Op>
__device__ __forceinline__ longlong2 cheb_apply1(const longlong2* cur, const longlong2* prev, int x, int dim,
                                                 const Op& op, const FxConstA& c, const long long* mb, long long m_s) {
  longlong2 y;
  if constexpr (FAMILY == kFamilySpin) y = fx_apply_spin(cur, prev, x, op, c, mb);
  else y = fx_apply_dia(cur, prev, x, dim, op, c);
  if (m_s != 0) {
    const longlong2 v = cur[x];
    y.x += fx_mulhi(m_s, v.x << c.pk);
    y.y += fx_mulhi(m_s, v.y << c.pk);
  }
  return y;
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
  // vectors: three slots of the fixed-point workspace
  longlong2* V[3] = {p.qbasis, p.qbasis + dim, p.qbasis + 2 * (size_t)dim};
  int sA = 0, sB = 1;
  const int sC = 2;  // the sum

  // exchange by warp 0 after all element work of the CTA; every thread learns
  // the outcome from S.abort_flag
  auto exchange1 = [&](bool fence) -> bool {
    __syncthreads();
    if (warp == 0) {
      const unsigned mine[1] = {0u};
      ChebNone acc;
      const bool ok = ctl_exchange<1>(rec + (size_t)slot * 4 * G, mine, tag0 + (++gen), fence, &st->status,
                                      p.timeout_ns, t_wait, acc);
      if (lane == 0 && !ok) S.abort_flag = 1;
    } else {
      ++gen;
    }
    slot ^= 1;
    __syncthreads();
    return S.abort_flag == 0;
  };

  // ---------------- psi: NaN check and ||psi||^2 -> E; convert to v_0
  {
    if (tid == 0) S.abort_flag = 0;
    double s2 = 0.0;
    unsigned long long mx = 0;
    for (int x = wx0; x < wxe; x += wstep) {
      const double2 v = p.psi[x];
      const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFULL;
      const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFULL;
      mx = max(mx, max(a, b));
      s2 = fma(v.x, v.x, fma(v.y, v.y, s2));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = m2 > mx ? m2 : mx;
    }
    if (lane == 0) {
      S.wsum[warp] = s2;
      S.wmax[warp] = mx;
    }
    __syncthreads();
    if (warp == 0) {
      double cs = lane < NW ? S.wsum[lane] : 0.0;
      unsigned long long cm = lane < NW ? S.wmax[lane] : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        cs += __shfl_xor_sync(0xffffffffu, cs, o);
        const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, cm, o);
        cm = m2 > cm ? m2 : cm;
      }
      const unsigned long long cb = (unsigned long long)__double_as_longlong(cs);
      const unsigned mine[4] = {(unsigned)cb, (unsigned)(cb >> 32), (unsigned)cm, (unsigned)(cm >> 32)};
      ChebSumMax acc;
      const bool ok = ctl_exchange<4>(rec + (size_t)slot * 4 * G, mine, tag0 + (++gen), false, &st->status,
                                      p.timeout_ns, t_wait, acc);
      double ts = acc.s;
      unsigned long long tm = acc.m;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ts += __shfl_xor_sync(0xffffffffu, ts, o);
        const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, tm, o);
        tm = m2 > tm ? m2 : tm;
      }
      if (lane == 0) {
        if (!ok) {
          S.abort_flag = 1;
        } else if (tm >= 0x7FF0000000000000ULL || !(ts < 1e300)) {
          atomicCAS(&st->status, 0, (int)CFET_ENAN);
          S.abort_flag = 1;
        } else {
          S.E = fx_exp_for(32.0 * sqrt(ts), kFxBits);
        }
      }
    } else {
      ++gen;
    }
    slot ^= 1;
    __syncthreads();
    if (S.abort_flag) return;
    const double sc = fx_scale2(1.0, -S.E);
    for (int x = wx0; x < wxe; x += wstep) {
      const double2 v = p.psi[x];
      V[sA][x] = make_longlong2(__double2ll_rn(v.x * sc), __double2ll_rn(v.y * sc));
    }
    if (!exchange1(true)) return;
  }
  const int E = S.E;

  long long n_app = 0;
  int max_k = 0;
  double max_tail = 0.0;
  for (long long e = 0; e < p.nexp; ++e) {
    const long long eg = p.exp_base + e;
    const double* R = p.cheb + eg * kChebRec;
    const int K = (int)R[2];
    const double* rk = p.cheb_coef + (long long)R[3];
    const bool last_exp = e == p.nexp - 1;
    // ---- constants of this exponential (warp 0)
    if (tid < ncoef) S.scal[tid] = p.scal[e * ncoef + tid];
    __syncthreads();
    if (warp == 0) {
      if constexpr (FAMILY == kFamilySpin) {
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
      const double g1 = R[0], ba = R[1];
      bool ok = cheb_const<FAMILY>(S, 0, op, g1, ba, 0, E);
      ok = cheb_const<FAMILY>(S, 1, op, 2.0 * g1, 2.0 * ba, 1, E) && ok;
      if (lane == 0) {
        // the sum lives at exponent E + ea with |mantissa| < 2^57
        const int ea = fx_exp_for(R[4] * kChebA, kFxBits);
        S.ea = ea;
        S.K = K;
        // conversion v_0 = rot(sum) * 2^ea: products fx_mulhi(m, sum << 4) << L_rot
        const Mant mc = fx_mant(R[5]), ms = fx_mant(R[6]);
        int sc_ = mc.m ? -ea - mc.e - 60 : 1 << 20, ss_ = ms.m ? -ea - ms.e - 60 : 1 << 20;
        int L = 0;
        if (-sc_ > L) L = -sc_;
        if (-ss_ > L) L = -ss_;
        S.L_rot = L;
        S.m_cs = mc.m ? fx_fold(mc.m, sc_ + L) : 0;
        S.m_sn = ms.m ? fx_fold(ms.m, ss_ + L) : 0;
        if (!ok) {
          atomicCAS(&st->status, 0, (int)CFET_EINVAL);
          S.abort_flag = 1;
        }
      }
    }
    __syncthreads();
    if (S.abort_flag) return;
    const int ea = S.ea, L_rot = S.L_rot;
    const long long m_cs = S.m_cs, m_sn = S.m_sn;
    const long long t0 = sm_clock();
    // ---- terms k = 1..K (K = 0: the phase only)
    for (int k = (K == 0 ? 0 : 1); k <= K; ++k) {
      const bool last = k == K;
      const bool first = k <= 1;
      const FxConstA& c = S.c[first ? 0 : 1];
      const long long* mb = S.mb[first ? 0 : 1];
      const long long m_s = S.m_s[first ? 0 : 1];
      // v_{k-1} is in (k-1 even ? sA : sB), v_{k-2} in the other; y = v_k goes to v_{k-2}'s slot
      const longlong2* cur = V[((k - 1) & 1) ? sB : sA];
      longlong2* dst = V[((k - 1) & 1) ? sA : sB];
      const longlong2* prev = k >= 2 ? dst : cur;
      longlong2* acc = V[sC];
      const long long mr = cheb_rk(k == 0 ? 0.0 : __ldg(rk + k), ea, fx_norm_shift(kChebA));
      const long long m0 = cheb_rk(__ldg(rk), ea, fx_norm_shift(kChebA));
      const int py = fx_norm_shift(kChebA);
      for (int x = wx0; x < wxe; x += wstep) {
        long long ar, ai;
        if (k == 0) {
          const longlong2 v = V[sA][x];
          ar = fx_mulhi(m0, v.x << py);
          ai = fx_mulhi(m0, v.y << py);
        } else {
          const longlong2 y = cheb_apply1<FAMILY>(cur, prev, x, dim, op, c, mb, m_s);
          long long zr, zi;
          cheb_rot(k, y.x, y.y, zr, zi);
          if (first) {
            const longlong2 v = cur[x];
            ar = fx_mulhi(m0, v.x << py);
            ai = fx_mulhi(m0, v.y << py);
          } else {
            const longlong2 a = acc[x];
            ar = a.x;
            ai = a.y;
          }
          ar += fx_mulhi(mr, zr << py);
          ai += fx_mulhi(mr, zi << py);
          if (!last) {
            dst[x] = y;
            acc[x] = make_longlong2(ar, ai);
          }
        }
        if (last) {
          // v_0 of the next exponential: (cos - i sin)(ar + i ai) 2^ea at exponent E
          const long long nr = (fx_mulhi(m_cs, ar << 4) - fx_mulhi(m_sn, ai << 4)) << L_rot;
          const long long ni = (fx_mulhi(m_sn, ar << 4) + fx_mulhi(m_cs, ai << 4)) << L_rot;
          if (k == 0) V[sA][x] = make_longlong2(nr, ni);
          else dst[x] = make_longlong2(nr, ni);
          if (last_exp) {
            const double osc = fx_scale2(1.0, E);
            p.psi[x] = make_double2(__ll2double_rn(nr) * osc, __ll2double_rn(ni) * osc);
          }
        }
      }
      if (!(last && last_exp)) {
        if (!exchange1(true)) return;
      }
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
  if (tid == 0) {
    atomicAdd((unsigned long long*)&st->phase_ns[0], (unsigned long long)(t_loop / G));
    atomicMax(&st->phase_max_ns[0], t_loop);
    atomicAdd((unsigned long long*)&st->phase_ns[5], (unsigned long long)(t_wait / G));
    atomicMax(&st->phase_max_ns[5], t_wait);
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

int max_coresident_blocks_cheb(int family, int block) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(k_cheb_fx<kFamilySpin, OpSpinFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_cheb_fx<kFamilyDia, OpDiaFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaError_t e;
  if (family == kFamilySpin)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cheb_fx<kFamilySpin, OpSpinFx>, block,
                                                      sizeof(SmemCheb));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cheb_fx<kFamilyDia, OpDiaFx>, block,
                                                      sizeof(SmemCheb));
  if (e != cudaSuccess) return -1;
  return per * nsm;
}

}  // namespace cfet
