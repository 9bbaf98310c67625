// Mixed-precision persistent Lanczos kernel (sm_103a): complex64 Krylov
// vectors, FP64-class reductions and FP64 scalar work.
//
// Same method and decisions as k_propagate (kernels.cu) and k_propagate_fx
// (kernels_fx.cu): the stage exponential exp(-i tau H_j) psi of a CFET step
// (Alvermann & Fehske, arXiv:1102.5071, Sec. 4 Eq. (Ucf), Sec. 7
// Eq. (OmGLeg)) by the Lanczos / Krylov method of Sec. 8.1 with the
// a-posteriori estimate, adaptive Krylov dimension and substepping.
//
// Number format.  The Krylov vectors q_i are complex64 (8 B per element, half
// the bytes of complex128) and the operator apply, the three-term recurrence
// and the reconstruction run in FP32 (the GB300 FP32 rate is 64x its FP64
// rate).  Everything that decides the method stays FP64-class:
//   * alpha_k, ||w||^2 and ||psi||^2 are compensated FP32 dot products per
//     thread (error-free product by FMA and error-free sum, i.e. the Dot2
//     scheme of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005),
//     combined as float-float pairs over the warp and in FP64 over the CTA
//     and the grid, in one fixed order (every CTA holds bit-identical sums);
//   * the stage and Lanczos scalars, the tridiagonal exponential, the error
//     estimate and all decisions are FP64-class on the control warp (taken in
//     FP32 or integers only where scalar_bounds.cuh shows the FP64 decision
//     for certain);
//   * psi enters and leaves as complex128; in between it is held as q_1.
// The result differs from the FP64 method by FP32 rounding of the vectors
// (relative 2^-24 per element and operation), not by the Krylov decisions.
//
// Work split: NW worker warps do element work only; one control warp does
// the reductions, the bounded grid barrier, the per-pass scalars and the
// small exponential (the estimate of iteration k runs while the workers
// already apply H for iteration k+1, as in the fixed-point kernel).
//
// Long chains: the TILED instantiation applies H in window passes over
// shared-memory tiles moved by TMA (tiled_common.cuh) instead of element by
// element; its window 0 also does the previous iteration's orthogonalisation
// step, so it has one grid exchange per iteration less.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cfet_internal.h"
#include "device_common.cuh"
#include "tiled_common.cuh"

namespace cfet {

// ------------------------------------------------------------------ compensated sums
// (s, c): running sum s and accumulated rounding errors c.  The _rn
// intrinsics keep the compiler from contracting the error-free steps.
__device__ __forceinline__ void ff_two_sum(float& s, float& c, float p) {
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, e);
}
__device__ __forceinline__ void ff_add_prod(float& s, float& c, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);  // a b = p + e exactly
  ff_two_sum(s, c, p);
  c = __fadd_rn(c, e);
}
// Warp sum of (s, c) pairs (lane 0 result).
__device__ __forceinline__ void ff_warp_sum(float& s, float& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, s, o);
    const float c2 = __shfl_down_sync(0xffffffffu, c, o);
    ff_two_sum(s, c, s2);
    c = __fadd_rn(c, c2);
  }
}

// ------------------------------------------------------------------ shared state
struct CConst {
  // phase A: u = s_k H_j q_k - beta_{k-1} s_{k-1} q_{k-1}
  float cz, ch, cx, cp;          // spin: c0 s_k, 2 J c0 s_k, uniform field s_k, -beta s_{k-1}
  float co[1 + kMaxDrives];      // dia: c_o s_k per operator
  int use_prev;
};

struct SmemC {
  float ws[3][32], wc[3][32];    // per-warp compensated partials of the workers (up to 3 sums)
  double alpha[kMaxKrylov + 2];
  double beta[kMaxKrylov + 2];
  double scale[kMaxKrylov + 3];  // 1 / ||q_i||
  double yr[kMaxKrylov], yi[kMaxKrylov];
  double tr[kMaxKrylov], ti[kMaxKrylov];
  float cr[kMaxKrylov], ci[kMaxKrylov];  // reconstruction coefficients
  double scal[1 + kMaxDrives];
  double bsite_raw[kMaxSites];
  float bx[kMaxSites];           // non-uniform fields: b_i s_k
  CConst ca;
  float am;                      // phase B: -alpha_k s_k
  double wnorm2;                 // ||w||^2 of the current iteration (from the phase-A sums)
  double qnorm2[kMaxKrylov + 3]; // ||q_i||^2 of the stored vectors (reduced after they are written)
  int abort_flag, stop_prev, accept_now, pend, y_ready, acc_h;
  int tma_fail;                  // tiled apply: a tile wait gave up
  double err_now, err_prev;
  double beta0;
  LeadAcc lead;                  // running FP32 bounds of the current T_k for the estimate's screens
  GershAcc gfull;                // rows whose couplings are all known
};

// ------------------------------------------------------------------ applies
__device__ __forceinline__ float2 c_apply_spin(const float2* __restrict__ q, const float2* __restrict__ qm, int x,
                                               const OpSpinC& op, const CConst& c, const float* bx) {
  const int N = op.N, L = op.lo_bits;
  const float dz = __ldg(op.dz_lo + (x & ((1 << L) - 1))) + __ldg(op.dz_hi + (x >> (L - 1)));
  const float d = c.cz * dz;
  const float2 v = q[x];
  float ur = d * v.x, ui = d * v.y;
  float hr = 0.f, hi = 0.f;
  const unsigned anti = ((unsigned)x ^ ((unsigned)x >> 1)) & ((1u << (N - 1)) - 1u);
#pragma unroll 4
  for (int i = 0; i < N - 1; ++i) {  // antiparallel bonds only (predicated)
    if ((anti >> i) & 1u) {
      const float2 w = q[x ^ (3 << i)];
      hr += w.x;
      hi += w.y;
    }
  }
  ur = fmaf(c.ch, hr, ur);
  ui = fmaf(c.ch, hi, ui);
  if (op.uniform) {
    float xr = 0.f, xi = 0.f;
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const float2 w = q[x ^ (1 << i)];
      xr += w.x;
      xi += w.y;
    }
    ur = fmaf(c.cx, xr, ur);
    ui = fmaf(c.cx, xi, ui);
  } else {
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const float2 w = q[x ^ (1 << i)];
      ur = fmaf(bx[i], w.x, ur);
      ui = fmaf(bx[i], w.y, ui);
    }
  }
  if (c.use_prev) {
    const float2 w = qm[x];
    ur = fmaf(c.cp, w.x, ur);
    ui = fmaf(c.cp, w.y, ui);
  }
  return make_float2(ur, ui);
}

// Two elements x and x2 per call: the neighbour loads of both are issued in
// the same loop iterations (twice the independent requests per warp).
__device__ __forceinline__ void c_apply_spin2(const float2* __restrict__ q, const float2* __restrict__ qm, int x,
                                              int x2, const OpSpinC& op, const CConst& c, const float* bx,
                                              float2& r1, float2& r2) {
  const int N = op.N, L = op.lo_bits;
  const float d1 = c.cz * (__ldg(op.dz_lo + (x & ((1 << L) - 1))) + __ldg(op.dz_hi + (x >> (L - 1))));
  const float d2 = c.cz * (__ldg(op.dz_lo + (x2 & ((1 << L) - 1))) + __ldg(op.dz_hi + (x2 >> (L - 1))));
  const float2 v1 = q[x], v2 = q[x2];
  float ur1 = d1 * v1.x, ui1 = d1 * v1.y, ur2 = d2 * v2.x, ui2 = d2 * v2.y;
  float hr1 = 0.f, hi1 = 0.f, hr2 = 0.f, hi2 = 0.f;
  const unsigned mask = (1u << (N - 1)) - 1u;
  const unsigned anti1 = ((unsigned)x ^ ((unsigned)x >> 1)) & mask;
  const unsigned anti2 = ((unsigned)x2 ^ ((unsigned)x2 >> 1)) & mask;
#pragma unroll 4
  for (int i = 0; i < N - 1; ++i) {
    if ((anti1 >> i) & 1u) {
      const float2 w = q[x ^ (3 << i)];
      hr1 += w.x;
      hi1 += w.y;
    }
    if ((anti2 >> i) & 1u) {
      const float2 w = q[x2 ^ (3 << i)];
      hr2 += w.x;
      hi2 += w.y;
    }
  }
  ur1 = fmaf(c.ch, hr1, ur1);
  ui1 = fmaf(c.ch, hi1, ui1);
  ur2 = fmaf(c.ch, hr2, ur2);
  ui2 = fmaf(c.ch, hi2, ui2);
  if (op.uniform) {
    float xr1 = 0.f, xi1 = 0.f, xr2 = 0.f, xi2 = 0.f;
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const float2 w1 = q[x ^ (1 << i)];
      const float2 w2 = q[x2 ^ (1 << i)];
      xr1 += w1.x;
      xi1 += w1.y;
      xr2 += w2.x;
      xi2 += w2.y;
    }
    ur1 = fmaf(c.cx, xr1, ur1);
    ui1 = fmaf(c.cx, xi1, ui1);
    ur2 = fmaf(c.cx, xr2, ur2);
    ui2 = fmaf(c.cx, xi2, ui2);
  } else {
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const float2 w1 = q[x ^ (1 << i)];
      const float2 w2 = q[x2 ^ (1 << i)];
      ur1 = fmaf(bx[i], w1.x, ur1);
      ui1 = fmaf(bx[i], w1.y, ui1);
      ur2 = fmaf(bx[i], w2.x, ur2);
      ui2 = fmaf(bx[i], w2.y, ui2);
    }
  }
  if (c.use_prev) {
    const float2 w1 = qm[x], w2 = qm[x2];
    ur1 = fmaf(c.cp, w1.x, ur1);
    ui1 = fmaf(c.cp, w1.y, ui1);
    ur2 = fmaf(c.cp, w2.x, ur2);
    ui2 = fmaf(c.cp, w2.y, ui2);
  }
  r1 = make_float2(ur1, ui1);
  r2 = make_float2(ur2, ui2);
}

__device__ __forceinline__ float2 c_apply_dia(const float2* __restrict__ q, const float2* __restrict__ qm, int r,
                                              int dim, const OpDiaC& op, const CConst& c) {
  float ur = 0.f, ui = 0.f;
  for (int o = 0; o < op.nops; ++o) {
    float ar = 0.f, ai = 0.f;
    const int d0 = op.dfirst[o], d1 = d0 + op.dcount[o];
    for (int d = d0; d < d1; ++d) {
      const long long cidx = (long long)r + __ldg(op.off + d);
      if (cidx >= 0 && cidx < dim) {
        const float a = __ldg(op.val + (size_t)d * dim + r);
        const float2 w = q[cidx];
        ar = fmaf(a, w.x, ar);
        ai = fmaf(a, w.y, ai);
      }
    }
    ur = fmaf(c.co[o], ar, ur);
    ui = fmaf(c.co[o], ai, ui);
  }
  if (c.use_prev) {
    const float2 w = qm[r];
    ur = fmaf(c.cp, w.x, ur);
    ui = fmaf(c.cp, w.y, ui);
  }
  return make_float2(ur, ui);
}

// CSR: per operator the row's sum of val * q in FP32 (complex values of
// Hermitian operators), then the operator's scalar.
__device__ __forceinline__ float2 c_apply_csr(const float2* __restrict__ q, const float2* __restrict__ qm, int r,
                                              int dim, const OpCsrC& op, const CConst& c) {
  float ur = 0.f, ui = 0.f;
  for (int o = 0; o < op.nops; ++o) {
    const int* rp = op.rp + (size_t)o * (dim + 1);
    const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
    float ar = 0.f, ai = 0.f;
    if (op.vi) {
      for (int e = e0; e < e1; ++e) {
        const float a = __ldg(op.vr + e), b = __ldg(op.vi + e);
        const float2 w = q[__ldg(op.col + e)];
        ar = fmaf(a, w.x, fmaf(-b, w.y, ar));
        ai = fmaf(a, w.y, fmaf(b, w.x, ai));
      }
    } else {
      for (int e = e0; e < e1; ++e) {
        const float a = __ldg(op.vr + e);
        const float2 w = q[__ldg(op.col + e)];
        ar = fmaf(a, w.x, ar);
        ai = fmaf(a, w.y, ai);
      }
    }
    ur = fmaf(c.co[o], ar, ur);
    ui = fmaf(c.co[o], ai, ui);
  }
  if (c.use_prev) {
    const float2 w = qm[r];
    ur = fmaf(c.cp, w.x, ur);
    ui = fmaf(c.cp, w.y, ui);
  }
  return make_float2(ur, ui);
}

__device__ __forceinline__ float2 c_apply_sparse(const float2* __restrict__ q, const float2* __restrict__ qm, int r,
                                                 int dim, const OpDiaC& op, const CConst& c) {
  return c_apply_dia(q, qm, r, dim, op, c);
}
__device__ __forceinline__ float2 c_apply_sparse(const float2* __restrict__ q, const float2* __restrict__ qm, int r,
                                                 int dim, const OpCsrC& op, const CConst& c) {
  return c_apply_csr(q, qm, r, dim, op, c);
}

// ------------------------------------------------------------------ control warp
// Worker warps: compensated per-warp partial of sum j into shared memory.
__device__ __forceinline__ void c_worker_partial(SmemC& S, float s, float c, int j = 0) {
  ff_warp_sum(s, c);
  if ((threadIdx.x & 31) == 0) {
    S.ws[j][threadIdx.x >> 5] = s;
    S.wc[j][threadIdx.x >> 5] = c;
  }
}

// Float-float accumulation of the exchanged CTA partials (fixed order per lane).
template <int NS>
struct FFAcc {
  float s[NS], c[NS];
  __device__ void reset() {
    for (int j = 0; j < NS; ++j) s[j] = c[j] = 0.f;
  }
  __device__ void add(const unsigned (&v)[2 * NS]) {
    for (int j = 0; j < NS; ++j) {
      ff_two_sum(s[j], c[j], __uint_as_float(v[2 * j]));
      c[j] = __fadd_rn(c[j], __uint_as_float(v[2 * j + 1]));
    }
  }
};

// Control warp: publish the CTA's float-float partials of NS sums, exchange
// records with every CTA (the grid barrier), and return the global sums,
// accumulated in one fixed order and rounded to FP64 once, to all lanes.
// Keeping the chain in FP32 pairs avoids long dependent sequences on the
// 1/64-rate FP64 units.  NS = 0: a pure grid barrier.
template <int NS>
__device__ bool c_ctl_reduce(SmemC& S, int NW, unsigned long long* part, unsigned tag, bool fence, int* status,
                             long long timeout_ns, double* sum, long long& spin) {
  const int lane = threadIdx.x & 31;
  constexpr int W = NS > 0 ? 2 * NS : 1;
  unsigned mine[W];
  mine[0] = 0u;
  for (int j = 0; j < NS; ++j) {
    float s = lane < NW ? S.ws[j][lane] : 0.f, c = lane < NW ? S.wc[j][lane] : 0.f;
    ff_warp_sum(s, c);
    mine[2 * j] = __float_as_uint(__shfl_sync(0xffffffffu, s, 0));
    mine[2 * j + 1] = __float_as_uint(__shfl_sync(0xffffffffu, c, 0));
  }
  if constexpr (NS > 0) {
    FFAcc<NS> acc;
    if (!ctl_exchange<W>(part, mine, tag, fence, status, timeout_ns, spin, acc)) return false;
    for (int j = 0; j < NS; ++j) {
      float s = acc.s[j], c = acc.c[j];
      ff_warp_sum(s, c);
      sum[j] = (double)__shfl_sync(0xffffffffu, s, 0) + (double)__shfl_sync(0xffffffffu, c, 0);
    }
  } else {
    struct NoAcc {
      __device__ void reset() {}
      __device__ void add(const unsigned (&)[1]) {}
    } acc;
    if (!ctl_exchange<1>(part, mine, tag, fence, status, timeout_ns, spin, acc)) return false;
  }
  return true;
}

// Phase-A constants for iteration `it` (lane 0 scalars, per-site table over lanes).
template <int FAMILY, class Op>
__device__ void c_const_a(SmemC& S, const Op& op, int it) {
  const int lane = threadIdx.x & 31;
  const double sk = S.scale[it];
  if (lane == 0) {
    CConst& c = S.ca;
    if constexpr (FAMILY == kFamilySpin) {
      const double cz = S.scal[0] * sk;
      c.cz = (float)cz;
      c.ch = (float)(cz * op.J2);
      c.cx = (float)(S.bsite_raw[0] * sk);
    } else {
      for (int o = 0; o < op.nops; ++o) c.co[o] = (float)(S.scal[o] * sk);
    }
    c.cp = it > 1 ? (float)(-S.beta[it - 1] * S.scale[it - 1]) : 0.f;
    c.use_prev = it > 1;
  }
  if constexpr (FAMILY == kFamilySpin) {
    if (!op.uniform)
      for (int i = lane; i < op.N; i += 32) S.bx[i] = (float)(S.bsite_raw[i] * sk);
  }
}

// Error estimate of iteration k (control warp), with the FP32 screen of
// fx_estimate: above thr without the FP64 small exponential when it can.
__device__ double c_estimate(SmemC& S, int k, double ts, double thr) {
  const int dec = krylov_lead_decide(S.lead, k, ts, S.beta0, S.beta[k], thr);
  if (dec == 0) return 2.0 * thr + 1e-300;
  const double scale = S.beta0 * S.beta[k];
  if (dec < 0 && small_expm_rejects32(k, S.alpha + 1, S.beta + 1, ts, scale, thr)) return 2.0 * thr + 1e-300;
  small_expm_e1(k, S.alpha + 1, S.beta + 1, ts, S.yr, S.yi, S.tr, S.ti);
  const double yr = S.yr[k - 1], yi = S.yi[k - 1];
  return scale * sqrt(fma(yr, yr, yi * yi));
}

// ------------------------------------------------------------------ tiled apply (large chains)
// Window tiling of tiled_common.cuh with tiles of 2^12 complex64 elements
// moved by TMA.  Each of kTmaStages stages holds the q tile and the tile of
// the vector each element reads for itself (q_{k-1} in window 0, the partial
// u after it): 64 KB per stage.  One worker (the producer) keeps two tiles in
// flight ahead of the others: it arms the stage's mbarrier with the bytes of
// both loads and issues them, and once the workers have written a tile's
// results (in place over its own-element buffer) it stores that buffer with a
// bulk tensor store.  The loop touches global memory only for the diagonal
// tables; the last window also takes <q, u> and ||u||^2.
constexpr int kTileBits = kC64TileBits;
constexpr int kTileElems = 1 << kTileBits;
constexpr unsigned kTileBytes = kTileElems * sizeof(float2);

struct TmaPass {
  const unsigned char* maps;  // kTmaMapBytes per window
  unsigned long long* bar;    // [kTmaStages] in shared memory
  float2* stage;              // [kTmaStages][2][kTileElems] in shared memory
  int* fail;                  // shared flag: a wait gave up
  unsigned* phase;            // parity bits of the stages (per thread, identical in all workers)
  int* status;
  long long timeout_ns;
};

// Bounded wait for a stage's tile; false (status CFET_ETIMEOUT) when it gave up.
__device__ bool tile_wait(unsigned long long* bar, unsigned parity, int* status, long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = global_timer_ns();
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 255u) == 0u) {
      if (ld_volatile_i32(status) != 0) return false;
      if (global_timer_ns() - t0 > timeout_ns) {
        atomicCAS(status, 0, (int)CFET_ETIMEOUT);
        return false;
      }
    }
  }
  return true;
}

// One window pass of this CTA's worker threads over its tiles (vectors are
// basis indices: iq the applied q, ia the own-element input, iu the output).
// ORTH (window 0 from the second iteration on): the q tile holds u_{k-1} and
// the aux tile q_{k-1}; the pass first forms q_k = w_{k-1} = u_{k-1} + am q_{k-1}
// in place (the orthogonalisation step of iteration k-1, with ||w||^2 into
// s2/c2), applies H to it and stores both w (over u_{k-1}) and the result.
template <bool FIRST, bool LAST, bool ORTH = false>
__device__ void c_tiled_pass(const TmaPass& T, const OpSpinC& op, const CConst& c, const float* bx, int iq, int ia,
                             int iu, const TileWin& W, int w, int nworkers, float& s0, float& c0, float& s1,
                             float& c1, float am = 0.f, float* s2 = nullptr, float* c2 = nullptr) {
  static_assert(!ORTH || FIRST, "the orthogonalisation step runs in window 0");
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const int ntiles = 1 << (op.N - kTileBits);
  const bool aux = !FIRST || c.use_prev;
  const unsigned bytes = aux ? 2 * kTileBytes : kTileBytes;
  const void* map = T.maps + (size_t)w * kTmaMapBytes;
  const bool prod = tid == 0;
  auto issue = [&](int k, int t) {  // producer: tile t into stage k % kTmaStages
    const int st = k % kTmaStages;
    float2* qb = T.stage + (size_t)st * 2 * kTileElems;
    mbar_arrive_expect_tx(T.bar + st, bytes);
    tile_load(qb, map, FIRST, W, op.N, t, iq, T.bar + st);
    if (aux) tile_load(qb + kTileElems, map, FIRST, W, op.N, t, ia, T.bar + st);
  };
  if (prod) {
    fence_proxy_async_all();  // vectors written by generic stores before the exchange, read by TMA now
    for (int k = 0; k < kTmaStages - 1; ++k)
      if (blockIdx.x + k * G < ntiles) issue(k, blockIdx.x + k * G);
  }
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; ++k, t += G) {
    const int st = k % kTmaStages;
    float2* cur = T.stage + (size_t)st * 2 * kTileElems;
    float2* acur = T.stage + (size_t)st * 2 * kTileElems + kTileElems;
    const unsigned par = (*T.phase >> st) & 1u;
    *T.phase ^= 1u << st;
    if (!tile_wait(T.bar + st, par, T.status, T.timeout_ns)) *T.fail = 1;
    if constexpr (ORTH) {
      if (!*T.fail) {
        float4* w4 = reinterpret_cast<float4*>(cur);
        const float4* p4 = reinterpret_cast<const float4*>(acur);
        for (int jp = tid; jp < kTileElems / 2; jp += nworkers) {
          const float4 uu = w4[jp], qq = p4[jp];
          const float4 wv = make_float4(fmaf(am, qq.x, uu.x), fmaf(am, qq.y, uu.y), fmaf(am, qq.z, uu.z),
                                        fmaf(am, qq.w, uu.w));
          w4[jp] = wv;
          ff_add_prod(*s2, *c2, wv.x, wv.x);
          ff_add_prod(*s2, *c2, wv.y, wv.y);
          ff_add_prod(*s2, *c2, wv.z, wv.z);
          ff_add_prod(*s2, *c2, wv.w, wv.w);
        }
      }
      workers_sync(nworkers);  // every w of the tile written before its neighbours are read
    }
    if (!*T.fail) {
      // Element pairs (2 jp, 2 jp + 1) of the tile: a flip or hop of any bit
      // above bit 0 moves both elements of a pair to the two elements of
      // another pair, so each such neighbour pair is one 16-byte load; the
      // flip of bit 0 swaps the pair, and the hop of bond (0, 1) takes one
      // element of pair jp ^ 1.
      const float4* cur4 = reinterpret_cast<const float4*>(cur);
      float4* acur4 = reinterpret_cast<float4*>(acur);
      for (int jp = tid; jp < kTileElems / 2; jp += nworkers) {
        const int j = 2 * jp;
        const float4 v = cur4[jp];
        float ur0, ui0, ur1, ui1;
        float hr0 = 0.f, hi0 = 0.f, hr1 = 0.f, hi1 = 0.f, fr0 = 0.f, fi0 = 0.f, fr1 = 0.f, fi1 = 0.f;
        if (FIRST) {
          const int x = (t << kTileBits) | j;  // even
          const int L = op.lo_bits;
          const float2 dlo = *reinterpret_cast<const float2*>(op.dz_lo + (x & ((1 << L) - 1)));
          const float dhi = __ldg(op.dz_hi + (x >> (L - 1)));
          const float d0 = c.cz * (dlo.x + dhi), d1 = c.cz * (dlo.y + dhi);
          ur0 = d0 * v.x;
          ui0 = d0 * v.y;
          ur1 = d1 * v.z;
          ui1 = d1 * v.w;
          const unsigned anti = ((unsigned)j ^ ((unsigned)j >> 1)) & ((1u << (kTileBits - 1)) - 1u);
          {  // bond (0, 1): element 0 hops when bit 1 is set, element 1 when it is clear
            const float4 w = cur4[jp ^ 1];
            if ((j >> 1) & 1) {
              hr0 += w.z;
              hi0 += w.w;
            } else {
              hr1 += w.x;
              hi1 += w.y;
            }
          }
#pragma unroll
          for (int i = 1; i < kTileBits - 1; ++i)
            if ((anti >> i) & 1u) {
              const float4 w = cur4[jp ^ (3 << (i - 1))];
              hr0 += w.x;
              hi0 += w.y;
              hr1 += w.z;
              hi1 += w.w;
            }
          if (op.uniform) {
            fr0 = v.z;  // flip of bit 0
            fi0 = v.w;
            fr1 = v.x;
            fi1 = v.y;
#pragma unroll
            for (int i = 1; i < kTileBits; ++i) {
              const float4 w = cur4[jp ^ (1 << (i - 1))];
              fr0 += w.x;
              fi0 += w.y;
              fr1 += w.z;
              fi1 += w.w;
            }
          } else {
            ur0 = fmaf(bx[0], v.z, ur0);
            ui0 = fmaf(bx[0], v.w, ui0);
            ur1 = fmaf(bx[0], v.x, ur1);
            ui1 = fmaf(bx[0], v.y, ui1);
#pragma unroll
            for (int i = 1; i < kTileBits; ++i) {
              const float4 w = cur4[jp ^ (1 << (i - 1))];
              ur0 = fmaf(bx[i], w.x, ur0);
              ui0 = fmaf(bx[i], w.y, ui0);
              ur1 = fmaf(bx[i], w.z, ur1);
              ui1 = fmaf(bx[i], w.w, ui1);
            }
          }
          if (c.use_prev) {
            const float4 w = acur4[jp];
            ur0 = fmaf(c.cp, w.x, ur0);
            ui0 = fmaf(c.cp, w.y, ui0);
            ur1 = fmaf(c.cp, w.z, ur1);
            ui1 = fmaf(c.cp, w.w, ui1);
          }
        } else {
          // the window's bits are slot bits c .. c + width - 1, pair bits c - 1 ..
          const float4 a = acur4[jp];
          ur0 = a.x;
          ui0 = a.y;
          ur1 = a.z;
          ui1 = a.w;
          const unsigned jh = (unsigned)j >> W.c;  // bits b0 .. b0+width-1 of x
          const unsigned anti = (jh ^ (jh >> 1)) & ((1u << (W.width - 1)) - 1u);
          for (int i = 0; i < W.width - 1; ++i)
            if ((anti >> i) & 1u) {
              const float4 w = cur4[jp ^ (3 << (W.c - 1 + i))];
              hr0 += w.x;
              hi0 += w.y;
              hr1 += w.z;
              hi1 += w.w;
            }
          if (op.uniform) {
            for (int i = 1; i < W.width; ++i) {
              const float4 w = cur4[jp ^ (1 << (W.c - 1 + i))];
              fr0 += w.x;
              fi0 += w.y;
              fr1 += w.z;
              fi1 += w.w;
            }
          } else {
            for (int i = 1; i < W.width; ++i) {
              const float4 w = cur4[jp ^ (1 << (W.c - 1 + i))];
              const float b = bx[W.b0 + i];
              ur0 = fmaf(b, w.x, ur0);
              ui0 = fmaf(b, w.y, ui0);
              ur1 = fmaf(b, w.z, ur1);
              ui1 = fmaf(b, w.w, ui1);
            }
          }
        }
        ur0 = fmaf(c.ch, hr0, ur0);
        ui0 = fmaf(c.ch, hi0, ui0);
        ur1 = fmaf(c.ch, hr1, ur1);
        ui1 = fmaf(c.ch, hi1, ui1);
        if (op.uniform) {
          ur0 = fmaf(c.cx, fr0, ur0);
          ui0 = fmaf(c.cx, fi0, ui0);
          ur1 = fmaf(c.cx, fr1, ur1);
          ui1 = fmaf(c.cx, fi1, ui1);
        }
        acur4[jp] = make_float4(ur0, ui0, ur1, ui1);  // the own pair only: read above by this thread
        if (LAST) {
          ff_add_prod(s0, c0, v.x, ur0);
          ff_add_prod(s0, c0, v.y, ui0);
          ff_add_prod(s0, c0, v.z, ur1);
          ff_add_prod(s0, c0, v.w, ui1);
          ff_add_prod(s1, c1, ur0, ur0);
          ff_add_prod(s1, c1, ui0, ui0);
          ff_add_prod(s1, c1, ur1, ur1);
          ff_add_prod(s1, c1, ui1, ui1);
        }
      }
    }
    fence_proxy_async_smem();  // the results, written by generic stores, are read by the TMA store
    workers_sync(nworkers);
    if (*T.fail) break;
    if (prod) {
      tile_store(map, FIRST, W, op.N, t, iu, acur);
      if constexpr (ORTH) tile_store(map, FIRST, W, op.N, t, iq, cur);
      bulk_commit();
      const int tn = t + (kTmaStages - 1) * G;
      if (tn < ntiles) {
        bulk_wait_read_1();  // the stage to refill was stored from at tile k - 1
        issue(k + kTmaStages - 1, tn);
      }
    }
  }
  if (prod) {
    bulk_wait_all();         // u written before the exchange that follows
    fence_proxy_async_all();
    if (*T.fail) {           // tiles still in flight: wait for them, again with a limit
      for (int s2 = 0; s2 < kTmaStages; ++s2) {
        const unsigned par = (*T.phase >> s2) & 1u;
        tile_wait(T.bar + s2, par, T.status, T.timeout_ns);
      }
    }
  }
  workers_sync(nworkers);
}

// ------------------------------------------------------------------ the kernel
// TILED: the window-tiled apply of long spin chains (a separate instantiation,
// so that the element-wise kernel carries none of its code).
template <int FAMILY, class Op, bool TILED = false>
__global__ void __launch_bounds__(CFET_CTL_MAX_THREADS, 1) k_propagate_c64(PropParams p, Op op) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemC& S = *reinterpret_cast<SmemC*>(smem_raw);
  const int tid = threadIdx.x;
  const int NW = (int)(blockDim.x >> 5) - 1;
  const bool ctl = (tid >> 5) == NW;
  const int lane = tid & 31;
  const bool lead = ctl && lane == 0;
  const int dim = p.dim;
  const int G = gridDim.x;
  const int chunk = (dim + G - 1) / G;  // one contiguous chunk per CTA
  const int wstep = NW * 32;
  const int wx0 = blockIdx.x * chunk + tid;
  const int wxe = min(dim, (blockIdx.x + 1) * chunk);
  const int ncoef = 1 + p.nV;
  // record exchange: three slots (phase A, phase B, reconstruction) of one
  // float-float pair (two tagged words) per CTA; tags continue across launches
  const unsigned tag0 = (unsigned)ld_volatile_i32((const int*)&p.st->tag_base);
  unsigned gen = 0;
  unsigned long long* partA = reinterpret_cast<unsigned long long*>(p.partials);  // 3 sums: 6 words (stride 8)
  unsigned long long* partB = partA + 8 * G;                                        // 1 sum: 2 words
  unsigned long long* partR = partA + 16 * G;                                       // 1 sum: 2 words
  unsigned long long* partW = partA + 24 * G;  // window barriers of the tiled apply: two 1-word slots
  // tiled apply: windows and the tile buffers behind SmemC
  TileWin win[kTiledMaxWindows] = {};
  int nwin = 1;
  if constexpr (TILED) {
    nwin = tiled_windows<kTileBits>(op.N, win);
  }
  // tiled apply: the stages' mbarriers and tile buffers behind SmemC
  unsigned char* tiles_base = smem_raw + ((sizeof(SmemC) + 127) & ~size_t(127));
  unsigned tph = 0;  // parities of the stages' mbarriers (the same in every worker)
  const TmaPass TP{p.tmaps, reinterpret_cast<unsigned long long*>(tiles_base),
                   reinterpret_cast<float2*>(tiles_base + 128), &S.tma_fail, &tph, &p.st->status, p.timeout_ns};
  if constexpr (TILED) {
    if (tid == 0) {  // ordered before any use by the CTA barriers of the conversion pass
      for (int s2 = 0; s2 < kTmaStages; ++s2) mbar_init(TP.bar + s2, 1);
      S.tma_fail = 0;
      mbar_init_fence();
    }
  }
  int wslot = 0;
  DevStatus* st = p.st;
  const bool glead = (blockIdx.x == 0) && lead;
  long long tacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long twe = 0;  // thread 0: end of its last worker loop
  const bool fixed_k = p.tol <= 0.0;
  const bool forced = p.f_nsub != nullptr;
  long long fpos = st->forced_pos;
  long long rpos = st->rec_pos;
  long long n_app = 0, n_sub = 0;
  int max_k = 0;
  double max_err = 0.0;

  auto Q = [&](int i) -> float2* { return p.qbasis32 + (size_t)(i - 1) * dim; };

  // ---------------- psi (complex128) -> q_1 (complex64), ||q_1||^2, finiteness
  {
    if (!ctl) {
      float s = 0.f, c = 0.f;
      int bad = 0;
      for (int x = wx0; x < wxe; x += wstep) {
        const double2 v = p.psi[x];
        bad |= !(isfinite(v.x) && isfinite(v.y));
        const float2 f = make_float2((float)v.x, (float)v.y);
        Q(1)[x] = f;
        ff_add_prod(s, c, f.x, f.x);
        ff_add_prod(s, c, f.y, f.y);
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) atomicCAS(&st->status, 0, (int)CFET_ENAN);
      c_worker_partial(S, s, c);
    }
    __syncthreads();
    if (ctl) {
      double sum[1];
      if (!c_ctl_reduce<1>(S, NW, partR, tag0 + (++gen), true, &st->status, p.timeout_ns, sum, tacc[5])) {
        if (lane == 0) S.abort_flag = 1;
      } else if (lane == 0) {
        S.abort_flag = ld_volatile_i32(&st->status) != 0;
        S.beta0 = sqrt(sum[0]);
        S.qnorm2[1] = sum[0];
      }
    }
    __syncthreads();
    if (S.abort_flag) return;
  }

  for (long long e = 0; e < p.nexp; ++e) {
    if (tid < ncoef) S.scal[tid] = p.scal[e * ncoef + tid];
    __syncthreads();
    if constexpr (FAMILY == kFamilySpin) {
      if (ctl && lane < op.N) {
        double bi = 0.0;
        for (int k = 0; k < p.nV; ++k) bi = fma(S.scal[1 + k], __ldg(op.xf + k * op.N + lane), bi);
        S.bsite_raw[lane] = bi;
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
          c_const_a<FAMILY>(S, op, 1);
        }
        __syncthreads();
        int it = 1;
        for (;; ++it) {
          // -------- phase A(it); deferred estimate of it-1 on the control warp
          const int pend = S.pend;
          if (!ctl) {
            const CConst& c = S.ca;
            const float2* q = Q(it);
            const float2* qm = it > 1 ? Q(it - 1) : q;
            float2* u = Q(it + 1);
            // <q,u> and ||u||^2: with ||q||^2 (reduced when q was written) they
            // give alpha and ||u - alpha s q||^2, so the decisions need not wait
            // for the orthogonalisation pass
            float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;
            const long long tw0 = sm_clock();
            int x = wx0;
            if constexpr (TILED) {
              {  // window passes, grid exchanges between them (control warp)
                for (int w = 0; w < nwin; ++w) {
                  // basis indices: q_it is vector it - 1, q_{it-1} vector it - 2, u vector it
                  // (from it = 2 on, window 0 first turns u_{it-1} in vector
                  // it - 1 into q_it = u_{it-1} - alpha s q_{it-1}: ORTH)
                  const int iq = it - 1, ia = w == 0 ? (it > 1 ? it - 2 : 0) : it, iu = it;
                  if (w == 0) {
                    const float am = S.am;
                    if (nwin == 1) {
                      if (it > 1)
                        c_tiled_pass<true, true, true>(TP, op, c, S.bx, iq, ia, iu, win[0], 0, wstep, s0, c0, s1, c1,
                                                       am, &s2, &c2);
                      else
                        c_tiled_pass<true, true>(TP, op, c, S.bx, iq, ia, iu, win[0], 0, wstep, s0, c0, s1, c1);
                    } else {
                      if (it > 1)
                        c_tiled_pass<true, false, true>(TP, op, c, S.bx, iq, ia, iu, win[0], 0, wstep, s0, c0, s1, c1,
                                                        am, &s2, &c2);
                      else
                        c_tiled_pass<true, false>(TP, op, c, S.bx, iq, ia, iu, win[0], 0, wstep, s0, c0, s1, c1);
                    }
                  } else if (w == nwin - 1) {
                    c_tiled_pass<false, true>(TP, op, c, S.bx, iq, ia, iu, win[w], w, wstep, s0, c0, s1, c1);
                  } else {
                    c_tiled_pass<false, false>(TP, op, c, S.bx, iq, ia, iu, win[w], w, wstep, s0, c0, s1, c1);
                  }
                  if (w + 1 < nwin) {
                    window_written_sync();    // all threads: window w written
                    window_exchanged_sync();  // all threads: the grid exchange passed
                  }
                }
                x = wxe;  // nothing left for the element loops
              }
            }
            // spin apply on two elements per thread and loop iteration (twice the
            // independent neighbour loads per warp)
            if constexpr (FAMILY == kFamilySpin) {
              for (; x + wstep < wxe; x += 2 * wstep) {
                float2 h1, h2;
                c_apply_spin2(q, qm, x, x + wstep, op, c, S.bx, h1, h2);
                u[x] = h1;
                u[x + wstep] = h2;
                const float2 v1 = q[x], v2 = q[x + wstep];
                ff_add_prod(s0, c0, v1.x, h1.x);
                ff_add_prod(s0, c0, v1.y, h1.y);
                ff_add_prod(s0, c0, v2.x, h2.x);
                ff_add_prod(s0, c0, v2.y, h2.y);
                ff_add_prod(s1, c1, h1.x, h1.x);
                ff_add_prod(s1, c1, h1.y, h1.y);
                ff_add_prod(s1, c1, h2.x, h2.x);
                ff_add_prod(s1, c1, h2.y, h2.y);
              }
            }
            for (; x < wxe; x += wstep) {
              float2 hv;
              if constexpr (FAMILY == kFamilySpin) hv = c_apply_spin(q, qm, x, op, c, S.bx);
              else hv = c_apply_sparse(q, qm, x, dim, op, c);
              u[x] = hv;
              const float2 v = q[x];
              ff_add_prod(s0, c0, v.x, hv.x);
              ff_add_prod(s0, c0, v.y, hv.y);
              ff_add_prod(s1, c1, hv.x, hv.x);
              ff_add_prod(s1, c1, hv.y, hv.y);
            }
            c_worker_partial(S, s0, c0, 0);
            c_worker_partial(S, s1, c1, 1);
            if constexpr (TILED) c_worker_partial(S, s2, c2, 2);  // ||q_it||^2 of the w stored in window 0
            if (tid == 0) {
              twe = sm_clock();
              tacc[0] += twe - tw0;
            }
          } else {
            if (pend) {
              const long long te0 = sm_clock();
              const double err = c_estimate(S, it - 1, remaining, p.tol * remaining / p.tau);
              if (lane == 0) {
                S.err_prev = err;
                S.stop_prev = err <= p.tol * remaining / p.tau;
                S.y_ready = S.stop_prev;
                tacc[6] += sm_clock() - te0;
              }
              __syncwarp();
            }
            if constexpr (TILED) {
              {  // grid exchanges between the window passes of the workers
                for (int w = 0; w + 1 < nwin; ++w) {
                  window_written_sync();
                  double none[1];
                  const bool ok = !S.abort_flag && c_ctl_reduce<0>(S, NW, partW + (size_t)wslot * G, tag0 + (++gen),
                                                                   true, &st->status, p.timeout_ns, none, tacc[5]);
                  __syncwarp();
                  if (!ok && lane == 0) S.abort_flag = 1;
                  wslot ^= 1;
                  window_exchanged_sync();
                }
              }
            }
          }
          __syncthreads();
          if (ctl) {
            const long long tc0 = sm_clock(), sp0 = tacc[5];
            double sum[3];
            // (the tiled apply leaves u written by other CTAs: fence; it also
            // carries ||q_it||^2 of the w that its window 0 stored)
            constexpr bool kMayTile = TILED;
            if ((kMayTile && S.abort_flag) ||
                !c_ctl_reduce<TILED ? 3 : 2>(S, NW, partA, tag0 + (++gen), kMayTile, &st->status, p.timeout_ns,
                                             sum, tacc[5])) {
              if (lane == 0) S.abort_flag = 1;
            } else if (lane == 0 && !S.stop_prev) {
              if (TILED && it > 1) S.qnorm2[it] = sum[2];
              // q_it holds the Lanczos vector v_it times 1/scale[it]:
              // alpha = <v, u>,  ||w||^2 = ||u - alpha v||^2
              //       = ||u||^2 - alpha^2 (2 - s^2 ||q||^2)
              // (the stored q is a unit vector only to FP32 rounding, which the
              // last factor keeps out of the cancellation)
              const double s_it = S.scale[it];
              const double alpha = sum[0] * s_it;
              S.alpha[it] = alpha;
              S.am = (float)(-alpha * s_it);
              S.wnorm2 = sum[1] - alpha * alpha * (2.0 - s_it * s_it * S.qnorm2[it]);
            }
            if (lane == 0) tacc[1] += sm_clock() - tc0 - (tacc[5] - sp0);
          }
          __syncthreads();
          if (tid == 0) tacc[7] += sm_clock() - twe;
          if (S.abort_flag) return;
          if (S.stop_prev) {  // the deferred estimate accepted it-1
            it -= 1;
            acc_err = S.err_prev;
            break;
          }
          // -------- phase B(it): w = u - alpha s_it q_it on the workers (the
          // tiled form does it in the next iteration's window 0); beta (known
          // from the phase-A sums), the decisions and the next iteration's
          // constants on the control warp at the same time
          if (!ctl) {
            if constexpr (!TILED) {
              const float am = S.am;
              const float2* q = Q(it);
              float2* u = Q(it + 1);
              float s0 = 0.f, c0 = 0.f;  // ||w||^2 of the stored w, for the next iteration
              const long long tw0 = sm_clock();
              int x = wx0;
              // four elements per step with every load issued first (more bytes
              // in flight per thread); the sums keep the order of the plain loop
              for (; x + 3 * wstep < wxe; x += 4 * wstep) {
                float2 v[4], uu[4];
  #pragma unroll
                for (int j = 0; j < 4; ++j) {
                  v[j] = q[x + j * wstep];
                  uu[j] = u[x + j * wstep];
                }
  #pragma unroll
                for (int j = 0; j < 4; ++j) {
                  const float2 w = make_float2(fmaf(am, v[j].x, uu[j].x), fmaf(am, v[j].y, uu[j].y));
                  u[x + j * wstep] = w;
                  ff_add_prod(s0, c0, w.x, w.x);
                  ff_add_prod(s0, c0, w.y, w.y);
                }
              }
              for (; x < wxe; x += wstep) {
                const float2 v = q[x];
                const float2 uu = u[x];
                const float2 w = make_float2(fmaf(am, v.x, uu.x), fmaf(am, v.y, uu.y));
                u[x] = w;
                ff_add_prod(s0, c0, w.x, w.x);
                ff_add_prod(s0, c0, w.y, w.y);
              }
              c_worker_partial(S, s0, c0, 0);
              if (tid == 0) {
                twe = sm_clock();
                tacc[2] += twe - tw0;
              }
            }
          } else {
            const long long tc0 = sm_clock();
            // beta and 1/beta from one reciprocal square root (a rounding-level
            // negative ||w||^2 is an exact breakdown)
            const double wn = S.wnorm2;
            const double rb = wn > 0.0 ? rsqrt(wn) : 0.0;
            const double b = wn > 0.0 ? wn * rb : 0.0;
            const double prev_b = it > 1 ? S.beta[it - 1] : 0.0;
            const bool breakdown =
                sb_no_breakdown(b, S.alpha[it], prev_b) != 1 && b <= 1e-13 * (fabs(S.alpha[it]) + prev_b + 1.0);
            int gate = -1;
            if (lane == 0) {
              S.beta[it] = b;
              S.scale[it + 1] = rb;
              gate = krylov_bounds_update(S, it, remaining);
            }
            gate = __shfl_sync(0xffffffffu, gate, 0);
            __syncwarp();
            int acc_flag = 0, pend_next = 0;
            double err = 0.0;
            if (forced) {
              acc_flag = (it == kf);
            } else if (fixed_k) {
              acc_flag = (it == p.m_max) || breakdown;
            } else if (breakdown) {
              acc_flag = 1;
            } else if (it >= p.m_min &&
                       (gate >= 0 ? gate == 1
                                  : fabs(remaining) * gersh_width(it, S.alpha + 1, S.beta + 1) <= 2.0 * it)) {
              if (it < klimit) {
                pend_next = 1;  // estimate runs during the next apply
              } else {
                err = c_estimate(S, it, remaining, p.tol * remaining / p.tau);
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
            if (!acc_flag && it < klimit) c_const_a<FAMILY>(S, op, it + 1);
            if (lane == 0) tacc[3] += sm_clock() - tc0;
          }
          __syncthreads();
          const bool last_it = S.accept_now || it >= klimit;
          if (!TILED && !last_it) {
            // every CTA's w must be visible before the next apply reads it; the
            // exchange also carries ||w||^2 of the stored w
            if (ctl) {
              double wsum[1];
              if (!c_ctl_reduce<1>(S, NW, partB, tag0 + (++gen), true, &st->status, p.timeout_ns, wsum, tacc[5])) {
                if (lane == 0) S.abort_flag = 1;
              } else if (lane == 0) {
                S.qnorm2[it + 1] = wsum[0];
              }
            }
            __syncthreads();
          }
          if (tid == 0) tacc[7] += sm_clock() - twe;
          if (S.abort_flag) return;
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
              const double ts = ldexp(remaining, -h);
              if (!(fabs(ts) * width <= 2.0 * it)) continue;
              err = c_estimate(S, it, ts, p.tol * ts / p.tau);
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
      const double ts = ldexp(remaining, -acc_h);
      const bool final_rec = last_exp && acc_h == 0;
      if (acc_k > 0) {
        // -------- reconstruct q_1 <- beta0 sum_i y_i s_i q_i
        if (ctl) {
          const long long tr0 = sm_clock();
          if (!S.y_ready) small_expm_e1(acc_k, S.alpha + 1, S.beta + 1, ts, S.yr, S.yi, S.tr, S.ti);
          __syncwarp();
          for (int i = lane; i < acc_k; i += 32) {
            const double f = beta0 * S.scale[i + 1];
            S.cr[i] = (float)(f * S.yr[i]);
            S.ci[i] = (float)(f * S.yi[i]);
          }
          if (lane == 0) tacc[6] += sm_clock() - tr0;
        }
        __syncthreads();
        if (!ctl) {
          float s = 0.f, cc = 0.f;
          const long long tw0 = sm_clock();
          for (int x = wx0; x < wxe; x += wstep) {
            float re = 0.f, im = 0.f;
            int i = 0;
            for (; i + 3 < acc_k; i += 4) {  // four basis loads in flight before their use (same order)
              float2 v[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) v[j] = Q(i + j + 1)[x];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float cr = S.cr[i + j], ci = S.ci[i + j];
                re = fmaf(cr, v[j].x, fmaf(-ci, v[j].y, re));
                im = fmaf(cr, v[j].y, fmaf(ci, v[j].x, im));
              }
            }
            for (; i < acc_k; ++i) {
              const float2 v = Q(i + 1)[x];
              const float cr = S.cr[i], ci = S.ci[i];
              re = fmaf(cr, v.x, fmaf(-ci, v.y, re));
              im = fmaf(cr, v.y, fmaf(ci, v.x, im));
            }
            Q(1)[x] = make_float2(re, im);
            if (final_rec) p.psi[x] = make_double2((double)re, (double)im);
            ff_add_prod(s, cc, re, re);
            ff_add_prod(s, cc, im, im);
          }
          c_worker_partial(S, s, cc);
          if (tid == 0) {
              twe = sm_clock();
              tacc[4] += twe - tw0;
            }
        }
        __syncthreads();
        if (ctl) {
          double sum[1];
          if (!c_ctl_reduce<1>(S, NW, partR, tag0 + (++gen), true, &st->status, p.timeout_ns, sum, tacc[5])) {
            if (lane == 0) S.abort_flag = 1;
          } else if (lane == 0) {
            S.beta0 = sqrt(sum[0]);
            S.qnorm2[1] = sum[0];
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

// ------------------------------------------------------------------ launchers
size_t c64_tiled_smem_bytes() {
  return ((sizeof(SmemC) + 127) & ~size_t(127)) + 128 + (size_t)kTmaStages * 2 * kTileBytes;
}

template <int FAMILY, class Op>
static int launch_prop_c64(const PropParams& p, const Op& op, int grid, int block, void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = p.tiled ? c64_tiled_smem_bytes() : sizeof(SmemC);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if constexpr (FAMILY == kFamilySpin) {
    if (p.tiled) return (int)cudaLaunchKernelEx(&cfg, k_propagate_c64<FAMILY, Op, true>, p, op);
  }
  return (int)cudaLaunchKernelEx(&cfg, k_propagate_c64<FAMILY, Op>, p, op);
}

int launch_propagate_spin_c64(const PropParams& p, const OpSpinC& op, int grid, int block, void* stream) {
  return launch_prop_c64<kFamilySpin>(p, op, grid, block, stream);
}
int launch_propagate_dia_c64(const PropParams& p, const OpDiaC& op, int grid, int block, void* stream) {
  return launch_prop_c64<kFamilyDia>(p, op, grid, block, stream);
}
int launch_propagate_csr_c64(const PropParams& p, const OpCsrC& op, int grid, int block, void* stream) {
  return launch_prop_c64<kFamilyCsr>(p, op, grid, block, stream);
}

int max_coresident_blocks_c64(int family, int block, bool tiled) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // a few KB of shared memory: leave the unified storage to L1 (a tiled launch
  // asks for its tile buffers and gets the shared-memory split it needs)
  cudaFuncSetAttribute(k_propagate_c64<kFamilySpin, OpSpinC>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_propagate_c64<kFamilyDia, OpDiaC>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_propagate_c64<kFamilyCsr, OpCsrC>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_propagate_c64<kFamilySpin, OpSpinC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)c64_tiled_smem_bytes());
  cudaError_t e;
  if (family == kFamilySpin)
    e = tiled ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate_c64<kFamilySpin, OpSpinC, true>, block,
                                                              c64_tiled_smem_bytes())
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate_c64<kFamilySpin, OpSpinC>, block, sizeof(SmemC));
  else if (family == kFamilyCsr)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate_c64<kFamilyCsr, OpCsrC>, block,
                                                      sizeof(SmemC));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate_c64<kFamilyDia, OpDiaC>, block,
                                                      sizeof(SmemC));
  if (e != cudaSuccess) return -1;
  return per * nsm;
}

}  // namespace cfet
