// Fixed-point persistent Lanczos kernel (sm_103a).
//
// Same method and decisions as k_propagate (kernels.cu): the stage
// exponential exp(-i tau H_j) psi of a CFET step (Alvermann & Fehske,
// arXiv:1102.5071, Sec. 4 Eq. (Ucf), Sec. 7 Eq. (OmGLeg)) by the Lanczos /
// Krylov method of Sec. 8.1 with the a-posteriori estimate, adaptive Krylov
// dimension and substepping.  Two things differ.
//
// Number format.  On GB300 FP64 runs at 1/64 of the FP32 rate while 32-bit
// integer add/logic/multiply-add run at full or half rate, so every Krylov
// vector q_i is stored as int64 (re, im) mantissas with one exponent per
// vector (value = M * 2^E_i, |M| < 2^57):
//   * neighbour sums of the apply are exact integer additions (up to 32
//     terms stay below 2^62);
//   * a product of a real scalar (or a per-element table value) with a stored
//     value or sum takes the high 64 bits of a 64x64 product of operands
//     normalised to 62 bits, shifted (rounding) once to the result exponent;
//   * the result exponent of each new vector comes from a rigorous bound
//     built from the scalars and the measured maxima of the inputs, so no
//     value overflows; the resolution is 2^-57 of that bound;
//   * alpha, ||w||^2 and ||psi||^2 are exact 128-bit sums, reduced exactly
//     over the CTA and the grid (order-independent, deterministic) and
//     rounded to FP64 once.
//
// Work split.  Each CTA has NW worker warps doing only integer element work
// and one control warp doing all scalar work: the global reductions, the grid
// barrier, the per-pass constants, and the small tridiagonal exponential of
// the error estimate (FP64 where the result must be exact; bounds and certain
// decisions in integer and FP32 arithmetic, scalar_bounds.cuh, because one
// FP64 warp instruction costs 64 cycles here).  The error estimate of iteration k runs
// on the control warp while the workers already compute the apply of
// iteration k+1; if it accepts k, that apply is discarded.  The accepted
// estimate's y = exp(-i tau T_k) e_1 is reused for the reconstruction.
//
// Long chains.  The TILED instantiation replaces the element-wise spin apply
// by window passes over shared-memory tiles moved by TMA (tiled_common.cuh)
// separated by grid exchanges, for chains whose vectors leave L2.  Small
// problems.  The SMALL instantiation runs one CTA with the whole Krylov basis
// in shared memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cfet_internal.h"
#include "device_common.cuh"
#include "fx_common.cuh"
#include "tiled_common.cuh"

namespace cfet {

// ------------------------------------------------------------------ shared state
struct SmemFx {
  // per-warp partials of the workers
  unsigned long long wlo[32];
  long long whi[32];
  long long wmx[32];
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
  // running FP32 bounds of the current T_k for the estimate's screens
  LeadAcc lead;
  GershAcc gfull;  // rows whose couplings are all known
  int gate_it;     // FP32 gate of the current iteration (1, 0, -1: FP64 needed)
  int tma_fail;    // tiled apply: a tile wait gave up
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

// Control warp: a grid-wide exchange of one tagged word per CTA (a barrier),
// with the fences that make the vectors written before it visible after it.
__device__ bool fx_ctl_barrier(unsigned long long* part, unsigned tag, int* status, long long timeout_ns,
                               long long& spin) {
  struct NoAcc {
    __device__ void reset() {}
    __device__ void add(const unsigned (&)[1]) {}
  } acc;
  const unsigned mine[1] = {0u};
  return ctl_exchange<1>(part, mine, tag, true, status, timeout_ns, spin, acc);
}

// ------------------------------------------------------------------ tiled apply (long chains)
// Window tiling of tiled_common.cuh with tiles of 2^11 elements (32 KB of
// int64 pairs), moved by TMA: one tensor map per window over the whole Krylov
// basis (two 8-byte words per element), three pipeline stages of a q tile and
// a tile of the vector each element reads for itself (q_{k-1} in window 0, the
// partial u after it), 192 KB, one mbarrier per stage.  Worker thread 0 issues
// the loads two tiles ahead; once the workers have written a tile's results
// (in place over its own-element tile) it stores that tile with a bulk tensor
// store.  Every window adds its terms in the format of the apply above (exact
// integer neighbour sums, one rounded product per sum and window), so the
// result differs from the element-wise apply by the rounding of the extra
// products (units of the last place of u).  The last window takes <q, u>
// exactly and max |u|.
constexpr int kFxTileElems = 1 << kFxTileBits;
constexpr unsigned kFxTileBytes = kFxTileElems * sizeof(longlong2);

size_t fx_tiled_smem_bytes();

struct FxTma {
  const unsigned char* maps;  // kTmaMapBytes per window
  unsigned long long* bar;    // [kTmaStages] in shared memory
  longlong2* stage;           // [kTmaStages][2][kFxTileElems] in shared memory
  int* fail;                  // shared flag: a wait gave up
  unsigned* phase;            // parity bits of the stages (per thread, identical in all workers)
  int* status;
  long long timeout_ns;
};

// Bounded wait for a stage's tile; false (status CFET_ETIMEOUT) when it gave up.
__device__ bool fx_tile_wait(unsigned long long* bar, unsigned parity, int* status, long long timeout_ns) {
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

// One window pass of this CTA's worker threads over its tiles (basis indices:
// iq the applied q, ia the own-element input, iu the output).
template <bool FIRST, bool LAST>
__device__ void fx_tiled_pass(const FxTma& T, const OpSpinFx& op, const FxConstA& c, const long long* mb, int iq,
                              int ia, int iu, const TileWin& W, int w, int nworkers, __int128& a2, long long& mx) {
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const int ntiles = 1 << (op.N - kFxTileBits);
  const bool aux = !FIRST || c.use_prev;
  const unsigned bytes = aux ? 2 * kFxTileBytes : kFxTileBytes;
  const void* map = T.maps + (size_t)w * kTmaMapBytes;
  const bool prod = tid == 0;
  auto issue = [&](int k, int t) {  // producer: tile t into stage k % kTmaStages
    const int st = k % kTmaStages;
    longlong2* qb = T.stage + (size_t)st * 2 * kFxTileElems;
    mbar_arrive_expect_tx(T.bar + st, bytes);
    tile_load_t<kFxTileBits, 2>(qb, map, FIRST, W, op.N, t, iq, T.bar + st);
    if (aux) tile_load_t<kFxTileBits, 2>(qb + kFxTileElems, map, FIRST, W, op.N, t, ia, T.bar + st);
  };
  if (prod) {
    fence_proxy_async_all();  // vectors written by generic stores before the exchange, read by TMA now
    for (int k = 0; k < kTmaStages - 1; ++k)
      if (blockIdx.x + k * G < ntiles) issue(k, blockIdx.x + k * G);
  }
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; ++k, t += G) {
    const int st = k % kTmaStages;
    const longlong2* cur = T.stage + (size_t)st * 2 * kFxTileElems;
    longlong2* acur = T.stage + (size_t)st * 2 * kFxTileElems + kFxTileElems;
    const unsigned par = (*T.phase >> st) & 1u;
    *T.phase ^= 1u << st;
    if (!fx_tile_wait(T.bar + st, par, T.status, T.timeout_ns)) *T.fail = 1;
    if (!*T.fail) {
      for (int j = tid; j < kFxTileElems; j += nworkers) {
        long long ur, ui, hr = 0, hi = 0;
        const longlong2 v = cur[j];
        if (FIRST) {
          const int x = (t << kFxTileBits) | j;
          const int L = op.lo_bits;
          const long long dz = __ldg(op.DZ_lo + (x & ((1 << L) - 1))) + __ldg(op.DZ_hi + (x >> (L - 1)));
          const long long Dp = fx_mulhi(c.m_cz, dz << 1) << 3;
          ur = fx_mulhi(Dp, v.x << c.pk);
          ui = fx_mulhi(Dp, v.y << c.pk);
          const unsigned anti = ((unsigned)j ^ ((unsigned)j >> 1)) & ((1u << (kFxTileBits - 1)) - 1u);
#pragma unroll
          for (int i = 0; i < kFxTileBits - 1; ++i)
            if ((anti >> i) & 1u) {
              const longlong2 wv = cur[j ^ (3 << i)];
              hr += wv.x;
              hi += wv.y;
            }
          if (op.uniform) {
            long long xr = 0, xi = 0;
#pragma unroll
            for (int i = 0; i < kFxTileBits; ++i) {
              const longlong2 wv = cur[j ^ (1 << i)];
              xr += wv.x;
              xi += wv.y;
            }
            ur += fx_mulhi(c.m_x, xr << c.px);
            ui += fx_mulhi(c.m_x, xi << c.px);
          } else {
#pragma unroll
            for (int i = 0; i < kFxTileBits; ++i) {
              const longlong2 wv = cur[j ^ (1 << i)];
              ur += fx_mulhi(mb[i], wv.x << c.pk);
              ui += fx_mulhi(mb[i], wv.y << c.pk);
            }
          }
          if (c.use_prev) {
            const longlong2 wv = acur[j];
            ur += fx_mulhi(c.m_p, wv.x << c.pp);
            ui += fx_mulhi(c.m_p, wv.y << c.pp);
          }
        } else {
          const longlong2 a = acur[j];
          ur = a.x;
          ui = a.y;
          const unsigned jh = (unsigned)j >> W.c;  // bits b0 .. b0+width-1 of x
          const unsigned anti = (jh ^ (jh >> 1)) & ((1u << (W.width - 1)) - 1u);
          for (int i = 0; i < W.width - 1; ++i)
            if ((anti >> i) & 1u) {
              const longlong2 wv = cur[j ^ (3 << (W.c + i))];
              hr += wv.x;
              hi += wv.y;
            }
          if (op.uniform) {
            long long xr = 0, xi = 0;
            for (int i = 1; i < W.width; ++i) {
              const longlong2 wv = cur[j ^ (1 << (W.c + i))];
              xr += wv.x;
              xi += wv.y;
            }
            ur += fx_mulhi(c.m_x, xr << c.px);
            ui += fx_mulhi(c.m_x, xi << c.px);
          } else {
            for (int i = 1; i < W.width; ++i) {
              const longlong2 wv = cur[j ^ (1 << (W.c + i))];
              ur += fx_mulhi(mb[W.b0 + i], wv.x << c.pk);
              ui += fx_mulhi(mb[W.b0 + i], wv.y << c.pk);
            }
          }
        }
        ur += fx_mulhi(c.m_hop, hr << c.ph);
        ui += fx_mulhi(c.m_hop, hi << c.ph);
        acur[j] = make_longlong2(ur, ui);  // the own element only: read above by this thread
        if (LAST) {
          a2 += (__int128)v.x * ur + (__int128)v.y * ui;
          mx = max(mx, fx_absmax(ur, ui));
        }
      }
    }
    fence_proxy_async_smem();  // the results, written by generic stores, are read by the TMA store
    workers_sync(nworkers);
    if (*T.fail) break;
    if (prod) {
      tile_store_t<kFxTileBits, 2>(map, FIRST, W, op.N, t, iu, acur);
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
        fx_tile_wait(T.bar + s2, par, T.status, T.timeout_ns);
      }
    }
  }
  workers_sync(nworkers);
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
    B += (fabs(cz) * op.maxdz + fabs(ch) * op.nbond + bsum) * Akr;
    const int Eu = fx_exp_for(B, kFxBits);
    const Mant mcz = fx_mant(cz);
    const int ED = fx_exp_for(fabs(cz) * op.maxdz, 59);
    c.m_cz = mcz.m;
    c.s_d = ED - mcz.e - (op.E_dz - 1) - 64;
    c.s_diag = Eu - (ED - 3) - (Ek - c.pk) - 64;
    c.m_cz = fx_fold(mcz.m, c.s_d + c.s_diag);
    const Mant mh = fx_mant(ch);
    c.ph = fx_norm_shift((op.N > 1 ? op.nbond : 1.0) * Ak);
    c.m_hop = mh.m;
    c.s_hop = Eu - mh.e - (Ek - c.ph) - 64;
    c.m_hop = fx_fold(c.m_hop, c.s_hop);
    if (op.uniform) {
      const Mant mx = fx_mant(S.bsite_raw[0] * sk);
      c.px = fx_norm_shift(op.nsite * Ak);
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
// y = exp(-i ts T_k) e_1 left in S.yr/S.yi.  When the FP32 screen shows that
// err exceeds the threshold thr, the FP64 evaluation is skipped and a value
// above thr is returned (S.yr/S.yi then stay untouched).
__device__ double fx_estimate(SmemFx& S, int k, double ts, double thr) {
  const int dec = krylov_lead_decide(S.lead, k, ts, S.beta0, S.beta[k], thr);
  if (dec == 0) return 2.0 * thr + 1e-300;
  const double scale = S.beta0 * S.beta[k];
  if (dec < 0 && small_expm_rejects32(k, S.alpha + 1, S.beta + 1, ts, scale, thr)) return 2.0 * thr + 1e-300;
  small_expm_e1(k, S.alpha + 1, S.beta + 1, ts, S.yr, S.yi, S.tr, S.ti);
  const double yr = S.yr[k - 1], yi = S.yi[k - 1];
  return scale * sqrt(fma(yr, yr, yi * yi));
}

// ------------------------------------------------------------------ the kernel
// TILED: the window-tiled apply of long spin chains (a separate instantiation,
// so that the element-wise kernel carries none of its code).  SMALL: one CTA
// with the Krylov basis in shared memory (separate too, so that the other
// instantiations keep global-memory loads for the vectors).
template <int FAMILY, class Op, bool TILED = false, bool SMALL = false>
__global__ void __launch_bounds__(CFET_CTL_MAX_THREADS, 1) k_propagate_fx(PropParams p, Op op) {
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
  unsigned long long* partA = reinterpret_cast<unsigned long long*>(p.partials);
  unsigned long long* partB = partA + 8 * G;
  unsigned long long* partR = partA + 16 * G;
  unsigned long long* partW = partA + 24 * G;  // window exchanges of the tiled apply: two 1-word slots
  // tiled apply: windows and the tile buffers behind SmemFx
  TileWin win[kTiledMaxWindows] = {};
  int nwin = 1;
  if constexpr (TILED) {
    nwin = tiled_windows<kFxTileBits>(op.N, win);
  }
  // behind SmemFx: the shared-memory basis of one-CTA launches, or the tiled
  // apply's stage mbarriers (128 bytes) and tile buffers
  unsigned char* const tiles_base = smem_raw + ((sizeof(SmemFx) + 127) & ~size_t(127));
  longlong2* tbuf = reinterpret_cast<longlong2*>(tiles_base);
  unsigned tph = 0;  // parities of the stages' mbarriers (the same in every worker)
  const FxTma TP{p.tmaps, reinterpret_cast<unsigned long long*>(tiles_base),
                 reinterpret_cast<longlong2*>(tiles_base + 128), &S.tma_fail, &tph, &p.st->status, p.timeout_ns};
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

  // one-CTA launches of small problems keep the basis in shared memory (a
  // separate instantiation: the others keep global-memory loads)
  longlong2* const qb = SMALL ? tbuf : p.qbasis;
  auto Q = [&](int i) -> longlong2* { return qb + (size_t)(i - 1) * dim; };

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
          fx_const_a<FAMILY>(S, op, 1);
        }
        __syncthreads();
        int it = 1;
        for (;; ++it) {
          // -------- phase A(it) on the workers; deferred estimate of it-1 on the control warp
          const int pend = S.pend;
          if (!ctl) {
            const FxConstA& c = S.ca;
            const longlong2* q = Q(it);
            const longlong2* qm = it > 1 ? Q(it - 1) : q;
            longlong2* u = Q(it + 1);
            __int128 a2 = 0;
            long long mx = 0;
            const long long tw0 = sm_clock();
            int x = wx0;
            if constexpr (TILED) {
              {  // window passes, grid exchanges between them (control warp)
                for (int w = 0; w < nwin; ++w) {
                  // basis indices: q_it is vector it - 1, q_{it-1} vector it - 2, u vector it
                  const int iq = it - 1, ia = w == 0 ? (it > 1 ? it - 2 : 0) : it, iu = it;
                  if (w == 0) {
                    if (nwin == 1)
                      fx_tiled_pass<true, true>(TP, op, c, S.mb, iq, ia, iu, win[0], 0, wstep, a2, mx);
                    else
                      fx_tiled_pass<true, false>(TP, op, c, S.mb, iq, ia, iu, win[0], 0, wstep, a2, mx);
                  } else if (w == nwin - 1) {
                    fx_tiled_pass<false, true>(TP, op, c, S.mb, iq, ia, iu, win[w], w, wstep, a2, mx);
                  } else {
                    fx_tiled_pass<false, false>(TP, op, c, S.mb, iq, ia, iu, win[w], w, wstep, a2, mx);
                  }
                  if (w + 1 < nwin) {
                    window_written_sync();    // all threads: window w written
                    window_exchanged_sync();  // all threads: the grid exchange passed
                  }
                }
                x = wxe;  // nothing left for the element loops
              }
            }
            if constexpr (FAMILY == kFamilySpin) {
              for (; x + wstep < wxe; x += 2 * wstep) {
                longlong2 h1, h2;
                fx_apply_spin2(q, qm, x, x + wstep, op, c, S.mb, h1, h2);
                u[x] = h1;
                u[x + wstep] = h2;
                const longlong2 v1 = q[x], v2 = q[x + wstep];
                a2 += (__int128)v1.x * h1.x + (__int128)v1.y * h1.y;
                a2 += (__int128)v2.x * h2.x + (__int128)v2.y * h2.y;
                mx = max(mx, max(fx_absmax(h1.x, h1.y), fx_absmax(h2.x, h2.y)));
              }
            }
            for (; x < wxe; x += wstep) {
              longlong2 hv;
              if constexpr (FAMILY == kFamilySpin) hv = fx_apply_spin(q, qm, x, op, c, S.mb);
              else hv = fx_apply_sparse(q, qm, x, dim, op, c);
              u[x] = hv;
              const longlong2 v = q[x];
              a2 += (__int128)v.x * hv.x + (__int128)v.y * hv.y;
              mx = max(mx, fx_absmax(hv.x, hv.y));
            }
            fx_worker_partial(S, a2, mx);
            if (tid == 0) {
              twe = sm_clock();
              tacc[0] += twe - tw0;
            }
          } else {
            if (pend) {
              const long long te0 = sm_clock();
              const double err = fx_estimate(S, it - 1, remaining, p.tol * remaining / p.tau);
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
                  const bool ok = !S.abort_flag && fx_ctl_barrier(partW + (size_t)wslot * G, tag0 + (++gen),
                                                                  &st->status, p.timeout_ns, tacc[5]);
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
            double sum;
            long long mxi;
            // (the tiled apply leaves u written by other CTAs: fence)
            constexpr bool kMayTile = TILED;
            if ((kMayTile && S.abort_flag) ||
                !fx_ctl_reduce(S, NW, partA, tag0 + (++gen), kMayTile, &st->status, p.timeout_ns,
                               sum, mxi, tacc[5])) {
              if (lane == 0) S.abort_flag = 1;
            } else if (lane == 0 && !S.stop_prev) {
              const double s_it = S.scale[it];
              const double alpha = fx_scale2(sum, S.E[it] + S.Eu) * s_it;
              S.alpha[it] = alpha;
              // phase-B constants: w = u - alpha s_it q_it
              const double am = alpha * s_it;
              const double Bw = fx_scale2(sb_ll_to_double_up(mxi), S.Eu) + fabs(am) * fx_scale2(S.A[it], S.E[it]);
              const int Ew = fx_exp_for(Bw, kFxBits);
              const Mant ma = fx_mant(-am);
              const int pk = fx_norm_shift(S.A[it]);
              S.Ew = Ew;
              S.sh_u = Ew - S.Eu;
              S.m_a = ma.m;
              S.pk_b = pk;
              S.s_a = Ew - ma.e - (S.E[it] - pk) - 64;
              S.m_a = fx_fold(ma.m, S.s_a);
              if (mxi >= (1LL << 60)) {  // fixed-point range exceeded (not expected)
                atomicCAS(&st->status, 0, (int)CFET_ENAN);
                S.abort_flag = 1;
              }
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
          // -------- phase B(it): w = u - alpha s_it q_it, beta = ||w||
          if (!ctl) {
            const int sh_u = S.sh_u, pk = S.pk_b;
            const long long m_a = S.m_a;
            const longlong2* q = Q(it);
            longlong2* u = Q(it + 1);
            __int128 b2 = 0;
            long long mx = 0;
            const long long tw0 = sm_clock();
            int x = wx0;
            // two elements per step with every load issued first (exact sums:
            // the order does not matter)
            for (; x + wstep < wxe; x += 2 * wstep) {
              const longlong2 v0 = q[x], v1 = q[x + wstep];
              const longlong2 u0 = u[x], u1 = u[x + wstep];
              const long long wr0 = fx_rshr(u0.x, sh_u) + fx_mulhi(m_a, v0.x << pk);
              const long long wi0 = fx_rshr(u0.y, sh_u) + fx_mulhi(m_a, v0.y << pk);
              const long long wr1 = fx_rshr(u1.x, sh_u) + fx_mulhi(m_a, v1.x << pk);
              const long long wi1 = fx_rshr(u1.y, sh_u) + fx_mulhi(m_a, v1.y << pk);
              u[x] = make_longlong2(wr0, wi0);
              u[x + wstep] = make_longlong2(wr1, wi1);
              b2 += (__int128)wr0 * wr0 + (__int128)wi0 * wi0;
              b2 += (__int128)wr1 * wr1 + (__int128)wi1 * wi1;
              mx = max(mx, max(fx_absmax(wr0, wi0), fx_absmax(wr1, wi1)));
            }
            for (; x < wxe; x += wstep) {
              const longlong2 v = q[x];
              const longlong2 uu = u[x];
              const long long wr = fx_rshr(uu.x, sh_u) + fx_mulhi(m_a, v.x << pk);
              const long long wi = fx_rshr(uu.y, sh_u) + fx_mulhi(m_a, v.y << pk);
              u[x] = make_longlong2(wr, wi);
              b2 += (__int128)wr * wr + (__int128)wi * wi;
              mx = max(mx, fx_absmax(wr, wi));
            }
            fx_worker_partial(S, b2, mx);
            if (tid == 0) {
              twe = sm_clock();
              tacc[2] += twe - tw0;
            }
          } else if (lane == 0) {
            // meanwhile: running bounds of T_it (alpha_it and beta_{it-1} are
            // known) and the FP32 gate of its estimate
            S.gate_it = krylov_bounds_update(S, it, remaining);
          }
          __syncthreads();
          if (ctl) {
            const long long tc0 = sm_clock(), sp0 = tacc[5];
            double sum;
            long long mxi;
            if (!fx_ctl_reduce(S, NW, partB, tag0 + (++gen), true, &st->status, p.timeout_ns, sum, mxi, tacc[5])) {
              if (lane == 0) S.abort_flag = 1;
            } else {
              // beta and 1/beta from one reciprocal square root
              const double rb = __double_as_longlong(sum) > 0 ? rsqrt(sum) : 0.0;
              const double b = fx_scale2(sum * rb, S.Ew);
              const double prev_b = it > 1 ? S.beta[it - 1] : 0.0;
              const bool breakdown =
                  sb_no_breakdown(b, S.alpha[it], prev_b) != 1 && b <= 1e-13 * (fabs(S.alpha[it]) + prev_b + 1.0);
              const int gate = S.gate_it;
              if (lane == 0) {
                S.beta[it] = b;
                S.scale[it + 1] = fx_scale2(rb, -S.Ew);
                S.E[it + 1] = S.Ew;
                S.A[it + 1] = sb_ll_to_double_up(mxi);
              }
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
                  err = fx_estimate(S, it, remaining, p.tol * remaining / p.tau);
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
              if (!acc_flag && it < klimit) fx_const_a<FAMILY>(S, op, it + 1);
            }
            if (lane == 0) tacc[3] += sm_clock() - tc0 - (tacc[5] - sp0);
          }
          __syncthreads();
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
              const double ts = fx_scale2(remaining, -h);
              if (!(fabs(ts) * width <= 2.0 * it)) continue;
              err = fx_estimate(S, it, ts, p.tol * ts / p.tau);
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
          // (cr + i ci)(vr + i vi) with three products; the sums (< 2^63) are
          // halved to stay in fx_mulhi's operand range
          auto term = [&](int i, const longlong2 v, long long& re, long long& im) {
            const int pi = S.cp[i];
            const long long cr = S.crm[i], ci = S.cim[i];
            const long long vr = v.x << pi, vi = v.y << pi;
            const long long p1 = fx_mulhi(cr, vr), p2 = fx_mulhi(ci, vi);
            const long long p3 = fx_mulhi((cr + ci) >> 1, (vr + vi) >> 1) << 2;
            re += p1 - p2;
            im += p3 - p1 - p2;
          };
          for (int x = wx0; x < wxe; x += wstep) {
            long long re = 0, im = 0;
            int i = 0;
            for (; i + 3 < acc_k; i += 4) {  // four basis loads in flight before their use
              longlong2 v[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) v[j] = Q(i + j + 1)[x];
#pragma unroll
              for (int j = 0; j < 4; ++j) term(i + j, v[j], re, im);
            }
            for (; i < acc_k; ++i) term(i, Q(i + 1)[x], re, im);
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

// ------------------------------------------------------------------ launchers
template <int FAMILY, class Op>
static int launch_prop_fx(const PropParams& p, const Op& op, int grid, int block, void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = p.tiled ? fx_tiled_smem_bytes() : p.small ? fx_small_smem_bytes(p.dim, p.m_max) : sizeof(SmemFx);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if constexpr (FAMILY == kFamilySpin) {
    if (p.tiled) return (int)cudaLaunchKernelEx(&cfg, k_propagate_fx<FAMILY, Op, true>, p, op);
  }
  if (p.small) return (int)cudaLaunchKernelEx(&cfg, k_propagate_fx<FAMILY, Op, false, true>, p, op);
  return (int)cudaLaunchKernelEx(&cfg, k_propagate_fx<FAMILY, Op>, p, op);
}

int launch_propagate_spin_fx(const PropParams& p, const OpSpinFx& op, int grid, int block, void* stream) {
  return launch_prop_fx<kFamilySpin>(p, op, grid, block, stream);
}
int launch_propagate_dia_fx(const PropParams& p, const OpDiaFx& op, int grid, int block, void* stream) {
  return launch_prop_fx<kFamilyDia>(p, op, grid, block, stream);
}
int launch_propagate_csr_fx(const PropParams& p, const OpCsrFx& op, int grid, int block, void* stream) {
  return launch_prop_fx<kFamilyCsr>(p, op, grid, block, stream);
}

size_t fx_tiled_smem_bytes() {
  return ((sizeof(SmemFx) + 127) & ~size_t(127)) + 128 + (size_t)kTmaStages * 2 * kFxTileBytes;
}

// Shared memory of a one-CTA launch that holds q_1 .. q_{m_max+1} (0 when it
// does not fit in an SM's shared memory).
size_t fx_small_smem_bytes(int dim, int m_max) {
  const size_t b = ((sizeof(SmemFx) + 127) & ~size_t(127)) + (size_t)(m_max + 1) * dim * sizeof(longlong2);
  return b <= kFxSmallSmemMax ? b : 0;
}

int fx_small_prepare(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_propagate_fx<kFamilySpin, OpSpinFx, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_propagate_fx<kFamilyDia, OpDiaFx, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_propagate_fx<kFamilyCsr, OpCsrFx, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return (int)e;
}

int max_coresident_blocks_fx(int family, int block, bool tiled) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // the element-wise kernel needs only a few KB of shared memory: leave the
  // rest of the unified L1/shared storage to L1, which holds each CTA's chunk
  // (a tiled launch asks for its tile buffers and gets the split it needs)
  cudaFuncSetAttribute(k_propagate_fx<kFamilySpin, OpSpinFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_propagate_fx<kFamilyDia, OpDiaFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_propagate_fx<kFamilyCsr, OpCsrFx>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_propagate_fx<kFamilySpin, OpSpinFx, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fx_tiled_smem_bytes());
  cudaError_t e;
  if (family == kFamilySpin)
    e = tiled ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate_fx<kFamilySpin, OpSpinFx, true>, block,
                                                              fx_tiled_smem_bytes())
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate_fx<kFamilySpin, OpSpinFx>, block, sizeof(SmemFx));
  else if (family == kFamilyCsr)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate_fx<kFamilyCsr, OpCsrFx>, block,
                                                      sizeof(SmemFx));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate_fx<kFamilyDia, OpDiaFx>, block,
                                                      sizeof(SmemFx));
  if (e != cudaSuccess) return -1;
  return per * nsm;
}

}  // namespace cfet
