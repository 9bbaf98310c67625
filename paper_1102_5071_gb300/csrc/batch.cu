// Batched CFET propagation of many driven XXZ chains of uneven size in one
// persistent launch (sm_103a).
//
// Each instance runs the method of the single-instance kernels: CFET steps
// (Alvermann & Fehske, arXiv:1102.5071, Sec. 4 Eq. (Ucf)) with stage
// operators from the Gauss-Legendre rule (Sec. 7, Eq. (OmGLeg)), each stage
// exponential by the Lanczos / Krylov method of Sec. 8.1 with the
// a-posteriori estimate, adaptive Krylov dimension and substepping, in FP64
// (complex128 vectors) or mixed precision (complex64 vectors, compensated
// FP64-class reductions, FP64 scalars).
//
// Schedule.  The grid is a set of thread-block clusters of cluster_size CTAs
// that take work items from a global counter until none is left (no grid-wide
// synchronisation).  A work item is either
//   * one large instance spread over all CTAs of the cluster: every CTA owns a
//     contiguous chunk of each vector, the partial sums of a reduction are
//     exchanged through distributed shared memory after a cluster barrier and
//     added in rank order, so that every CTA holds identical scalars and takes
//     identical decisions; or
//   * up to cluster_size small instances, one per CTA, each with CTA-local
//     reductions.
// The host orders the items by decreasing work (longest first) and picks the
// cluster size, CTA size and the size threshold of the first kind, by
// measurement (cfet_batch_tune) or from the caller.  Warp 0 of every CTA does
// the FP64 scalar work (tridiagonal exponential, estimate, decisions) while
// the other CTAs resident on the SM keep the memory system busy.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "cfet_internal.h"
#include "device_common.cuh"

namespace cg = cooperative_groups;

namespace cfet {
namespace {

constexpr int kBatchMaxSites = 24;

struct BInst {
  int N, L, uniform, dim;
  double J2;
  const void* dz;       // dz_lo [2^L] then dz_hi [2^(N-L+1)] (double or float)
  const double* a;      // [N] X-field coefficients
  double2* psi;         // caller's state
  void* basis;          // (m_max + 1) * dim vector elements
  const double* scal;   // [nexp * 2]: c0, c1 per stage exponential
  long long f_nsub, f_kh;  // offsets into the forced decision arrays (-1: none)
  long long r_nsub, r_kh;  // offsets into the record arrays (-1: none)
  long long r_cap;
};

struct BItem {
  int coop;     // 1: one instance over the whole cluster; 0: one instance per CTA
  int n;        // instances in the item
  int inst[8];
};

struct BStat {
  long long n_exp, n_sub, n_app;
  int max_k, status;
  double max_err;
  int rec_overflow, pad;
};

struct BParams {
  const BInst* inst;
  const BItem* items;
  int nitems;
  int* queue;
  long long nexp;
  double tau, tol;
  int m_min, m_max, max_substeps, pad;
  const int* f_nsub; const int* f_k; const int* f_h;
  int* r_nsub; int* r_k; int* r_h;
  BStat* stat;
};

// ------------------------------------------------------------------ number formats
// FP64: complex128 vectors, FP64 sums.
struct FmtF64 {
  using V = double2;
  using T = double;
  struct Acc {
    double s;
  };
  static __device__ __forceinline__ V make(T x, T y) { return make_double2(x, y); }
  static __device__ __forceinline__ V from64(double2 v) { return v; }
  static __device__ __forceinline__ Acc zero() { return Acc{0.0}; }
  static __device__ __forceinline__ void add_prod(Acc& a, T x, T y) { a.s = fma(x, y, a.s); }
  static __device__ __forceinline__ void add(Acc& a, const Acc& b) { a.s += b.s; }
  static __device__ __forceinline__ Acc shfl_down(const Acc& a, int o) {
    return Acc{__shfl_down_sync(0xffffffffu, a.s, o)};
  }
  static __device__ __forceinline__ double value(const Acc& a) { return a.s; }
};

// complex64 vectors; per-thread Dot2 (error-free product and sum), float-float
// across threads, rounded to FP64 once.
struct FmtC64 {
  using V = float2;
  using T = float;
  struct Acc {
    float s, c;
  };
  static __device__ __forceinline__ V make(T x, T y) { return make_float2(x, y); }
  static __device__ __forceinline__ V from64(double2 v) { return make_float2((float)v.x, (float)v.y); }
  static __device__ __forceinline__ Acc zero() { return Acc{0.f, 0.f}; }
  static __device__ __forceinline__ void two_sum(Acc& a, float p) {
    const float t = __fadd_rn(a.s, p);
    const float z = __fsub_rn(t, a.s);
    const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(p, z));
    a.s = t;
    a.c = __fadd_rn(a.c, e);
  }
  static __device__ __forceinline__ void add_prod(Acc& a, T x, T y) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    two_sum(a, p);
    a.c = __fadd_rn(a.c, e);
  }
  static __device__ __forceinline__ void add(Acc& a, const Acc& b) {
    two_sum(a, b.s);
    a.c = __fadd_rn(a.c, b.c);
  }
  static __device__ __forceinline__ Acc shfl_down(const Acc& a, int o) {
    return Acc{__shfl_down_sync(0xffffffffu, a.s, o), __shfl_down_sync(0xffffffffu, a.c, o)};
  }
  static __device__ __forceinline__ double value(const Acc& a) { return (double)a.s + (double)a.c; }
};

template <class Fmt>
struct SmemB {
  typename Fmt::Acc wacc[32];
  typename Fmt::Acc cta[2];           // this CTA's partial, two alternating slots
  double result;
  double alpha[kMaxKrylov + 2];
  double beta[kMaxKrylov + 2];
  double scale[kMaxKrylov + 3];
  double yr[kMaxKrylov], yi[kMaxKrylov];
  double tr[kMaxKrylov], ti[kMaxKrylov];
  typename Fmt::T cr[kMaxKrylov], ci[kMaxKrylov];
  typename Fmt::T bx[kBatchMaxSites];  // per-site field times the current scale
  double bsite[kBatchMaxSites];        // per-site field of the stage
  typename Fmt::T cz, ch, cx, cp, am;
  int use_prev;
  int accept_now, acc_h, y_ready;
  double err_now;
  int item;
};

// ------------------------------------------------------------------ reductions
// Sum over the CTA (and over the cluster when coop) of per-thread partials;
// the result is returned to every thread of the CTA.  Every CTA of a cluster
// adds the partials in rank order, so all hold the same value.
template <class Fmt>
__device__ double batch_reduce(SmemB<Fmt>& S, typename Fmt::Acc a, int& slot, bool coop, cg::cluster_group& cl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) Fmt::add(a, Fmt::shfl_down(a, o));
  if (lane == 0) S.wacc[warp] = a;
  __syncthreads();
  if (warp == 0) {
    a = lane < nw ? S.wacc[lane] : Fmt::zero();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Fmt::add(a, Fmt::shfl_down(a, o));
    if (lane == 0) S.cta[slot] = a;
  }
  if (coop) {
    cl.sync();  // release / acquire at cluster scope: partials and vector stores
    if (threadIdx.x == 0) {
      typename Fmt::Acc t = Fmt::zero();
      const int nb = (int)cl.num_blocks();
      for (int r = 0; r < nb; ++r) Fmt::add(t, *cl.map_shared_rank(&S.cta[slot], r));
      S.result = Fmt::value(t);
    }
  } else if (threadIdx.x == 0) {
    S.result = Fmt::value(S.cta[slot]);
  }
  __syncthreads();
  slot ^= 1;
  return S.result;
}

// ------------------------------------------------------------------ apply
template <class Fmt>
__device__ __forceinline__ typename Fmt::V batch_apply(const typename Fmt::V* __restrict__ q,
                                                       const typename Fmt::V* __restrict__ qm, int x, int N, int L,
                                                       int uniform, const typename Fmt::T* dz_lo,
                                                       const typename Fmt::T* dz_hi, const SmemB<Fmt>& S) {
  using T = typename Fmt::T;
  using V = typename Fmt::V;
  const T dz = dz_lo[x & ((1 << L) - 1)] + dz_hi[x >> (L - 1)];
  const T d = S.cz * dz;
  const V v = q[x];
  T ur = d * v.x, ui = d * v.y;
  T hr = 0, hi = 0;
  const unsigned anti = ((unsigned)x ^ ((unsigned)x >> 1)) & ((1u << (N - 1)) - 1u);
#pragma unroll 4
  for (int i = 0; i < N - 1; ++i) {  // antiparallel bonds only (predicated)
    if ((anti >> i) & 1u) {
      const V w = q[x ^ (3 << i)];
      hr += w.x;
      hi += w.y;
    }
  }
  ur = fma(S.ch, hr, ur);
  ui = fma(S.ch, hi, ui);
  if (uniform) {
    T xr = 0, xi = 0;
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const V w = q[x ^ (1 << i)];
      xr += w.x;
      xi += w.y;
    }
    ur = fma(S.cx, xr, ur);
    ui = fma(S.cx, xi, ui);
  } else {
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const V w = q[x ^ (1 << i)];
      ur = fma(S.bx[i], w.x, ur);
      ui = fma(S.bx[i], w.y, ui);
    }
  }
  if (S.use_prev) {
    const V w = qm[x];
    ur = fma(S.cp, w.x, ur);
    ui = fma(S.cp, w.y, ui);
  }
  return Fmt::make(ur, ui);
}

// ------------------------------------------------------------------ one instance
template <class Fmt>
__device__ void run_instance(const BParams& P, int ii, int part, int nparts, bool coop, SmemB<Fmt>& S,
                             cg::cluster_group& cl) {
  using V = typename Fmt::V;
  using T = typename Fmt::T;
  using Acc = typename Fmt::Acc;
  const BInst I = P.inst[ii];
  const int tid = threadIdx.x, lane = tid & 31;
  const bool w0 = tid < 32;                   // scalar warp
  const bool lead = (tid == 0) && part == 0;  // writes results of the instance
  const int dim = I.dim, N = I.N;
  const int chunk = (((dim + nparts - 1) / nparts) + 31) & ~31;
  const int x0 = part * chunk + tid, xe = min(dim, (part + 1) * chunk);
  const int step = blockDim.x;
  const T* dz_lo = reinterpret_cast<const T*>(I.dz);
  const T* dz_hi = dz_lo + (1 << I.L);
  V* basis = reinterpret_cast<V*>(I.basis);
  auto Q = [&](int i) -> V* { return basis + (size_t)(i - 1) * dim; };
  const bool fixed_k = P.tol <= 0.0;
  const bool forced = I.f_nsub >= 0;
  long long fpos = 0, rpos = 0;
  long long n_app = 0, n_sub = 0;
  int max_k = 0, status = 0;
  double max_err = 0.0;
  int slot = 0;

  // psi (complex128) -> q_1, ||q_1||^2 (non-finite input gives a non-finite sum)
  double beta0;
  {
    Acc a = Fmt::zero();
    for (int x = x0; x < xe; x += step) {
      const V f = Fmt::from64(I.psi[x]);
      Q(1)[x] = f;
      Fmt::add_prod(a, f.x, f.x);
      Fmt::add_prod(a, f.y, f.y);
    }
    const double s = batch_reduce<Fmt>(S, a, slot, coop, cl);
    if (!isfinite(s)) status = CFET_ENAN;
    beta0 = sqrt(s);
  }

  for (long long e = 0; e < P.nexp && status == 0; ++e) {
    const double c0 = I.scal[2 * e], c1 = I.scal[2 * e + 1];
    if (tid < N) S.bsite[tid] = c1 * I.a[tid];
    __syncthreads();
    const bool last_exp = (e == P.nexp - 1);
    const int nforced = forced ? P.f_nsub[I.f_nsub + e] : 0;
    double remaining = P.tau;
    int nsub_e = 0;
    while (true) {
      if (nsub_e >= P.max_substeps || (forced && nsub_e >= nforced)) {
        status = CFET_EKRYLOV;
        break;
      }
      int kf = -1, hf = 0;
      if (forced) {
        kf = P.f_k[I.f_kh + fpos];
        hf = P.f_h[I.f_kh + fpos];
      }
      int acc_k = 0, acc_h = 0;
      double acc_err = 0.0;
      if (beta0 != 0.0) {
        const int klimit = forced ? kf : P.m_max;
        if (tid == 0) S.scale[1] = 1.0 / beta0;
        int it = 1;
        bool accepted = false;
        for (;; ++it) {
          // constants of u = s_it H_j q_it - beta_{it-1} s_{it-1} q_{it-1}
          if (tid == 0) {
            const double sk = S.scale[it];
            const double cz = c0 * sk;
            S.cz = (T)cz;
            S.ch = (T)(cz * I.J2);
            S.cx = (T)(S.bsite[0] * sk);
            S.cp = it > 1 ? (T)(-S.beta[it - 1] * S.scale[it - 1]) : (T)0;
            S.use_prev = it > 1;
          }
          if (!I.uniform && tid < N) S.bx[tid] = (T)(S.bsite[tid] * S.scale[it]);
          __syncthreads();
          Acc a = Fmt::zero();
          {
            const V* q = Q(it);
            const V* qm = it > 1 ? Q(it - 1) : q;
            V* u = Q(it + 1);
            for (int x = x0; x < xe; x += step) {
              const V hv = batch_apply<Fmt>(q, qm, x, N, I.L, I.uniform, dz_lo, dz_hi, S);
              u[x] = hv;
              const V v = q[x];
              Fmt::add_prod(a, v.x, hv.x);
              Fmt::add_prod(a, v.y, hv.y);
            }
          }
          const double s_it = S.scale[it];
          const double alpha = batch_reduce<Fmt>(S, a, slot, coop, cl) * s_it;
          if (tid == 0) {
            S.alpha[it] = alpha;
            S.am = (T)(-alpha * s_it);
          }
          __syncthreads();
          a = Fmt::zero();
          {
            const T am = S.am;
            const V* q = Q(it);
            V* u = Q(it + 1);
            for (int x = x0; x < xe; x += step) {
              const V v = q[x];
              const V uu = u[x];
              const V w = Fmt::make(fma(am, v.x, uu.x), fma(am, v.y, uu.y));
              u[x] = w;
              Fmt::add_prod(a, w.x, w.x);
              Fmt::add_prod(a, w.y, w.y);
            }
          }
          const double bsum = batch_reduce<Fmt>(S, a, slot, coop, cl);
          if (w0) {
            const double b = sqrt(bsum);
            const double prev_b = it > 1 ? S.beta[it - 1] : 0.0;
            const bool breakdown =
                sb_no_breakdown(b, S.alpha[it], prev_b) != 1 && b <= 1e-13 * (fabs(S.alpha[it]) + prev_b + 1.0);
            if (lane == 0) {
              S.beta[it] = b;
              S.scale[it + 1] = 1.0 / b;
            }
            __syncwarp();
            int acc_flag = 0;
            double err = 0.0;
            if (forced) {
              acc_flag = (it == kf);
            } else if (fixed_k) {
              acc_flag = (it == P.m_max) || breakdown;
            } else if (breakdown) {
              acc_flag = 1;
            } else if (it >= P.m_min && gersh_gate(it, S.alpha + 1, S.beta + 1, remaining)) {
              const double thr = P.tol * remaining / P.tau;
              if (krylov_lead_rejects(it, S.alpha + 1, S.beta + 1, remaining, beta0 * b, thr)) {
                err = 2.0 * thr + 1e-300;
              } else {
                small_expm_e1(it, S.alpha + 1, S.beta + 1, remaining, S.yr, S.yi, S.tr, S.ti);
                err = beta0 * b * hypot(S.yr[it - 1], S.yi[it - 1]);
                acc_flag = err <= thr;
              }
            }
            if (lane == 0) {
              S.accept_now = acc_flag;
              S.err_now = err;
              S.y_ready = acc_flag && !forced && !fixed_k && !breakdown;
            }
          }
          __syncthreads();
          if (S.accept_now) {
            accepted = true;
            acc_err = S.err_now;
            break;
          }
          if (it >= klimit) break;
        }
        acc_k = it;
        if (forced) {
          acc_h = hf;
        } else if (!accepted) {
          if (w0) {
            int hh = 0;
            double err = 0.0;
            const double width = gersh_width(it, S.alpha + 1, S.beta + 1);
            for (int h = 1; h <= 40; ++h) {
              const double ts = ldexp(remaining, -h);
              if (!(fabs(ts) * width <= 2.0 * it)) continue;
              small_expm_e1(it, S.alpha + 1, S.beta + 1, ts, S.yr, S.yi, S.tr, S.ti);
              err = beta0 * S.beta[it] * hypot(S.yr[it - 1], S.yi[it - 1]);
              if (err <= P.tol * ts / P.tau) { hh = h; break; }
            }
            if (lane == 0) { S.acc_h = hh; S.err_now = err; S.y_ready = hh > 0; }
          }
          __syncthreads();
          acc_h = S.acc_h;
          acc_err = S.err_now;
          if (acc_h == 0) {
            status = CFET_EKRYLOV;
            break;
          }
        }
        n_app += acc_k;
      }
      const double ts = ldexp(remaining, -acc_h);
      if (acc_k > 0) {
        // reconstruct q_1 <- beta0 sum_i y_i s_i q_i
        if (w0) {
          if (!S.y_ready) small_expm_e1(acc_k, S.alpha + 1, S.beta + 1, ts, S.yr, S.yi, S.tr, S.ti);
          __syncwarp();
          for (int i = lane; i < acc_k; i += 32) {
            const double f = beta0 * S.scale[i + 1];
            S.cr[i] = (T)(f * S.yr[i]);
            S.ci[i] = (T)(f * S.yi[i]);
          }
        }
        __syncthreads();
        const bool final_rec = last_exp && acc_h == 0;
        Acc a = Fmt::zero();
        for (int x = x0; x < xe; x += step) {
          T re = 0, im = 0;
          for (int i = 0; i < acc_k; ++i) {
            const V v = Q(i + 1)[x];
            const T cr = S.cr[i], ci = S.ci[i];
            re = fma(cr, v.x, fma(-ci, v.y, re));
            im = fma(cr, v.y, fma(ci, v.x, im));
          }
          Q(1)[x] = Fmt::make(re, im);
          if (final_rec) I.psi[x] = make_double2((double)re, (double)im);
          Fmt::add_prod(a, re, re);
          Fmt::add_prod(a, im, im);
        }
        beta0 = sqrt(batch_reduce<Fmt>(S, a, slot, coop, cl));
      }
      if (lead && I.r_kh >= 0) {
        if (rpos < I.r_cap) {
          P.r_k[I.r_kh + rpos] = acc_k;
          P.r_h[I.r_kh + rpos] = acc_h;
        } else {
          P.stat[ii].rec_overflow = 1;
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
    if (lead && I.r_nsub >= 0) P.r_nsub[I.r_nsub + e] = nsub_e;
  }
  if (lead) {
    BStat& st = P.stat[ii];
    st.n_exp = P.nexp;
    st.n_sub = n_sub;
    st.n_app = n_app;
    st.max_k = max_k;
    st.max_err = max_err;
    st.status = status;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ the kernel
template <class Fmt>
__global__ void __launch_bounds__(512) k_batch_propagate(BParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemB<Fmt>& S = *reinterpret_cast<SmemB<Fmt>*>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  while (true) {
    if (rank == 0 && threadIdx.x == 0) S.item = atomicAdd(P.queue, 1);
    cl.sync();
    const int item = *cl.map_shared_rank(&S.item, 0);
    if (item >= P.nitems) break;
    const BItem& it = P.items[item];
    if (it.coop) {
      run_instance<Fmt>(P, it.inst[0], rank, (int)cl.num_blocks(), true, S, cl);
    } else if (rank < it.n) {
      run_instance<Fmt>(P, it.inst[rank], 0, 1, false, S, cl);
    }
    cl.sync();  // the item is done in every CTA before rank 0 takes the next
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <class Fmt>
int launch_batch(const BParams& p, int clusters, int cluster_size, int threads, void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * cluster_size);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = sizeof(SmemB<Fmt>);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster_size;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_batch_propagate<Fmt>, p);
}

template <class Fmt>
int max_clusters(int cluster_size, int threads) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster_size);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = sizeof(SmemB<Fmt>);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster_size;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_batch_propagate<Fmt>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace
}  // namespace cfet

// ============================================================================
// C ABI
using namespace cfet;

struct cfet_batch {
  int device = 0;
  int n = 0;
  int precision = CFET_PREC_F64;
  cfet_options opt{};
  std::string err;
  std::vector<cfet_chain> chains;          // h / a pointers replaced by owned copies
  std::vector<std::vector<double>> h, a;
  std::vector<int> dims;
  std::vector<BInst> inst;                 // host copy (device pointers)
  void* d_tables = nullptr;                // all dz tables
  double* d_a = nullptr;                   // all X-field coefficients
  void* d_basis = nullptr;                 // all Krylov bases
  BInst* d_inst = nullptr;
  BItem* d_items = nullptr;
  int* d_queue = nullptr;
  BStat* d_stat = nullptr;
  BStat* h_stat = nullptr;                 // pinned
  double* d_scal = nullptr;
  double* h_scal = nullptr;                // pinned
  size_t scal_cap = 0;
  int* d_dec = nullptr;
  size_t dec_cap = 0;
  double2* d_tune_psi = nullptr;           // tuning states
  cfet_batch_plan plan{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

thread_local std::string g_batch_err;

cfet_status bfail(cfet_batch* b, cfet_status s, const std::string& m) {
  if (b) b->err = m; else g_batch_err = m;
  return s;
}

cfet_status bcuda(cfet_batch* b, cudaError_t e, const char* where) {
  return bfail(b, e == cudaErrorMemoryAllocation ? CFET_ENOMEM : CFET_ECUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

#define BCK(call, where)                                     \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return bcuda(b, _e, where);       \
  } while (0)

void free_batch(cfet_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaFree(b->d_tables); cudaFree(b->d_a); cudaFree(b->d_basis); cudaFree(b->d_inst); cudaFree(b->d_items);
  cudaFree(b->d_queue); cudaFree(b->d_stat); cudaFree(b->d_scal); cudaFree(b->d_dec); cudaFree(b->d_tune_psi);
  if (b->h_stat) cudaFreeHost(b->h_stat);
  if (b->h_scal) cudaFreeHost(b->h_scal);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  delete b;
}

bool is_fin(double v) { return std::isfinite(v); }

// Work items for a plan: instances with at least coop_min_sites sites alone on a
// cluster, the rest grouped cluster_size at a time with equal sizes together;
// items in order of decreasing work (longest first).
std::vector<BItem> make_items(const cfet_batch* b, const cfet_batch_plan& pl) {
  std::vector<int> order(b->n);
  for (int i = 0; i < b->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->dims[x] > b->dims[y]; });
  std::vector<BItem> items;
  std::vector<double> work;
  std::vector<int> small;
  for (int i : order) {
    if (pl.cluster_size > 1 && b->chains[i].nsites >= pl.coop_min_sites) {
      BItem it{};
      it.coop = 1;
      it.n = 1;
      it.inst[0] = i;
      items.push_back(it);
      work.push_back((double)b->dims[i] / pl.cluster_size);
    } else {
      small.push_back(i);
    }
  }
  for (size_t s = 0; s < small.size(); s += pl.cluster_size) {
    BItem it{};
    it.coop = 0;
    it.n = (int)std::min<size_t>(pl.cluster_size, small.size() - s);
    for (int r = 0; r < it.n; ++r) it.inst[r] = small[s + r];
    items.push_back(it);
    work.push_back((double)b->dims[small[s]]);
  }
  std::vector<int> idx(items.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return work[x] > work[y]; });
  std::vector<BItem> out;
  for (int i : idx) out.push_back(items[i]);
  return out;
}

cfet_status ensure_scal(cfet_batch* b, size_t n) {
  if (n <= b->scal_cap) return CFET_OK;
  cudaFree(b->d_scal);
  if (b->h_scal) cudaFreeHost(b->h_scal);
  b->d_scal = nullptr; b->h_scal = nullptr; b->scal_cap = 0;
  BCK(cudaMalloc(&b->d_scal, n * sizeof(double)), "cudaMalloc(scalars)");
  BCK(cudaMallocHost(&b->h_scal, n * sizeof(double)), "cudaMallocHost(scalars)");
  b->scal_cap = n;
  return CFET_OK;
}

// One launch over the batch with plan pl; psi_ptrs: device pointers per
// instance.  forced / record: per-instance decision logs (host) or NULL.
cfet_status run_batch(cfet_batch* b, const cfet_batch_plan& pl, double2* const* psi_ptrs, double t0, double dt,
                      int64_t nsteps, int32_t order, double tol, cudaStream_t s, const cfet_decisions* forced,
                      cfet_decisions* record, cfet_stats* stats, float* ms) {
  const int id = default_scheme_for_order(order);
  if (!id) return bfail(b, CFET_EINVAL, "order must be 2, 4, 6 or 8");
  SchemeData sd;
  build_scheme(id, &sd);
  const long long nexp = nsteps * (long long)sd.s;
  // stage scalars (host): c0 = sum_m g_{j,m}, c1 = sum_m g_{j,m} f(t + x_m dt)
  cfet_status st = ensure_scal(b, (size_t)b->n * nexp * 2);
  if (st != CFET_OK) return st;
  for (int i = 0; i < b->n; ++i) {
    const cfet_chain& c = b->chains[i];
    double* row = b->h_scal + (size_t)i * nexp * 2;
    for (long long n = 0; n < nsteps; ++n) {
      double fv[4];
      for (int m = 0; m < sd.M; ++m) {
        const double t = t0 + (double)n * dt + sd.x[m] * dt;
        fv[m] = c.f ? c.f(t, c.user) : c.A * std::cos(c.omega * t + c.phase);
        if (!is_fin(fv[m])) return bfail(b, CFET_EINVAL, "drive returned a non-finite value");
      }
      for (int jj = 0; jj < sd.s; ++jj) {
        const int j = sd.s - 1 - jj;  // exp(Omega_s) acts first
        double c0 = 0.0, c1 = 0.0;
        for (int m = 0; m < sd.M; ++m) {
          c0 += sd.g[j][m];
          c1 += sd.g[j][m] * fv[m];
        }
        row[2 * (n * sd.s + jj)] = c0;
        row[2 * (n * sd.s + jj) + 1] = c1;
      }
    }
  }
  // decisions
  std::vector<long long> f_nsub(b->n, -1), f_kh(b->n, -1), r_nsub(b->n, -1), r_kh(b->n, -1), r_cap(b->n, 0);
  std::vector<int> blob;
  long long fk_total = 0, rk_total = 0;
  if (forced) {
    for (int i = 0; i < b->n; ++i) {
      const cfet_decisions& d = forced[i];
      if (d.n_exp != nexp || !d.n_sub || !d.k || !d.h || d.len < nexp)
        return bfail(b, CFET_EINVAL, "forced decisions do not cover nsteps * s exponentials");
      long long tot = 0;
      for (long long e = 0; e < nexp; ++e) {
        if (d.n_sub[e] < 1) return bfail(b, CFET_EINVAL, "forced decisions: n_sub < 1");
        tot += d.n_sub[e];
      }
      if (tot != d.len) return bfail(b, CFET_EINVAL, "forced decisions: len mismatch");
      for (long long q = 0; q < tot; ++q)
        if (d.k[q] < 1 || d.k[q] > b->opt.m_max || d.h[q] < 0 || d.h[q] > 60)
          return bfail(b, CFET_EINVAL, "forced decisions: k or h out of range");
      fk_total += tot;
    }
  }
  if (record) {
    for (int i = 0; i < b->n; ++i) {
      const cfet_decisions& d = record[i];
      if (d.n_exp != nexp || !d.n_sub || !d.k || !d.h || d.cap < 0)
        return bfail(b, CFET_EINVAL, "record must cover nsteps * s exponentials");
      rk_total += d.cap;
    }
  }
  // layout: [f_nsub (n*nexp) | f_k | f_h | r_nsub (n*nexp) | r_k | r_h]
  const size_t nf = forced ? (size_t)b->n * nexp + 2 * fk_total : 0;
  const size_t nr = record ? (size_t)b->n * nexp + 2 * rk_total : 0;
  if (nf + nr > b->dec_cap) {
    cudaFree(b->d_dec);
    b->d_dec = nullptr;
    b->dec_cap = 0;
    BCK(cudaMalloc(&b->d_dec, (nf + nr) * sizeof(int)), "cudaMalloc(decisions)");
    b->dec_cap = nf + nr;
  }
  BParams p{};
  if (forced) {
    blob.resize(nf);
    long long pos = 0;
    for (int i = 0; i < b->n; ++i) {
      f_nsub[i] = (long long)i * nexp;
      f_kh[i] = pos;
      for (long long e = 0; e < nexp; ++e) blob[(size_t)i * nexp + e] = forced[i].n_sub[e];
      for (long long q = 0; q < forced[i].len; ++q) {
        blob[(size_t)b->n * nexp + pos + q] = forced[i].k[q];
        blob[(size_t)b->n * nexp + fk_total + pos + q] = forced[i].h[q];
      }
      pos += forced[i].len;
    }
    BCK(cudaMemcpy(b->d_dec, blob.data(), nf * sizeof(int), cudaMemcpyHostToDevice), "decision upload");
    p.f_nsub = b->d_dec;
    p.f_k = b->d_dec + (size_t)b->n * nexp;
    p.f_h = p.f_k + fk_total;
  }
  if (record) {
    int* r = b->d_dec + nf;
    long long pos = 0;
    for (int i = 0; i < b->n; ++i) {
      r_nsub[i] = (long long)i * nexp;
      r_kh[i] = pos;
      r_cap[i] = record[i].cap;
      pos += record[i].cap;
    }
    p.r_nsub = r;
    p.r_k = r + (size_t)b->n * nexp;
    p.r_h = p.r_k + rk_total;
  }
  // instance table for this call
  std::vector<BInst> inst = b->inst;
  for (int i = 0; i < b->n; ++i) {
    inst[i].psi = psi_ptrs[i];
    inst[i].scal = b->d_scal + (size_t)i * nexp * 2;
    inst[i].f_nsub = f_nsub[i];
    inst[i].f_kh = f_kh[i];
    inst[i].r_nsub = r_nsub[i];
    inst[i].r_kh = r_kh[i];
    inst[i].r_cap = r_cap[i];
  }
  const std::vector<BItem> items = make_items(b, pl);
  const int maxc = b->precision == CFET_PREC_C64 ? max_clusters<FmtC64>(pl.cluster_size, pl.threads)
                                                 : max_clusters<FmtF64>(pl.cluster_size, pl.threads);
  if (maxc < 1) return bfail(b, CFET_EINVAL, "plan cannot be launched (no cluster fits on the device)");
  const int clusters = std::min<int>((int)items.size(), maxc);
  // the previous launch may still read the tables: order on the stream
  BCK(cudaMemcpyAsync(b->d_scal, b->h_scal, (size_t)b->n * nexp * 2 * sizeof(double), cudaMemcpyHostToDevice, s),
      "scalar upload");
  BCK(cudaMemcpyAsync(b->d_inst, inst.data(), inst.size() * sizeof(BInst), cudaMemcpyHostToDevice, s),
      "instance upload");
  BCK(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice, s),
      "item upload");
  BCK(cudaMemsetAsync(b->d_queue, 0, sizeof(int), s), "queue reset");
  BCK(cudaMemsetAsync(b->d_stat, 0, (size_t)b->n * sizeof(BStat), s), "stat reset");
  p.inst = b->d_inst;
  p.items = b->d_items;
  p.nitems = (int)items.size();
  p.queue = b->d_queue;
  p.nexp = nexp;
  p.tau = dt;
  p.tol = tol;
  p.m_min = b->opt.m_min;
  p.m_max = b->opt.m_max;
  p.max_substeps = b->opt.max_substeps;
  p.stat = b->d_stat;
  BCK(cudaEventRecord(b->ev0, s), "event");
  const int e = b->precision == CFET_PREC_C64
                    ? launch_batch<FmtC64>(p, clusters, pl.cluster_size, pl.threads, s)
                    : launch_batch<FmtF64>(p, clusters, pl.cluster_size, pl.threads, s);
  if (e != cudaSuccess) return bcuda(b, (cudaError_t)e, "batch kernel launch");
  BCK(cudaEventRecord(b->ev1, s), "event");
  BCK(cudaMemcpyAsync(b->h_stat, b->d_stat, (size_t)b->n * sizeof(BStat), cudaMemcpyDeviceToHost, s),
      "stat read-back");
  BCK(cudaStreamSynchronize(s), "stream synchronize");
  if (ms) BCK(cudaEventElapsedTime(ms, b->ev0, b->ev1), "event time");
  if (record) {
    std::vector<int> rb(nr);
    BCK(cudaMemcpy(rb.data(), b->d_dec + nf, nr * sizeof(int), cudaMemcpyDeviceToHost), "record read-back");
    for (int i = 0; i < b->n; ++i) {
      long long len = 0;
      for (long long q = 0; q < nexp; ++q) {
        record[i].n_sub[q] = rb[(size_t)i * nexp + q];
        len += record[i].n_sub[q];
      }
      for (long long q = 0; q < record[i].cap && q < len; ++q) {
        record[i].k[q] = rb[(size_t)b->n * nexp + r_kh[i] + q];
        record[i].h[q] = rb[(size_t)b->n * nexp + rk_total + r_kh[i] + q];
      }
      record[i].len = len;
    }
  }
  int worst = 0;
  for (int i = 0; i < b->n; ++i) {
    const BStat& bs = b->h_stat[i];
    if (stats) {
      std::memset(&stats[i], 0, sizeof(cfet_stats));
      stats[i].n_exp = bs.n_exp;
      stats[i].n_substeps = bs.n_sub;
      stats[i].n_applies = bs.n_app;
      stats[i].max_k = bs.max_k;
      stats[i].status = bs.status;
      stats[i].max_err_est = bs.max_err;
    }
    if (bs.status != 0 && worst == 0) worst = bs.status;
  }
  if (worst == CFET_EKRYLOV) return bfail(b, CFET_EKRYLOV, "a stage exponential exceeded max_substeps");
  if (worst == CFET_ENAN) return bfail(b, CFET_ENAN, "an instance's psi is not finite");
  if (worst != 0) return bfail(b, (cfet_status)worst, "device error");
  return CFET_OK;
}

}  // namespace

extern "C" {

const char* cfet_batch_last_error(const cfet_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

void cfet_batch_destroy(cfet_batch* b) { free_batch(b); }

cfet_status cfet_batch_create(cfet_batch** out, int32_t n, const cfet_chain* chains, const cfet_options* opt) {
  g_batch_err.clear();
  if (!out) return bfail(nullptr, CFET_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !chains) return bfail(nullptr, CFET_EINVAL, "need n >= 1 chains");
  cfet_options o;
  cfet_options_default(&o);
  o.precision = CFET_PREC_F64;  // the batch default
  if (opt) o = *opt;
  if (o.precision == CFET_PREC_DEFAULT) o.precision = CFET_PREC_F64;
  if (o.precision != CFET_PREC_F64 && o.precision != CFET_PREC_C64)
    return bfail(nullptr, CFET_EINVAL, "batch precision must be CFET_PREC_F64 or CFET_PREC_C64");
  if (o.m_max < 1 || o.m_max > kMaxKrylov) return bfail(nullptr, CFET_EINVAL, "m_max must be in [1, 64]");
  if (o.m_min < 1 || o.m_min > o.m_max) return bfail(nullptr, CFET_EINVAL, "m_min must be in [1, m_max]");
  if (o.max_substeps < 1) return bfail(nullptr, CFET_EINVAL, "max_substeps must be >= 1");
  for (int i = 0; i < n; ++i) {
    const cfet_chain& c = chains[i];
    if (c.nsites < 1 || c.nsites > kBatchMaxSites) return bfail(nullptr, CFET_EINVAL, "nsites must be in [1, 24]");
    if (!c.h || !c.a) return bfail(nullptr, CFET_EINVAL, "chain h or a is NULL");
    if (!is_fin(c.J) || !is_fin(c.Delta)) return bfail(nullptr, CFET_EINVAL, "chain J, Delta not finite");
    for (int s = 0; s < c.nsites; ++s)
      if (!is_fin(c.h[s]) || !is_fin(c.a[s])) return bfail(nullptr, CFET_EINVAL, "chain h or a not finite");
    if (!c.f && (!is_fin(c.A) || !is_fin(c.omega) || !is_fin(c.phase)))
      return bfail(nullptr, CFET_EINVAL, "built-in drive parameters not finite");
  }
  {
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || nd == 0) {
      cudaGetLastError();
      return bfail(nullptr, CFET_ENODEV, "no CUDA device available");
    }
  }
  cfet_batch* b = new cfet_batch();
  cudaGetDevice(&b->device);
  b->n = n;
  b->precision = o.precision;
  b->opt = o;
  const size_t esz = o.precision == CFET_PREC_C64 ? sizeof(float2) : sizeof(double2);
  const size_t tsz = o.precision == CFET_PREC_C64 ? sizeof(float) : sizeof(double);
#define BCKC(call, where)                      \
  do {                                         \
    cudaError_t _e = (call);                   \
    if (_e != cudaSuccess) {                   \
      cfet_status _s = bcuda(nullptr, _e, where); \
      free_batch(b);                           \
      return _s;                               \
    }                                          \
  } while (0)
  size_t ntab = 0, na = 0, nbasis = 0, nstate = 0;
  std::vector<size_t> tab_off(n), a_off(n), basis_off(n), state_off(n);
  std::vector<int> Ls(n);
  for (int i = 0; i < n; ++i) {
    const cfet_chain& c = chains[i];
    b->chains.push_back(c);
    b->h.emplace_back(c.h, c.h + c.nsites);
    b->a.emplace_back(c.a, c.a + c.nsites);
    const int N = c.nsites, L = N < 10 ? N : 10;
    Ls[i] = L;
    b->dims.push_back(1 << N);
    tab_off[i] = ntab;
    ntab += (size_t(1) << L) + (size_t(1) << (N - L + 1));
    a_off[i] = na;
    na += N;
    basis_off[i] = nbasis;
    nbasis += (size_t)(o.m_max + 1) * (1 << N);
    state_off[i] = nstate;
    nstate += (size_t)1 << N;
  }
  BCKC(cudaMalloc(&b->d_tables, ntab * tsz), "cudaMalloc(tables)");
  BCKC(cudaMalloc(&b->d_a, na * sizeof(double)), "cudaMalloc(fields)");
  BCKC(cudaMalloc(&b->d_basis, nbasis * esz), "cudaMalloc(Krylov bases)");
  BCKC(cudaMalloc(&b->d_inst, n * sizeof(BInst)), "cudaMalloc(instances)");
  BCKC(cudaMalloc(&b->d_items, n * sizeof(BItem)), "cudaMalloc(items)");
  BCKC(cudaMalloc(&b->d_queue, sizeof(int)), "cudaMalloc(queue)");
  BCKC(cudaMalloc(&b->d_stat, n * sizeof(BStat)), "cudaMalloc(stats)");
  BCKC(cudaMallocHost(&b->h_stat, n * sizeof(BStat)), "cudaMallocHost(stats)");
  BCKC(cudaEventCreate(&b->ev0), "event");
  BCKC(cudaEventCreate(&b->ev1), "event");
  // diagonal tables: the FP64 table kernel per instance, converted for complex64
  {
    double *d_h = nullptr, *d_lo = nullptr;
    size_t maxtab = 0;
    for (int i = 0; i < n; ++i) {
      const int N = chains[i].nsites, L = Ls[i];
      maxtab = std::max(maxtab, (size_t(1) << L) + (size_t(1) << (N - L + 1)));
    }
    BCKC(cudaMalloc(&d_h, kBatchMaxSites * sizeof(double)), "cudaMalloc(h)");
    BCKC(cudaMalloc(&d_lo, maxtab * sizeof(double)), "cudaMalloc(table scratch)");
    std::vector<double> tmp(maxtab);
    std::vector<float> tmpf(maxtab);
    for (int i = 0; i < n; ++i) {
      const int N = chains[i].nsites, L = Ls[i];
      const size_t nlo = size_t(1) << L, nt = nlo + (size_t(1) << (N - L + 1));
      BCKC(cudaMemcpy(d_h, b->h[i].data(), N * sizeof(double), cudaMemcpyHostToDevice), "upload h");
      const int e = launch_spin_tables(N, L, chains[i].J, chains[i].Delta, d_h, d_lo, d_lo + nlo, nullptr);
      BCKC((cudaError_t)e, "spin table kernel");
      BCKC(cudaMemcpy(tmp.data(), d_lo, nt * sizeof(double), cudaMemcpyDeviceToHost), "download table");
      if (o.precision == CFET_PREC_C64) {
        for (size_t k = 0; k < nt; ++k) tmpf[k] = (float)tmp[k];
        BCKC(cudaMemcpy((float*)b->d_tables + tab_off[i], tmpf.data(), nt * sizeof(float), cudaMemcpyHostToDevice),
             "upload table");
      } else {
        BCKC(cudaMemcpy((double*)b->d_tables + tab_off[i], tmp.data(), nt * sizeof(double), cudaMemcpyHostToDevice),
             "upload table");
      }
      BCKC(cudaMemcpy(b->d_a + a_off[i], b->a[i].data(), N * sizeof(double), cudaMemcpyHostToDevice), "upload a");
    }
    cudaFree(d_h);
    cudaFree(d_lo);
  }
  for (int i = 0; i < n; ++i) {
    const cfet_chain& c = chains[i];
    BInst I{};
    I.N = c.nsites;
    I.L = Ls[i];
    bool uniform = true;
    for (int s = 1; s < c.nsites; ++s)
      if (c.a[s] != c.a[0]) uniform = false;
    I.uniform = uniform ? 1 : 0;
    I.dim = 1 << c.nsites;
    I.J2 = 2.0 * c.J;
    I.dz = (const char*)b->d_tables + tab_off[i] * tsz;
    I.a = b->d_a + a_off[i];
    I.basis = (char*)b->d_basis + basis_off[i] * esz;
    I.f_nsub = I.f_kh = I.r_nsub = I.r_kh = -1;
    b->inst.push_back(I);
    b->chains[i].h = b->h[i].data();
    b->chains[i].a = b->a[i].data();
  }
  // default plan: clusters of 4 CTAs of 256 threads, instances of the
  // largest size present (when more than 12 sites) spread over a cluster
  int nmax = 0;
  for (int i = 0; i < n; ++i) nmax = std::max(nmax, chains[i].nsites);
  b->plan.cluster_size = 4;
  b->plan.threads = 256;
  b->plan.coop_min_sites = nmax > 12 ? nmax : kBatchMaxSites + 1;
  b->plan.tuned_ms = 0.f;
#undef BCKC
  *out = b;
  return CFET_OK;
}

cfet_status cfet_batch_get_plan(const cfet_batch* b, cfet_batch_plan* plan) {
  if (!b || !plan) return CFET_EINVAL;
  *plan = b->plan;
  return CFET_OK;
}

cfet_status cfet_batch_set_plan(cfet_batch* b, const cfet_batch_plan* plan) {
  if (!b || !plan) return CFET_EINVAL;
  const int cs = plan->cluster_size, th = plan->threads;
  if (cs != 1 && cs != 2 && cs != 4 && cs != 8) return bfail(b, CFET_EINVAL, "cluster_size must be 1, 2, 4 or 8");
  if (th != 128 && th != 256 && th != 512) return bfail(b, CFET_EINVAL, "threads must be 128, 256 or 512");
  b->plan = *plan;
  return CFET_OK;
}

cfet_status cfet_batch_propagate(cfet_batch* b, void* const* psi, double t0, double dt, int64_t nsteps, int32_t order,
                                 double krylov_tol, void* stream, const cfet_decisions* forced,
                                 cfet_decisions* record, cfet_stats* stats) {
  if (!b) return CFET_EINVAL;
  if (!psi) return bfail(b, CFET_EINVAL, "psi is NULL");
  for (int i = 0; i < b->n; ++i) {
    if (!psi[i]) return bfail(b, CFET_EINVAL, "psi[i] is NULL");
    if (reinterpret_cast<uintptr_t>(psi[i]) % 16 != 0) return bfail(b, CFET_EINVAL, "psi[i] is not 16-byte aligned");
  }
  if (!is_fin(t0) || !is_fin(dt) || dt == 0.0) return bfail(b, CFET_EINVAL, "t0, dt must be finite, dt != 0");
  if (!is_fin(krylov_tol)) return bfail(b, CFET_EINVAL, "krylov_tol not finite");
  if (nsteps < 0) return bfail(b, CFET_EINVAL, "nsteps must be >= 0");
  if (!default_scheme_for_order(order)) return bfail(b, CFET_EINVAL, "order must be 2, 4, 6 or 8");
  if (nsteps == 0) {
    if (stats) std::memset(stats, 0, (size_t)b->n * sizeof(cfet_stats));
    return CFET_OK;
  }
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, CFET_ECUDA, "cudaSetDevice");
  std::vector<double2*> ptrs(b->n);
  for (int i = 0; i < b->n; ++i) ptrs[i] = (double2*)psi[i];
  return run_batch(b, b->plan, ptrs.data(), t0, dt, nsteps, order, krylov_tol, (cudaStream_t)stream, forced, record,
                   stats, nullptr);
}

cfet_status cfet_batch_kernel_time_ms(cfet_batch* b, float* ms) {
  if (!b || !ms) return CFET_EINVAL;
  cudaError_t e = cudaEventElapsedTime(ms, b->ev0, b->ev1);
  if (e != cudaSuccess) return bcuda(b, e, "event time");
  return CFET_OK;
}

cfet_status cfet_batch_tune(cfet_batch* b, double t0, double dt, int32_t order, double krylov_tol, int64_t nsteps,
                            void* stream, cfet_batch_plan* chosen) {
  if (!b) return CFET_EINVAL;
  if (!is_fin(t0) || !is_fin(dt) || dt == 0.0 || !is_fin(krylov_tol) || nsteps < 1)
    return bfail(b, CFET_EINVAL, "tune: t0, dt, tol must be finite, dt != 0, nsteps >= 1");
  if (!default_scheme_for_order(order)) return bfail(b, CFET_EINVAL, "order must be 2, 4, 6 or 8");
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, CFET_ECUDA, "cudaSetDevice");
  // tuning states: normalised deterministic pseudo-random vectors, reset before
  // every candidate so that each one does the same work
  size_t total = 0;
  std::vector<size_t> off(b->n);
  for (int i = 0; i < b->n; ++i) {
    off[i] = total;
    total += (size_t)b->dims[i];
  }
  if (!b->d_tune_psi) BCK(cudaMalloc(&b->d_tune_psi, total * sizeof(double2)), "cudaMalloc(tuning states)");
  std::vector<double2> host(total);
  unsigned long long z = 0x9E3779B97F4A7C15ull;
  for (int i = 0; i < b->n; ++i) {
    double nrm = 0.0;
    for (int k = 0; k < b->dims[i]; ++k) {
      z ^= z << 13; z ^= z >> 7; z ^= z << 17;
      const double re = (double)(z >> 11) * 0x1.0p-53 - 0.5;
      z ^= z << 13; z ^= z >> 7; z ^= z << 17;
      const double im = (double)(z >> 11) * 0x1.0p-53 - 0.5;
      host[off[i] + k] = make_double2(re, im);
      nrm += re * re + im * im;
    }
    const double sc = 1.0 / std::sqrt(nrm);
    for (int k = 0; k < b->dims[i]; ++k) {
      host[off[i] + k].x *= sc;
      host[off[i] + k].y *= sc;
    }
  }
  std::vector<double2*> ptrs(b->n);
  for (int i = 0; i < b->n; ++i) ptrs[i] = b->d_tune_psi + off[i];
  int nmax = 0;
  for (int i = 0; i < b->n; ++i) nmax = std::max(nmax, b->chains[i].nsites);
  std::vector<cfet_batch_plan> cands;
  for (int cs : {1, 2, 4, 8})
    for (int th : {128, 256, 512}) {
      if (cs == 1) {
        cands.push_back(cfet_batch_plan{cs, th, kBatchMaxSites + 1, 0.f});
        continue;
      }
      for (int thr : {nmax - 1, nmax, kBatchMaxSites + 1}) {
        if (thr < 1) continue;
        cands.push_back(cfet_batch_plan{cs, th, thr, 0.f});
      }
    }
  cfet_batch_plan best{};
  float best_ms = 0.f;
  for (const cfet_batch_plan& c : cands) {
    BCK(cudaMemcpy(b->d_tune_psi, host.data(), total * sizeof(double2), cudaMemcpyHostToDevice), "tuning states");
    float ms = 0.f;
    cfet_status s = run_batch(b, c, ptrs.data(), t0, dt, nsteps, order, krylov_tol, (cudaStream_t)stream, nullptr,
                              nullptr, nullptr, &ms);
    if (s == CFET_EINVAL) continue;  // the plan does not fit on this device
    if (s != CFET_OK) return s;
    if (best_ms == 0.f || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  if (best_ms == 0.f) return bfail(b, CFET_ECUDA, "tune: no plan could be launched");
  best.tuned_ms = best_ms;
  b->plan = best;
  if (chosen) *chosen = best;
  return CFET_OK;
}

int32_t cfet_batch_size(const cfet_batch* b) { return b ? b->n : 0; }

}  // extern "C"
