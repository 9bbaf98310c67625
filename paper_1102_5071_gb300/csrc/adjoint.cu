// Backward (adjoint) sweep of the gradient of the fidelity loss
// L = 1 - |<phi|psi(T)>|^2 with respect to piecewise-constant drive amplitudes
// (FP64, sm_103a).  The paper has no gradients; the method is the chain rule
// through the CFET steps of Sec. 4 Eq. (Ucf) with the stage operators of
// Sec. 7 Eq. (OmGLeg):
//
//   d<phi|psi(T)>/dA_k = sum over stages (n, j) of segment k of
//       gamma_{n,j} <lambda_after| dE |psi_before>,
//   dE = d/dc exp(-i tau (c0 H0 + c V)) = -i tau int_0^1 e^{-i tau (1-s) H} V e^{-i tau s H} ds.
//
// With a(r) = e^{+i tau r H} psi_after (= e^{-i tau s H} psi_before, r = 1 - s)
// and b(r) = e^{+i tau r H} lambda_after the stage term is
//   -i tau int_0^1 <b(r)| V |a(r)> dr.
// Both families live in the Krylov spaces of psi_after and lambda_after
// (Sec. 8.1; a Krylov space does not depend on the time): a(r) =
// beta_a V_a exp(i tau r T_a) e_1 and likewise for b, so the integrand is
// y_b(r)^H W y_a(r) with W = V_b^H V V_a (k_b x k_a), integrated by
// Gauss-Legendre quadrature in r.  The same bases give psi_before = a(1) and
// lambda_before = b(1): the forward states are recovered by the inverse
// unitary step, and the driver replaces the recovered state by a stored
// checkpoint at every launch boundary (the drift is reported).
//
// One persistent cooperative launch undoes a range of stage exponentials.
// The Lanczos processes of psi and lambda run jointly (one pass, one pair of
// reductions per iteration for both); W takes one pass per psi vector.  All
// reductions are per-CTA trees, one partial per value and CTA, a bounded grid
// barrier and fixed-order sums, so every CTA holds identical scalars.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cfet_internal.h"
#include "device_common.cuh"

namespace cfet {
namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjWarps = kAdjThreads / 32;
constexpr int kAdjVals = 2 * kAdjMaxK + 2;  // values of one reduction, at most

struct SmemAdj {
  double red[kAdjWarps][kAdjVals];
  double res[kAdjVals];
  double alpha[2][kAdjMaxK + 2];
  double beta[2][kAdjMaxK + 2];
  double scale[2][kAdjMaxK + 3];
  double yr[2][kAdjMaxK], yi[2][kAdjMaxK];
  double tr[kAdjMaxK], ti[kAdjMaxK];
  double Wr[kAdjMaxK][kAdjMaxK], Wi[kAdjMaxK][kAdjMaxK];
  double cre[2][kAdjMaxK], cim[2][kAdjMaxK];
  double bsite_raw[kMaxSites];
  double bsite[2][kMaxSites];
  double beta0[2];
  int k[2], active[2];
  int nq;   // Gauss-Legendre nodes of this stage integral (0: beyond the largest rule)
  int ok;
};

// Grid sum of n <= kAdjVals values per thread; result in S.res (all threads).
__device__ bool adj_reduce(SmemAdj& S, const double* v, int n, double* part, unsigned& gen, const AdjParams& p) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = gridDim.x;
  for (int i = 0; i < n; ++i) {
    double x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) S.red[warp][i] = x;
  }
  __syncthreads();
  if ((int)threadIdx.x < n) {
    double s = 0.0;
    for (int w = 0; w < kAdjWarps; ++w) s += S.red[w][threadIdx.x];
    part[(size_t)threadIdx.x * G + blockIdx.x] = s;
  }
  if (!grid_barrier(p.bar, gen, &p.st->status, p.timeout_ns, &S.ok)) return false;
  for (int i = warp; i < n; i += kAdjWarps) {
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += __ldcg(part + (size_t)i * G + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) S.res[i] = s;
  }
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(kAdjThreads) k_adjoint(AdjParams p, OpSpin op) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemAdj& S = *reinterpret_cast<SmemAdj*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31;
  const int dim = p.dim, N = op.N;
  const int G = gridDim.x;
  const int stride = G * blockDim.x;
  const int x0 = blockIdx.x * blockDim.x + tid;
  const bool lead = blockIdx.x == 0 && tid == 0;
  const double tau = p.tau;
  const bool fixed_k = p.tol <= 0.0;
  unsigned gen = 0;
  int slot = 0;
  auto part = [&]() {
    double* q = p.partials + (size_t)slot * kAdjVals * G;
    slot ^= 1;
    return q;
  };
  auto Qv = [&](int pp, int i) -> double2* {
    return i == 1 ? (pp == 0 ? p.psi : p.lam) : (pp == 0 ? p.Vp : p.Vl) + (size_t)(i - 2) * dim;
  };
  double v[kAdjVals];
  long long n_app = 0;

  // ---- entry: checkpoint, adjoint initial state, overlap, norms
  {
    for (int i = 0; i < 5; ++i) v[i] = 0.0;
    for (int x = x0; x < dim; x += stride) {
      double2 a = p.psi[x];
      if (p.ckpt) {
        const double2 c = p.ckpt[x];
        const double dx = a.x - c.x, dy = a.y - c.y;
        v[0] = fma(dx, dx, fma(dy, dy, v[0]));
        a = c;
        p.psi[x] = a;
      }
      double2 l;
      if (p.phi) {
        l = p.phi[x];
        p.lam[x] = l;
        v[1] = fma(l.x, a.x, fma(l.y, a.y, v[1]));   // Re conj(phi) psi
        v[2] = fma(l.x, a.y, fma(-l.y, a.x, v[2]));  // Im conj(phi) psi
      } else {
        l = p.lam[x];
      }
      v[3] = fma(a.x, a.x, fma(a.y, a.y, v[3]));
      v[4] = fma(l.x, l.x, fma(l.y, l.y, v[4]));
    }
    if (!adj_reduce(S, v, 5, part(), gen, p)) return;
    if (lead) {
      if (p.phi) {
        p.out[0] = S.res[1];
        p.out[1] = S.res[2];
      }
      p.out[2] = fmax(p.out[2], sqrt(S.res[0]));
    }
    if (tid == 0) {
      S.beta0[0] = sqrt(S.res[3]);
      S.beta0[1] = sqrt(S.res[4]);
    }
    __syncthreads();
  }

  for (long long e = p.e_hi - 1; e >= p.e_lo; --e) {
    const double c0 = p.c0[e], c1 = p.c1[e];
    if (tid < N) S.bsite_raw[tid] = c1 * __ldg(op.xf + tid);
    if (tid < 2) {
      const double b0 = S.beta0[tid];
      if (!(b0 < 1e300)) atomicCAS(&p.st->status, 0, (int)CFET_ENAN);
      S.scale[tid][1] = b0 > 0.0 ? 1.0 / b0 : 0.0;
      S.active[tid] = b0 > 0.0;
      S.k[tid] = 0;
    }
    __syncthreads();
    if (ld_volatile_i32(&p.st->status) != 0) return;
    // ---- joint Lanczos of psi_after (0) and lambda_after (1) under H_j
    for (int it = 1; it <= p.m_max; ++it) {
      const int act0 = S.active[0], act1 = S.active[1];
      if (!act0 && !act1) break;
      if (tid < N) {
        S.bsite[0][tid] = S.bsite_raw[tid] * S.scale[0][it];
        S.bsite[1][tid] = S.bsite_raw[tid] * S.scale[1][it];
      }
      __syncthreads();
      v[0] = v[1] = 0.0;
      for (int pp = 0; pp < 2; ++pp) {
        if (!(pp == 0 ? act0 : act1)) continue;
        const double s_it = S.scale[pp][it];
        SpinScaled sc;
        sc.cz = c0 * s_it;
        sc.cxx = c0 * op.J2 * s_it;
        const double bm = it > 1 ? S.beta[pp][it - 1] * S.scale[pp][it - 1] : 0.0;
        const double2* q = Qv(pp, it);
        const double2* qm = it > 1 ? Qv(pp, it - 1) : q;
        double2* u = Qv(pp, it + 1);
        double acc = 0.0;
        for (int x = x0; x < dim; x += stride) {
          double2 hv = apply_spin_at(q, x, op, sc, S.bsite[pp]);
          if (it > 1) {
            const double2 w = qm[x];
            hv.x = fma(-bm, w.x, hv.x);
            hv.y = fma(-bm, w.y, hv.y);
          }
          u[x] = hv;
          const double2 a = q[x];
          acc = fma(a.x, hv.x, fma(a.y, hv.y, acc));
        }
        v[pp] = acc;
      }
      if (!adj_reduce(S, v, 2, part(), gen, p)) return;
      const double al0 = S.res[0] * S.scale[0][it], al1 = S.res[1] * S.scale[1][it];
      v[0] = v[1] = 0.0;
      for (int pp = 0; pp < 2; ++pp) {
        if (!(pp == 0 ? act0 : act1)) continue;
        const double s_it = S.scale[pp][it];
        const double am = -(pp == 0 ? al0 : al1) * s_it;
        const double2* q = Qv(pp, it);
        double2* u = Qv(pp, it + 1);
        double acc = 0.0;
        for (int x = x0; x < dim; x += stride) {
          const double2 a = q[x];
          double2 w = u[x];
          w.x = fma(am, a.x, w.x);
          w.y = fma(am, a.y, w.y);
          u[x] = w;
          acc = fma(w.x, w.x, fma(w.y, w.y, acc));
        }
        v[pp] = acc;
      }
      if (!adj_reduce(S, v, 2, part(), gen, p)) return;
      n_app += act0 + act1;
      if (tid < 32) {
        for (int pp = 0; pp < 2; ++pp) {
          if (!(pp == 0 ? act0 : act1)) continue;
          const double al = pp == 0 ? al0 : al1;
          const double b = sqrt(S.res[pp]);
          const double prev_b = it > 1 ? S.beta[pp][it - 1] : 0.0;
          const bool breakdown = b <= 1e-13 * (fabs(al) + prev_b + 1.0);
          if (lane == 0) {
            S.alpha[pp][it] = al;
            S.beta[pp][it] = b;
            S.scale[pp][it + 1] = b > 0.0 ? 1.0 / b : 0.0;
          }
          __syncwarp();
          int acc_flag = 0;
          if (fixed_k) {
            acc_flag = (it == p.m_max) || breakdown;
          } else if (breakdown) {
            acc_flag = 1;
          } else if (it >= p.m_min &&
                     fabs(tau) * gersh_width(it, S.alpha[pp] + 1, S.beta[pp] + 1) <= 2.0 * it) {
            small_expm_e1(it, S.alpha[pp] + 1, S.beta[pp] + 1, tau, S.yr[pp], S.yi[pp], S.tr, S.ti);
            const double err = S.beta0[pp] * b * hypot(S.yr[pp][it - 1], S.yi[pp][it - 1]);
            acc_flag = err <= p.tol;
          }
          if (lane == 0 && acc_flag) {
            S.active[pp] = 0;
            S.k[pp] = it;
          }
          __syncwarp();
        }
      }
      __syncthreads();
    }
    if (S.active[0] || S.active[1]) {  // the adjoint sweep takes no substeps
      if (lead) atomicCAS(&p.st->status, 0, (int)CFET_EKRYLOV);
      return;
    }
    const int kp = S.k[0], kl = S.k[1];
    // Rule of the stage integral: the integrand is a sum of e^{i om' r} with
    // |om'| <= om = |tau| (width_psi + width_lambda); the n-node rule on [0, 1]
    // integrates e^{i om r} to 1e-14 for om up to 1.25 (6), 10 (12), 39.5 (24)
    // and 114 (48 nodes).  Beyond that the sweep gives up (CFET_EKRYLOV);
    // every CTA takes the same decision (identical scalars).
    if (tid < 32) {
      int nq = 6;
      if (kp > 0 && kl > 0) {
        const double om = fabs(tau) * (gersh_width(kp, S.alpha[0] + 1, S.beta[0] + 1) +
                                       gersh_width(kl, S.alpha[1] + 1, S.beta[1] + 1));
        nq = om <= 1.25 ? 6 : (om <= 10.0 ? 12 : (om <= 39.5 ? 24 : (om <= 114.0 ? 48 : 0)));
      }
      if (lane == 0) S.nq = nq;
    }
    __syncthreads();
    if (S.nq == 0) {
      if (lead) atomicCAS(&p.st->status, 0, (int)CFET_EKRYLOV);
      return;
    }
    // ---- W[i][j] = <v_lambda_i | V | v_psi_j> (normalised vectors), V = sum_i a_i X_i
    for (int j = 1; j <= kp; ++j) {
      for (int i = 0; i < 2 * kl; ++i) v[i] = 0.0;
      const double2* qa = Qv(0, j);
      for (int x = x0; x < dim; x += stride) {
        double vr = 0.0, vi = 0.0;
        for (int s = 0; s < N; ++s) {
          const double2 w = qa[x ^ (1 << s)];
          const double as = __ldg(op.xf + s);
          vr = fma(as, w.x, vr);
          vi = fma(as, w.y, vi);
        }
        for (int i = 1; i <= kl; ++i) {
          const double2 l = Qv(1, i)[x];
          v[2 * (i - 1)] = fma(l.x, vr, fma(l.y, vi, v[2 * (i - 1)]));
          v[2 * (i - 1) + 1] = fma(l.x, vi, fma(-l.y, vr, v[2 * (i - 1) + 1]));
        }
      }
      if (!adj_reduce(S, v, 2 * kl, part(), gen, p)) return;
      if (tid < kl) {
        const double f = S.scale[1][tid + 1] * S.scale[0][j];
        S.Wr[tid][j - 1] = S.res[2 * tid] * f;
        S.Wi[tid][j - 1] = S.res[2 * tid + 1] * f;
      }
      __syncthreads();
    }
    // ---- stage integral (warp 0) and gradient accumulation
    if (tid < 32 && kp > 0 && kl > 0) {
      const int nq = S.nq;
      const int q0 = nq == 6 ? p.nq6 : (nq == 12 ? p.nq12 : (nq == 24 ? p.nq24 : p.nq48));
      double Ir = 0.0, Ii = 0.0;
      for (int q = 0; q < nq; ++q) {
        const double r = p.glx[q0 + q], wq = p.glw[q0 + q];
        // y(r) = exp(+i tau r T) e_1
        small_expm_e1(kp, S.alpha[0] + 1, S.beta[0] + 1, -tau * r, S.yr[0], S.yi[0], S.tr, S.ti);
        small_expm_e1(kl, S.alpha[1] + 1, S.beta[1] + 1, -tau * r, S.yr[1], S.yi[1], S.tr, S.ti);
        double ar = 0.0, ai = 0.0;
        if (lane < kl) {
          double tr_ = 0.0, ti_ = 0.0;  // (W y_psi)_lane
          for (int j = 0; j < kp; ++j) {
            tr_ += S.Wr[lane][j] * S.yr[0][j] - S.Wi[lane][j] * S.yi[0][j];
            ti_ += S.Wr[lane][j] * S.yi[0][j] + S.Wi[lane][j] * S.yr[0][j];
          }
          const double br = S.yr[1][lane], bi = S.yi[1][lane];  // conj(y_lambda) * t
          ar = br * tr_ + bi * ti_;
          ai = br * ti_ - bi * tr_;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          ar += __shfl_xor_sync(0xffffffffu, ar, o);
          ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        Ir = fma(wq, ar, Ir);
        Ii = fma(wq, ai, Ii);
        __syncwarp();
      }
      if (lead) {
        // term = -i tau beta0_psi beta0_lambda I
        const double f = tau * S.beta0[0] * S.beta0[1] * p.gam[e];
        const int sg = p.seg[e];
        p.grad[2 * sg] += f * Ii;
        p.grad[2 * sg + 1] -= f * Ir;
      }
    }
    // ---- psi_before = a(1), lambda_before = b(1)
    if (tid < 32) {
      for (int pp = 0; pp < 2; ++pp) {
        const int k = S.k[pp];
        if (k > 0) small_expm_e1(k, S.alpha[pp] + 1, S.beta[pp] + 1, -tau, S.yr[pp], S.yi[pp], S.tr, S.ti);
        __syncwarp();
        for (int i = lane; i < k; i += 32) {
          const double f = S.beta0[pp] * S.scale[pp][i + 1];
          S.cre[pp][i] = f * S.yr[pp][i];
          S.cim[pp][i] = f * S.yi[pp][i];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    v[0] = v[1] = 0.0;
    for (int x = x0; x < dim; x += stride) {
      for (int pp = 0; pp < 2; ++pp) {
        double re = 0.0, im = 0.0;
        for (int i = 0; i < S.k[pp]; ++i) {
          const double2 w = Qv(pp, i + 1)[x];
          const double cr = S.cre[pp][i], ci = S.cim[pp][i];
          re = fma(cr, w.x, fma(-ci, w.y, re));
          im = fma(cr, w.y, fma(ci, w.x, im));
        }
        Qv(pp, 1)[x] = make_double2(re, im);
        v[pp] = fma(re, re, fma(im, im, v[pp]));
      }
    }
    if (!adj_reduce(S, v, 2, part(), gen, p)) return;
    if (tid == 0) {
      S.beta0[0] = sqrt(S.res[0]);
      S.beta0[1] = sqrt(S.res[1]);
    }
    __syncthreads();
  }
  if (lead) p.out[3] += (double)n_app;
}

}  // namespace

int launch_adjoint_spin(const AdjParams& p, const OpSpin& op, int grid, int block, void* stream) {
  if (block != kAdjThreads) return (int)cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = sizeof(SmemAdj);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_adjoint, p, op);
}

int max_coresident_blocks_adjoint(int block) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adjoint, block, sizeof(SmemAdj)) != cudaSuccess)
    return -1;
  return per * nsm;
}

}  // namespace cfet
