// Device kernels of the CFET/Krylov propagator (FP64, sm_103a).
//
// Alvermann & Fehske, arXiv:1102.5071.  The hot path is the stage
// exponential exp(-i tau H_j) psi of a CFET step (Sec. 4, Eq. (Ucf); Sec. 7,
// Eq. (OmGLeg)), evaluated by the Lanczos/Krylov method of Sec. 8.1.  The
// stage operator H_j = c_0 H0 + sum_k c_k V_k is never formed: the apply
// functions take the per-stage scalars (Sec. 8, weighted sums keep the
// sparsity pattern).
//
// Structure: one persistent cooperative kernel per launch runs a sequence of
// stage exponentials.  Every CTA walks a grid-stride slice of the vectors;
// the two scalar reductions of a Lanczos iteration (alpha, beta) go through a
// per-CTA warp-shuffle/shared-memory tree, one partial per CTA in global
// memory, and a bounded grid barrier; every CTA then sums the partials in the
// same fixed order, so all CTAs hold bit-identical alpha/beta and take the
// same adaptive decisions without a broadcast.  Warp 0 of each CTA evaluates
// the small exponential exp(-i tau T_k) e_1 of the tridiagonal Lanczos matrix.
// Operator families: XXZ chain with X fields, DIA, CSR, general Pauli sums,
// and the chain in the interaction picture; optionally every Lanczos vector is
// re-orthogonalised against all earlier ones (classical Gram-Schmidt).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cfet_internal.h"
#include "device_common.cuh"

namespace cfet {

struct Coefs {
  double c[1 + kMaxDrives];
};

// ------------------------------------------------------------------ apply
// DIA family: sum_d coef[opidx[d]] * val[d][r] * v[r + off[d]], coef pre-scaled.
__device__ __forceinline__ double2 apply_dia_at(const double2* q, int r, int dim, const OpDia& op,
                                                const double* copf) {
  double2 acc = make_double2(0.0, 0.0);
  for (int d = 0; d < op.ndiag; ++d) {
    const long long c = (long long)r + __ldg(op.off + d);
    if (c >= 0 && c < dim) {
      const double a = copf[__ldg(op.opidx + d)] * __ldg(op.val + (size_t)d * dim + r);
      const double2 w = q[c];
      acc.x = fma(a, w.x, acc.x);
      acc.y = fma(a, w.y, acc.y);
    }
  }
  return acc;
}

// CSR family: sum_o copf[o] sum_{e in row r of o} val[e] v[col[e]], with the
// complex values (vr + i vi) of Hermitian operators, coef pre-scaled.
__device__ __forceinline__ double2 apply_csr_at(const double2* q, int r, int dim, const OpCsr& op,
                                                const double* copf) {
  double ar = 0.0, ai = 0.0;
  for (int o = 0; o < op.nops; ++o) {
    const int* rp = op.rp + (size_t)o * (dim + 1);
    const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
    double sr = 0.0, si = 0.0;
    if (op.vi) {
      for (int e = e0; e < e1; ++e) {
        const double a = __ldg(op.vr + e), b = __ldg(op.vi + e);
        const double2 w = q[__ldg(op.col + e)];
        sr = fma(a, w.x, fma(-b, w.y, sr));
        si = fma(a, w.y, fma(b, w.x, si));
      }
    } else {
      for (int e = e0; e < e1; ++e) {
        const double a = __ldg(op.vr + e);
        const double2 w = q[__ldg(op.col + e)];
        sr = fma(a, w.x, sr);
        si = fma(a, w.y, si);
      }
    }
    ar = fma(copf[o], sr, ar);
    ai = fma(copf[o], si, ai);
  }
  return make_double2(ar, ai);
}

// The two stored-matrix families behind one name (DIA, CSR).
__device__ __forceinline__ double2 apply_sparse_at(const double2* q, int r, int dim, const OpDia& op,
                                                   const double* copf) {
  return apply_dia_at(q, r, dim, op, copf);
}
__device__ __forceinline__ double2 apply_sparse_at(const double2* q, int r, int dim, const OpCsr& op,
                                                   const double* copf) {
  return apply_csr_at(q, r, dim, op, copf);
}

// Pauli-sum family at index y: for every group of strings with X mask xm,
// the partner y ^ xm weighted by sum_t pc[t] (-1)^popc((y ^ xm) & z_t), with
// the strings of odd popc(x & z) contributing an imaginary weight (the phase
// i^popc(x & z) of the string; its sign is folded into pc).
// The Z-only group may come from per-operator tables (scal: the stage
// scalars c_o); groups whose strings all have real phases take real products.
__device__ __forceinline__ double2 apply_pauli_at(const double2* q, int y, const OpPauli& op, const double* pc,
                                                  const double* scal) {
  double ar = 0.0, ai = 0.0;
  if (op.nd > 0) {
    double d = 0.0;
    for (int j = 0; j < op.nd; ++j) d = fma(scal[op.dop[j]], __ldg(op.dtab + ((size_t)j << op.N) + y), d);
    const double2 w = q[y];
    ar = d * w.x;
    ai = d * w.y;
  }
  int t = __ldg(op.gstart + op.g0);
  for (int g = op.g0; g < op.ngroups; ++g) {
    const unsigned b = (unsigned)y ^ __ldg(op.gx + g);
    const int t1 = __ldg(op.gstart + g + 1);
    const double2 w = q[b];
    if (__ldg(op.greal + g)) {
      double cr = 0.0;
      for (; t < t1; ++t) cr += (__popc(b & __ldg(op.tz + t)) & 1) ? -pc[t] : pc[t];
      ar = fma(cr, w.x, ar);
      ai = fma(cr, w.y, ai);
    } else {
      double cr = 0.0, ci = 0.0;
      for (; t < t1; ++t) {
        const double c = (__popc(b & __ldg(op.tz + t)) & 1) ? -pc[t] : pc[t];
        if (__ldg(op.tim + t)) ci += c;
        else cr += c;
      }
      ar = fma(cr, w.x, fma(-ci, w.y, ar));
      ai = fma(cr, w.y, fma(ci, w.x, ai));
    }
  }
  return make_double2(ar, ai);
}

// Diagonal tables of a Pauli-sum context: strings [0, n0) are the Z-only group.
__global__ void k_pauli_diag_table(OpPauli op, int n0, double* dtab) {
  const size_t dim = (size_t)1 << op.N;
  for (size_t y = (size_t)blockIdx.x * blockDim.x + threadIdx.x; y < dim; y += (size_t)gridDim.x * blockDim.x) {
    for (int j = 0; j < op.nd; ++j) {
      double s = 0.0;
      for (int t = 0; t < n0; ++t)
        if (op.top[t] == op.dop[j]) s += (__popc((unsigned)y & op.tz[t]) & 1) ? -op.tc[t] : op.tc[t];
      dtab[((size_t)j << op.N) + y] = s;
    }
  }
}

// Interaction-picture spin apply at index x (OpSpinIP): sum over the single
// flips and the antiparallel-bond hops of x of the stage weight of the local
// spin configuration times the partner's amplitude (complex products).
__device__ __forceinline__ double2 apply_spin_ip_at(const double2* q, int x, int N, const double2* W) {
  double ar = 0.0, ai = 0.0;
  const unsigned ux = (unsigned)x;
  for (int i = 0; i < N; ++i) {
    const int b = (ux >> i) & 1u;
    int n = 0;  // s_{i-1} + s_{i+1} over existing neighbours, s = 1 - 2 bit
    if (i > 0) n += 1 - 2 * (int)((ux >> (i - 1)) & 1u);
    if (i < N - 1) n += 1 - 2 * (int)((ux >> (i + 1)) & 1u);
    const double2 w = W[i * kIPWeightsPerSite + b * 5 + n + 2];
    const double2 v = q[x ^ (1 << i)];
    ar = fma(w.x, v.x, fma(-w.y, v.y, ar));
    ai = fma(w.x, v.y, fma(w.y, v.x, ai));
  }
  unsigned anti = (ux ^ (ux >> 1)) & ((1u << (N - 1)) - 1u);
  while (anti) {
    const int i = __ffs(anti) - 1;
    anti &= anti - 1u;
    const int b = (ux >> i) & 1u;
    int m = 0;  // s_{i-1} - s_{i+2} over existing sites
    if (i > 0) m += 1 - 2 * (int)((ux >> (i - 1)) & 1u);
    if (i + 2 < N) m -= 1 - 2 * (int)((ux >> (i + 2)) & 1u);
    const double2 w = W[N * kIPWeightsPerSite + i * kIPWeightsPerSite + b * 5 + m + 2];
    const double2 v = q[x ^ (3 << i)];
    ar = fma(w.x, v.x, fma(-w.y, v.y, ar));
    ai = fma(w.x, v.y, fma(w.y, v.x, ai));
  }
  return make_double2(ar, ai);
}

// Offset of the interaction-picture weight table behind SmemLayout (16-byte aligned).
template <class L>
__host__ __device__ constexpr size_t ip_table_offset() { return (sizeof(L) + 15) & ~size_t(15); }

// ------------------------------------------------------------------ shared layout
struct SmemLayout {
  double red[32];
  double alpha[kMaxKrylov + 1];
  double beta[kMaxKrylov + 1];   // beta[i] = ||w_i|| (1-based i)
  double scale[kMaxKrylov + 2];  // scale[i] = 1 / ||q_i||  (q_1 = psi)
  double yr[kMaxKrylov], yi[kMaxKrylov];
  double tr[kMaxKrylov], ti[kMaxKrylov];
  double cre[kMaxKrylov], cim[kMaxKrylov];
  double bsite[kMaxSites];      // spin: scaled per-site X coefficients
  double bsite_raw[kMaxSites];  // spin: sum_k c_k a_{k,i} for the current exponential
  double copf[1 + kMaxDrives];  // dia: scaled per-operator coefficients
  double scal[1 + kMaxDrives];  // current stage scalars
  double bcast[4];
  int dec[4];                   // decision broadcast: accepted, k, h, pad
  int ok;
};

// ------------------------------------------------------------------ the persistent kernel
template <int FAMILY, class Op>
__global__ void __launch_bounds__(256) k_propagate(PropParams p, Op op) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemLayout& S = *reinterpret_cast<SmemLayout*>(smem_raw);
  const int tid = threadIdx.x;
  const int dim = p.dim;
  const int stride = gridDim.x * blockDim.x;
  const int x0 = blockIdx.x * blockDim.x + tid;
  const int G = gridDim.x;
  const int ncoef = 1 + p.nV;
  unsigned gen = 0;
  // three partial slots (phase A, phase B, norm): two uses of one slot are
  // always separated by a grid barrier on another slot
  double* part0 = p.partials;
  double* part1 = p.partials + G;
  double* part2 = p.partials + 2 * G;
  DevStatus* st = p.st;
  const bool lead = (blockIdx.x == 0 && tid == 0);
  const bool fixed_k = p.tol <= 0.0;
  const bool forced = p.f_nsub != nullptr;

  long long fpos = st->forced_pos;
  long long rpos = st->rec_pos;
  long long n_app = 0, n_sub = 0;
  int max_k = 0;
  double max_err = 0.0;

  auto vec = [&](int i) -> double2* { return i == 1 ? p.psi : p.basis + (size_t)(i - 2) * dim; };

  // initial norm of psi
  {
    double acc = 0.0;
    for (int x = x0; x < dim; x += stride) {
      const double2 v = p.psi[x];
      acc = fma(v.x, v.x, fma(v.y, v.y, acc));
    }
    const double s = block_sum(acc, S.red);
    if (tid == 0) part2[blockIdx.x] = s;
    if (!grid_barrier(p.bar, gen, &st->status, p.timeout_ns, &S.ok)) return;
    if (tid < 32) {
      const double t = sum_partials(part2);
      if (tid == 0) S.bcast[0] = sqrt(t);
    }
    __syncthreads();
  }
  double beta0 = S.bcast[0];

  for (long long e = 0; e < p.nexp; ++e) {
    // stage scalars of this exponential
    if (tid < ncoef) S.scal[tid] = p.scal[e * ncoef + tid];
    __syncthreads();
    if constexpr (FAMILY == kFamilySpin) {
      if (tid < op.N) {
        double bi = 0.0;
        for (int k = 0; k < p.nV; ++k) bi = fma(S.scal[1 + k], __ldg(op.xf + k * op.N + tid), bi);
        S.bsite_raw[tid] = bi;
      }
      __syncthreads();
    }
    if constexpr (FAMILY == kFamilyPauli) {  // string coefficients c_{top[t]} tc[t] of this exponential
      double* pc = reinterpret_cast<double*>(smem_raw + ip_table_offset<SmemLayout>());
      for (int t = tid; t < op.nterms; t += blockDim.x) pc[t] = S.scal[__ldg(op.top + t)] * __ldg(op.tc + t);
      __syncthreads();
    }
    if constexpr (FAMILY == kFamilySpinIP) {  // this exponential's stage weights
      double2* Wt = reinterpret_cast<double2*>(smem_raw + ip_table_offset<SmemLayout>());
      const double2* src = op.w + (size_t)(p.exp_base + e) * op.nw;
      for (int i = tid; i < op.nw; i += blockDim.x) Wt[i] = src[i];
      __syncthreads();
    }
    const long long eg = p.exp_base + e;
    const int nforced = forced ? p.f_nsub[eg] : 0;
    double remaining = p.tau;
    int nsub_e = 0;
    while (true) {
      if (!(beta0 < 1e300) || beta0 != beta0) {
        if (lead) atomicCAS(&st->status, 0, (int)CFET_ENAN);
        return;
      }
      if (nsub_e >= p.max_substeps || (forced && nsub_e >= nforced)) {
        if (lead) atomicCAS(&st->status, 0, (int)CFET_EKRYLOV);
        return;
      }
      int kf = -1, hf = 0;
      if (forced) {
        kf = p.f_k[fpos];
        hf = p.f_h[fpos];
      }
      int acc_k = 0, acc_h = 0;
      double acc_err = 0.0;
      if (beta0 == 0.0) {
        // zero vector: exp(-i tau H) 0 = 0
        acc_k = 0;
      } else {
        if (tid == 0) S.scale[1] = 1.0 / beta0;
        __syncthreads();
        const int klimit = forced ? kf : p.m_max;
        bool accepted = false;
        int it = 1;
        for (;; ++it) {
          // ---------------- phase A: u = s_it H q_it - beta_{it-1} s_{it-1} q_{it-1}
          const double s_it = S.scale[it];
          const double2* q = vec(it);
          const double2* qm = it > 1 ? vec(it - 1) : nullptr;
          double2* u = vec(it + 1);
          const double bm = it > 1 ? S.beta[it - 1] * S.scale[it - 1] : 0.0;
          if constexpr (FAMILY == kFamilySpin) {
            if (tid < op.N) S.bsite[tid] = S.bsite_raw[tid] * s_it;
          } else {
            if (tid < ncoef) S.copf[tid] = S.scal[tid] * s_it;
          }
          __syncthreads();
          double acc = 0.0;
          if constexpr (FAMILY == kFamilySpin) {
            SpinScaled sc;
            sc.cz = S.scal[0] * s_it;
            sc.cxx = S.scal[0] * s_it * op.J2;
            for (int x = x0; x < dim; x += stride) {
              double2 hv = apply_spin_at(q, x, op, sc, S.bsite);
              if (qm) {
                const double2 w = qm[x];
                hv.x = fma(-bm, w.x, hv.x);
                hv.y = fma(-bm, w.y, hv.y);
              }
              u[x] = hv;
              const double2 v = q[x];
              acc = fma(v.x, hv.x, fma(v.y, hv.y, acc));
            }
          } else if constexpr (FAMILY == kFamilyPauli) {
            const double* pc = reinterpret_cast<const double*>(smem_raw + ip_table_offset<SmemLayout>());
            for (int x = x0; x < dim; x += stride) {
              double2 hv = apply_pauli_at(q, x, op, pc, S.scal);
              hv.x *= s_it;
              hv.y *= s_it;
              if (qm) {
                const double2 w = qm[x];
                hv.x = fma(-bm, w.x, hv.x);
                hv.y = fma(-bm, w.y, hv.y);
              }
              u[x] = hv;
              const double2 v = q[x];
              acc = fma(v.x, hv.x, fma(v.y, hv.y, acc));
            }
          } else if constexpr (FAMILY == kFamilySpinIP) {
            const double2* Wt = reinterpret_cast<const double2*>(smem_raw + ip_table_offset<SmemLayout>());
            for (int x = x0; x < dim; x += stride) {
              double2 hv = apply_spin_ip_at(q, x, op.N, Wt);
              hv.x *= s_it;
              hv.y *= s_it;
              if (qm) {
                const double2 w = qm[x];
                hv.x = fma(-bm, w.x, hv.x);
                hv.y = fma(-bm, w.y, hv.y);
              }
              u[x] = hv;
              const double2 v = q[x];
              acc = fma(v.x, hv.x, fma(v.y, hv.y, acc));
            }
          } else {
            for (int x = x0; x < dim; x += stride) {
              double2 hv = apply_sparse_at(q, x, dim, op, S.copf);
              if (qm) {
                const double2 w = qm[x];
                hv.x = fma(-bm, w.x, hv.x);
                hv.y = fma(-bm, w.y, hv.y);
              }
              u[x] = hv;
              const double2 v = q[x];
              acc = fma(v.x, hv.x, fma(v.y, hv.y, acc));
            }
          }
          {
            const double s = block_sum(acc, S.red);
            if (tid == 0) part0[blockIdx.x] = s;
          }
          if (!grid_barrier(p.bar, gen, &st->status, p.timeout_ns, &S.ok)) return;
          if (tid < 32) {
            const double t = sum_partials(part0);
            if (tid == 0) S.alpha[it] = t * s_it;
          }
          __syncthreads();
          // ---------------- phase B: w = u - alpha s_it q_it, beta = ||w||
          const double am = S.alpha[it] * s_it;
          acc = 0.0;
          for (int x = x0; x < dim; x += stride) {
            const double2 v = q[x];
            double2 w = u[x];
            w.x = fma(-am, v.x, w.x);
            w.y = fma(-am, v.y, w.y);
            u[x] = w;
            acc = fma(w.x, w.x, fma(w.y, w.y, acc));
          }
          {
            const double s = block_sum(acc, S.red);
            if (tid == 0) part1[blockIdx.x] = s;
          }
          if (!grid_barrier(p.bar, gen, &st->status, p.timeout_ns, &S.ok)) return;
          if (p.reorth) {
            // ---------------- full re-orthogonalisation (option): one classical
            // Gram-Schmidt sweep w <- w - sum_i v_i <v_i, w> over the stored
            // q_i = v_i / scale[i]; ||w||^2 is then taken again into part1
            double* partQ = p.partials + 3 * (size_t)G;  // 2 it doubles per CTA
            for (int i = 1; i <= it; ++i) {
              const double2* qi = vec(i);
              double ar = 0.0, ai = 0.0;
              for (int x = x0; x < dim; x += stride) {
                const double2 a = qi[x], w = u[x];
                ar = fma(a.x, w.x, fma(a.y, w.y, ar));   // conj(q_i) w
                ai = fma(a.x, w.y, fma(-a.y, w.x, ai));
              }
              const double sr = block_sum(ar, S.red);
              __syncthreads();
              const double si = block_sum(ai, S.red);
              if (tid == 0) {
                partQ[(size_t)(2 * (i - 1)) * G + blockIdx.x] = sr;
                partQ[(size_t)(2 * (i - 1) + 1) * G + blockIdx.x] = si;
              }
              __syncthreads();
            }
            if (!grid_barrier(p.bar, gen, &st->status, p.timeout_ns, &S.ok)) return;
            if (tid < 32) {
              for (int i = 1; i <= it; ++i) {
                const double sc2 = S.scale[i] * S.scale[i];
                const double cr = sum_partials(partQ + (size_t)(2 * (i - 1)) * G) * sc2;
                const double ci = sum_partials(partQ + (size_t)(2 * (i - 1) + 1) * G) * sc2;
                if (tid == 0) {
                  S.cre[i - 1] = cr;
                  S.cim[i - 1] = ci;
                }
              }
            }
            __syncthreads();
            acc = 0.0;
            for (int x = x0; x < dim; x += stride) {
              double2 w = u[x];
              for (int i = 1; i <= it; ++i) {
                const double2 a = vec(i)[x];
                const double cr = S.cre[i - 1], ci = S.cim[i - 1];
                w.x -= cr * a.x - ci * a.y;
                w.y -= cr * a.y + ci * a.x;
              }
              u[x] = w;
              acc = fma(w.x, w.x, fma(w.y, w.y, acc));
            }
            {
              const double s2 = block_sum(acc, S.red);
              if (tid == 0) part1[blockIdx.x] = s2;
            }
            if (!grid_barrier(p.bar, gen, &st->status, p.timeout_ns, &S.ok)) return;
          }
          // ---------------- decision (warp 0)
          if (tid < 32) {
            const double t = sum_partials(part1);
            const double b = sqrt(t);
            const double prev_b = it > 1 ? S.beta[it - 1] : 0.0;
            const bool breakdown =
                sb_no_breakdown(b, S.alpha[it], prev_b) != 1 && b <= 1e-13 * (fabs(S.alpha[it]) + prev_b + 1.0);
            int acc_flag = 0;
            double err = 0.0;
            if (forced) {
              acc_flag = (it == kf);
            } else if (fixed_k) {
              acc_flag = (it == p.m_max) || breakdown;
            } else if (breakdown) {
              acc_flag = 1;
            } else if (it >= p.m_min && gersh_gate(it, S.alpha + 1, S.beta + 1, remaining)) {
              // T_it: diagonal alpha[1..it], off-diagonal beta[1..it-1]; the
              // estimate is evaluated only where Eq. (KryErr) applies
              const double thr = p.tol * remaining / p.tau;
              if (krylov_lead_rejects(it, S.alpha + 1, S.beta + 1, remaining, beta0 * b, thr)) {
                err = 2.0 * thr + 1e-300;
              } else {
                small_expm_e1(it, S.alpha + 1, S.beta + 1, remaining, S.yr, S.yi, S.tr, S.ti);
                const double yk = hypot(S.yr[it - 1], S.yi[it - 1]);
                err = beta0 * b * yk;
                acc_flag = err <= thr;
              }
            }
            if (tid == 0) {
              S.beta[it] = b;
              S.scale[it + 1] = 1.0 / b;
              S.dec[0] = acc_flag;
              S.bcast[1] = err;
            }
          }
          __syncthreads();
          if (S.dec[0]) {
            accepted = true;
            acc_err = S.bcast[1];
            break;
          }
          if (it >= klimit) break;
        }
        acc_k = it;
        acc_h = 0;
        if (forced) {
          acc_h = hf;
        } else if (!accepted) {
          // halve the substep on the same basis (T_{m_max}) until the estimate
          // meets the proportional tolerance
          if (tid < 32) {
            int hh = 0;
            double err = 0.0;
            const double width = gersh_width(it, S.alpha + 1, S.beta + 1);
            for (int h = 1; h <= 40; ++h) {
              const double ts = ldexp(remaining, -h);
              if (!(fabs(ts) * width <= 2.0 * it)) continue;
              small_expm_e1(it, S.alpha + 1, S.beta + 1, ts, S.yr, S.yi, S.tr, S.ti);
              err = beta0 * S.beta[it] * hypot(S.yr[it - 1], S.yi[it - 1]);
              if (err <= p.tol * ts / p.tau) { hh = h; break; }
            }
            if (tid == 0) { S.dec[2] = hh; S.bcast[1] = err; }
          }
          __syncthreads();
          acc_h = S.dec[2];
          acc_err = S.bcast[1];
          if (acc_h == 0) {
            if (lead) atomicCAS(&st->status, 0, (int)CFET_EKRYLOV);
            return;
          }
        }
        n_app += it;
      }
      const double ts = ldexp(remaining, -acc_h);
      if (acc_k > 0) {
        // ---------------- reconstruct psi <- beta0 sum_i y_i q_i / ||q_i||
        if (tid < 32) {
          small_expm_e1(acc_k, S.alpha + 1, S.beta + 1, ts, S.yr, S.yi, S.tr, S.ti);
          for (int i = tid; i < acc_k; i += 32) {
            const double f = beta0 * S.scale[i + 1];
            S.cre[i] = f * S.yr[i];
            S.cim[i] = f * S.yi[i];
          }
        }
        __syncthreads();
        double acc = 0.0;
        for (int x = x0; x < dim; x += stride) {
          double re = 0.0, im = 0.0;
          for (int i = 0; i < acc_k; ++i) {
            const double2 v = vec(i + 1)[x];
            const double cr = S.cre[i], ci = S.cim[i];
            re = fma(cr, v.x, re);
            re = fma(-ci, v.y, re);
            im = fma(cr, v.y, im);
            im = fma(ci, v.x, im);
          }
          p.psi[x] = make_double2(re, im);
          acc = fma(re, re, fma(im, im, acc));
        }
        {
          const double s = block_sum(acc, S.red);
          if (tid == 0) part2[blockIdx.x] = s;
        }
        if (!grid_barrier(p.bar, gen, &st->status, p.timeout_ns, &S.ok)) return;
        if (tid < 32) {
          const double t = sum_partials(part2);
          if (tid == 0) S.bcast[0] = sqrt(t);
        }
        __syncthreads();
        beta0 = S.bcast[0];
      }
      // ---------------- bookkeeping (identical in every CTA; CTA 0 writes)
      if (lead) {
        if (p.r_k != nullptr) {
          if (rpos < p.r_cap) {
            p.r_k[rpos] = acc_k;
            p.r_h[rpos] = acc_h;
          } else {
            st->rec_overflow = 1;
          }
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
    if (lead && p.r_nsub != nullptr) p.r_nsub[eg] = nsub_e;
  }
  if (lead) {
    st->forced_pos = fpos;
    st->rec_pos = rpos;
    st->n_exp += p.nexp;
    st->n_sub += n_sub;
    st->n_app += n_app;
    if (max_k > st->max_k) st->max_k = max_k;
    if (max_err > st->max_err) st->max_err = max_err;
  }
}

// ------------------------------------------------------------------ standalone apply
template <int FAMILY, class Op>
__global__ void k_apply(Op op, int dim, Coefs c, int nV, const double2* __restrict__ vin, double2* __restrict__ vout) {
  __shared__ double bsite[kMaxSites];
  __shared__ double copf[1 + kMaxDrives];
  extern __shared__ double pc[];  // Pauli family: string coefficients
  if constexpr (FAMILY == kFamilyPauli) {
    for (int t = threadIdx.x; t < op.nterms; t += blockDim.x) pc[t] = c.c[op.top[t]] * op.tc[t];
  } else if constexpr (FAMILY == kFamilySpin) {
    if (threadIdx.x < (unsigned)op.N) {
      double bi = 0.0;
      for (int k = 0; k < nV; ++k) bi = fma(c.c[1 + k], op.xf[k * op.N + threadIdx.x], bi);
      bsite[threadIdx.x] = bi;
    }
  } else {
    if (threadIdx.x < (unsigned)(1 + nV)) copf[threadIdx.x] = c.c[threadIdx.x];
  }
  __syncthreads();
  const int stride = gridDim.x * blockDim.x;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += stride) {
    if constexpr (FAMILY == kFamilySpin) {
      SpinScaled sc;
      sc.cz = c.c[0];
      sc.cxx = c.c[0] * op.J2;
      vout[x] = apply_spin_at(vin, x, op, sc, bsite);
    } else if constexpr (FAMILY == kFamilyPauli) {
      vout[x] = apply_pauli_at(vin, x, op, pc, c.c);
    } else {
      vout[x] = apply_sparse_at(vin, x, dim, op, copf);
    }
  }
}

// Diagonal tables of the XXZ chain: dz(x) = dz_lo[x & (2^L-1)] + dz_hi[x >> (L-1)]
//   dz_lo: J Delta sum_{i < L-1} s_i s_{i+1} + sum_{i < L} h_i s_i
//   dz_hi: J Delta sum_{L-1 <= i < N-1} s_i s_{i+1} + sum_{L <= i < N} h_i s_i
// (the index of dz_hi holds bits L-1 .. N-1 of x).
__global__ void k_spin_tables(int N, int L, double J, double Delta, const double* h, double* dz_lo, double* dz_hi) {
  const int nlo = 1 << L, nhi = 1 << (N - L + 1);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nlo) {
    const int y = t;
    double v = 0.0;
    for (int i = 0; i + 1 < L; ++i) {
      const double si = 1.0 - 2.0 * ((y >> i) & 1), sj = 1.0 - 2.0 * ((y >> (i + 1)) & 1);
      v += J * Delta * si * sj;
    }
    for (int i = 0; i < L; ++i) v += h[i] * (1.0 - 2.0 * ((y >> i) & 1));
    dz_lo[t] = v;
  } else if (t < nlo + nhi) {
    const int y = t - nlo;  // bit j of y is bit (L-1+j) of x
    double v = 0.0;
    for (int i = L - 1; i + 1 < N; ++i) {
      const int j = i - (L - 1);
      const double si = 1.0 - 2.0 * ((y >> j) & 1), sj = 1.0 - 2.0 * ((y >> (j + 1)) & 1);
      v += J * Delta * si * sj;
    }
    for (int i = L; i < N; ++i) v += h[i] * (1.0 - 2.0 * ((y >> (i - (L - 1))) & 1));
    dz_hi[t - nlo] = v;
  }
}

// ------------------------------------------------------------------ launchers
size_t propagate_smem_bytes(int /*block*/) { return sizeof(SmemLayout); }

template <int FAMILY, class Op>
static int launch_prop(const PropParams& p, const Op& op, int grid, int block, void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = sizeof(SmemLayout);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_propagate<FAMILY, Op>, p, op);
}

int launch_propagate_spin(const PropParams& p, const OpSpin& op, int grid, int block, void* stream) {
  return launch_prop<kFamilySpin>(p, op, grid, block, stream);
}
int launch_propagate_dia(const PropParams& p, const OpDia& op, int grid, int block, void* stream) {
  return launch_prop<kFamilyDia>(p, op, grid, block, stream);
}
int launch_propagate_csr(const PropParams& p, const OpCsr& op, int grid, int block, void* stream) {
  return launch_prop<kFamilyCsr>(p, op, grid, block, stream);
}
int launch_propagate_pauli(const PropParams& p, const OpPauli& op, int grid, int block, void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = ip_table_offset<SmemLayout>() + (size_t)op.nterms * sizeof(double);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_propagate<kFamilyPauli, OpPauli>, p, op);
}
int launch_propagate_spin_ip(const PropParams& p, const OpSpinIP& op, int grid, int block, void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = ip_table_offset<SmemLayout>() + (size_t)op.nw * sizeof(double2);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_propagate<kFamilySpinIP, OpSpinIP>, p, op);
}

// psi[x] *= exp(i sign d(x) t[which]), d = diagonal of the XXZ chain H0
__global__ void k_phase_diag(double2* psi, OpSpin op, int dim, const double* t, int which, double sign) {
  const double tt = sign * t[which];
  const int L = op.lo_bits;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += gridDim.x * blockDim.x) {
    const double d = __ldg(op.dz_lo + (x & ((1 << L) - 1))) + __ldg(op.dz_hi + (x >> (L - 1)));
    double sn, cs;
    sincos(d * tt, &sn, &cs);
    const double2 v = psi[x];
    psi[x] = make_double2(cs * v.x - sn * v.y, sn * v.x + cs * v.y);
  }
}

int launch_phase_diag(double2* psi, const OpSpin& op, int dim, const double* t, int which, double sign, void* stream) {
  int g = (dim + 255) / 256;
  g = g < 1 ? 1 : (g > 4096 ? 4096 : g);
  k_phase_diag<<<g, 256, 0, (cudaStream_t)stream>>>(psi, op, dim, t, which, sign);
  return (int)cudaGetLastError();
}

int max_coresident_blocks(int family, int block) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (family == kFamilySpin)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate<kFamilySpin, OpSpin>, block, sizeof(SmemLayout));
  else if (family == kFamilyCsr)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate<kFamilyCsr, OpCsr>, block, sizeof(SmemLayout));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate<kFamilyDia, OpDia>, block, sizeof(SmemLayout));
  if (e != cudaSuccess) return -1;
  return per * nsm;
}

int max_coresident_blocks_ip(int block, int nw) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = ip_table_offset<SmemLayout>() + (size_t)nw * sizeof(double2);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate<kFamilySpinIP, OpSpinIP>, block, smem) !=
      cudaSuccess)
    return -1;
  return per * nsm;
}

int max_coresident_blocks_pauli(int block, int nterms) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = ip_table_offset<SmemLayout>() + (size_t)nterms * sizeof(double);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_propagate<kFamilyPauli, OpPauli>, block, smem) !=
      cudaSuccess)
    return -1;
  return per * nsm;
}

static int apply_grid(int dim, int block) {
  int g = (dim + block - 1) / block;
  return g < 1 ? 1 : (g > 65535 ? 65535 : g);
}

int launch_apply_spin(const OpSpin& op, int dim, const double* c, int nV, const double2* vin, double2* vout,
                      void* stream) {
  Coefs cc = {};
  for (int i = 0; i < 1 + nV; ++i) cc.c[i] = c[i];
  k_apply<kFamilySpin, OpSpin><<<apply_grid(dim, 256), 256, 0, (cudaStream_t)stream>>>(op, dim, cc, nV, vin, vout);
  return (int)cudaGetLastError();
}
int launch_apply_dia(const OpDia& op, int dim, const double* c, int nV, const double2* vin, double2* vout,
                     void* stream) {
  Coefs cc = {};
  for (int i = 0; i < 1 + nV; ++i) cc.c[i] = c[i];
  k_apply<kFamilyDia, OpDia><<<apply_grid(dim, 256), 256, 0, (cudaStream_t)stream>>>(op, dim, cc, nV, vin, vout);
  return (int)cudaGetLastError();
}
int launch_apply_csr(const OpCsr& op, int dim, const double* c, int nV, const double2* vin, double2* vout,
                     void* stream) {
  Coefs cc = {};
  for (int i = 0; i < 1 + nV; ++i) cc.c[i] = c[i];
  k_apply<kFamilyCsr, OpCsr><<<apply_grid(dim, 256), 256, 0, (cudaStream_t)stream>>>(op, dim, cc, nV, vin, vout);
  return (int)cudaGetLastError();
}
int launch_pauli_diag_table(const OpPauli& op, int n0, double* dtab, void* stream) {
  const size_t dim = (size_t)1 << op.N;
  size_t g = (dim + 255) / 256;
  if (g > 4096) g = 4096;
  k_pauli_diag_table<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(op, n0, dtab);
  return (int)cudaGetLastError();
}
int launch_apply_pauli(const OpPauli& op, int dim, const double* c, int nV, const double2* vin, double2* vout,
                       void* stream) {
  Coefs cc = {};
  for (int i = 0; i < 1 + nV; ++i) cc.c[i] = c[i];
  k_apply<kFamilyPauli, OpPauli><<<apply_grid(dim, 256), 256, (size_t)op.nterms * sizeof(double),
                                   (cudaStream_t)stream>>>(op, dim, cc, nV, vin, vout);
  return (int)cudaGetLastError();
}
int launch_spin_tables(int N, int L, double J, double Delta, const double* h, double* dz_lo, double* dz_hi,
                       void* stream) {
  const int n = (1 << L) + (1 << (N - L + 1));
  k_spin_tables<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(N, L, J, Delta, h, dz_lo, dz_hi);
  return (int)cudaGetLastError();
}

}  // namespace cfet

// ------------------------------------------------------------------ wait-limit self test
namespace cfet {
namespace {
// Two CTAs of one warp: CTA 0 enters a grid-wide wait (record exchange or
// grid barrier) that CTA 1 never joins; the wait gives up after timeout_ns,
// records CFET_ETIMEOUT and returns.  Exercises the bounded-wait path of the
// persistent kernels without a fault or a hang.
__global__ void k_wait_selftest(int which, unsigned long long* rec, unsigned* bar, int* status,
                                long long timeout_ns) {
  __shared__ int s_ok;
  if (blockIdx.x != 0) return;  // never publishes, never arrives
  if (which == 0) {
    struct NoAcc {
      __device__ void reset() {}
      __device__ void add(const unsigned (&)[1]) {}
    } acc;
    const unsigned mine[1] = {0u};
    long long spin = 0;
    ctl_exchange<1>(rec, mine, 1u, false, status, timeout_ns, spin, acc);
  } else {
    unsigned gen = 0;
    grid_barrier(bar, gen, status, timeout_ns, &s_ok);
  }
}
}  // namespace

int launch_wait_selftest(int which, unsigned long long* rec, unsigned* bar, int* status, long long timeout_ns) {
  k_wait_selftest<<<2, 32>>>(which, rec, bar, status, timeout_ns);
  return (int)cudaGetLastError();
}
// ||a - b||_2^2 partial sums: block j writes the sum over its grid-stride
// elements (tree in shared memory, fixed order) to part[j]; the host adds the
// partials in block order.  Used by the time-step selection (Sec. 6.6).
__global__ void __launch_bounds__(256) k_diff_norm2(const double2* __restrict__ a, const double2* __restrict__ b,
                                                    int n, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 x = a[i], y = b[i];
    const double dr = x.x - y.x, di = x.y - y.y;
    s = fma(dr, dr, fma(di, di, s));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

int launch_diff_norm2(const double2* a, const double2* b, int n, double* part, int nblk, void* stream) {
  k_diff_norm2<<<nblk, 256, 0, (cudaStream_t)stream>>>(a, b, n, part);
  return (int)cudaGetLastError();
}

// Copy-bandwidth probe: `reps` grid-stride copies of n 16-byte units inside
// one launch, alternating a -> b and b -> a (each copy reads what the
// previous one wrote, so none can be elided), four units in flight per
// thread.  With a and b together smaller than L2 this measures the L2-served
// copy rate; larger buffers give the DRAM copy rate.
__global__ void __launch_bounds__(512) k_copy_probe(int4* a, int4* b, long long n, int reps) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (int r = 0; r < reps; ++r) {
    const int4* src = (r & 1) ? b : a;
    int4* dst = (r & 1) ? a : b;
    long long i = t;
    for (; i + 3 * stride < n; i += 4 * stride) {
      const int4 v0 = src[i], v1 = src[i + stride], v2 = src[i + 2 * stride], v3 = src[i + 3 * stride];
      dst[i] = v0;
      dst[i + stride] = v1;
      dst[i + 2 * stride] = v2;
      dst[i + 3 * stride] = v3;
    }
    for (; i < n; i += stride) dst[i] = src[i];
  }
}

int launch_copy_probe(void* a, void* b, long long n16, int reps, int grid, void* stream) {
  k_copy_probe<<<grid, 512, 0, (cudaStream_t)stream>>>(static_cast<int4*>(a), static_cast<int4*>(b), n16, reps);
  return (int)cudaGetLastError();
}

}  // namespace cfet
