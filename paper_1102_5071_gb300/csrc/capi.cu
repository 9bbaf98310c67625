// C ABI of the CFET/Krylov propagator: contexts, argument validation, the
// per-step stage-scalar table, and the launch driver.
//
// Alvermann & Fehske, arXiv:1102.5071.  A CFET step (Sec. 4, Eq. (Ucf)) is
// exp(Omega_1) ... exp(Omega_s) with Omega_j = -i dt sum_m g_{j,m} H(t + x_m dt)
// (Sec. 7, Eq. (OmGLeg)).  For H(t) = H0 + sum_k f_k(t) V_k the host builds,
// for every step n and stage j, the scalars
//     c_{j,0} = sum_m g_{j,m},   c_{j,k} = sum_m g_{j,m} f_k(t0 + n dt + x_m dt),
// evaluating each drive once per node, orders the stage exponentials as they
// act on psi (exp(Omega_s) first, Sec. 2.2), uploads the table and runs the
// persistent device kernel over it.  The per-call launch sequence (table
// upload, state reset, persistent-kernel chunks, status read-back) is
// captured into a CUDA graph owned by the context and replayed; an unchanged
// topology only updates the executable graph in place.
#include <cuda.h>  // CUtensorMap and its enums (the encoder comes from the runtime's driver entry point)
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "cfet_internal.h"
#include "scalar_bounds.cuh"
#include "tiled_common.cuh"

using namespace cfet;

// TMA maps of the window-tiled complex64 apply over the Krylov basis of ctx
// (nvec vectors of 2^N elements), one per window, copied to device memory.
static cfet_status build_tile_maps(cfet_ctx* ctx, int N, int nvec, bool fx);

struct cfet_ctx {
  int device = 0;
  int family = 0;
  int dim = 0;
  int nV = 0;
  cfet_options opt{};
  int grid = 1, block = 256;
  // one-CTA fixed-point launches with the Krylov basis in shared memory: the
  // CTA's size (one worker thread per element, at most block - 32, plus the
  // control warp)
  bool small_fx = false;
  int small_block = 0;
  int precision = CFET_PREC_FX;
  std::string err;
  // drives
  std::vector<cfet_drive_fn> f;
  std::vector<void*> f_user;
  // operators
  OpSpin spin{};
  OpDia dia{};
  OpCsr csr{};
  OpCsrFx csr_fx{};
  OpCsrC csr_c{};
  void* d_csr = nullptr;       // one allocation: rp | col | vr | vi | VR | VI | vr32 | vi32
  // interaction picture: host copies of the chain (stage weight tables)
  double ip_J = 0.0, ip_Delta = 0.0;
  std::vector<double> ip_h, ip_xf;
  // Gershgorin intervals of H0 and of every V_k (Chebyshev stage exponentials)
  double op_lo[1 + kMaxDrives] = {}, op_hi[1 + kMaxDrives] = {};
  double* d_dz_lo = nullptr;
  double* d_dz_hi = nullptr;
  double* d_xf = nullptr;
  long long* d_off = nullptr;
  int* d_opidx = nullptr;
  double* d_val = nullptr;
  // workspace
  double2* d_basis = nullptr;
  // fixed-point path
  OpSpinFx spin_fx{};
  OpDiaFx dia_fx{};
  long long* d_DZ = nullptr;   // DZ_lo | DZ_hi
  long long* d_VAL = nullptr;
  longlong2* d_qbasis = nullptr;
  // mixed-precision path
  OpSpinC spin_c{};
  OpDiaC dia_c{};
  float* d_dz32 = nullptr;     // dz_lo | dz_hi in FP32
  float* d_val32 = nullptr;
  float2* d_qbasis32 = nullptr;
  bool tiled = false;          // window-tiled apply (long chains, complex64 and fixed point)
  unsigned char* d_tmaps = nullptr;  // complex64 tiled apply: one TMA map per window
  // Pauli-sum family (FP64): strings grouped by X mask
  OpPauli pauli{};
  void* d_pauli = nullptr;     // one allocation: gx | gstart | tz | top | tc | tim | greal
  double* d_pauli_dtab = nullptr;  // diagonal tables of the Z-only strings
  double* d_partials = nullptr;
  unsigned* d_bar = nullptr;
  DevStatus* d_st = nullptr;
  DevStatus* h_st = nullptr;  // pinned
  double* d_scal = nullptr;
  double* h_scal = nullptr;  // pinned
  size_t scal_cap = 0;
  double2* d_psi_e2e = nullptr;
  // decisions
  int* d_dec = nullptr;  // [f_nsub | f_k | f_h | r_nsub | r_k | r_h]
  size_t dec_cap = 0;    // ints
  // fidelity gradient (adjoint sweep) workspace
  double2* d_adj_ckpt = nullptr;   // checkpoints of the forward states
  size_t adj_ckpt_n = 0;
  double2* d_adj_vec = nullptr;    // psi, lambda, Krylov bases of both
  double* d_adj_part = nullptr;
  double* d_adj_tab = nullptr;     // c0 | c1 | gamma per exponential, then GL nodes and weights
  int* d_adj_seg = nullptr;
  size_t adj_tab_n = 0;
  double* d_adj_acc = nullptr;     // gradient accumulators [2 nseg] then out [4]
  int adj_nseg_cap = 0;
  int adj_grid = 0;
  // time-step selection: two trial states and the difference-norm partials
  double2* d_ts = nullptr;
  double* d_ts_part = nullptr;
  // graph driver
  struct GraphKey {  // everything the captured sequence depends on
    const void* psi = nullptr;
    const void* scal = nullptr;
    const void* dec = nullptr;
    long long nexp = -1, chunk = 0, flen = 0, rcap = 0;
    size_t table_bytes = 0, nf = 0;
    double tau = 0.0, tol = 0.0;
    int has_f = 0, has_r = 0;
    bool operator==(const GraphKey& o) const {
      return psi == o.psi && scal == o.scal && dec == o.dec && nexp == o.nexp && chunk == o.chunk &&
             flen == o.flen && rcap == o.rcap && table_bytes == o.table_bytes && nf == o.nf && tau == o.tau &&
             tol == o.tol && has_f == o.has_f && has_r == o.has_r;
    }
  } gkey;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev_done = nullptr;
  bool ev_pending = false;
  cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;  // kernel timing (inside the graph)
  bool timed = false;
};

namespace {

// Reduction / exchange scratch per CTA (8-byte words): the FP64 kernel uses 3
// partials, the control-warp kernels slots of tagged words: the two-pass
// fixed-point and complex64 kernels 3 slots of at most 8 words, the one-pass
// fixed-point kernel two 16-word slots and three 8-word slots.
constexpr size_t kPartialWordsPerCta = 56;
constexpr int kMaxCtlGrid = 256;  // 32 lanes x 8 records per lane of the exchange
// FP64 kernel with full re-orthogonalisation: 3 slots + 2 m_max Gram-Schmidt coefficients per CTA
static size_t partial_words_per_cta(const cfet_ctx* ctx) {
  const size_t need = ctx->opt.reorth ? 3 + 2 * (size_t)ctx->opt.m_max : 0;
  return need > kPartialWordsPerCta ? need : kPartialWordsPerCta;
}

thread_local std::string g_create_err;

cfet_status fail(cfet_ctx* ctx, cfet_status s, const std::string& msg) {
  if (ctx) ctx->err = msg; else g_create_err = msg;
  return s;
}

cfet_status cuda_fail(cfet_ctx* ctx, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(ctx, e == cudaErrorMemoryAllocation ? CFET_ENOMEM : CFET_ECUDA, m);
}

#define CK(call, where)                              \
  do {                                               \
    cudaError_t _e = (call);                         \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, where); \
  } while (0)

bool is_finite_d(double v) { return std::isfinite(v); }

cfet_status device_available(cfet_ctx* ctx) {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(ctx, CFET_ENODEV, "no CUDA device available");
  }
  return CFET_OK;
}

void free_ctx(cfet_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->ev_done) cudaEventDestroy(c->ev_done);
  if (c->ev_k0) cudaEventDestroy(c->ev_k0);
  if (c->ev_k1) cudaEventDestroy(c->ev_k1);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  cudaFree(c->d_dz_lo); cudaFree(c->d_dz_hi); cudaFree(c->d_xf);
  cudaFree(c->d_off); cudaFree(c->d_opidx); cudaFree(c->d_val);
  cudaFree(c->d_basis); cudaFree(c->d_partials); cudaFree(c->d_bar); cudaFree(c->d_st);
  cudaFree(c->d_scal); cudaFree(c->d_psi_e2e); cudaFree(c->d_dec);
  cudaFree(c->d_DZ); cudaFree(c->d_VAL); cudaFree(c->d_qbasis);
  cudaFree(c->d_dz32); cudaFree(c->d_val32); cudaFree(c->d_qbasis32);
  cudaFree(c->d_adj_ckpt); cudaFree(c->d_adj_vec); cudaFree(c->d_adj_part); cudaFree(c->d_adj_tab);
  cudaFree(c->d_adj_seg); cudaFree(c->d_adj_acc);
  cudaFree(c->d_ts); cudaFree(c->d_ts_part);
  cudaFree(c->d_pauli);
  cudaFree(c->d_pauli_dtab);
  cudaFree(c->d_tmaps);
  cudaFree(c->d_csr);
  if (c->h_st) cudaFreeHost(c->h_st);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  delete c;
}

cfet_status check_psi(cfet_ctx* ctx, const void* psi) {
  if (!psi) return fail(ctx, CFET_EINVAL, "psi is NULL");
  if (reinterpret_cast<uintptr_t>(psi) % 16 != 0) return fail(ctx, CFET_EINVAL, "psi is not 16-byte aligned");
  return CFET_OK;
}

cfet_status ensure_scal(cfet_ctx* ctx, size_t n) {
  if (n <= ctx->scal_cap) return CFET_OK;
  if (ctx->ev_pending) { cudaEventSynchronize(ctx->ev_done); ctx->ev_pending = false; }
  cudaFree(ctx->d_scal);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  ctx->d_scal = nullptr; ctx->h_scal = nullptr; ctx->scal_cap = 0;
  size_t cap = n < 1024 ? 1024 : n;
  CK(cudaMalloc(&ctx->d_scal, cap * sizeof(double)), "cudaMalloc(scalars)");
  CK(cudaMallocHost(&ctx->h_scal, cap * sizeof(double)), "cudaMallocHost(scalars)");
  ctx->scal_cap = cap;
  return CFET_OK;
}

cfet_status ensure_dec(cfet_ctx* ctx, size_t n_ints) {
  if (n_ints <= ctx->dec_cap) return CFET_OK;
  if (ctx->ev_pending) { cudaEventSynchronize(ctx->ev_done); ctx->ev_pending = false; }
  cudaFree(ctx->d_dec);
  ctx->d_dec = nullptr; ctx->dec_cap = 0;
  CK(cudaMalloc(&ctx->d_dec, n_ints * sizeof(int)), "cudaMalloc(decisions)");
  ctx->dec_cap = n_ints;
  return CFET_OK;
}

void fill_stats(const DevStatus& s, cfet_stats* out) {
  if (!out) return;
  out->n_exp = s.n_exp;
  out->n_substeps = s.n_sub;
  out->n_applies = s.n_app;
  out->max_k = s.max_k;
  out->status = s.status;
  out->max_err_est = s.max_err;
  for (int i = 0; i < 8; ++i) {
    out->phase_ns[i] = s.n_exp > 0 && s.phase_ns[i] > 0 ? s.phase_ns[i] : 0;
    out->phase_max_ns[i] = s.phase_max_ns[i];
  }
}

// One persistent launch over exponentials [e0, e0 + ne).
cfet_status launch_chunk(cfet_ctx* ctx, const PropParams& base, long long e0, long long ne, cudaStream_t s) {
  PropParams p = base;
  p.scal = base.scal + (size_t)e0 * (1 + ctx->nV);
  p.nexp = ne;
  p.exp_base = e0;
  int e;
  if (p.ip_w) {
    OpSpinIP op{ctx->spin.N, p.ip_nw, p.ip_w};
    e = launch_propagate_spin_ip(p, op, ctx->grid, ctx->block, s);
  } else if (ctx->opt.expm == CFET_EXPM_CHEBYSHEV)
    e = ctx->family == kFamilySpin  ? launch_cheb_spin_fx(p, ctx->spin_fx, ctx->grid, cheb_threads(ctx->block - 32), s)
        : ctx->family == kFamilyCsr ? launch_cheb_csr_fx(p, ctx->csr_fx, ctx->grid, cheb_threads(ctx->block - 32), s)
                                    : launch_cheb_dia_fx(p, ctx->dia_fx, ctx->grid, cheb_threads(ctx->block - 32), s);
  else if (ctx->precision == CFET_PREC_FX) {
    const int b = ctx->small_fx ? ctx->small_block : ctx->block;
    e = ctx->family == kFamilySpin  ? launch_propagate_spin_fx(p, ctx->spin_fx, ctx->grid, b, s)
        : ctx->family == kFamilyCsr ? launch_propagate_csr_fx(p, ctx->csr_fx, ctx->grid, b, s)
                                    : launch_propagate_dia_fx(p, ctx->dia_fx, ctx->grid, b, s);
  }
  else if (ctx->precision == CFET_PREC_C64)
    e = ctx->family == kFamilySpin  ? launch_propagate_spin_c64(p, ctx->spin_c, ctx->grid, ctx->block, s)
        : ctx->family == kFamilyCsr ? launch_propagate_csr_c64(p, ctx->csr_c, ctx->grid, ctx->block, s)
                                    : launch_propagate_dia_c64(p, ctx->dia_c, ctx->grid, ctx->block, s);
  else if (ctx->family == kFamilyPauli)
    e = launch_propagate_pauli(p, ctx->pauli, ctx->grid, ctx->block, s);
  else
    e = ctx->family == kFamilySpin  ? launch_propagate_spin(p, ctx->spin, ctx->grid, ctx->block, s)
        : ctx->family == kFamilyCsr ? launch_propagate_csr(p, ctx->csr, ctx->grid, ctx->block, s)
                                    : launch_propagate_dia(p, ctx->dia, ctx->grid, ctx->block, s);
  if (e != cudaSuccess) return cuda_fail(ctx, (cudaError_t)e, "persistent kernel launch");
  return CFET_OK;
}

// Issue the whole device sequence of one propagation on stream s.
cfet_status issue_sequence(cfet_ctx* ctx, const PropParams& base, long long nexp, long long chunk,
                           size_t table_bytes, cudaStream_t s, bool timed) {
  CK(cudaMemcpyAsync(ctx->d_scal, ctx->h_scal, table_bytes, cudaMemcpyHostToDevice, s), "scalar upload");
  CK(cudaMemsetAsync(ctx->d_st, 0, sizeof(DevStatus), s), "status reset");
  CK(cudaMemsetAsync(ctx->d_bar, 0, 2 * sizeof(unsigned), s), "barrier reset");
  // exchange records of the control-warp kernels: no stale tag may survive
  CK(cudaMemsetAsync(ctx->d_partials, 0, partial_words_per_cta(ctx) * (size_t)ctx->grid * sizeof(double), s),
     "exchange reset");
  if (timed) CK(cudaEventRecordWithFlags(ctx->ev_k0, s, cudaEventRecordExternal), "timing event");
  if (base.ip_w) {  // into the interaction picture at t0
    const int e = launch_phase_diag(base.psi, ctx->spin, ctx->dim, base.ip_times, 0, 1.0, s);
    if (e != cudaSuccess) return cuda_fail(ctx, (cudaError_t)e, "phase kernel launch");
  }
  for (long long e0 = 0; e0 < nexp; e0 += chunk) {
    const long long ne = (nexp - e0) < chunk ? (nexp - e0) : chunk;
    cfet_status st = launch_chunk(ctx, base, e0, ne, s);
    if (st != CFET_OK) return st;
  }
  if (base.ip_w) {  // back to the Schroedinger picture at t_end
    const int e = launch_phase_diag(base.psi, ctx->spin, ctx->dim, base.ip_times, 1, -1.0, s);
    if (e != cudaSuccess) return cuda_fail(ctx, (cudaError_t)e, "phase kernel launch");
  }
  if (timed) CK(cudaEventRecordWithFlags(ctx->ev_k1, s, cudaEventRecordExternal), "timing event");
  CK(cudaMemcpyAsync(ctx->h_st, ctx->d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s), "status read-back");
  return CFET_OK;
}

PropParams base_params(cfet_ctx* ctx, double2* psi, double tau, double tol) {
  PropParams p{};
  p.dim = ctx->dim;
  p.nV = ctx->nV;
  p.psi = psi;
  p.basis = ctx->d_basis;
  p.scal = ctx->d_scal;
  p.tau = tau;
  p.tol = tol;
  p.m_min = ctx->opt.m_min;
  p.m_max = ctx->opt.m_max;
  p.max_substeps = ctx->opt.max_substeps;
  p.partials = ctx->d_partials;
  p.bar = ctx->d_bar;
  p.st = ctx->d_st;
  p.timeout_ns = (long long)(ctx->opt.barrier_timeout_s * 1e9);
  p.qbasis = ctx->d_qbasis;
  p.qbasis32 = ctx->d_qbasis32;
  p.tiled = ctx->tiled ? 1 : 0;
  p.tmaps = ctx->d_tmaps;
  p.reorth = ctx->opt.reorth;
  p.small = ctx->small_fx ? 1 : 0;
  return p;
}

// Chebyshev records (kChebRec doubles each) and concatenated coefficients of
// nexp stage exponentials exp(-i tau H_e) whose scalar rows (1 + nV doubles
// each) are `rows`: spectral interval of H_e by Weyl's inequality from the
// operators' Gershgorin intervals, a = half width, b = centre, K and r_k from
// the Bessel tail bound (chebyshev.cpp).
constexpr size_t kMaxChebCoef = size_t(1) << 27;
cfet_status build_cheb(cfet_ctx* ctx, const double* rows, long long nexp, double tau, double tol,
                       std::vector<double>& rec, std::vector<double>& coef) {
  const int ncoef = 1 + ctx->nV;
  const long long kcap = (long long)ctx->opt.m_max * ctx->opt.max_substeps;
  rec.assign((size_t)nexp * kChebRec, 0.0);
  coef.clear();
  std::vector<double> r;
  for (long long e = 0; e < nexp; ++e) {
    double lo = 0.0, hi = 0.0;
    stage_interval(ncoef, ctx->op_lo, ctx->op_hi, rows + e * ncoef, &lo, &hi);
    const double a = 0.5 * (hi - lo), b = 0.5 * (hi + lo);
    double* R = rec.data() + (size_t)e * kChebRec;
    double tail = 0.0;
    int K = 0;
    if (a > 0.0) {
      if (std::fabs(b) > 1.5 * a)
        return fail(ctx, CFET_EINVAL, "Chebyshev: spectral centre |b| > 1.5 a (shift H0 by a multiple of the identity)");
      if (!(std::fabs(tau * a) <= 1e8)) return fail(ctx, CFET_EKRYLOV, "Chebyshev: dt * a too large");
      K = cheb_series(tau * a, tol, &r, &tail);
      if (K > kcap) return fail(ctx, CFET_EKRYLOV, "Chebyshev: a stage exponential needs more than m_max * max_substeps terms");
      R[0] = 1.0 / a;
      R[1] = b / a;
    } else {
      r.assign(1, 1.0);
    }
    double sum = 0.0;
    for (double v : r) sum += std::fabs(v);
    R[2] = (double)K;
    R[3] = (double)coef.size();
    R[4] = sum;
    R[5] = std::cos(tau * b);
    R[6] = -std::sin(tau * b);
    R[7] = tail;
    coef.insert(coef.end(), r.begin(), r.end());
    if (coef.size() > kMaxChebCoef)
      return fail(ctx, CFET_EINVAL, "Chebyshev: more than 2^27 coefficients in one call; propagate in shorter calls");
  }
  return CFET_OK;
}

// Append the Chebyshev table behind the nexp scalar rows in ctx->h_scal;
// returns the total table length (doubles) in *n.
cfet_status stage_cheb_table(cfet_ctx* ctx, long long nexp, double tau, double tol, size_t* n) {
  const size_t nrows = (size_t)nexp * (1 + ctx->nV);
  std::vector<double> rows(ctx->h_scal, ctx->h_scal + nrows), rec, coef;
  cfet_status s = build_cheb(ctx, rows.data(), nexp, tau, tol, rec, coef);
  if (s != CFET_OK) return s;
  *n = nrows + rec.size() + coef.size();
  if ((s = ensure_scal(ctx, *n)) != CFET_OK) return s;
  std::memcpy(ctx->h_scal, rows.data(), nrows * sizeof(double));
  std::memcpy(ctx->h_scal + nrows, rec.data(), rec.size() * sizeof(double));
  std::memcpy(ctx->h_scal + nrows + rec.size(), coef.data(), coef.size() * sizeof(double));
  return CFET_OK;
}

void set_cheb_params(cfet_ctx* ctx, PropParams& p, long long nexp) {
  p.cheb = ctx->d_scal + (size_t)nexp * (1 + ctx->nV);
  p.cheb_coef = p.cheb + (size_t)nexp * kChebRec;
}

// Interaction-picture stage weights of one CFET step from t (Secs. 9.3, 9.4):
// for every stage (execution order, exp(Omega_s) first) the table of OpSpinIP,
//   flip  of site i, spin bit b, n = s_{i-1} + s_{i+1}:
//         sum_m g_{j,m} b_i(t_m) e^{i 2 s (h_i + J Delta n) t_m},  b_i(t) = sum_k f_k(t) a_{k,i}
//   hop   of bond (i, i+1), bit b of site i, m = s_{i-1} - s_{i+2}:
//         sum_m g_{j,m} 2J e^{i 2 s (h_i - h_{i+1} + J Delta m) t_m},
// s = 1 - 2b; the exponents are d(x) - d(partner) for the diagonal d of H0.
// fval: drives at the nodes, [m * nV + k].
void ip_step_weights(const cfet_ctx* ctx, const SchemeData& sd, double t, double dt, const std::vector<double>& fval,
                     double* out) {
  const int N = ctx->spin.N, nV = ctx->nV;
  const double JD = ctx->ip_J * ctx->ip_Delta;
  const int nw = kIPWeightsPerSite * (2 * N - 1);
  std::vector<double> tm(sd.M), bs((size_t)sd.M * N, 0.0);
  for (int m = 0; m < sd.M; ++m) {
    tm[m] = t + sd.x[m] * dt;
    for (int i = 0; i < N; ++i)
      for (int k = 0; k < nV; ++k) bs[(size_t)m * N + i] += fval[(size_t)m * nV + k] * ctx->ip_xf[(size_t)k * N + i];
  }
  for (int jj = 0; jj < sd.s; ++jj) {
    const int j = sd.s - 1 - jj;
    double* w = out + (size_t)jj * nw * 2;
    for (int i = 0; i < N; ++i)
      for (int b = 0; b < 2; ++b)
        for (int n = -2; n <= 2; ++n) {
          const double dd = 2.0 * (1 - 2 * b) * (ctx->ip_h[i] + JD * n);
          double re = 0.0, im = 0.0;
          for (int m = 0; m < sd.M; ++m) {
            const double a = sd.g[j][m] * bs[(size_t)m * N + i];
            re += a * std::cos(dd * tm[m]);
            im += a * std::sin(dd * tm[m]);
          }
          const size_t idx = (size_t)i * kIPWeightsPerSite + b * 5 + (n + 2);
          w[2 * idx] = re;
          w[2 * idx + 1] = im;
        }
    for (int i = 0; i + 1 < N; ++i)
      for (int b = 0; b < 2; ++b)
        for (int mm = -2; mm <= 2; ++mm) {
          const double dd = 2.0 * (1 - 2 * b) * (ctx->ip_h[i] - ctx->ip_h[i + 1] + JD * mm);
          double re = 0.0, im = 0.0;
          for (int m = 0; m < sd.M; ++m) {
            const double a = sd.g[j][m] * 2.0 * ctx->ip_J;
            re += a * std::cos(dd * tm[m]);
            im += a * std::sin(dd * tm[m]);
          }
          const size_t idx = (size_t)N * kIPWeightsPerSite + (size_t)i * kIPWeightsPerSite + b * 5 + (mm + 2);
          w[2 * idx] = re;
          w[2 * idx + 1] = im;
        }
  }
}

cfet_status finish(cfet_ctx* ctx, cudaStream_t s, cfet_stats* stats) {
  CK(cudaStreamSynchronize(s), "stream synchronize");
  ctx->ev_pending = false;
  fill_stats(*ctx->h_st, stats);
  const int code = ctx->h_st->status;
  if (code == CFET_EKRYLOV) return fail(ctx, CFET_EKRYLOV, "stage exponential exceeded max_substeps");
  if (code == CFET_ETIMEOUT) return fail(ctx, CFET_ETIMEOUT, "device grid barrier timed out");
  if (code == CFET_ENAN) return fail(ctx, CFET_ENAN, "psi norm is not finite");
  if (code != 0) return fail(ctx, (cfet_status)code, "device error");
  return CFET_OK;
}

// Gauss-Legendre nodes and weights on [0, 1] by Newton's method on the
// Legendre polynomial P_n (three-term recurrence); weights 1 / ((1 - z^2) P_n'(z)^2).
void gauss_legendre_01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), p1 = 0.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0;
      p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-15) break;
    }
    {
      double p0 = 1.0;
      p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Piecewise-constant drive amplitude: f(t) = amps[k] cos(omega t + phase), k the
// segment of the step that contains t.
struct PwcDrive {
  const double* amps;
  int nseg;
  double omega, phase, t0, dt;
  long long steps_per_seg;
};

double pwc_eval(double t, void* user) {
  const PwcDrive* d = static_cast<const PwcDrive*>(user);
  long long n = (long long)std::floor((t - d->t0) / d->dt);
  long long k = n / d->steps_per_seg;
  if (k < 0) k = 0;
  if (k >= d->nseg) k = d->nseg - 1;
  return d->amps[k] * std::cos(d->omega * t + d->phase);
}

// ---------------------------------------------------------------- CSR operators
// Structure and Hermiticity of one CSR operator (NULL when acceptable).
// Duplicate entries of a row are summed; every stored (r, c) must have its
// mirror (c, r) with the conjugate value, to 1e-13 of the largest entry (an
// entry without a mirror must be that small itself); the diagonal is real.
const char* csr_check(const cfet_op& o, int dim) {
  if (!o.row_ptr || !o.col_idx || (!o.csr_re && o.row_ptr[dim] > 0)) return "CSR: missing arrays";
  if (o.row_ptr[0] != 0) return "CSR: row_ptr[0] must be 0";
  for (int r = 0; r < dim; ++r)
    if (o.row_ptr[r + 1] < o.row_ptr[r]) return "CSR: row_ptr must be non-decreasing";
  const int64_t nnz = o.row_ptr[dim];
  if (nnz >= 0x7fffffffLL) return "CSR: too many stored entries";
  struct E {
    int r, c;
    double re, im;
  };
  std::vector<E> es;
  es.reserve((size_t)nnz);
  double amax = 0.0;
  for (int r = 0; r < dim; ++r)
    for (int64_t e = o.row_ptr[r]; e < o.row_ptr[r + 1]; ++e) {
      const int c = o.col_idx[e];
      if (c < 0 || c >= dim) return "CSR: column index out of range";
      const double re = o.csr_re[e], im = o.csr_im ? o.csr_im[e] : 0.0;
      if (!is_finite_d(re) || !is_finite_d(im)) return "CSR: value not finite";
      es.push_back({r, c, re, im});
      amax = std::fmax(amax, std::fabs(re) + std::fabs(im));
    }
  auto key_less = [](const E& a, const E& b) { return a.r != b.r ? a.r < b.r : a.c < b.c; };
  std::sort(es.begin(), es.end(), key_less);
  std::vector<E> m;  // duplicates summed
  m.reserve(es.size());
  for (const E& x : es) {
    if (!m.empty() && m.back().r == x.r && m.back().c == x.c) {
      m.back().re += x.re;
      m.back().im += x.im;
    } else {
      m.push_back(x);
    }
  }
  const double tol = 1e-13 * amax;
  for (const E& x : m) {
    E key{x.c, x.r, 0.0, 0.0};
    auto it = std::lower_bound(m.begin(), m.end(), key, key_less);
    double wr = 0.0, wi = 0.0;
    if (it != m.end() && it->r == x.c && it->c == x.r) {
      wr = it->re;
      wi = it->im;
    }
    if (std::fabs(x.re - wr) > tol || std::fabs(x.im + wi) > tol) return "CSR: operator is not Hermitian";
  }
  return nullptr;
}

// Device copies of the CSR operators of a context: FP64 values, fixed-point
// values with one exponent per operator (row sums of |re| + |im| below 2^62),
// FP32 values; one allocation.
cfet_status csr_upload(cfet_ctx* ctx, const cfet_op* H0, int nV, const cfet_op* V) {
  const int dim = ctx->dim;
  const int nops = 1 + nV;
  bool cplx = false;
  std::vector<int> rp((size_t)nops * (dim + 1));
  size_t nnz = 0;
  for (int k = -1; k < nV; ++k) {
    const cfet_op& o = k < 0 ? *H0 : V[k];
    const int64_t n = o.row_ptr[dim];
    for (int r = 0; r <= dim; ++r) rp[(size_t)(k + 1) * (dim + 1) + r] = (int)(nnz + o.row_ptr[r]);
    if (o.csr_im)
      for (int64_t e = 0; e < n; ++e) cplx = cplx || o.csr_im[e] != 0.0;
    nnz += (size_t)n;
  }
  const size_t n1 = nnz > 0 ? nnz : 1;
  std::vector<int> col(n1, 0);
  std::vector<double> vr(n1, 0.0), vi(cplx ? n1 : 0, 0.0);
  std::vector<long long> VR(n1, 0), VI(cplx ? n1 : 0, 0);
  std::vector<float> vr32(n1, 0.f), vi32(cplx ? n1 : 0, 0.f);
  OpCsrFx& fx = ctx->csr_fx;
  size_t at = 0;
  for (int k = -1; k < nV; ++k) {
    const cfet_op& o = k < 0 ? *H0 : V[k];
    const int oi = k + 1;
    double mrow = 0.0;
    for (int r = 0; r < dim; ++r) {
      double rs = 0.0;
      for (int64_t e = o.row_ptr[r]; e < o.row_ptr[r + 1]; ++e)
        rs += std::fabs(o.csr_re[e]) + (o.csr_im ? std::fabs(o.csr_im[e]) : 0.0);
      mrow = std::fmax(mrow, rs);
    }
    mrow *= 1.0 + 1e-12;
    int E_op = 0;
    if (mrow > 0.0) {
      int ex = 0;
      std::frexp(mrow, &ex);  // mrow < 2^ex
      E_op = ex - 62;
    }
    fx.E_op[oi] = E_op;
    fx.maxrow[oi] = mrow;
    const int64_t n = o.row_ptr[dim];
    for (int64_t e = 0; e < n; ++e, ++at) {
      col[at] = o.col_idx[e];
      vr[at] = o.csr_re[e];
      VR[at] = std::llrint(std::ldexp(o.csr_re[e], -E_op));
      vr32[at] = (float)o.csr_re[e];
      if (cplx) {
        const double im = o.csr_im ? o.csr_im[e] : 0.0;
        vi[at] = im;
        VI[at] = std::llrint(std::ldexp(im, -E_op));
        vi32[at] = (float)im;
      }
    }
    csr_interval(o.row_ptr, o.col_idx, o.csr_re, o.csr_im, dim, &ctx->op_lo[oi], &ctx->op_hi[oi]);
  }
  // layout: rp | col | vr | vi | VR | VI | vr32 | vi32, 16-byte aligned pieces
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  const size_t nv = cplx ? n1 : 0;
  const size_t o_rp = 0, o_col = o_rp + al(rp.size() * sizeof(int)), o_vr = o_col + al(n1 * sizeof(int));
  const size_t o_vi = o_vr + al(n1 * sizeof(double)), o_VR = o_vi + al(nv * sizeof(double));
  const size_t o_VI = o_VR + al(n1 * sizeof(long long)), o_v32 = o_VI + al(nv * sizeof(long long));
  const size_t o_i32 = o_v32 + al(n1 * sizeof(float)), bytes = o_i32 + al(nv * sizeof(float));
  std::vector<unsigned char> blob(bytes, 0);
  std::memcpy(blob.data() + o_rp, rp.data(), rp.size() * sizeof(int));
  std::memcpy(blob.data() + o_col, col.data(), n1 * sizeof(int));
  std::memcpy(blob.data() + o_vr, vr.data(), n1 * sizeof(double));
  std::memcpy(blob.data() + o_VR, VR.data(), n1 * sizeof(long long));
  std::memcpy(blob.data() + o_v32, vr32.data(), n1 * sizeof(float));
  if (cplx) {
    std::memcpy(blob.data() + o_vi, vi.data(), nv * sizeof(double));
    std::memcpy(blob.data() + o_VI, VI.data(), nv * sizeof(long long));
    std::memcpy(blob.data() + o_i32, vi32.data(), nv * sizeof(float));
  }
  cudaError_t ce = cudaMalloc(&ctx->d_csr, bytes);
  if (ce == cudaSuccess) ce = cudaMemcpy(ctx->d_csr, blob.data(), bytes, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "CSR upload");
  unsigned char* b = static_cast<unsigned char*>(ctx->d_csr);
  const int* d_rp = reinterpret_cast<const int*>(b + o_rp);
  const int* d_col = reinterpret_cast<const int*>(b + o_col);
  ctx->csr = OpCsr{nops, d_rp, d_col, reinterpret_cast<const double*>(b + o_vr),
                   cplx ? reinterpret_cast<const double*>(b + o_vi) : nullptr};
  fx.nops = nops;
  fx.rp = d_rp;
  fx.col = d_col;
  fx.VR = reinterpret_cast<const long long*>(b + o_VR);
  fx.VI = cplx ? reinterpret_cast<const long long*>(b + o_VI) : nullptr;
  ctx->csr_c = OpCsrC{nops, d_rp, d_col, reinterpret_cast<const float*>(b + o_v32),
                      cplx ? reinterpret_cast<const float*>(b + o_i32) : nullptr};
  return CFET_OK;
}

}  // namespace

// ============================================================================
extern "C" {

void cfet_options_default(cfet_options* opt) {
  if (!opt) return;
  opt->m_max = 16;
  opt->m_min = 2;
  opt->max_substeps = 64;
  opt->block_size = 0;
  opt->grid_size = 0;
  opt->steps_per_launch = 256;
  opt->barrier_timeout_s = 2.0;
  opt->precision = CFET_PREC_DEFAULT;  // fixed point; FP64 for Pauli sums
  opt->expm = CFET_EXPM_KRYLOV;
  opt->picture = CFET_PICTURE_SCHROEDINGER;
  opt->reorth = 0;
  opt->apply_form = CFET_APPLY_AUTO;
}

cfet_status cfet_scheme_info(int32_t scheme, int32_t* order, int32_t* s, int32_t* M, double* f, double* x,
                             double* w, double* g, int32_t capacity) {
  SchemeData d;
  if (!build_scheme(scheme, &d)) return CFET_EINVAL;
  if (order) *order = d.order;
  if (s) *s = d.s;
  if (M) *M = d.M;
  const int need = d.s * d.M;
  if ((f || g) && capacity < need) return CFET_EINVAL;
  if ((x || w) && capacity < d.M) return CFET_EINVAL;
  for (int i = 0; i < d.s; ++i)
    for (int m = 0; m < d.M; ++m) {
      if (f) f[i * d.M + m] = d.f[i][m];
      if (g) g[i * d.M + m] = d.g[i][m];
    }
  for (int m = 0; m < d.M; ++m) {
    if (x) x[m] = d.x[m];
    if (w) w[m] = d.w[m];
  }
  return CFET_OK;
}

const char* cfet_last_error(const cfet_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int64_t cfet_dim(const cfet_ctx* ctx) { return ctx ? ctx->dim : 0; }
int32_t cfet_num_drives(const cfet_ctx* ctx) { return ctx ? ctx->nV : 0; }

cfet_status cfet_create(cfet_ctx** out, const cfet_op* H0, int32_t nV, const cfet_op* V, const cfet_drive_fn* f,
                        void* const* f_user, const cfet_options* opt) {
  cfet_ctx* ctx = nullptr;
  g_create_err.clear();
  if (!out) return fail(nullptr, CFET_EINVAL, "out is NULL");
  *out = nullptr;
  if (!H0) return fail(nullptr, CFET_EINVAL, "H0 is NULL");
  if (nV < 0 || nV > kMaxDrives) return fail(nullptr, CFET_EINVAL, "nV must be in [0, 8]");
  if (nV > 0 && (!V || !f)) return fail(nullptr, CFET_EINVAL, "V and f are required when nV > 0");
  for (int k = 0; k < nV; ++k)
    if (!f[k]) return fail(nullptr, CFET_EINVAL, "drive callback is NULL");
  cfet_options o;
  cfet_options_default(&o);
  if (opt) o = *opt;
  if (o.m_max < 1 || o.m_max > kMaxKrylov) return fail(nullptr, CFET_EINVAL, "m_max must be in [1, 64]");
  if (o.m_min < 1 || o.m_min > o.m_max) return fail(nullptr, CFET_EINVAL, "m_min must be in [1, m_max]");
  if (o.max_substeps < 1) return fail(nullptr, CFET_EINVAL, "max_substeps must be >= 1");
  // a Pauli sum anywhere makes the context a Pauli-sum context (FP64 only)
  bool pauli = H0->kind == CFET_OP_PAULI;
  for (int k = 0; k < nV; ++k) pauli = pauli || V[k].kind == CFET_OP_PAULI;
  if (o.precision == CFET_PREC_DEFAULT) o.precision = pauli ? CFET_PREC_F64 : CFET_PREC_FX;
  if (pauli && o.precision != CFET_PREC_F64)
    return fail(nullptr, CFET_EINVAL, "Pauli-sum operators compute in CFET_PREC_F64 only");
  if (o.precision != CFET_PREC_F64 && o.precision != CFET_PREC_FX && o.precision != CFET_PREC_C64)
    return fail(nullptr, CFET_EINVAL, "precision must be CFET_PREC_F64, CFET_PREC_FX or CFET_PREC_C64");
  if (o.expm != CFET_EXPM_KRYLOV && o.expm != CFET_EXPM_CHEBYSHEV)
    return fail(nullptr, CFET_EINVAL, "expm must be CFET_EXPM_KRYLOV or CFET_EXPM_CHEBYSHEV");
  if (o.expm == CFET_EXPM_CHEBYSHEV && o.precision != CFET_PREC_FX)
    return fail(nullptr, CFET_EINVAL, "CFET_EXPM_CHEBYSHEV requires CFET_PREC_FX");
  if (o.picture != CFET_PICTURE_SCHROEDINGER && o.picture != CFET_PICTURE_INTERACTION)
    return fail(nullptr, CFET_EINVAL, "picture must be CFET_PICTURE_SCHROEDINGER or CFET_PICTURE_INTERACTION");
  if (o.picture == CFET_PICTURE_INTERACTION &&
      (o.precision != CFET_PREC_F64 || o.expm != CFET_EXPM_KRYLOV || H0->kind != CFET_OP_XXZ_CHAIN || pauli))
    return fail(nullptr, CFET_EINVAL, "CFET_PICTURE_INTERACTION requires an XXZ chain, CFET_PREC_F64 and CFET_EXPM_KRYLOV");
  if (o.reorth != 0 && o.reorth != 1) return fail(nullptr, CFET_EINVAL, "reorth must be 0 or 1");
  if (o.reorth && (o.precision != CFET_PREC_F64 || o.expm != CFET_EXPM_KRYLOV))
    return fail(nullptr, CFET_EINVAL, "reorth requires CFET_PREC_F64 and CFET_EXPM_KRYLOV");
  if (o.apply_form != CFET_APPLY_AUTO && o.apply_form != CFET_APPLY_ELEMENTWISE && o.apply_form != CFET_APPLY_TILED)
    return fail(nullptr, CFET_EINVAL, "apply_form must be CFET_APPLY_AUTO, CFET_APPLY_ELEMENTWISE or CFET_APPLY_TILED");
  if (o.block_size == 0) o.block_size = (o.precision == CFET_PREC_F64) ? 256 : 384;
  {
    // FP64 kernel: block_size threads (<= 256); fixed-point and mixed-precision
    // kernels: 2 * block_size workers + one control warp (<= 1024 threads)
    // (the latter are compiled for at most CFET_CTL_MAX_THREADS threads per CTA)
    const int lim = (o.precision == CFET_PREC_F64) ? 256 : ((CFET_CTL_MAX_THREADS - 32) / 2) & ~31;
    if (o.block_size < 32 || o.block_size > lim || o.block_size % 32)
      return fail(nullptr, CFET_EINVAL, "block_size must be a multiple of 32 in [32, 256] (FP64) or [32, 384]");
  }
  if (o.grid_size < 0) return fail(nullptr, CFET_EINVAL, "grid_size must be >= 0");
  if (o.steps_per_launch <= 0) o.steps_per_launch = 256;
  if (!(o.barrier_timeout_s > 0.0) || !is_finite_d(o.barrier_timeout_s))
    return fail(nullptr, CFET_EINVAL, "barrier_timeout_s must be positive");


  int family = 0, dim = 0, nsites = 0;
  // Pauli-sum family: every operator expanded into strings (x, z, coefficient, operator)
  struct PString {
    unsigned x, z;
    double c;
    int op;
  };
  std::vector<PString> strings;
  if (pauli) {
    family = kFamilyPauli;
    nsites = H0->nsites;
    if (nsites < 1 || nsites > kMaxSites) return fail(nullptr, CFET_EINVAL, "nsites must be in [1, 30]");
    for (int k = -1; k < nV; ++k) {
      const cfet_op& o2 = k < 0 ? *H0 : V[k];
      if (o2.nsites != nsites || o2.dim != (int64_t(1) << nsites))
        return fail(nullptr, CFET_EINVAL, "Pauli sums: every operator on the same chain, dim = 2^nsites");
      const int oi = k + 1;
      if (o2.kind == CFET_OP_PAULI) {
        if (o2.nterms < 0 || (o2.nterms > 0 && (!o2.xmask || !o2.zmask || !o2.coeff)))
          return fail(nullptr, CFET_EINVAL, "Pauli sum: nterms < 0 or missing arrays");
        if (strings.size() + (size_t)o2.nterms > (size_t)kMaxPauliTerms)
          return fail(nullptr, CFET_EINVAL, "Pauli sums: more than 4096 strings");
        for (int t = 0; t < o2.nterms; ++t) {
          if ((o2.xmask[t] | o2.zmask[t]) >> nsites) return fail(nullptr, CFET_EINVAL, "Pauli sum: mask beyond nsites");
          if (!is_finite_d(o2.coeff[t])) return fail(nullptr, CFET_EINVAL, "Pauli sum: coefficient not finite");
          strings.push_back({(unsigned)o2.xmask[t], (unsigned)o2.zmask[t], o2.coeff[t], oi});
        }
      } else if (o2.kind == CFET_OP_XXZ_CHAIN) {
        if (!o2.site_coeff || !is_finite_d(o2.J) || !is_finite_d(o2.Delta))
          return fail(nullptr, CFET_EINVAL, "XXZ chain: missing or non-finite parameters");
        for (int i = 0; i + 1 < nsites; ++i) {
          const unsigned b = 3u << i;
          strings.push_back({b, 0u, o2.J, oi});              // X_i X_{i+1}
          strings.push_back({b, b, o2.J, oi});               // Y_i Y_{i+1} = i^2 X X Z Z
          strings.push_back({0u, b, o2.J * o2.Delta, oi});   // Z_i Z_{i+1}
        }
        for (int i = 0; i < nsites; ++i) {
          if (!is_finite_d(o2.site_coeff[i])) return fail(nullptr, CFET_EINVAL, "XXZ chain: h not finite");
          strings.push_back({0u, 1u << i, o2.site_coeff[i], oi});
        }
      } else if (o2.kind == CFET_OP_X_FIELD) {
        if (!o2.site_coeff) return fail(nullptr, CFET_EINVAL, "X field: site_coeff is NULL");
        for (int i = 0; i < nsites; ++i) {
          if (!is_finite_d(o2.site_coeff[i])) return fail(nullptr, CFET_EINVAL, "X field coefficient not finite");
          strings.push_back({1u << i, 0u, o2.site_coeff[i], oi});
        }
      } else {
        return fail(nullptr, CFET_EINVAL, "Pauli sums combine only with XXZ chains and X fields");
      }
    }
    if (strings.size() > (size_t)kMaxPauliTerms) return fail(nullptr, CFET_EINVAL, "Pauli sums: more than 4096 strings");
    dim = 1 << nsites;
  } else if (H0->kind == CFET_OP_XXZ_CHAIN) {
    family = kFamilySpin;
    nsites = H0->nsites;
    if (nsites < 1 || nsites > kMaxSites) return fail(nullptr, CFET_EINVAL, "nsites must be in [1, 30]");
    if (H0->dim != (int64_t(1) << nsites)) return fail(nullptr, CFET_EINVAL, "XXZ chain: dim must be 2^nsites");
    if (!H0->site_coeff) return fail(nullptr, CFET_EINVAL, "XXZ chain: site_coeff (h) is NULL");
    if (!is_finite_d(H0->J) || !is_finite_d(H0->Delta)) return fail(nullptr, CFET_EINVAL, "XXZ chain: J, Delta not finite");
    for (int i = 0; i < nsites; ++i)
      if (!is_finite_d(H0->site_coeff[i])) return fail(nullptr, CFET_EINVAL, "XXZ chain: h not finite");
    for (int k = 0; k < nV; ++k) {
      if (V[k].kind != CFET_OP_X_FIELD || V[k].nsites != nsites || V[k].dim != H0->dim || !V[k].site_coeff)
        return fail(nullptr, CFET_EINVAL, "drive operators of an XXZ chain must be X fields of the same chain");
      for (int i = 0; i < nsites; ++i)
        if (!is_finite_d(V[k].site_coeff[i])) return fail(nullptr, CFET_EINVAL, "X field coefficient not finite");
    }
    dim = (int)H0->dim;
  } else if (H0->kind == CFET_OP_DIA) {
    family = kFamilyDia;
    if (H0->dim < 1 || H0->dim > 0x7fffffffLL) return fail(nullptr, CFET_EINVAL, "DIA: dim must be in [1, 2^31)");
    dim = (int)H0->dim;
    int total = 0;
    for (int k = -1; k < nV; ++k) {
      const cfet_op& o2 = k < 0 ? *H0 : V[k];
      if (o2.kind != CFET_OP_DIA || o2.dim != H0->dim)
        return fail(nullptr, CFET_EINVAL, "drive operators of a DIA operator must be DIA of the same dimension");
      if (o2.ndiag < 1 || !o2.offsets || !o2.values) return fail(nullptr, CFET_EINVAL, "DIA: missing diagonals");
      for (int d = 0; d < o2.ndiag; ++d)
        if (o2.offsets[d] <= -(int64_t)dim || o2.offsets[d] >= (int64_t)dim)
          return fail(nullptr, CFET_EINVAL, "DIA: offset out of range");
      for (int64_t i = 0; i < (int64_t)o2.ndiag * dim; ++i)
        if (!is_finite_d(o2.values[i])) return fail(nullptr, CFET_EINVAL, "DIA: value not finite");
      total += o2.ndiag;
    }
    if (total > kMaxDiag) return fail(nullptr, CFET_EINVAL, "DIA: more than 32 diagonals in total");
  } else if (H0->kind == CFET_OP_CSR) {
    family = kFamilyCsr;
    if (H0->dim < 1 || H0->dim >= 0x7fffffffLL) return fail(nullptr, CFET_EINVAL, "CSR: dim must be in [1, 2^31 - 1)");
    dim = (int)H0->dim;
    int64_t total = 0;
    for (int k = -1; k < nV; ++k) {
      const cfet_op& o2 = k < 0 ? *H0 : V[k];
      if (o2.kind != CFET_OP_CSR || o2.dim != H0->dim)
        return fail(nullptr, CFET_EINVAL, "drive operators of a CSR operator must be CSR of the same dimension");
      const char* why = csr_check(o2, dim);
      if (why) return fail(nullptr, CFET_EINVAL, why);
      total += o2.row_ptr[dim];
    }
    if (total >= 0x7fffffffLL) return fail(nullptr, CFET_EINVAL, "CSR: more than 2^31 - 2 stored entries in total");
  } else {
    return fail(nullptr, CFET_EINVAL, "H0 must be an XXZ chain, a Pauli sum, a DIA or a CSR operator");
  }
  {
    cfet_status s = device_available(nullptr);
    if (s != CFET_OK) return s;
  }

  ctx = new cfet_ctx();
  cudaGetDevice(&ctx->device);
  ctx->family = family;
  ctx->dim = dim;
  ctx->nV = nV;
  ctx->opt = o;
  // FP64 kernel: block_size threads; fixed-point and mixed-precision kernels:
  // 2 * block_size worker threads plus one control warp (default 768 + 32,
  // one CTA per SM)
  const bool ctl_warp = o.precision != CFET_PREC_F64;
  ctx->block = ctl_warp ? 2 * o.block_size + 32 : o.block_size;
  ctx->precision = o.precision;
  for (int k = 0; k < nV; ++k) {
    ctx->f.push_back(f[k]);
    ctx->f_user.push_back(f_user ? f_user[k] : nullptr);
  }
#define CKC(call, where)                                         \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) {                                     \
      cfet_status _s = cuda_fail(nullptr, _e, where);            \
      free_ctx(ctx);                                             \
      return _s;                                                 \
    }                                                            \
  } while (0)

  if (family == kFamilyPauli) {
    // group the strings by X mask (stable: the order within a group is the input order)
    std::stable_sort(strings.begin(), strings.end(), [](const PString& a, const PString& b) { return a.x < b.x; });
    const int nt = (int)strings.size();
    std::vector<unsigned> gx, tz(nt);
    std::vector<int> gstart, top(nt);
    std::vector<double> tc(nt);
    std::vector<unsigned char> tim(nt);
    for (int t = 0; t < nt; ++t) {
      const PString& ps = strings[t];
      if (t == 0 || ps.x != strings[t - 1].x) {
        gx.push_back(ps.x);
        gstart.push_back(t);
      }
      const int ph = __builtin_popcount(ps.x & ps.z) & 3;  // the string's phase i^ph
      tz[t] = ps.z;
      top[t] = ps.op;
      tc[t] = ph >= 2 ? -ps.c : ps.c;
      tim[t] = (unsigned char)(ph & 1);
    }
    gstart.push_back(nt);
    const int ng = (int)gx.size();
    // one allocation, 8-byte aligned pieces
    const size_t o_gx = 0, o_gs = o_gx + 8 * ((ng * sizeof(unsigned) + 7) / 8);
    const size_t o_tz = o_gs + 8 * (((ng + 1) * sizeof(int) + 7) / 8);
    const size_t o_top = o_tz + 8 * ((nt * sizeof(unsigned) + 7) / 8);
    const size_t o_tc = o_top + 8 * ((nt * sizeof(int) + 7) / 8);
    const size_t o_tim = o_tc + (size_t)nt * sizeof(double);
    const size_t o_gre = o_tim + 8 * (((size_t)nt + 7) / 8);
    const size_t bytes = o_gre + (size_t)ng + 8;
    std::vector<unsigned char> greal(ng, 1);
    for (int g = 0; g < ng; ++g)
      for (int t = gstart[g]; t < gstart[g + 1]; ++t)
        if (tim[t]) greal[g] = 0;
    std::vector<unsigned char> blob(bytes, 0);
    if (ng) std::memcpy(blob.data() + o_gx, gx.data(), ng * sizeof(unsigned));
    std::memcpy(blob.data() + o_gs, gstart.data(), (ng + 1) * sizeof(int));
    if (nt) {
      std::memcpy(blob.data() + o_tz, tz.data(), nt * sizeof(unsigned));
      std::memcpy(blob.data() + o_top, top.data(), nt * sizeof(int));
      std::memcpy(blob.data() + o_tc, tc.data(), nt * sizeof(double));
      std::memcpy(blob.data() + o_tim, tim.data(), nt);
    }
    if (ng) std::memcpy(blob.data() + o_gre, greal.data(), ng);
    CKC(cudaMalloc(&ctx->d_pauli, bytes), "cudaMalloc(Pauli tables)");
    CKC(cudaMemcpy(ctx->d_pauli, blob.data(), bytes, cudaMemcpyHostToDevice), "upload Pauli tables");
    unsigned char* base = (unsigned char*)ctx->d_pauli;
    ctx->pauli.N = nsites;
    ctx->pauli.ngroups = ng;
    ctx->pauli.nterms = nt;
    ctx->pauli.gx = (const unsigned*)(base + o_gx);
    ctx->pauli.gstart = (const int*)(base + o_gs);
    ctx->pauli.tz = (const unsigned*)(base + o_tz);
    ctx->pauli.top = (const int*)(base + o_top);
    ctx->pauli.tc = (const double*)(base + o_tc);
    ctx->pauli.tim = base + o_tim;
    ctx->pauli.greal = base + o_gre;
    ctx->pauli.g0 = 0;
    ctx->pauli.nd = 0;
    ctx->pauli.dtab = nullptr;
    // Z-only strings (group 0 when its X mask is 0): per-operator tables over
    // all indices when they take at most 2 GiB
    if (ng > 0 && gx[0] == 0u) {
      const int n0 = gstart[1];
      bool has[1 + kMaxDrives] = {};
      for (int t = 0; t < n0; ++t) has[top[t]] = true;
      int nd = 0;
      for (int o2 = 0; o2 <= nV; ++o2)
        if (has[o2]) ctx->pauli.dop[nd++] = o2;
      if (nd > 0 && (size_t)nd * ((size_t)1 << nsites) * sizeof(double) <= (size_t(2) << 30)) {
        CKC(cudaMalloc(&ctx->d_pauli_dtab, (size_t)nd * ((size_t)1 << nsites) * sizeof(double)),
            "cudaMalloc(Pauli diagonal tables)");
        ctx->pauli.nd = nd;
        const int e = launch_pauli_diag_table(ctx->pauli, n0, ctx->d_pauli_dtab, nullptr);
        const cudaError_t es = cudaDeviceSynchronize();
        CKC((cudaError_t)e, "Pauli diagonal table kernel");
        CKC(es, "Pauli diagonal table kernel");
        ctx->pauli.dtab = ctx->d_pauli_dtab;
        ctx->pauli.g0 = 1;
      }
    }
  }
  if (family == kFamilySpin) {
    const int N = nsites;
    const int L = N < 10 ? N : 10;
    const size_t nlo = size_t(1) << L, nhi = size_t(1) << (N - L + 1);
    double* d_h = nullptr;
    CKC(cudaMalloc(&ctx->d_dz_lo, nlo * sizeof(double)), "cudaMalloc(dz_lo)");
    CKC(cudaMalloc(&ctx->d_dz_hi, nhi * sizeof(double)), "cudaMalloc(dz_hi)");
    CKC(cudaMalloc(&d_h, N * sizeof(double)), "cudaMalloc(h)");
    CKC(cudaMemcpy(d_h, H0->site_coeff, N * sizeof(double), cudaMemcpyHostToDevice), "upload h");
    int e = launch_spin_tables(N, L, H0->J, H0->Delta, d_h, ctx->d_dz_lo, ctx->d_dz_hi, nullptr);
    cudaError_t es = cudaDeviceSynchronize();
    cudaFree(d_h);
    CKC((cudaError_t)e, "spin table kernel");
    CKC(es, "spin table kernel");
    std::vector<double> xf((size_t)(nV > 0 ? nV : 1) * N, 0.0);
    for (int k = 0; k < nV; ++k)
      for (int i = 0; i < N; ++i) xf[(size_t)k * N + i] = V[k].site_coeff[i];
    CKC(cudaMalloc(&ctx->d_xf, xf.size() * sizeof(double)), "cudaMalloc(xf)");
    CKC(cudaMemcpy(ctx->d_xf, xf.data(), xf.size() * sizeof(double), cudaMemcpyHostToDevice), "upload xf");
    ctx->spin.N = N;
    ctx->spin.lo_bits = L;
    ctx->spin.J2 = 2.0 * H0->J;
    ctx->spin.dz_lo = ctx->d_dz_lo;
    ctx->spin.dz_hi = ctx->d_dz_hi;
    ctx->spin.xf = ctx->d_xf;
    // fixed-point diagonal tables: DZ = round(dz * 2^-E_dz), |DZ_lo + DZ_hi| < 2^61
    std::vector<double> lo(nlo), hi(nhi);
    CKC(cudaMemcpy(lo.data(), ctx->d_dz_lo, nlo * sizeof(double), cudaMemcpyDeviceToHost), "download dz_lo");
    CKC(cudaMemcpy(hi.data(), ctx->d_dz_hi, nhi * sizeof(double), cudaMemcpyDeviceToHost), "download dz_hi");
    double mlo = 0.0, mhi = 0.0;
    for (double v : lo) mlo = std::fmax(mlo, std::fabs(v));
    for (double v : hi) mhi = std::fmax(mhi, std::fabs(v));
    const double maxdz = (mlo + mhi) * (1.0 + 1e-12);
    int E_dz = 0;
    if (maxdz > 0.0) {
      int ex = 0;
      std::frexp(maxdz, &ex);          // maxdz < 2^ex
      E_dz = ex - 60;                  // |DZ| < 2^60 each
    }
    std::vector<long long> dz((size_t)nlo + nhi);
    for (size_t i = 0; i < nlo; ++i) dz[i] = std::llrint(std::ldexp(lo[i], -E_dz));
    for (size_t i = 0; i < nhi; ++i) dz[nlo + i] = std::llrint(std::ldexp(hi[i], -E_dz));
    CKC(cudaMalloc(&ctx->d_DZ, dz.size() * sizeof(long long)), "cudaMalloc(DZ)");
    CKC(cudaMemcpy(ctx->d_DZ, dz.data(), dz.size() * sizeof(long long), cudaMemcpyHostToDevice), "upload DZ");
    bool uniform = true;
    for (int k = 0; k < nV; ++k)
      for (int i = 1; i < N; ++i)
        if (V[k].site_coeff[i] != V[k].site_coeff[0]) uniform = false;
    ctx->spin_fx.N = N;
    ctx->spin_fx.lo_bits = L;
    ctx->spin_fx.E_dz = E_dz;
    ctx->spin_fx.uniform = uniform ? 1 : 0;
    ctx->spin_fx.DZ_lo = ctx->d_DZ;
    ctx->spin_fx.DZ_hi = ctx->d_DZ + nlo;
    ctx->spin_fx.maxdz = maxdz;
    ctx->spin_fx.nbond = (double)(N - 1);
    ctx->spin_fx.nsite = (double)N;
    ctx->spin_fx.J2 = 2.0 * H0->J;
    ctx->spin_fx.xf = ctx->d_xf;
    // FP32 diagonal tables of the mixed-precision path
    std::vector<float> dz32((size_t)nlo + nhi);
    for (size_t i = 0; i < nlo; ++i) dz32[i] = (float)lo[i];
    for (size_t i = 0; i < nhi; ++i) dz32[nlo + i] = (float)hi[i];
    CKC(cudaMalloc(&ctx->d_dz32, dz32.size() * sizeof(float)), "cudaMalloc(dz32)");
    CKC(cudaMemcpy(ctx->d_dz32, dz32.data(), dz32.size() * sizeof(float), cudaMemcpyHostToDevice), "upload dz32");
    ctx->spin_c.N = N;
    ctx->spin_c.lo_bits = L;
    ctx->spin_c.uniform = uniform ? 1 : 0;
    ctx->spin_c.J2 = 2.0 * H0->J;
    ctx->spin_c.dz_lo = ctx->d_dz32;
    ctx->spin_c.dz_hi = ctx->d_dz32 + nlo;
    ctx->spin_c.xf = ctx->d_xf;
    spin_h0_interval(N, H0->J, H0->Delta, H0->site_coeff, &ctx->op_lo[0], &ctx->op_hi[0]);
    ctx->ip_J = H0->J;
    ctx->ip_Delta = H0->Delta;
    ctx->ip_h.assign(H0->site_coeff, H0->site_coeff + N);
    ctx->ip_xf = xf;
    for (int k = 0; k < nV; ++k) xfield_interval(N, V[k].site_coeff, &ctx->op_lo[1 + k], &ctx->op_hi[1 + k]);
  } else if (family == kFamilyDia) {
    std::vector<long long> off;
    std::vector<int> opidx;
    for (int k = -1; k < nV; ++k) {
      const cfet_op& o2 = k < 0 ? *H0 : V[k];
      for (int d = 0; d < o2.ndiag; ++d) {
        off.push_back(o2.offsets[d]);
        opidx.push_back(k + 1);
      }
    }
    const int nd = (int)off.size();
    CKC(cudaMalloc(&ctx->d_off, nd * sizeof(long long)), "cudaMalloc(offsets)");
    CKC(cudaMalloc(&ctx->d_opidx, nd * sizeof(int)), "cudaMalloc(opidx)");
    CKC(cudaMalloc(&ctx->d_val, (size_t)nd * dim * sizeof(double)), "cudaMalloc(values)");
    CKC(cudaMemcpy(ctx->d_off, off.data(), nd * sizeof(long long), cudaMemcpyHostToDevice), "upload offsets");
    CKC(cudaMemcpy(ctx->d_opidx, opidx.data(), nd * sizeof(int), cudaMemcpyHostToDevice), "upload opidx");
    size_t row = 0;
    for (int k = -1; k < nV; ++k) {
      const cfet_op& o2 = k < 0 ? *H0 : V[k];
      CKC(cudaMemcpy(ctx->d_val + row * dim, o2.values, (size_t)o2.ndiag * dim * sizeof(double),
                     cudaMemcpyHostToDevice), "upload values");
      row += o2.ndiag;
    }
    ctx->dia.ndiag = nd;
    ctx->dia.off = ctx->d_off;
    ctx->dia.opidx = ctx->d_opidx;
    ctx->dia.val = ctx->d_val;
    // fixed-point values: one exponent per operator, |VAL| < 2^62; row bound
    OpDiaFx& fx = ctx->dia_fx;
    fx.ndiag = nd;
    fx.nops = 1 + nV;
    fx.off = ctx->d_off;
    fx.opidx = ctx->d_opidx;
    std::vector<long long> VAL((size_t)nd * dim);
    std::vector<float> val32((size_t)nd * dim);
    OpDiaC& dc = ctx->dia_c;
    dc.ndiag = nd;
    dc.nops = 1 + nV;
    dc.off = ctx->d_off;
    int dcur = 0;
    for (int k = -1; k < nV; ++k) {
      const cfet_op& o2 = k < 0 ? *H0 : V[k];
      const int oi = k + 1;
      double vmax = 0.0;
      std::vector<double> rowsum(dim, 0.0);
      for (int d = 0; d < o2.ndiag; ++d)
        for (int r = 0; r < dim; ++r) {
          const long long c = (long long)r + o2.offsets[d];
          const double v = (c >= 0 && c < dim) ? std::fabs(o2.values[(size_t)d * dim + r]) : 0.0;
          vmax = std::fmax(vmax, v);
          rowsum[r] += v;
        }
      int E_op = 0;
      if (vmax > 0.0) {
        int ex = 0;
        std::frexp(vmax * (1.0 + 1e-12), &ex);
        E_op = ex - 62;
      }
      double mrow = 0.0;
      for (double v : rowsum) mrow = std::fmax(mrow, v);
      fx.E_op[oi] = E_op;
      fx.maxrow[oi] = mrow * (1.0 + 1e-12);
      fx.dfirst[oi] = dcur;
      fx.dcount[oi] = o2.ndiag;
      dc.dfirst[oi] = dcur;
      dc.dcount[oi] = o2.ndiag;
      for (int d = 0; d < o2.ndiag; ++d, ++dcur)
        for (int r = 0; r < dim; ++r) {
          const long long c = (long long)r + o2.offsets[d];
          const double v = (c >= 0 && c < dim) ? o2.values[(size_t)d * dim + r] : 0.0;
          VAL[(size_t)dcur * dim + r] = std::llrint(std::ldexp(v, -E_op));
          val32[(size_t)dcur * dim + r] = (float)v;
        }
    }
    CKC(cudaMalloc(&ctx->d_VAL, VAL.size() * sizeof(long long)), "cudaMalloc(VAL)");
    CKC(cudaMemcpy(ctx->d_VAL, VAL.data(), VAL.size() * sizeof(long long), cudaMemcpyHostToDevice), "upload VAL");
    fx.VAL = ctx->d_VAL;
    CKC(cudaMalloc(&ctx->d_val32, val32.size() * sizeof(float)), "cudaMalloc(val32)");
    CKC(cudaMemcpy(ctx->d_val32, val32.data(), val32.size() * sizeof(float), cudaMemcpyHostToDevice),
        "upload val32");
    dc.val = ctx->d_val32;
    for (int k = -1; k < nV; ++k) {
      const cfet_op& o2 = k < 0 ? *H0 : V[k];
      dia_interval(o2.offsets, o2.values, o2.ndiag, dim, &ctx->op_lo[k + 1], &ctx->op_hi[k + 1]);
    }
  }
  if (family == kFamilyCsr) {
    cfet_status cs = csr_upload(ctx, H0, nV, V);
    if (cs != CFET_OK) {
      free_ctx(ctx);
      return cs;
    }
  }
  // long chains: the window-tiled apply of the complex64 and fixed-point
  // Krylov kernels
  if (family == kFamilySpin && (ctx->precision == CFET_PREC_C64 || ctx->precision == CFET_PREC_FX)) {
    const int min_sites = ctx->precision == CFET_PREC_C64 ? kC64TiledMinSites : kFxTiledMinSites;
    const bool want_tiled = o.apply_form == CFET_APPLY_AUTO ? nsites >= min_sites : o.apply_form == CFET_APPLY_TILED;
    ctx->tiled = want_tiled && nsites >= kTiledMinSites && nsites <= kTiledMaxSites;
  }
  // persistent grid: co-resident maximum, no more CTAs than needed to give
  // every thread at least one element
  int maxg = ctx->precision == CFET_PREC_FX    ? max_coresident_blocks_fx(family, ctx->block, ctx->tiled)
                   : ctx->precision == CFET_PREC_C64 ? max_coresident_blocks_c64(family, ctx->block, ctx->tiled)
                   : family == kFamilyPauli          ? max_coresident_blocks_pauli(ctx->block, ctx->pauli.nterms)
                                                     : max_coresident_blocks(family, ctx->block);
  if (maxg < 1) {
    free_ctx(ctx);
    return fail(nullptr, CFET_ECUDA, "occupancy query failed for the persistent kernel");
  }
  if (o.picture == CFET_PICTURE_INTERACTION) {  // the interaction-picture form of the FP64 kernel
    const int mi = max_coresident_blocks_ip(ctx->block, kIPWeightsPerSite * (2 * nsites - 1));
    if (mi < 1) {
      free_ctx(ctx);
      return fail(nullptr, CFET_ECUDA, "occupancy query failed for the interaction-picture kernel");
    }
    if (mi < maxg) maxg = mi;
  }
  if (o.expm == CFET_EXPM_CHEBYSHEV) {  // the Chebyshev kernel: the same workers, no control warp
    const int mc = max_coresident_blocks_cheb(family, cheb_threads(ctx->block - 32));
    if (mc < 1) {
      free_ctx(ctx);
      return fail(nullptr, CFET_ECUDA, "occupancy query failed for the Chebyshev kernel");
    }
    if (mc < maxg) maxg = mc;
  }
  // element threads per CTA (the fixed-point kernel adds one control warp)
  const int workers = ctl_warp ? ctx->block - 32 : ctx->block;
  int want = (dim + workers - 1) / workers;
  if (o.grid_size > 0) want = o.grid_size;
  ctx->grid = want < maxg ? want : maxg;
  if (ctl_warp && ctx->grid > kMaxCtlGrid) ctx->grid = kMaxCtlGrid;  // record exchange limit
  if (ctx->grid < 1) ctx->grid = 1;

  if (ctx->precision == CFET_PREC_FX && o.expm == CFET_EXPM_KRYLOV && ctx->grid == 1 && !ctx->tiled) {
    // a single CTA: the basis fits in its shared memory for small problems
    const size_t sb = fx_small_smem_bytes(dim, o.m_max);
    if (sb > 0 && fx_small_prepare(sb) == 0) {
      ctx->small_fx = true;
      ctx->small_block = 32 + std::min(ctx->block - 32, (dim + 31) / 32 * 32);
    }
  }
  if (ctx->precision == CFET_PREC_FX)  // basis q_1..q_{m_max+1}; the Chebyshev kernel's three vectors
    CKC(cudaMalloc(&ctx->d_qbasis, (size_t)std::max(o.m_max + 1, 3) * dim * sizeof(longlong2)),
        "cudaMalloc(Krylov basis)");
  else if (ctx->precision == CFET_PREC_C64)
    CKC(cudaMalloc(&ctx->d_qbasis32, (size_t)(o.m_max + 1) * dim * sizeof(float2)), "cudaMalloc(Krylov basis)");
  if ((ctx->precision == CFET_PREC_C64 || ctx->precision == CFET_PREC_FX) && ctx->tiled) {
    const cfet_status ts = build_tile_maps(ctx, nsites, o.m_max + 1, ctx->precision == CFET_PREC_FX);
    if (ts != CFET_OK) {
      free_ctx(ctx);
      return ts;
    }
  }
  else
    CKC(cudaMalloc(&ctx->d_basis, (size_t)o.m_max * dim * sizeof(double2)), "cudaMalloc(Krylov basis)");
  if (ctx->precision == CFET_PREC_FX) {
    // exact per-thread sums stay below 2^127 for at most 4096 elements per thread
    const long long per_thread = ((long long)dim + (long long)ctx->grid * workers - 1) / ((long long)ctx->grid * workers);
    if (per_thread > 4096) {
      free_ctx(ctx);
      return fail(nullptr, CFET_EINVAL, "fixed-point precision: dimension too large for the grid, use CFET_PREC_F64");
    }
  }
  CKC(cudaMalloc(&ctx->d_partials, partial_words_per_cta(ctx) * (size_t)ctx->grid * sizeof(double)),
      "cudaMalloc(partials)");
  CKC(cudaMalloc(&ctx->d_bar, 2 * sizeof(unsigned)), "cudaMalloc(barrier)");
  CKC(cudaMemset(ctx->d_bar, 0, 2 * sizeof(unsigned)), "barrier init");
  CKC(cudaMalloc(&ctx->d_st, sizeof(DevStatus)), "cudaMalloc(status)");
  CKC(cudaMemset(ctx->d_st, 0, sizeof(DevStatus)), "status init");
  CKC(cudaMallocHost(&ctx->h_st, sizeof(DevStatus)), "cudaMallocHost(status)");
  std::memset(ctx->h_st, 0, sizeof(DevStatus));
  CKC(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "capture stream");
  CKC(cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming), "event");
  CKC(cudaEventCreate(&ctx->ev_k0), "event");
  CKC(cudaEventCreate(&ctx->ev_k1), "event");
#undef CKC
  *out = ctx;
  return CFET_OK;
}

void cfet_destroy(cfet_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->ev_pending) cudaEventSynchronize(ctx->ev_done);
  free_ctx(ctx);
}

cfet_status cfet_apply(cfet_ctx* ctx, const double* c, const void* v_in, void* v_out, void* stream) {
  if (!ctx) return CFET_EINVAL;
  if (!c) return fail(ctx, CFET_EINVAL, "coefficients are NULL");
  for (int i = 0; i <= ctx->nV; ++i)
    if (!is_finite_d(c[i])) return fail(ctx, CFET_EINVAL, "coefficient not finite");
  cfet_status s = check_psi(ctx, v_in);
  if (s != CFET_OK) return s;
  if ((s = check_psi(ctx, v_out)) != CFET_OK) return s;
  const char* a = (const char*)v_in;
  const char* b = (const char*)v_out;
  const size_t bytes = (size_t)ctx->dim * sizeof(double2);
  if (a < b + bytes && b < a + bytes) return fail(ctx, CFET_EINVAL, "v_in and v_out overlap");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  int e = ctx->family == kFamilySpin
              ? launch_apply_spin(ctx->spin, ctx->dim, c, ctx->nV, (const double2*)v_in, (double2*)v_out, stream)
          : ctx->family == kFamilyPauli
              ? launch_apply_pauli(ctx->pauli, ctx->dim, c, ctx->nV, (const double2*)v_in, (double2*)v_out, stream)
          : ctx->family == kFamilyCsr
              ? launch_apply_csr(ctx->csr, ctx->dim, c, ctx->nV, (const double2*)v_in, (double2*)v_out, stream)
              : launch_apply_dia(ctx->dia, ctx->dim, c, ctx->nV, (const double2*)v_in, (double2*)v_out, stream);
  if (e != cudaSuccess) return cuda_fail(ctx, (cudaError_t)e, "apply kernel launch");
  return CFET_OK;
}

cfet_status cfet_expv(cfet_ctx* ctx, const double* c, double tau, void* psi, double tol, void* stream,
                      cfet_stats* stats) {
  if (!ctx) return CFET_EINVAL;
  if (!c) return fail(ctx, CFET_EINVAL, "coefficients are NULL");
  for (int i = 0; i <= ctx->nV; ++i)
    if (!is_finite_d(c[i])) return fail(ctx, CFET_EINVAL, "coefficient not finite");
  if (!is_finite_d(tau) || tau == 0.0) return fail(ctx, CFET_EINVAL, "tau must be finite and non-zero");
  if (!is_finite_d(tol)) return fail(ctx, CFET_EINVAL, "tol not finite");
  cfet_status s = check_psi(ctx, psi);
  if (s != CFET_OK) return s;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if ((s = ensure_scal(ctx, 1 + ctx->nV)) != CFET_OK) return s;
  if (ctx->ev_pending) { cudaEventSynchronize(ctx->ev_done); ctx->ev_pending = false; }
  for (int i = 0; i <= ctx->nV; ++i) ctx->h_scal[i] = c[i];
  size_t table_n = 1 + ctx->nV;
  const bool cheb = ctx->opt.expm == CFET_EXPM_CHEBYSHEV;
  if (cheb && (s = stage_cheb_table(ctx, 1, tau, tol, &table_n)) != CFET_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  PropParams p = base_params(ctx, (double2*)psi, tau, tol);
  if (cheb) set_cheb_params(ctx, p, 1);
  if ((s = issue_sequence(ctx, p, 1, 1, table_n * sizeof(double), st, false)) != CFET_OK) return s;
  CK(cudaEventRecord(ctx->ev_done, st), "event record");
  ctx->ev_pending = true;
  if (stats) return finish(ctx, st, stats);
  return CFET_OK;
}

cfet_status cfet_propagate_ex(cfet_ctx* ctx, void* psi, double t0, double dt, int64_t nsteps, int32_t order,
                              int32_t scheme, double krylov_tol, void* stream, const cfet_decisions* forced,
                              cfet_decisions* record, cfet_stats* stats) {
  if (!ctx) return CFET_EINVAL;
  cfet_status s = check_psi(ctx, psi);
  if (s != CFET_OK) return s;
  if (!is_finite_d(t0) || !is_finite_d(dt) || dt == 0.0) return fail(ctx, CFET_EINVAL, "t0, dt must be finite, dt != 0");
  if (!is_finite_d(krylov_tol)) return fail(ctx, CFET_EINVAL, "krylov_tol not finite");
  if (nsteps < 0) return fail(ctx, CFET_EINVAL, "nsteps must be >= 0");
  int id = scheme;
  if (id == CFET_SCHEME_DEFAULT) {
    id = default_scheme_for_order(order);
    if (!id) return fail(ctx, CFET_EINVAL, "order must be 2, 4, 6 or 8");
  }
  SchemeData sd;
  if (!build_scheme(id, &sd)) return fail(ctx, CFET_EINVAL, "unknown scheme id");
  if (scheme != CFET_SCHEME_DEFAULT && order != 0 && order != sd.order)
    return fail(ctx, CFET_EINVAL, "order does not match the scheme");
  if (nsteps == 0) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    return CFET_OK;
  }
  const long long nexp = nsteps * (long long)sd.s;
  const int ncoef = 1 + ctx->nV;
  const bool cheb = ctx->opt.expm == CFET_EXPM_CHEBYSHEV;
  if (cheb && (forced || record))
    return fail(ctx, CFET_EINVAL, "Chebyshev stage exponentials take no Krylov decision logs");
  if (forced) {
    if (forced->n_exp != nexp || !forced->n_sub || !forced->k || !forced->h || forced->len < nexp)
      return fail(ctx, CFET_EINVAL, "forced decisions do not cover nsteps * s exponentials");
    long long tot = 0;
    for (long long e = 0; e < nexp; ++e) {
      if (forced->n_sub[e] < 1) return fail(ctx, CFET_EINVAL, "forced decisions: n_sub < 1");
      tot += forced->n_sub[e];
    }
    if (tot != forced->len || tot > forced->cap) return fail(ctx, CFET_EINVAL, "forced decisions: len mismatch");
    for (long long i = 0; i < tot; ++i)
      if (forced->k[i] < 1 || forced->k[i] > ctx->opt.m_max || forced->h[i] < 0 || forced->h[i] > 60)
        return fail(ctx, CFET_EINVAL, "forced decisions: k or h out of range");
  }
  if (record && (record->n_exp != nexp || !record->n_sub || !record->k || !record->h || record->cap < 0))
    return fail(ctx, CFET_EINVAL, "record must cover nsteps * s exponentials");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if ((s = ensure_scal(ctx, (size_t)nexp * ncoef)) != CFET_OK) return s;
  // decision buffers: [f_nsub nexp | f_k len | f_h len | r_nsub nexp | r_k cap | r_h cap]
  const size_t flen = forced ? (size_t)forced->len : 0;
  const size_t rcap = record ? (size_t)record->cap : 0;
  const size_t nf = forced ? (size_t)nexp + 2 * flen : 0;
  const size_t nr = record ? (size_t)nexp + 2 * rcap : 0;
  if (nf + nr > 0 && (s = ensure_dec(ctx, nf + nr)) != CFET_OK) return s;
  // the previous call's graph may still read the pinned table
  if (ctx->ev_pending) { cudaEventSynchronize(ctx->ev_done); ctx->ev_pending = false; }

  const bool ip = ctx->opt.picture == CFET_PICTURE_INTERACTION;
  const int ipnw = ip ? kIPWeightsPerSite * (2 * ctx->spin.N - 1) : 0;
  std::vector<double> ipw(ip ? (size_t)nexp * ipnw * 2 : 0);
  // ---- stage scalars (host): drives at the Gauss-Legendre nodes of each step
  std::vector<double> fval((size_t)sd.M * (ctx->nV > 0 ? ctx->nV : 1));
  for (long long n = 0; n < nsteps; ++n) {
    const double t = t0 + (double)n * dt;
    for (int m = 0; m < sd.M; ++m)
      for (int k = 0; k < ctx->nV; ++k) {
        const double v = ctx->f[k](t + sd.x[m] * dt, ctx->f_user[k]);
        if (!is_finite_d(v)) return fail(ctx, CFET_EINVAL, "drive returned a non-finite value");
        fval[(size_t)m * ctx->nV + k] = v;
      }
    if (ip) ip_step_weights(ctx, sd, t, dt, fval, ipw.data() + (size_t)n * sd.s * ipnw * 2);
    for (int jj = 0; jj < sd.s; ++jj) {
      const int j = sd.s - 1 - jj;  // exp(Omega_s) acts first
      double* row = ctx->h_scal + ((size_t)n * sd.s + jj) * ncoef;
      double c0 = 0.0;
      for (int m = 0; m < sd.M; ++m) c0 += sd.g[j][m];
      row[0] = c0;
      for (int k = 0; k < ctx->nV; ++k) {
        double ck = 0.0;
        for (int m = 0; m < sd.M; ++m) ck += sd.g[j][m] * fval[(size_t)m * ctx->nV + k];
        row[1 + k] = ck;
      }
    }
  }
  size_t table_n = (size_t)nexp * ncoef;
  if (cheb && (s = stage_cheb_table(ctx, nexp, dt, krylov_tol, &table_n)) != CFET_OK) return s;
  size_t ip_off_t = 0, ip_off_w = 0;
  if (ip) {  // [rows][pad][t0, t_end][weights], the weights 16-byte aligned
    ip_off_t = (table_n + 1) & ~size_t(1);
    ip_off_w = ip_off_t + 2;
    const size_t total = ip_off_w + ipw.size();
    std::vector<double> rows(ctx->h_scal, ctx->h_scal + table_n);
    if ((s = ensure_scal(ctx, total)) != CFET_OK) return s;
    std::memcpy(ctx->h_scal, rows.data(), rows.size() * sizeof(double));
    ctx->h_scal[ip_off_t] = t0;
    ctx->h_scal[ip_off_t + 1] = t0 + (double)nsteps * dt;
    std::memcpy(ctx->h_scal + ip_off_w, ipw.data(), ipw.size() * sizeof(double));
    table_n = total;
  }
  // ---- forced decisions blob (host staging)
  std::vector<int> fblob;
  if (forced) {
    fblob.resize(nf);
    for (long long e = 0; e < nexp; ++e) fblob[e] = forced->n_sub[e];
    for (size_t i = 0; i < flen; ++i) {
      fblob[nexp + i] = forced->k[i];
      fblob[nexp + flen + i] = forced->h[i];
    }
  }
  if (forced) CK(cudaMemcpy(ctx->d_dec, fblob.data(), nf * sizeof(int), cudaMemcpyHostToDevice), "decision upload");
  PropParams p = base_params(ctx, (double2*)psi, dt, krylov_tol);
  if (cheb) set_cheb_params(ctx, p, nexp);
  if (ip) {
    p.ip_times = ctx->d_scal + ip_off_t;
    p.ip_w = reinterpret_cast<const double2*>(ctx->d_scal + ip_off_w);
    p.ip_nw = ipnw;
  }
  if (forced) {
    p.f_nsub = ctx->d_dec;
    p.f_k = ctx->d_dec + nexp;
    p.f_h = ctx->d_dec + nexp + flen;
  }
  if (record) {
    int* r = ctx->d_dec + nf;
    p.r_nsub = r;
    p.r_k = r + nexp;
    p.r_h = r + nexp + rcap;
    p.r_cap = (long long)rcap;
  }
  const long long chunk = (long long)ctx->opt.steps_per_launch * sd.s;
  cudaStream_t user = (cudaStream_t)stream;
  // ---- capture the launch sequence and replay it on the caller's stream; an
  // unchanged sequence (same buffers, sizes and scalars; the stage table is
  // re-read from the pinned buffer by the graph's own copy) is relaunched as is
  cfet_ctx::GraphKey key;
  key.psi = psi;
  key.scal = ctx->d_scal;
  key.dec = ctx->d_dec;
  key.nexp = nexp;
  key.chunk = chunk;
  key.flen = (long long)flen;
  key.rcap = (long long)rcap;
  key.table_bytes = table_n * sizeof(double);
  key.nf = nf;
  key.tau = dt;
  key.tol = krylov_tol;
  key.has_f = forced != nullptr;
  key.has_r = record != nullptr;
  if (!(ctx->gexec && key == ctx->gkey)) {
    ctx->gkey = cfet_ctx::GraphKey();
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    s = issue_sequence(ctx, p, nexp, chunk, table_n * sizeof(double), ctx->cap_stream, true);
    cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (s != CFET_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (ec != cudaSuccess) return cuda_fail(ctx, ec, "end capture");
    bool updated = false;
    if (ctx->gexec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(ctx->gexec, graph, &info) == cudaSuccess) updated = true;
      else {
        cudaGetLastError();
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
      }
    }
    if (!updated) {
      cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, graph, 0);
      if (ei != cudaSuccess) {
        cudaGraphDestroy(graph);
        ctx->gexec = nullptr;
        return cuda_fail(ctx, ei, "graph instantiate");
      }
    }
    cudaGraphDestroy(graph);
    ctx->gkey = key;
  }
  CK(cudaGraphLaunch(ctx->gexec, user), "graph launch");
  ctx->timed = true;
  CK(cudaEventRecord(ctx->ev_done, user), "event record");
  ctx->ev_pending = true;
  if (!stats && !record) return CFET_OK;
  cfet_stats tmp;
  s = finish(ctx, user, stats ? stats : &tmp);
  if (record) {
    // copy decisions back (device -> host), synchronous
    const DevStatus& hs = *ctx->h_st;
    const long long len = hs.rec_pos < (long long)rcap ? hs.rec_pos : (long long)rcap;
    int* r = ctx->d_dec + nf;
    CK(cudaMemcpy(record->n_sub, r, nexp * sizeof(int), cudaMemcpyDeviceToHost), "record n_sub");
    if (len > 0) {
      CK(cudaMemcpy(record->k, r + nexp, len * sizeof(int), cudaMemcpyDeviceToHost), "record k");
      CK(cudaMemcpy(record->h, r + nexp + rcap, len * sizeof(int), cudaMemcpyDeviceToHost), "record h");
    }
    record->len = hs.rec_pos;
    if (s == CFET_OK && hs.rec_overflow) return fail(ctx, CFET_EINVAL, "decision record capacity too small");
  }
  return s;
}

cfet_status cfet_propagate(cfet_ctx* ctx, void* psi, double t0, double dt, int64_t nsteps, int32_t order,
                           double krylov_tol, void* stream, cfet_stats* stats) {
  return cfet_propagate_ex(ctx, psi, t0, dt, nsteps, order, CFET_SCHEME_DEFAULT, krylov_tol, stream, nullptr,
                           nullptr, stats);
}

cfet_status cfet_propagate_host(cfet_ctx* ctx, void* psi_host, double t0, double dt, int64_t nsteps, int32_t order,
                                double krylov_tol, void* stream, cfet_stats* stats) {
  if (!ctx) return CFET_EINVAL;
  if (!psi_host) return fail(ctx, CFET_EINVAL, "psi_host is NULL");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t bytes = (size_t)ctx->dim * sizeof(double2);
  if (!ctx->d_psi_e2e) CK(cudaMalloc(&ctx->d_psi_e2e, bytes), "cudaMalloc(psi staging)");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(ctx->d_psi_e2e, psi_host, bytes, cudaMemcpyHostToDevice, st), "psi upload");
  cfet_stats tmp;
  cfet_status s = cfet_propagate(ctx, ctx->d_psi_e2e, t0, dt, nsteps, order, krylov_tol, stream,
                                 stats ? stats : &tmp);
  if (s != CFET_OK) return s;
  CK(cudaMemcpyAsync(psi_host, ctx->d_psi_e2e, bytes, cudaMemcpyDeviceToHost, st), "psi download");
  CK(cudaStreamSynchronize(st), "stream synchronize");
  return CFET_OK;
}

cfet_status cfet_kernel_time_ms(cfet_ctx* ctx, float* ms) {
  if (!ctx || !ms) return CFET_EINVAL;
  if (!ctx->timed) return fail(ctx, CFET_EINVAL, "no timed propagation yet");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(cudaEventSynchronize(ctx->ev_k1), "event synchronize");
  CK(cudaEventElapsedTime(ms, ctx->ev_k0, ctx->ev_k1), "event elapsed");
  return CFET_OK;
}

cfet_status cfet_sync(cfet_ctx* ctx, void* stream, cfet_stats* stats) {
  if (!ctx) return CFET_EINVAL;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  return finish(ctx, (cudaStream_t)stream, stats);
}

// Host check of the window tiling of the long-chain kernels (tiled_common.cuh,
// tiles of 2^tile_bits elements): every element in exactly one tile slot per
// window, every flip and every bond in exactly one window, the 16-byte copy
// units of complex64 tiles (element pairs) contiguous and aligned, and the
// window count within its bound.
extern "C++" {
// TMA geometry of window w of a window-tiled apply: tiles of 2^TB elements
// of wpe 8-byte words (complex64: TB 12, one word; fixed point: TB 11, an int64
// pair), a map over the whole Krylov basis of nvec contiguous vectors, so that
// the vector index continues the outermost dimension, all in words.  Window 0
// views the basis as rows of 256 words (box: one tile's rows); window w >= 1
// splits the index into its bits [0, c) (2^c wpe words, as 256 x 2^c wpe / 256
// beyond 256 words: a box dimension holds at most 256), [c, b0), the window's
// bits [b0, b0 + width) and the rest (box: the low bits x 1 x 2^width x 1).
struct TileMapGeom {
  int rank;
  uint64_t dims[5];
  uint64_t strides[4];  // bytes, dimensions 1 .. rank - 1
  uint32_t box[5];
};
static void tile_map_geometry(int N, int TB, int wpe, int w, const TileWin& W, int nvec, TileMapGeom* g) {
  const uint64_t e = 8 * (uint64_t)wpe, dim = uint64_t(1) << N, nv = (uint64_t)nvec;
  const int rs = wpe == 2 ? 7 : 8;  // log2 of the elements per 256-word row
  if (w == 0) {
    *g = TileMapGeom{2, {256, (dim >> rs) * nv, 0, 0, 0}, {256 * 8, 0, 0, 0},
                     {256, (uint32_t)(1u << (TB - rs)), 0, 0, 0}};
    return;
  }
  const int c = W.c, b0 = W.b0, wd = W.width;
  const uint64_t lo = (uint64_t(1) << c) * (uint64_t)wpe, mid = uint64_t(1) << (b0 - c), win = uint64_t(1) << wd;
  const uint64_t rest = (uint64_t(1) << (N - b0 - wd)) * nv;
  const uint64_t s_mid = (uint64_t(1) << c) * e, s_win = (uint64_t(1) << b0) * e, s_rest = (uint64_t(1) << (b0 + wd)) * e;
  if (lo <= 256)
    *g = TileMapGeom{4, {lo, mid, win, rest, 0}, {s_mid, s_win, s_rest, 0}, {(uint32_t)lo, 1, (uint32_t)win, 1, 0}};
  else
    *g = TileMapGeom{5, {256, lo >> 8, mid, win, rest}, {256 * 8, s_mid, s_win, s_rest},
                     {256, (uint32_t)(lo >> 8), 1, (uint32_t)win, 1}};
}
// Coordinates of tile t of vector v (as the kernels' tile_load_t / tile_store_t).
static void tile_map_coords(int N, int TB, int wpe, int w, const TileWin& W, int t, int v, int* c) {
  const int rs = wpe == 2 ? 7 : 8;
  if (w == 0) {
    c[0] = 0; c[1] = (t << (TB - rs)) + v * (1 << (N - rs));
    return;
  }
  const int nb = W.b0 - W.c, tl = t & ((1 << nb) - 1), th = (t >> nb) + v * (1 << (N - W.b0 - W.width));
  if (W.c <= rs) {
    c[0] = 0; c[1] = tl; c[2] = 0; c[3] = th;
  } else {
    c[0] = 0; c[1] = 0; c[2] = tl; c[3] = 0; c[4] = th;
  }
}
// Word (index within the basis, in 8-byte words) that box word j of the box at
// coordinates c holds: the box is laid out in shared memory with dimension 0
// fastest.
static int64_t tile_map_element(const TileMapGeom& g, const int* c, int j) {
  int64_t off = 0, stride = 1;  // stride in elements of the current dimension
  for (int d = 0; d < g.rank; ++d) {
    const int64_t idx = (int64_t)c[d] + (j % (int)g.box[d]);
    j /= (int)g.box[d];
    if (idx >= (int64_t)g.dims[d]) return -1;
    off += idx * stride;
    if (d + 1 < g.rank) stride = (int64_t)(g.strides[d] / 8);
  }
  return off;
}
// Constraints of a tiled TMA map: rank <= 5, box dimensions in [1, 256], inner
// box a multiple of 16 bytes, strides multiples of 16 bytes below 2^40.
static bool tile_map_valid(const TileMapGeom& g) {
  if (g.rank < 1 || g.rank > 5 || (g.box[0] * 8) % 16 != 0) return false;
  for (int d = 0; d < g.rank; ++d)
    if (g.box[d] < 1 || g.box[d] > 256 || g.dims[d] < 1 || g.dims[d] > (uint64_t(1) << 32)) return false;
  for (int d = 0; d + 1 < g.rank; ++d)
    if (g.strides[d] % 16 != 0 || g.strides[d] >= (uint64_t(1) << 40)) return false;
  return true;
}

template <int TB>
static bool check_tiling(int N, int64_t* checked) {
  TileWin W[kTiledMaxWindows] = {};
  const int nwin = tiled_windows<TB>(N, W);
  const int64_t dim = int64_t(1) << N;
  const int ntiles = 1 << (N - TB);
  std::vector<unsigned char> seen((size_t)dim);
  std::vector<int> flips(N, 0), bonds(N, 0);
  for (int w = 0; w < nwin; ++w) {
    std::fill(seen.begin(), seen.end(), 0);
    if (w == 0) {
      for (int i = 0; i < TB; ++i) ++flips[i];
      for (int i = 0; i + 1 < TB; ++i) ++bonds[i];
    } else {
      if (W[w].width < 2 || W[w].c < 1 || W[w].c + W[w].width != TB) return false;
      for (int i = 1; i < W[w].width; ++i) ++flips[W[w].b0 + i];
      for (int i = 0; i + 1 < W[w].width; ++i) ++bonds[W[w].b0 + i];
    }
    for (int t = 0; t < ntiles; ++t)
      for (int j = 0; j < (1 << TB); ++j) {
        const int64_t x = w == 0 ? ((int64_t)t << TB) | j : tile_x(W[w], t, j);
        if (x < 0 || x >= dim || seen[(size_t)x]) return false;
        seen[(size_t)x] = 1;
        if (w > 0) {
          // copy units: slots j, j + 1 (j even) hold x, x + 1
          if ((j & 1) == 0 && tile_x(W[w], t, j + 1) != x + 1) return false;
          // the window's own bits: slot j ^ 2^(c+i) holds x ^ 2^(b0+i)
          for (int i = 0; i < W[w].width; ++i)
            if (tile_x(W[w], t, j ^ (1 << (W[w].c + i))) != (x ^ (int64_t(1) << (W[w].b0 + i)))) return false;
        }
        ++*checked;
      }
    {  // the TMA boxes hold the same slots (complex64: TB 12, one word per element; fixed point: TB 11, two)
      const int wpe = TB == kC64TileBits ? 1 : 2;
      TileMapGeom g;
      tile_map_geometry(N, TB, wpe, w, W[w], 3, &g);
      if (!tile_map_valid(g)) return false;
      int64_t boxn = 1;
      for (int d = 0; d < g.rank; ++d) boxn *= g.box[d];
      if (boxn != (int64_t(1) << TB) * wpe) return false;
      for (int v = 0; v < 3; v += 2)
        for (int t = 0; t < ntiles; ++t) {
          int c[5];
          tile_map_coords(N, TB, wpe, w, W[w], t, v, c);
          for (int d = 0; d < g.rank; ++d)
            if (c[d] < 0 || (d == 0 && c[d] != 0)) return false;
          for (int jw = 0; jw < (1 << TB) * wpe; ++jw) {
            const int j = jw / wpe;
            const int64_t x = w == 0 ? ((int64_t)t << TB) | j : tile_x(W[w], t, j);
            if (tile_map_element(g, c, jw) != (x + (int64_t)v * dim) * wpe + jw % wpe) return false;
          }
        }
    }
  }
  for (int i = 0; i < N; ++i)
    if (flips[i] != 1) return false;
  for (int i = 0; i + 1 < N; ++i)
    if (bonds[i] != 1) return false;
  return true;
}
}  // extern "C++"

extern "C++" {
static cfet_status build_tile_maps(cfet_ctx* ctx, int N, int nvec, bool fx) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return fail(nullptr, CFET_ECUDA, "cuTensorMapEncodeTiled is not available");
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  TileWin W[kTiledMaxWindows] = {};
  const int TB = fx ? kFxTileBits : kC64TileBits, wpe = fx ? 2 : 1;
  const int nwin = fx ? tiled_windows<kFxTileBits>(N, W) : tiled_windows<kC64TileBits>(N, W);
  void* base = fx ? (void*)ctx->d_qbasis : (void*)ctx->d_qbasis32;
  std::vector<CUtensorMap> maps(nwin);
  for (int w = 0; w < nwin; ++w) {
    TileMapGeom g;
    tile_map_geometry(N, TB, wpe, w, W[w], nvec, &g);
    if (!tile_map_valid(g)) return fail(nullptr, CFET_EINVAL, "tiled apply: invalid TMA geometry");
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = encode(&maps[w], CU_TENSOR_MAP_DATA_TYPE_INT64, (cuuint32_t)g.rank, base, g.dims,
                              g.strides, g.box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(nullptr, CFET_ECUDA, "cuTensorMapEncodeTiled failed for the tiled apply");
  }
  static_assert(sizeof(CUtensorMap) == kTmaMapBytes, "tensor map size");
  cudaError_t e = cudaMalloc(&ctx->d_tmaps, (size_t)nwin * sizeof(CUtensorMap));
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->d_tmaps, maps.data(), (size_t)nwin * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "upload of the TMA maps");
  return CFET_OK;
}
}  // extern "C++"

cfet_status cfet_selftest_tiling(int32_t nsites, int32_t tile_bits, int64_t* checked) {
  if (!checked) return fail(nullptr, CFET_EINVAL, "checked is NULL");
  *checked = 0;
  if ((tile_bits != 11 && tile_bits != 12) || nsites < tile_bits || nsites > kTiledMaxSites || nsites > 27)
    return fail(nullptr, CFET_EINVAL, "tiling self-test: tile_bits 11 or 12, nsites in [tile_bits, 27]");
  const bool ok = tile_bits == 11 ? check_tiling<11>(nsites, checked) : check_tiling<12>(nsites, checked);
  if (!ok) return fail(nullptr, CFET_ECUDA, "tiling self-test: window tiling inconsistent");
  return CFET_OK;
}

cfet_status cfet_selftest_i128_to_double(const uint64_t* lo, const int64_t* hi, int64_t n, int32_t shift,
                                         double* out) {
  if (!lo || !hi || !out || n < 0 || shift < -200 || shift > 200)
    return fail(nullptr, CFET_EINVAL, "selftest: lo, hi, out required, n >= 0, shift in [-200, 200]");
  for (int64_t i = 0; i < n; ++i) out[i] = sb_i128_to_double(lo[i], hi[i], shift);
  return CFET_OK;
}

cfet_status cfet_selftest_ll_to_double_up(const int64_t* v, int64_t n, double* out) {
  if (!v || !out || n < 0) return fail(nullptr, CFET_EINVAL, "selftest: v, out required, n >= 0");
  for (int64_t i = 0; i < n; ++i) out[i] = sb_ll_to_double_up(v[i]);
  return CFET_OK;
}

cfet_status cfet_selftest_krylov_bounds(int32_t k, const double* a, const double* b, double ts, double* log2_bounds,
                                        int32_t* gate) {
  if (k < 1 || k > kMaxKrylov || !a || (k > 1 && !b) || !log2_bounds || !gate)
    return fail(nullptr, CFET_EINVAL, "selftest: k in [1, 64], a, b, log2_bounds and gate required");
  LeadAcc s;
  sb_lead_init(s);
  GershAcc g;
  sb_gersh_init(g);
  for (int r = 0; r < k; ++r) {
    sb_lead_row(s, r, k, a, b);
    sb_gersh_row(g, r, k, a, b);
  }
  float lo, hi;
  sb_lead_log2_bounds(s, k, ts, lo, hi);
  log2_bounds[0] = lo;
  log2_bounds[1] = hi;
  *gate = sb_gersh_gate(g, k, ts);
  return CFET_OK;
}

cfet_status cfet_selftest_wait_timeout(int32_t which, double timeout_s, int32_t* device_status) {
  if ((which != 0 && which != 1) || !(timeout_s > 0.0) || timeout_s > 10.0 || !device_status)
    return fail(nullptr, CFET_EINVAL, "selftest: which in {0, 1}, timeout in (0, 10] s, device_status required");
  cfet_status s = device_available(nullptr);
  if (s != CFET_OK) return s;
  unsigned long long* rec = nullptr;
  unsigned* bar = nullptr;
  int* st = nullptr;
  cudaError_t e = cudaMalloc(&rec, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&bar, 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&st, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(rec, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(bar, 0, 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(st, 0, sizeof(int));
  if (e == cudaSuccess) e = (cudaError_t)launch_wait_selftest(which, rec, bar, st, (long long)(timeout_s * 1e9));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(rec);
  cudaFree(bar);
  cudaFree(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "wait self test");
  *device_status = h;
  return h == CFET_ETIMEOUT ? CFET_OK : fail(nullptr, CFET_ECUDA, "wait self test: the wait did not time out");
}

cfet_status cfet_probe_copy_gbs(void* a, void* b, int64_t bytes, int32_t reps, void* stream, double* gbs) {
  if (!gbs) return fail(nullptr, CFET_EINVAL, "copy probe: gbs is NULL");
  *gbs = 0.0;
  if (!a || !b || a == b || bytes < 16 || (bytes % 16) != 0 || reps < 1 || reps > 100000 ||
      (reinterpret_cast<uintptr_t>(a) % 16) != 0 || (reinterpret_cast<uintptr_t>(b) % 16) != 0)
    return fail(nullptr, CFET_EINVAL, "copy probe: two distinct 16-byte aligned buffers, bytes a positive "
                                      "multiple of 16, reps in [1, 100000]");
  cfet_status s = device_available(nullptr);
  if (s != CFET_OK) return s;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = (cudaError_t)launch_copy_probe(a, b, bytes / 16, 1, 4 * nsm, cs);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
  if (e == cudaSuccess) e = (cudaError_t)launch_copy_probe(a, b, bytes / 16, reps, 4 * nsm, cs);
  if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "copy probe");
  *gbs = ms > 0.0f ? 2.0 * (double)bytes * reps / (ms * 1e-3) / 1e9 : 0.0;
  return CFET_OK;
}

cfet_status cfet_fidelity_grad(cfet_ctx* ctx, const void* psi0, const void* phi, double t0, double dt,
                               int64_t nsteps, int32_t order, double krylov_tol, int32_t nseg, const double* amps,
                               double omega, double phase, int64_t checkpoint_every, void* stream, double* loss,
                               double* grad, cfet_grad_stats* gstats) {
  if (ctx && (ctx->opt.expm != CFET_EXPM_KRYLOV || ctx->opt.picture != CFET_PICTURE_SCHROEDINGER))
    return fail(ctx, CFET_EINVAL, "fidelity gradient: the context must use CFET_EXPM_KRYLOV, Schroedinger picture");
  if (!ctx) return CFET_EINVAL;
  if (ctx->family != kFamilySpin || ctx->nV != 1)
    return fail(ctx, CFET_EINVAL, "fidelity gradient: needs an XXZ chain with exactly one X-field drive");
  cfet_status s = check_psi(ctx, psi0);
  if (s != CFET_OK) return s;
  if ((s = check_psi(ctx, phi)) != CFET_OK) return s;
  if (!loss || !grad || !amps) return fail(ctx, CFET_EINVAL, "loss, grad and amps are required");
  if (!is_finite_d(t0) || !is_finite_d(dt) || dt == 0.0 || !is_finite_d(krylov_tol) || !is_finite_d(omega) ||
      !is_finite_d(phase))
    return fail(ctx, CFET_EINVAL, "t0, dt, tol, omega, phase must be finite, dt != 0");
  if (nsteps < 1 || nseg < 1 || nsteps % nseg != 0)
    return fail(ctx, CFET_EINVAL, "nsteps must be a positive multiple of nseg");
  for (int k = 0; k < nseg; ++k)
    if (!is_finite_d(amps[k])) return fail(ctx, CFET_EINVAL, "amplitude not finite");
  if (checkpoint_every < 1) return fail(ctx, CFET_EINVAL, "checkpoint_every must be >= 1");
  if (ctx->opt.m_max > kAdjMaxK) return fail(ctx, CFET_EINVAL, "fidelity gradient: m_max must be <= 16");
  const int id = default_scheme_for_order(order);
  if (!id) return fail(ctx, CFET_EINVAL, "order must be 2, 4, 6 or 8");
  SchemeData sd;
  build_scheme(id, &sd);
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const int dim = ctx->dim;
  const long long nexp = nsteps * (long long)sd.s;
  const long long nch = (nsteps + checkpoint_every - 1) / checkpoint_every;
  // ---- workspace
  if (ctx->ev_pending) { cudaEventSynchronize(ctx->ev_done); ctx->ev_pending = false; }
  if ((size_t)(nch + 1) > ctx->adj_ckpt_n) {
    cudaFree(ctx->d_adj_ckpt);
    ctx->d_adj_ckpt = nullptr;
    ctx->adj_ckpt_n = 0;
    CK(cudaMalloc(&ctx->d_adj_ckpt, (size_t)(nch + 1) * dim * sizeof(double2)), "cudaMalloc(checkpoints)");
    ctx->adj_ckpt_n = (size_t)(nch + 1);
  }
  if (!ctx->d_adj_vec) {
    CK(cudaMalloc(&ctx->d_adj_vec, (size_t)(2 + 2 * kAdjMaxK) * dim * sizeof(double2)), "cudaMalloc(adjoint)");
    int g = max_coresident_blocks_adjoint(256);
    if (g < 1) return fail(ctx, CFET_ECUDA, "occupancy query failed for the adjoint kernel");
    const int want = (dim + 255) / 256;
    ctx->adj_grid = want < g ? want : g;
    CK(cudaMalloc(&ctx->d_adj_part, 2 * (2 * kAdjMaxK + 2) * (size_t)ctx->adj_grid * sizeof(double)),
       "cudaMalloc(adjoint partials)");
  }
  const int nql = 6 + 12 + 24 + 48;
  if ((size_t)(3 * nexp + 2 * nql) > ctx->adj_tab_n) {
    cudaFree(ctx->d_adj_tab);
    cudaFree(ctx->d_adj_seg);
    ctx->d_adj_tab = nullptr;
    ctx->d_adj_seg = nullptr;
    ctx->adj_tab_n = 0;
    CK(cudaMalloc(&ctx->d_adj_tab, (size_t)(3 * nexp + 2 * nql) * sizeof(double)), "cudaMalloc(adjoint tables)");
    CK(cudaMalloc(&ctx->d_adj_seg, (size_t)nexp * sizeof(int)), "cudaMalloc(adjoint tables)");
    ctx->adj_tab_n = (size_t)(3 * nexp + 2 * nql);
  }
  if (nseg > ctx->adj_nseg_cap) {
    cudaFree(ctx->d_adj_acc);
    ctx->d_adj_acc = nullptr;
    ctx->adj_nseg_cap = 0;
    CK(cudaMalloc(&ctx->d_adj_acc, (2 * (size_t)nseg + 4) * sizeof(double)), "cudaMalloc(gradient)");
    ctx->adj_nseg_cap = nseg;
  }
  double2* d_psi = ctx->d_adj_vec;
  double2* d_lam = ctx->d_adj_vec + dim;
  double2* d_Vp = ctx->d_adj_vec + 2 * (size_t)dim;
  double2* d_Vl = d_Vp + (size_t)kAdjMaxK * dim;
  // ---- per-exponential tables (application order) and quadrature rules
  const long long sps = nsteps / nseg;
  std::vector<double> tab(3 * nexp + 2 * nql);
  std::vector<int> segv(nexp);
  for (long long n = 0; n < nsteps; ++n) {
    const double t = t0 + (double)n * dt;
    for (int jj = 0; jj < sd.s; ++jj) {
      const int j = sd.s - 1 - jj;  // exp(Omega_s) acts first
      double c0 = 0.0, gm = 0.0;
      for (int m = 0; m < sd.M; ++m) {
        c0 += sd.g[j][m];
        gm += sd.g[j][m] * std::cos(omega * (t + sd.x[m] * dt) + phase);
      }
      const long long e = n * sd.s + jj;
      const int k = (int)(n / sps);
      tab[e] = c0;
      tab[nexp + e] = amps[k] * gm;
      tab[2 * nexp + e] = gm;
      segv[e] = k;
    }
  }
  double* glx = tab.data() + 3 * nexp;
  double* glw = glx + nql;
  gauss_legendre_01(6, glx, glw);
  gauss_legendre_01(12, glx + 6, glw + 6);
  gauss_legendre_01(24, glx + 18, glw + 18);
  gauss_legendre_01(48, glx + 42, glw + 42);
  CK(cudaMemcpyAsync(ctx->d_adj_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st),
     "adjoint table upload");
  CK(cudaMemcpyAsync(ctx->d_adj_seg, segv.data(), segv.size() * sizeof(int), cudaMemcpyHostToDevice, st),
     "adjoint table upload");
  // ---- forward pass with checkpoints (the context's own propagator)
  cudaEvent_t e0, e1, e2;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  CK(cudaEventCreate(&e2), "event");
  struct EvGuard {
    cudaEvent_t a, b, c;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); cudaEventDestroy(c); }
  } evg{e0, e1, e2};
  CK(cudaEventRecord(e0, st), "event");
  CK(cudaMemcpyAsync(d_psi, psi0, (size_t)dim * sizeof(double2), cudaMemcpyDeviceToDevice, st), "copy psi0");
  CK(cudaMemcpyAsync(ctx->d_adj_ckpt, psi0, (size_t)dim * sizeof(double2), cudaMemcpyDeviceToDevice, st),
     "checkpoint");
  PwcDrive pd{amps, nseg, omega, phase, t0, dt, sps};
  const cfet_drive_fn f_saved = ctx->f[0];
  void* const u_saved = ctx->f_user[0];
  ctx->f[0] = pwc_eval;
  ctx->f_user[0] = &pd;
  long long fwd_app = 0;
  for (long long c = 0; c < nch; ++c) {
    const long long n0 = c * checkpoint_every;
    const long long nc = (nsteps - n0) < checkpoint_every ? (nsteps - n0) : checkpoint_every;
    cfet_stats fs;
    s = cfet_propagate_ex(ctx, d_psi, t0 + (double)n0 * dt, dt, nc, order, CFET_SCHEME_DEFAULT, krylov_tol, stream,
                          nullptr, nullptr, &fs);
    if (s != CFET_OK) break;
    fwd_app += fs.n_applies;
    cudaError_t ce = cudaMemcpyAsync(ctx->d_adj_ckpt + (size_t)(c + 1) * dim, d_psi, (size_t)dim * sizeof(double2),
                                     cudaMemcpyDeviceToDevice, st);
    if (ce != cudaSuccess) {
      s = cuda_fail(ctx, ce, "checkpoint");
      break;
    }
  }
  ctx->f[0] = f_saved;
  ctx->f_user[0] = u_saved;
  if (s != CFET_OK) return s;
  CK(cudaEventRecord(e1, st), "event");
  // ---- backward sweep, one launch per checkpoint interval
  CK(cudaMemsetAsync(ctx->d_adj_acc, 0, (2 * (size_t)nseg + 4) * sizeof(double), st), "gradient reset");
  CK(cudaMemsetAsync(ctx->d_st, 0, sizeof(DevStatus), st), "status reset");
  for (long long c = nch - 1; c >= 0; --c) {
    const long long n0 = c * checkpoint_every;
    const long long n1 = (n0 + checkpoint_every) < nsteps ? (n0 + checkpoint_every) : nsteps;
    AdjParams p{};
    p.dim = dim;
    p.m_min = ctx->opt.m_min;
    p.m_max = ctx->opt.m_max;
    p.tau = dt;
    p.tol = krylov_tol;
    p.psi = d_psi;
    p.ckpt = ctx->d_adj_ckpt + (size_t)(c + 1) * dim;
    p.lam = d_lam;
    p.phi = (c == nch - 1) ? (const double2*)phi : nullptr;
    p.Vp = d_Vp;
    p.Vl = d_Vl;
    p.c0 = ctx->d_adj_tab;
    p.c1 = ctx->d_adj_tab + nexp;
    p.gam = ctx->d_adj_tab + 2 * nexp;
    p.seg = ctx->d_adj_seg;
    p.e_lo = n0 * sd.s;
    p.e_hi = n1 * sd.s;
    p.nq6 = 0;
    p.nq12 = 6;
    p.nq24 = 18;
    p.nq48 = 42;
    p.glx = ctx->d_adj_tab + 3 * nexp;
    p.glw = p.glx + nql;
    p.grad = ctx->d_adj_acc;
    p.out = ctx->d_adj_acc + 2 * nseg;
    p.partials = ctx->d_adj_part;
    p.bar = ctx->d_bar;
    p.st = ctx->d_st;
    p.timeout_ns = (long long)(ctx->opt.barrier_timeout_s * 1e9);
    CK(cudaMemsetAsync(ctx->d_bar, 0, 2 * sizeof(unsigned), st), "barrier reset");
    const int e = launch_adjoint_spin(p, ctx->spin, ctx->adj_grid, 256, st);
    if (e != cudaSuccess) return cuda_fail(ctx, (cudaError_t)e, "adjoint kernel launch");
  }
  CK(cudaEventRecord(e2, st), "event");
  std::vector<double> acc(2 * (size_t)nseg + 4);
  CK(cudaMemcpyAsync(acc.data(), ctx->d_adj_acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
     "gradient read-back");
  CK(cudaMemcpyAsync(ctx->h_st, ctx->d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, st), "status read-back");
  CK(cudaStreamSynchronize(st), "stream synchronize");
  const int code = ctx->h_st->status;
  if (code == CFET_EKRYLOV)
    return fail(ctx, CFET_EKRYLOV, "adjoint sweep: a stage exponential needs more than m_max Krylov vectors");
  if (code == CFET_ETIMEOUT) return fail(ctx, CFET_ETIMEOUT, "device grid barrier timed out");
  if (code == CFET_ENAN) return fail(ctx, CFET_ENAN, "state not finite");
  if (code != 0) return fail(ctx, (cfet_status)code, "device error");
  const double ore = acc[2 * nseg], oim = acc[2 * nseg + 1];
  *loss = 1.0 - (ore * ore + oim * oim);
  for (int k = 0; k < nseg; ++k) grad[k] = -2.0 * (ore * acc[2 * k] + oim * acc[2 * k + 1]);
  if (gstats) {
    gstats->overlap_re = ore;
    gstats->overlap_im = oim;
    gstats->max_drift = acc[2 * nseg + 2];
    gstats->n_applies_forward = fwd_app;
    gstats->n_applies_backward = (int64_t)acc[2 * nseg + 3];
    cudaEventElapsedTime(&gstats->forward_ms, e0, e1);
    cudaEventElapsedTime(&gstats->backward_ms, e1, e2);
  }
  return CFET_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ time-step selection (Sec. 6.6)
namespace {

// CFET order of (order, scheme) as cfet_propagate_ex resolves them; 0 if invalid.
int resolve_order(int32_t order, int32_t scheme) {
  int id = scheme;
  if (id == CFET_SCHEME_DEFAULT) id = default_scheme_for_order(order);
  SchemeData sd;
  if (!id || !build_scheme(id, &sd)) return 0;
  if (scheme != CFET_SCHEME_DEFAULT && order != 0 && order != sd.order) return 0;
  return sd.order;
}

cfet_status ensure_ts(cfet_ctx* ctx) {
  if (!ctx->d_ts) CK(cudaMalloc(&ctx->d_ts, 2 * (size_t)ctx->dim * sizeof(double2)), "cudaMalloc(trial states)");
  if (!ctx->d_ts_part) CK(cudaMalloc(&ctx->d_ts_part, kDiffBlocks * sizeof(double)), "cudaMalloc(partials)");
  return CFET_OK;
}

// ||a - b||_2 (synchronises the stream)
cfet_status diff_norm(cfet_ctx* ctx, const double2* a, const double2* b, cudaStream_t s, double* out) {
  int e = launch_diff_norm2(a, b, ctx->dim, ctx->d_ts_part, kDiffBlocks, s);
  if (e != cudaSuccess) return cuda_fail(ctx, (cudaError_t)e, "difference norm kernel");
  double part[kDiffBlocks];
  CK(cudaMemcpyAsync(part, ctx->d_ts_part, sizeof(part), cudaMemcpyDeviceToHost, s), "partials read-back");
  CK(cudaStreamSynchronize(s), "stream synchronize");
  double sum = 0.0;
  for (int i = 0; i < kDiffBlocks; ++i) sum += part[i];
  *out = std::sqrt(sum);
  return CFET_OK;
}

void add_stats(cfet_stats* acc, const cfet_stats& s) {
  acc->n_exp += s.n_exp;
  acc->n_substeps += s.n_substeps;
  acc->n_applies += s.n_applies;
  if (s.max_k > acc->max_k) acc->max_k = s.max_k;
  if (s.max_err_est > acc->max_err_est) acc->max_err_est = s.max_err_est;
}

// one or more CFET steps of x (device) from t with step h, stats accumulated
cfet_status run_steps(cfet_ctx* ctx, double2* x, double t, double h, int64_t n, int32_t order, int32_t scheme,
                      double tol, void* stream, cfet_stats* acc) {
  cfet_stats st;
  cfet_status s = cfet_propagate_ex(ctx, x, t, h, n, order, scheme, tol, stream, nullptr, nullptr, &st);
  if (s == CFET_OK) add_stats(acc, st);
  return s;
}

}  // namespace

extern "C" {

cfet_status cfet_error_constant(cfet_ctx* ctx, const void* psi0, double t0, double T, int64_t n1, int32_t order,
                                int32_t scheme, double krylov_tol, double ratio, void* stream, double* c,
                                double* diff, double* dt2) {
  if (!ctx) return CFET_EINVAL;
  cfet_status s = check_psi(ctx, psi0);
  if (s != CFET_OK) return s;
  const int N = resolve_order(order, scheme);
  if (!N) return fail(ctx, CFET_EINVAL, "order / scheme invalid");
  if (!is_finite_d(t0) || !is_finite_d(T) || !(T > 0.0)) return fail(ctx, CFET_EINVAL, "T must be finite and > 0");
  if (n1 < 1) return fail(ctx, CFET_EINVAL, "n1 must be >= 1");
  if (!is_finite_d(ratio) || !(ratio > 1.0)) return fail(ctx, CFET_EINVAL, "ratio must be > 1");
  if (!c) return fail(ctx, CFET_EINVAL, "c is NULL");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if ((s = ensure_ts(ctx)) != CFET_OK) return s;
  int64_t n2 = (int64_t)std::llround((double)n1 * std::pow(ratio, 1.0 / N));
  if (n2 <= n1) n2 = n1 + 1;
  const double h1 = T / (double)n1, h2 = T / (double)n2;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)ctx->dim * sizeof(double2);
  double2* x1 = ctx->d_ts;
  double2* x2 = ctx->d_ts + ctx->dim;
  CK(cudaMemcpyAsync(x1, psi0, bytes, cudaMemcpyDeviceToDevice, st), "copy psi0");
  CK(cudaMemcpyAsync(x2, psi0, bytes, cudaMemcpyDeviceToDevice, st), "copy psi0");
  cfet_stats acc{};
  if ((s = run_steps(ctx, x1, t0, h1, n1, order, scheme, krylov_tol, stream, &acc)) != CFET_OK) return s;
  if ((s = run_steps(ctx, x2, t0, h2, n2, order, scheme, krylov_tol, stream, &acc)) != CFET_OK) return s;
  double e = 0.0;
  if ((s = diff_norm(ctx, x1, x2, st, &e)) != CFET_OK) return s;
  *c = e / (T * std::fabs(std::pow(h1, N) - std::pow(h2, N)));
  if (diff) *diff = e;
  if (dt2) *dt2 = h2;
  return CFET_OK;
}

cfet_status cfet_select_dt(cfet_ctx* ctx, const void* psi0, double t0, double T, double target, double T_probe,
                           int64_t n_probe, int32_t order, int32_t scheme, double krylov_tol, double ratio,
                           void* stream, double* dt, int64_t* nsteps, double* c) {
  if (!ctx) return CFET_EINVAL;
  if (!is_finite_d(T) || !(T > 0.0) || !is_finite_d(target) || !(target > 0.0))
    return fail(ctx, CFET_EINVAL, "T and target must be finite and > 0");
  if (!dt || !nsteps) return fail(ctx, CFET_EINVAL, "dt / nsteps is NULL");
  double cc = 0.0;
  cfet_status s = cfet_error_constant(ctx, psi0, t0, T_probe, n_probe, order, scheme, krylov_tol, ratio, stream, &cc,
                                      nullptr, nullptr);
  if (s != CFET_OK) return s;
  const int N = resolve_order(order, scheme);
  if (c) *c = cc;
  if (!(cc > 0.0)) {
    *dt = T;
    *nsteps = 1;
    return CFET_OK;
  }
  const double h = std::pow(target / (cc * T), 1.0 / N);
  const double n = std::ceil(T / h);
  if (!(n <= 9.0e15)) return fail(ctx, CFET_EINVAL, "selected step too small");
  *nsteps = (int64_t)n;
  *dt = T / n;
  return CFET_OK;
}

cfet_status cfet_propagate_adaptive(cfet_ctx* ctx, void* psi, double t0, double T, int32_t order, int32_t scheme,
                                    double krylov_tol, double target, double h0, double h_min, double h_max,
                                    int64_t max_steps, const double* forced_h, int64_t n_forced, double* h_log,
                                    int64_t h_cap, int64_t* n_steps, int64_t* n_trials, void* stream,
                                    cfet_stats* stats) {
  if (!ctx) return CFET_EINVAL;
  cfet_status s = check_psi(ctx, psi);
  if (s != CFET_OK) return s;
  const int N = resolve_order(order, scheme);
  if (!N) return fail(ctx, CFET_EINVAL, "order / scheme invalid");
  if (!is_finite_d(t0) || !is_finite_d(T) || !(T > 0.0)) return fail(ctx, CFET_EINVAL, "T must be finite and > 0");
  cfet_stats acc{};
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  double2* x = (double2*)psi;
  if (forced_h) {
    if (n_forced < 0) return fail(ctx, CFET_EINVAL, "n_forced < 0");
    for (int64_t i = 0; i < n_forced; ++i)
      if (!is_finite_d(forced_h[i]) || !(forced_h[i] > 0.0)) return fail(ctx, CFET_EINVAL, "forced step not > 0");
    double t = t0;
    for (int64_t i = 0; i < n_forced; ++i) {
      if ((s = run_steps(ctx, x, t, forced_h[i] / 2.0, 2, order, scheme, krylov_tol, stream, &acc)) != CFET_OK)
        return s;
      t += forced_h[i];
    }
    if (n_steps) *n_steps = n_forced;
    if (n_trials) *n_trials = 0;
    if (stats) *stats = acc;
    return CFET_OK;
  }
  if (!is_finite_d(target) || !(target > 0.0)) return fail(ctx, CFET_EINVAL, "target must be > 0");
  if (!(h_min > 0.0) || !(h0 >= h_min) || !(h_max >= h0) || !is_finite_d(h_max))
    return fail(ctx, CFET_EINVAL, "steps must satisfy 0 < h_min <= h0 <= h_max < inf");
  if (max_steps < 1) return fail(ctx, CFET_EINVAL, "max_steps must be >= 1");
  if ((s = ensure_ts(ctx)) != CFET_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)ctx->dim * sizeof(double2);
  double2* x1 = ctx->d_ts;
  double2* x2 = ctx->d_ts + ctx->dim;
  const double t_end = t0 + T;
  double t = t0, h = h0;
  int64_t ns = 0, nt = 0;
  while (t_end - t > 1e-12 * std::fmax(1.0, std::fabs(t_end))) {
    if (ns >= max_steps) return fail(ctx, CFET_EKRYLOV, "adaptive stepping: more than max_steps steps");
    const double rem = t_end - t;
    h = std::fmin(h, rem);
    ++nt;
    CK(cudaMemcpyAsync(x1, x, bytes, cudaMemcpyDeviceToDevice, st), "copy state");
    CK(cudaMemcpyAsync(x2, x, bytes, cudaMemcpyDeviceToDevice, st), "copy state");
    if ((s = run_steps(ctx, x1, t, h, 1, order, scheme, krylov_tol, stream, &acc)) != CFET_OK) return s;
    if ((s = run_steps(ctx, x2, t, h / 2.0, 2, order, scheme, krylov_tol, stream, &acc)) != CFET_OK) return s;
    double e = 0.0;
    if ((s = diff_norm(ctx, x1, x2, st, &e)) != CFET_OK) return s;
    const double c = e / (h * (std::pow(h, N) - std::pow(h / 2.0, N)));
    if (c * T * std::pow(h / 2.0, N) <= target || h <= h_min) {
      CK(cudaMemcpyAsync(x, x2, bytes, cudaMemcpyDeviceToDevice, st), "accept state");
      t = h < rem ? t + h : t_end;
      if (h_log && ns < h_cap) h_log[ns] = h;
      ++ns;
    }
    const double h_new = c <= 0.0 ? 2.0 * h : std::fmin(2.0 * h, 1.8 * std::pow(target / (c * T), 1.0 / N));
    h = std::fmin(std::fmax(h_new, h_min), h_max);
  }
  CK(cudaStreamSynchronize(st), "stream synchronize");
  if (n_steps) *n_steps = ns;
  if (n_trials) *n_trials = nt;
  if (stats) *stats = acc;
  return CFET_OK;
}

}  // extern "C"
