/*
 * cfet.h -- C ABI of the GB300 (sm_103a) commutator-free exponential
 * time-propagator (CFET) library.
 *
 * The library propagates a wave function psi under the time-dependent
 * Schroedinger equation  i d/dt psi = H(t) psi  (Sec. 1 of Alvermann & Fehske,
 * arXiv:1102.5071) with
 *
 *     H(t) = H0 + sum_{k=1..nV} f_k(t) V_k .
 *
 * One CFET time step from t to t+dt is the product of s exponentials
 * (Sec. 4, Eq. (Ucf)); by Gauss-Legendre quadrature each exponential is
 * exp(-i dt H_j) with the weighted sum  H_j = sum_m g_{j,m} H(t + x_m dt)
 * (Sec. 7, Eq. (OmGLeg)), i.e.
 *
 *     H_j = c_{j,0} H0 + sum_k c_{j,k} V_k,
 *     c_{j,0} = sum_m g_{j,m},   c_{j,k} = sum_m g_{j,m} f_k(t + x_m dt),
 *
 * so H_j is never formed: the apply kernels take the per-stage scalars c_{j,*}
 * (Sec. 8: weighted sums keep the sparsity pattern of H).  Each exponential
 * acting on psi is evaluated by a Lanczos/Krylov loop on the device (Sec. 8.1)
 * with an a-posteriori error estimate, adaptive Krylov dimension and time
 * substepping.  exp(Omega_s) is applied first and exp(Omega_1) last (Sec. 2.2).
 *
 * Conventions common to every entry point:
 *  - All vectors are complex128 (interleaved re, im doubles), 16-byte aligned,
 *    length `dim`, in DEVICE memory owned by the caller, unless an argument
 *    says "host".  psi is updated in place and is not renormalised.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    stream-ordered.  A call that returns device results to the host
 *    (non-NULL stats, decision logs, cfet_propagate_host) synchronises the
 *    stream before returning; otherwise the call returns after enqueueing.
 *  - Every entry point validates its arguments first.  On CFET_EINVAL no device
 *    work has been issued.  The text of the last error of a context is
 *    available from cfet_last_error().
 *  - The library never falls back to a CPU path: without a usable CUDA device
 *    every call that would compute returns CFET_ENODEV.
 *  - Device-side waits (grid barriers of the persistent kernel) are bounded by
 *    cfet_options.barrier_timeout_s; on expiry the kernel records
 *    CFET_ETIMEOUT, leaves psi in an unspecified state and returns.
 */
#ifndef CFET_H
#define CFET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cfet_status {
  CFET_OK = 0,
  CFET_EINVAL = 1,    /* invalid argument (no device work issued)            */
  CFET_ENOMEM = 2,    /* device or pinned-host allocation failed              */
  CFET_ECUDA = 3,     /* a CUDA runtime call failed                           */
  CFET_EKRYLOV = 4,   /* a stage exponential needed more than max_substeps    */
  CFET_ETIMEOUT = 5,  /* a device grid barrier exceeded its wait limit        */
  CFET_ENAN = 6,      /* psi norm not finite at the start of an exponential   */
  CFET_ENODEV = 7     /* no CUDA device usable by this library                */
} cfet_status;

/* ------------------------------------------------------------------------ */
/* Operators                                                                 */
/* ------------------------------------------------------------------------ */
/* Spin-1/2 chains use the basis index x in [0, 2^nsites); bit i of x is site
 * i; bit value 0 is spin up (sigma_z = +1).  With the Pauli matrices of
 * Sec. 6.2:  Z_i|x> = (1-2 b_i)|x>,  X_i|x> = |x ^ 2^i>,
 * Y_i|x> = i (1-2 b_i) |x ^ 2^i>.                                           */
enum {
  /* open XXZ chain (the spin chain of Sec. 11.1, Eq. (SpinChain1), with an
   * Ising anisotropy and site fields):
   *   H = sum_{i<N-1} [ J (X_i X_{i+1} + Y_i Y_{i+1}) + J*Delta Z_i Z_{i+1} ]
   *       + sum_i h_i Z_i
   * uses: nsites, J, Delta, site_coeff = h[nsites] (host, copied).          */
  CFET_OP_XXZ_CHAIN = 1,
  /* transverse field  V = sum_i a_i X_i ;  uses nsites, site_coeff = a[nsites]
   * (host, copied).  Only valid as a drive operator V_k of an XXZ chain.    */
  CFET_OP_X_FIELD = 2,
  /* real banded operator in DIA form:
   *   (D v)[r] = sum_d values[d*dim + r] * v[r + offsets[d]]
   * terms with r + offsets[d] outside [0, dim) are absent.  uses dim, ndiag,
   * offsets[ndiag] (host, int64, copied), values[ndiag*dim] (host, copied,
   * row-aligned).  The caller guarantees the operator is symmetric.        */
  CFET_OP_DIA = 3,
  /* real combination of Pauli strings on a chain of nsites spins:
   *   P = sum_t coeff[t] * i^popc(xmask[t] & zmask[t]) * X^xmask[t] Z^zmask[t]
   * (X^x Z^z = product over the set bits; the phase makes every string a
   * tensor product of X, Y = i X Z and Z on the sites of x | z, hence
   * Hermitian); (P v)[y] = sum_t coeff[t] i^popc(x&z) (-1)^popc((y^x)&z)
   * v[y ^ x].  uses nsites, dim = 2^nsites, nterms, xmask[nterms],
   * zmask[nterms] (bits below nsites only), coeff[nterms] (host, copied).
   * When H0 or any V_k is a Pauli sum, every operator of the context must be
   * a Pauli sum, an XXZ chain or an X field of the same chain (the latter two
   * are expanded into Pauli strings), the total number of strings is at most
   * 4096, and the context computes in CFET_PREC_F64 (CFET_PREC_DEFAULT
   * selects it; CFET_PREC_FX and CFET_PREC_C64 give CFET_EINVAL).           */
  CFET_OP_PAULI = 4,
  /* general sparse Hermitian operator in compressed sparse row form (Sec. 8:
   * the stage operator is a weighted sum of the operators, applied term by
   * term with the stage scalars, so it keeps their sparsity and is never
   * formed):
   *   (A v)[r] = sum_{e = row_ptr[r]}^{row_ptr[r+1]-1}
   *              (csr_re[e] + i csr_im[e]) * v[col_idx[e]]
   * uses dim, row_ptr[dim + 1] (host, int64, row_ptr[0] = 0, non-decreasing),
   * col_idx[nnz] (host, int32, each in [0, dim); duplicates within a row are
   * summed), csr_re[nnz] and csr_im[nnz] (host, copied; csr_im = NULL for a
   * real symmetric operator), nnz = row_ptr[dim].  The operator must be
   * Hermitian: every entry's mirror holds the conjugate value to 1e-13 of
   * the largest entry (checked at create, else CFET_EINVAL).  When H0 is CSR,
   * every V_k must be CSR of the same dim; at most 2^31 - 2 stored entries
   * over all operators.  Every precision and both stage-exponential methods
   * apply.                                                                  */
  CFET_OP_CSR = 5
};

typedef struct cfet_op {
  int32_t kind;               /* CFET_OP_*                                   */
  int32_t nsites;             /* spin operators: chain length, dim = 2^nsites */
  int64_t dim;                /* Hilbert-space dimension                      */
  double J, Delta;            /* XXZ_CHAIN couplings                          */
  const double* site_coeff;   /* XXZ_CHAIN: h_i; X_FIELD: a_i  (host)         */
  int32_t ndiag;              /* DIA: number of stored diagonals              */
  const int64_t* offsets;     /* DIA: offsets[ndiag] (host)                   */
  const double* values;       /* DIA: values[ndiag*dim] (host)                */
  int32_t nterms;             /* PAULI: number of strings                     */
  const uint64_t* xmask;      /* PAULI: X part of string t (host)             */
  const uint64_t* zmask;      /* PAULI: Z part of string t (host)             */
  const double* coeff;        /* PAULI: real coefficient of string t (host)   */
  const int64_t* row_ptr;     /* CSR: row_ptr[dim + 1] (host)                 */
  const int32_t* col_idx;     /* CSR: col_idx[row_ptr[dim]] (host)            */
  const double* csr_re;       /* CSR: real parts of the entries (host)        */
  const double* csr_im;       /* CSR: imaginary parts (host) or NULL (real)   */
} cfet_op;

/* Drive f_k(t), called on the host only at the Gauss-Legendre nodes
 * t + x_m dt of each step while cfet_propagate builds its stage scalars.   */
typedef double (*cfet_drive_fn)(double t, void* user);

/* ------------------------------------------------------------------------ */
/* Schemes (coefficient tables of Secs. 4.2-4.4, 5.2-5.3)                    */
/* ------------------------------------------------------------------------ */
enum {
  CFET_SCHEME_DEFAULT = 0,    /* default for the order: 2->CF2:1, 4->CF4:2,
                                 6->CF6:5Opt, 8->CF8:11                       */
  CFET_SCHEME_CF2_1 = 1,      /* Eq. (UCF2)                                   */
  CFET_SCHEME_CF4_2 = 2,      /* Table 4thCFET, Eq. (UCF4:2)                  */
  CFET_SCHEME_CF4_3 = 3,      /* Table 4thCFET                                */
  CFET_SCHEME_CF4_3OPT = 4,   /* Table 4thCFETOpt, Eq. (CF4Optimal)           */
  CFET_SCHEME_CF6_4 = 5,      /* Table 6thCFET                                */
  CFET_SCHEME_CF6_5 = 6,      /* Table 6thCFET                                */
  CFET_SCHEME_CF6_5B = 7,     /* Table 6thCFET (Blanes-Moan)                  */
  CFET_SCHEME_CF6_6 = 8,      /* Table 6thCFET                                */
  CFET_SCHEME_CF6_5IMP = 9,   /* Table 6thCFETOpt                             */
  CFET_SCHEME_CF6_5OPT = 10,  /* Table 6thCFETOpt (recommended, Sec. 12)      */
  CFET_SCHEME_CF6_6OPT = 11,  /* Table 6thCFETOpt                             */
  CFET_SCHEME_CF8_11 = 12     /* Table 8thCoeff                               */
};

/* Coefficients of scheme `scheme` (a CFET_SCHEME_* id, not DEFAULT) as used
 * by the device path.  Writes order, s (exponentials), M (Gauss-Legendre
 * points = Legendre terms), and, where the pointers are non-NULL and the
 * capacities suffice, f[s*M] (full table after rule (R1), Eq. (FSymm)),
 * x[M], w[M] (Table tab:GaussLeg) and g[s*M] (g_{i,m} of Sec. 7), row-major.
 * Host only; no device needed.  Returns CFET_EINVAL for an unknown id or too
 * small a capacity.                                                         */
cfet_status cfet_scheme_info(int32_t scheme, int32_t* order, int32_t* s, int32_t* M,
                             double* f, double* x, double* w, double* g, int32_t capacity);

/* Chebyshev expansion coefficients of exp(-i z x) on [-1, 1] (Jacobi-Anger;
 * the CFET_EXPM_CHEBYSHEV path): r[k] = (2 - delta_k0) J_k(z), k = 0..K, with
 * K the smallest order whose tail bound 2 sum_{k>K} |J_k(z)| is <= tol
 * (2^-52 for tol <= 0).  The Bessel values come from Miller's backward
 * recurrence normalised by J_0 + 2 sum J_{2k} = 1.  r may be NULL (query K
 * and the tail only); otherwise cap >= K + 1 is required.  Host only; no
 * device needed.  Errors: CFET_EINVAL (non-finite z or tol, |z| > 1e8, cap
 * too small).                                                               */
cfet_status cfet_chebyshev_coefficients(double z, double tol, int32_t cap, double* r, int32_t* K, double* tail);

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct cfet_options {
  int32_t m_max;             /* Krylov dimension limit (default 16, <= 64)    */
  int32_t m_min;             /* first dimension tested (default 2, >= 1)      */
  int32_t max_substeps;      /* per stage exponential (default 64)            */
  int32_t block_size;        /* 0 = auto; FP64 kernel: threads per CTA (256);
                                fixed-point and mixed-precision kernels:
                                2 x block_size worker threads + one control
                                warp (384 -> 800, the largest allowed)        */
  int32_t grid_size;         /* CTAs of the persistent kernel (0 = auto,
                                capped at the co-resident maximum)            */
  int32_t steps_per_launch;  /* CFET steps per persistent launch (0 = 256)    */
  double barrier_timeout_s;  /* device barrier wait limit (default 2.0 s)     */
  int32_t precision;         /* CFET_PREC_* (default CFET_PREC_DEFAULT: the
                                fixed point, FP64 for Pauli sums)              */
  int32_t expm;              /* CFET_EXPM_* (default CFET_EXPM_KRYLOV)        */
  int32_t picture;           /* CFET_PICTURE_* (default SCHROEDINGER)         */
  int32_t reorth;            /* 1: full re-orthogonalisation of every Lanczos
                                vector (one classical Gram-Schmidt sweep
                                against all earlier ones before beta_k);
                                CFET_PREC_F64 and CFET_EXPM_KRYLOV only
                                (otherwise CFET_EINVAL).  Default 0: the
                                three-term recurrence alone.                  */
  int32_t apply_form;        /* CFET_APPLY_* (default CFET_APPLY_AUTO): how the
                                fixed-point and complex64 kernels apply an
                                XXZ chain (see below)                         */
} cfet_options;

/* Number format of the Krylov vectors on the device.  All keep alpha, beta,
 * the tridiagonal exponential and all decisions in FP64.
 *  CFET_PREC_F64: complex128 vectors, FP64 arithmetic throughout.
 *  CFET_PREC_FX : int64 (re, im) mantissas with one exponent per vector
 *                 (|mantissa| < 2^57), exact integer neighbour sums, exact
 *                 64x64->128-bit scalar products, exact 128-bit dot products;
 *                 resolution finer than FP64 relative to each vector's
 *                 largest entry.  Uses integer units instead of the FP64
 *                 units, which run at 1/64 of the FP32 rate on GB300.
 *  CFET_PREC_C64: complex64 vectors (half the bytes), FP32 apply, recurrence
 *                 and reconstruction; alpha, ||w||^2 and ||psi||^2 are
 *                 compensated (float-float) per thread and FP64 across
 *                 threads.  psi stays complex128 at the boundary.  Results
 *                 carry FP32 rounding (relative ~1e-7 per stage exponential),
 *                 so Krylov tolerances below ~1e-7 no longer bound the
 *                 error; meant for targets of about 1e-6.
 * CFET_PREC_FX and CFET_PREC_C64 on XXZ chains of 23 or more sites (Krylov
 * bases far beyond the 129 MB L2) apply H in passes over shared-memory tiles
 * (2^11 fixed-point or 2^12 complex64 elements), one pass per window of index
 * bits, instead of gathering far-bit neighbours from DRAM.                  */
enum { CFET_PREC_DEFAULT = 0, CFET_PREC_F64 = 1, CFET_PREC_FX = 2, CFET_PREC_C64 = 3 };

/* cfet_options.apply_form: the form of the XXZ-chain apply in the fixed-point
 * and complex64 Krylov kernels.
 *  AUTO        : element-wise below 23 sites, window-tiled from 23 sites.
 *  ELEMENTWISE : every element gathers its neighbours from global memory.
 *  TILED       : window passes over shared-memory tiles; chains of 13..30
 *                sites (other sizes, operators and precisions keep the
 *                element-wise form).  Any other value: CFET_EINVAL.         */
enum { CFET_APPLY_AUTO = 0, CFET_APPLY_ELEMENTWISE = 1, CFET_APPLY_TILED = 2 };

/* How cfet_propagate evaluates each stage exponential exp(-i dt H_j) psi.
 *  KRYLOV    : the Lanczos/Krylov loop (Sec. 8.1) with the a-posteriori error
 *              estimate, adaptive dimension and substeps (every precision).
 *  CHEBYSHEV : the Chebyshev technique named in Sec. 8.1 (Tal-Ezer-Kosloff):
 *              exp(-i dt H_j) psi = exp(-i dt b) sum_{k<=K} (2 - delta_k0)
 *              (-i)^k J_k(dt a) T_k((H_j - b) / a) psi, where [b - a, b + a]
 *              bounds the spectrum of H_j (Gershgorin intervals of H0 and of
 *              each V_k combined by Weyl's inequality) and K is the smallest
 *              order whose Bessel tail bound 2 sum_{k>K} |J_k(dt a)| is at most
 *              krylov_tol (2^-52 for krylov_tol <= 0).  Fixed-point precision
 *              only (CFET_PREC_FX, the default); no decision logs (forced /
 *              record must be NULL); K <= m_max * max_substeps per
 *              exponential (else CFET_EKRYLOV before any device work);
 *              |b| <= 1.5 a required (else CFET_EINVAL).  cfet_stats: n_substeps
 *              = n_exp, n_applies = sum of K, max_k = largest K, max_err_est =
 *              largest tail bound.                                          */
enum {
  CFET_EXPM_KRYLOV = 0,
  CFET_EXPM_CHEBYSHEV = 1
};

/* Picture of the CFET stepping in cfet_propagate / cfet_propagate_ex.
 *  SCHROEDINGER : the stage operators of H(t) itself.
 *  INTERACTION  : the interaction picture of the diagonal H_d of H0
 *                 (Secs. 9.3, 9.4): psi^I(t) = e^{i H_d t} psi(t) is
 *                 propagated with H^I(t) = e^{i H_d t} (H(t) - H_d) e^{-i H_d t},
 *                 whose stage operators sum_m g_{j,m} H^I(t + x_m dt) have the
 *                 off-diagonal pattern of H with entries multiplied by phases
 *                 e^{i (d(x) - d(y)) t_m}; psi enters and leaves in the
 *                 Schroedinger picture (time measured from t = 0).  Removes the
 *                 diagonal from the Krylov matrices at the price of faster time
 *                 dependence.  XXZ chains only, CFET_PREC_F64 and
 *                 CFET_EXPM_KRYLOV only (else CFET_EINVAL at create);
 *                 cfet_apply and cfet_expv of such a context still act in the
 *                 Schroedinger picture; cfet_fidelity_grad is refused.      */
enum {
  CFET_PICTURE_SCHROEDINGER = 0,
  CFET_PICTURE_INTERACTION = 1
};

typedef struct cfet_stats {
  int64_t n_exp;             /* stage exponentials evaluated                  */
  int64_t n_substeps;        /* Krylov substeps (>= n_exp)                    */
  int64_t n_applies;         /* H_j v applications (Lanczos iterations)       */
  int32_t max_k;             /* largest Krylov dimension used                 */
  int32_t status;            /* device status word (a cfet_status)            */
  double max_err_est;        /* largest accepted error estimate               */
  /* Trace of the fixed-point and mixed-precision kernels, SM clock cycles
   * per CTA (mean over CTAs
   * in phase_ns, largest CTA in phase_max_ns; zero for the FP64 kernel):
   * [0] worker loops of the apply passes, [1] control-warp work after them
   * (reduction, scalar constants; barrier wait excluded), [2] worker loops of
   * the orthogonalisation passes, [3] control work after them (reduction,
   * error estimate, decisions, constants), [4] worker loops of the
   * reconstructions, [5] time spent waiting in grid barriers, [6] control
   * work overlapped with the worker loops (speculative error estimates,
   * reconstruction coefficients), [7] time the workers wait at CTA barriers
   * for the control warp (after their loops, until released).               */
  int64_t phase_ns[8];
  int64_t phase_max_ns[8];
} cfet_stats;

/* Per-exponential Krylov decisions, host arrays owned by the caller.  One
 * record per (sub)step, in execution order: k = Krylov dimension, h = number
 * of halvings (substep length = remaining time / 2^h).  n_sub[e] counts the
 * records of stage exponential e.  As input (`forced`) the device replays the
 * records instead of testing its error estimate; as output (`record`) it
 * receives the decisions taken.                                              */
typedef struct cfet_decisions {
  int64_t n_exp;             /* exponentials covered (n_sub has this length)  */
  int32_t* n_sub;            /* [n_exp]                                       */
  int32_t* k;                /* [cap]                                         */
  int32_t* h;                /* [cap]                                         */
  int64_t cap;               /* capacity of k and h                           */
  int64_t len;               /* records provided (forced) / written (record)  */
} cfet_decisions;

typedef struct cfet_ctx cfet_ctx;

/* Fill *opt with the defaults listed above.                                 */
void cfet_options_default(cfet_options* opt);

/* Create a propagation context for H(t) = H0 + sum_k f_k(t) V_k.
 *  out     : receives the context (owned by the library; cfet_destroy frees)
 *  H0      : XXZ_CHAIN or DIA operator
 *  nV, V   : drive operators (X_FIELD for an XXZ chain, DIA for a DIA H0),
 *            all with H0's dimension; nV <= 8
 *  f, f_user: nV drive callbacks and their user pointers (f_user may be NULL)
 *  opt     : options (NULL = defaults)
 * Copies all operator data to the device and allocates the Krylov workspace
 * on the current CUDA device: m_max x dim x 16 bytes (FP64), (m_max + 1) x
 * dim x 16 bytes (fixed point) or x 8 bytes (complex64).  Errors: CFET_EINVAL
 * (inconsistent operators or options), CFET_ENOMEM, CFET_ENODEV.            */
cfet_status cfet_create(cfet_ctx** out, const cfet_op* H0, int32_t nV, const cfet_op* V,
                        const cfet_drive_fn* f, void* const* f_user, const cfet_options* opt);

void cfet_destroy(cfet_ctx* ctx);

/* Text of the last error recorded on ctx (or of the last failed create when
 * ctx is NULL).  Valid until the next call on the same context.             */
const char* cfet_last_error(const cfet_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Hot path                                                                  */
/* ------------------------------------------------------------------------ */
/* Stage operator apply (Sec. 8):  v_out = (c[0] H0 + sum_k c[1+k] V_k) v_in.
 * c: host array of 1+nV doubles.  v_in, v_out: device, dim complex128, must
 * not overlap.  Always evaluated in FP64, whatever ctx's precision.        */
cfet_status cfet_apply(cfet_ctx* ctx, const double* c, const void* v_in, void* v_out, void* stream);

/* One stage exponential psi <- exp(-i tau (c[0] H0 + sum_k c[1+k] V_k)) psi by
 * the device Lanczos loop (Sec. 8.1) in ctx's precision, with Krylov
 * tolerance tol (tol <= 0: fixed Krylov dimension m_max, no substeps).
 * stats may be NULL.                                                         */
cfet_status cfet_expv(cfet_ctx* ctx, const double* c, double tau, void* psi, double tol,
                      void* stream, cfet_stats* stats);

/* nsteps CFET steps of length dt from time t0 with the default scheme of
 * `order` (2, 4, 6 or 8): psi(t0 + nsteps dt) <- U psi(t0), in ctx's
 * precision (psi is complex128 at the boundary in every precision).  Step n uses
 * t0 + n dt, so a run can be resumed exactly from (psi, t0 + n dt).
 * krylov_tol: absolute Krylov tolerance per stage exponential (<= 0: fixed
 * dimension m_max).  stats may be NULL (then the call does not synchronise). */
cfet_status cfet_propagate(cfet_ctx* ctx, void* psi, double t0, double dt, int64_t nsteps,
                           int32_t order, double krylov_tol, void* stream, cfet_stats* stats);

/* As cfet_propagate with an explicit scheme id (CFET_SCHEME_*; DEFAULT uses
 * `order`), optional forced decisions to replay and optional decision record.
 * forced->n_exp and record->n_exp must equal nsteps * s when given.         */
cfet_status cfet_propagate_ex(cfet_ctx* ctx, void* psi, double t0, double dt, int64_t nsteps,
                              int32_t order, int32_t scheme, double krylov_tol, void* stream,
                              const cfet_decisions* forced, cfet_decisions* record,
                              cfet_stats* stats);

/* End-to-end form: psi_host (host memory, dim complex128, pinned or pageable)
 * is copied to a context-owned device buffer, propagated, and copied back;
 * synchronises the stream before returning.                                  */
cfet_status cfet_propagate_host(cfet_ctx* ctx, void* psi_host, double t0, double dt, int64_t nsteps,
                                int32_t order, double krylov_tol, void* stream, cfet_stats* stats);

/* Device status of the last propagation on ctx: synchronises `stream` and
 * returns the recorded cfet_status (stats may be NULL).                     */
cfet_status cfet_sync(cfet_ctx* ctx, void* stream, cfet_stats* stats);

/* Device time in milliseconds of the persistent-kernel launches of the last
 * cfet_propagate / cfet_propagate_ex call on ctx (CUDA events recorded inside
 * the launch graph, immediately before the first and after the last kernel
 * launch).  Synchronises on those events.                                   */
cfet_status cfet_kernel_time_ms(cfet_ctx* ctx, float* ms);

/* Allocation-free stage exponential for a small driven XXZ chain (no
 * counterpart in the paper; it exists for callers that cannot allocate
 * device memory, e.g. code whose device memory is entirely owned by another
 * allocator or a fixed up-front budget, and latency-critical loops that must
 * not take the implicit device synchronisation of cudaMalloc/cudaFree):
 *     psi <- exp(-i tau (c0 H0 + c1 sum_i a_i X_i)) psi,
 * H0 the open XXZ chain of CFET_OP_XXZ_CHAIN with couplings J, Delta and
 * fields h.  nsites in [1, 12] (dim <= 4096), m_max in [1, 32]; larger sizes
 * return CFET_EINVAL.  h[nsites], a[nsites]: host arrays.  psi: device,
 * complex128[2^nsites], in/out.  Same Krylov rule as cfet_expv (tol <= 0:
 * fixed dimension m_max).  Allocates nothing: all scratch memory lives in one
 * static device array of about 2.1 MiB that every GPU loading this library
 * holds until process exit.  The first call on a device resolves that
 * array's device address (once per device, with the device current); make
 * that first call before any stream capture.  Every call reuses the same
 * array, so calls that overlap on the GPU (other streams, other host threads)
 * race; serialise them.  Synchronises `stream` and returns the device status;
 * stats may be NULL.                                                        */
cfet_status cfet_expv_chain_static(int32_t nsites, double J, double Delta, const double* h, const double* a,
                                   double c0, double c1, double tau, void* psi, double tol, int32_t m_max,
                                   void* stream, cfet_stats* stats);

/* ------------------------------------------------------------------------ */
/* Time-step selection (Sec. 6.6)                                            */
/* ------------------------------------------------------------------------ */
/* The error model of an Nth-order CFET is eps = c T dt^N.  These calls
 * estimate c from two propagations and pick dt for an accuracy goal; each
 * propagation is a cfet_propagate_ex call of ctx (its precision and stage
 * exponential method).  order / scheme as in cfet_propagate_ex (N is the
 * scheme's order).  All three synchronise `stream`.  Device memory of
 * 2 x dim x 16 bytes is allocated on first use and kept by ctx.            */

/* c from two runs of psi0 (device, unchanged) over [t0, t0 + T]: n1 steps of
 * dt1 = T / n1 and n2 = round(n1 ratio^(1/N)) (at least n1 + 1) steps of
 * dt2 = T / n2, c = ||x1(T) - x2(T)||_2 / (T |dt1^N - dt2^N|) (the two grids
 * meet at the end of the interval; the paper suggests ratio 2 ... 3).
 * Outputs: c; diff (the norm; may be NULL); dt2 (may be NULL).  Errors:
 * CFET_EINVAL (T <= 0, n1 < 1, ratio <= 1, invalid order), the errors of
 * cfet_propagate_ex.                                                       */
cfet_status cfet_error_constant(cfet_ctx* ctx, const void* psi0, double t0, double T, int64_t n1, int32_t order,
                                int32_t scheme, double krylov_tol, double ratio, void* stream, double* c,
                                double* diff, double* dt2);

/* Step for the goal `target` over a run of length T: c from
 * cfet_error_constant over [t0, t0 + T_probe] with n_probe steps, then
 * dt = (target / (c T))^(1/N) shortened to T / ceil(T / dt).  Outputs dt,
 * nsteps (= T / dt), c (may be NULL); c = 0 gives dt = T.                  */
cfet_status cfet_select_dt(cfet_ctx* ctx, const void* psi0, double t0, double T, double target, double T_probe,
                           int64_t n_probe, int32_t order, int32_t scheme, double krylov_tol, double ratio,
                           void* stream, double* dt, int64_t* nsteps, double* c);

/* Adaptive propagation of psi (device, in place) over [t0, t0 + T]: from the
 * state at t with trial step h, one step of h and two of h/2; the local
 * constant c = ||x_h - x_{h/2}|| / (h (h^N - (h/2)^N)); the step is accepted
 * (psi <- the two-half-step result) when c T (h/2)^N <= target or h <= h_min;
 * the next trial step is min(2h, 1.8 (target / (c T))^(1/N)) clipped to
 * [h_min, h_max] and to the remaining time.  forced_h: NULL, or n_forced
 * accepted steps to replay (two steps of h/2 each, no estimate).  h_log:
 * NULL or h_cap doubles receiving the accepted steps; n_steps, n_trials (may
 * be NULL): accepted and tried steps; stats: summed over every propagation
 * (may be NULL).  Errors: CFET_EINVAL (T <= 0, target <= 0, not
 * 0 < h_min <= h0 <= h_max), CFET_EKRYLOV (more than max_steps accepted
 * steps), the errors of cfet_propagate_ex.                                 */
cfet_status cfet_propagate_adaptive(cfet_ctx* ctx, void* psi, double t0, double T, int32_t order, int32_t scheme,
                                    double krylov_tol, double target, double h0, double h_min, double h_max,
                                    int64_t max_steps, const double* forced_h, int64_t n_forced, double* h_log,
                                    int64_t h_cap, int64_t* n_steps, int64_t* n_trials, void* stream,
                                    cfet_stats* stats);

/* ------------------------------------------------------------------------ */
/* Batched propagation of many driven XXZ chains                            */
/* ------------------------------------------------------------------------ */
/* Many independent instances of uneven Hilbert dimension, each a CFET
 * propagation exactly as cfet_propagate (Sec. 4 Eq. (Ucf), Sec. 7
 * Eq. (OmGLeg), Sec. 8.1 Krylov with its own adaptive dimensions and
 * substeps), run in one persistent launch (no counterpart in the paper).
 *
 * One instance: the open XXZ chain of CFET_OP_XXZ_CHAIN (nsites, J, Delta,
 * h[nsites]) driven by f(t) sum_i a_i X_i.  The drive is the host callback
 * f(t, user) when f is non-NULL, else the built-in A cos(omega t + phase)
 * (evaluated on the host in FP64, once per Gauss-Legendre node and step).
 * h and a are copied at create.                                             */
typedef struct cfet_chain {
  int32_t nsites;            /* [1, 24]                                      */
  double J, Delta;
  const double* h;           /* [nsites]                                     */
  const double* a;           /* [nsites]                                     */
  cfet_drive_fn f;           /* NULL: built-in cosine drive                  */
  void* user;
  double A, omega, phase;
} cfet_chain;

typedef struct cfet_batch cfet_batch;  /* opaque, owned by the library     */

/* Schedule of a batched launch.  The grid is a set of thread-block clusters
 * of cluster_size CTAs with `threads` threads each that take work items in
 * order of decreasing work.  An instance with at least coop_min_sites sites
 * is one item spread over all CTAs of a cluster (cluster-wide reductions in
 * distributed shared memory); smaller instances are grouped cluster_size to
 * an item, one per CTA.  tuned_ms: kernel time of the tuning run that chose
 * the plan (0 when set by hand or default).                                 */
typedef struct cfet_batch_plan {
  int32_t cluster_size;      /* 1, 2, 4 or 8                                 */
  int32_t threads;           /* 128, 256 or 512                              */
  int32_t coop_min_sites;
  float tuned_ms;
} cfet_batch_plan;

/* Create a batch of n chains.  opt: m_max, m_min, max_substeps as for
 * cfet_create; precision CFET_PREC_F64 (also for CFET_PREC_DEFAULT and a
 * NULL opt) or CFET_PREC_C64 (CFET_PREC_FX: CFET_EINVAL); other fields
 * ignored.  The library owns all device memory
 * (Krylov bases of (m_max + 1) x 2^nsites elements per instance).  Errors:
 * CFET_EINVAL (argument), CFET_ENODEV, CFET_ENOMEM; message in
 * cfet_batch_last_error(NULL).                                              */
cfet_status cfet_batch_create(cfet_batch** out, int32_t n, const cfet_chain* chains, const cfet_options* opt);
void cfet_batch_destroy(cfet_batch* b);
const char* cfet_batch_last_error(const cfet_batch* b);
int32_t cfet_batch_size(const cfet_batch* b);

/* nsteps CFET steps of order `order` (2, 4, 6, 8; default schemes as
 * cfet_propagate) from t0 with step dt for every instance.  psi: host array
 * of n device pointers, psi[i] complex128[2^nsites_i], 16-byte aligned,
 * caller-owned, updated in place.  forced / record: NULL or arrays of n
 * decision logs as in cfet_propagate_ex (per instance).  stats: NULL or
 * cfet_stats[n].  Synchronises `stream`.  Returns the first non-OK device
 * status over the instances (CFET_EKRYLOV, CFET_ENAN); the per-instance
 * statuses are in stats.                                                    */
cfet_status cfet_batch_propagate(cfet_batch* b, void* const* psi, double t0, double dt, int64_t nsteps,
                                 int32_t order, double krylov_tol, void* stream, const cfet_decisions* forced,
                                 cfet_decisions* record, cfet_stats* stats);

/* Autotuner: runs nsteps steps of the given propagation on internal states
 * (normalised pseudo-random vectors, reset before every candidate) for every
 * candidate plan (cluster size 1, 2, 4, 8 x 128, 256, 512 threads x three
 * thresholds) that fits on the device, keeps the fastest as the batch's plan
 * and returns it in `chosen` (may be NULL).  Caller states are not touched. */
cfet_status cfet_batch_tune(cfet_batch* b, double t0, double dt, int32_t order, double krylov_tol, int64_t nsteps,
                            void* stream, cfet_batch_plan* chosen);
cfet_status cfet_batch_get_plan(const cfet_batch* b, cfet_batch_plan* plan);
cfet_status cfet_batch_set_plan(cfet_batch* b, const cfet_batch_plan* plan);

/* Device time in milliseconds of the last batched launch.                  */
cfet_status cfet_batch_kernel_time_ms(cfet_batch* b, float* ms);

/* ------------------------------------------------------------------------ */
/* Gradient of the fidelity loss (adjoint sweep)                             */
/* ------------------------------------------------------------------------ */
typedef struct cfet_grad_stats {
  double overlap_re, overlap_im;   /* <phi|psi(T)>                            */
  double max_drift;                /* largest ||psi_recovered - checkpoint||  */
  int64_t n_applies_forward;       /* H applications of the forward pass      */
  int64_t n_applies_backward;      /* H applications of the adjoint sweep      */
  float forward_ms, backward_ms;   /* device time of both passes              */
} cfet_grad_stats;

/* L = 1 - |<phi|psi(T)>|^2 and dL/dA_k for the drive of ctx's single X field
 * replaced by the piecewise-constant amplitude f(t) = amps[k] cos(omega t +
 * phase) on segment k (nseg segments of nsteps / nseg CFET steps each, so
 * the Gauss-Legendre nodes of a step lie in one segment); psi(T) is the CFET
 * propagation of psi0 over nsteps steps of dt from t0 (order 2, 4, 6, 8;
 * Sec. 4 Eq. (Ucf), Sec. 7 Eq. (OmGLeg)).  No counterpart in the paper.
 * The forward pass runs ctx's propagator (its precision) and stores psi every
 * checkpoint_every steps; the backward sweep (FP64) undoes each stage
 * exponential with the inverse unitary step in the Krylov space of the
 * current state while propagating the adjoint state, and takes each stage's
 * derivative d/dc exp(-i dt (c0 H0 + c V)) as the exact time integral of
 * e^{i r H} V e^{i r H}-type terms inside the two Krylov spaces (Gauss-Legendre
 * in r); at every checkpoint the recovered state is replaced by the stored one
 * (max_drift reports the largest difference).  Requirements: ctx is an XXZ
 * chain with exactly one X-field drive operator, ctx's m_max <= 16, every
 * stage exponential of the sweep needs no substeps (else CFET_EKRYLOV).
 * psi0, phi: device complex128[dim], unchanged.  amps: host [nseg].  loss:
 * host scalar; grad: host [nseg].  Synchronises `stream`; gstats may be NULL.
 * Device memory of about (nsteps / checkpoint_every + 34) x dim x 16 bytes is
 * allocated on first use and kept by ctx.                                    */
cfet_status cfet_fidelity_grad(cfet_ctx* ctx, const void* psi0, const void* phi, double t0, double dt,
                               int64_t nsteps, int32_t order, double krylov_tol, int32_t nseg, const double* amps,
                               double omega, double phase, int64_t checkpoint_every, void* stream, double* loss,
                               double* grad, cfet_grad_stats* gstats);

/* Diagnostic of the bounded device waits (no counterpart in the paper): two
 * CTAs, of which one enters a grid-wide wait that the other never joins —
 * which = 0: the record exchange of the fixed-point / complex64 kernels,
 * 1: the grid barrier of the FP64 kernel.  The wait must give up after
 * timeout_s (in (0, 10] s), record CFET_ETIMEOUT and return; no fault, no
 * hang.  Returns CFET_OK when the device status read back (device_status) is
 * CFET_ETIMEOUT, CFET_ECUDA otherwise.  Synchronises the device.            */
cfet_status cfet_selftest_wait_timeout(int32_t which, double timeout_s, int32_t* device_status);

/* Copy-bandwidth probe (no counterpart in the paper; the measured
 * denominator of the L2 roofline): one launch of `reps` grid-stride copies of
 * `bytes` bytes, alternating a -> b and b -> a, timed with CUDA events on
 * `stream`; *gbs = 2 bytes reps / time in GB/s (read + write).  a, b: two
 * distinct caller-owned device buffers of at least `bytes` bytes, 16-byte
 * aligned; their contents are overwritten.  Buffers that fit in L2 together
 * give the L2-served copy rate, larger ones the DRAM rate.  Synchronises
 * `stream`.  Errors: CFET_EINVAL (NULL or equal pointers, misalignment,
 * bytes not a positive multiple of 16, reps outside [1, 100000]),
 * CFET_ENODEV, CFET_ECUDA.                                                  */
cfet_status cfet_probe_copy_gbs(void* a, void* b, int64_t bytes, int32_t reps, void* stream, double* gbs);

/* Host-only check (no device needed) of the index arithmetic of the
 * window-tiled apply of long chains (CFET_PREC_FX uses tile_bits 11,
 * CFET_PREC_C64 12): for an nsites chain, every basis index appears in
 * exactly one tile slot per window, every single-site flip and every bond
 * (i, i+1) is applied in exactly one window, and tile slots pair up into
 * contiguous 16-byte copy units.  *checked receives the number of
 * (window, index) pairs visited.  Returns CFET_EINVAL for tile_bits other
 * than 11, 12 or nsites outside [tile_bits, 27], CFET_ECUDA when the tiling
 * is inconsistent.                                                          */
cfet_status cfet_selftest_tiling(int32_t nsites, int32_t tile_bits, int64_t* checked);

/* Host-only checks (no device needed) of the scalar helpers that the
 * control warps of the persistent kernels use instead of FP64 instructions
 * (the same source compiled for the host).
 *
 * cfet_selftest_i128_to_double: out[i] = (hi[i] 2^64 + lo[i]) 2^shift, the
 * two's-complement 128-bit integers rounded to the nearest double (ties to
 * even), for i < n; shift in [-200, 200].  This is how the exact 128-bit
 * reductions of the fixed-point kernels become FP64 values.
 *
 * cfet_selftest_krylov_bounds: for the k x k real symmetric tridiagonal T_k
 * with diagonal a[0..k-1] and couplings b[0..k-2] (the Lanczos matrix of
 * Sec. 8.1) and the step ts:
 *   log2_bounds[0] = a certified lower bound of log2 |e_{k-1}^T exp(-i ts T_k) e_0|
 *     (leading Taylor term |ts|^{k-1} prod b_j / (k-1)! times
 *     2 - exp(g), g = |ts| D + (|ts| B)^2 / k, D = half the spread of the
 *     diagonal, B = max b_j, all roundings taken off), or -1e30 when that bound
 *     is void; log2_bounds[1] = a certified upper bound (the leading term times
 *     exp(g)), or 1e30; the kernels reject k without evaluating the
 *     exponential when beta0 beta_k times the lower bound exceeds the
 *     estimate's threshold, and skip the FP32 screen when the upper bound
 *     already meets it;
 *   *gate = 1 when |ts| w <= 2k, 0 when |ts| w > 2k for certain (w the
 *     Gershgorin width of T_k, the gate of the estimate), -1 when the FP32
 *     evaluation cannot decide (the kernels then evaluate it in FP64).
 * k in [1, 64]; CFET_EINVAL otherwise or for NULL pointers.                 */
cfet_status cfet_selftest_i128_to_double(const uint64_t* lo, const int64_t* hi, int64_t n, int32_t shift,
                                         double* out);
/* cfet_selftest_ll_to_double_up: out[i] = the smallest double not below v[i]
 * (v[i] >= 0; 0 for v[i] <= 0), for i < n: the conversion of the fixed-point
 * kernels' int64 maxima, which enter the exponent bounds and must not round
 * down.  CFET_EINVAL for NULL pointers or n < 0.                            */
cfet_status cfet_selftest_ll_to_double_up(const int64_t* v, int64_t n, double* out);
cfet_status cfet_selftest_krylov_bounds(int32_t k, const double* a, const double* b, double ts, double* log2_bounds,
                                        int32_t* gate);

/* Dimension and drive-operator count of ctx (for bindings).                 */
int64_t cfet_dim(const cfet_ctx* ctx);
int32_t cfet_num_drives(const cfet_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* CFET_H */
