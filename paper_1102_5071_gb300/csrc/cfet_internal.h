// Internal declarations shared by the host C-ABI code and the device kernels.
#pragma once

#include <cstdint>
#include <vector>

#include <vector_types.h>

#include "../../include/cfet.h"

namespace cfet {

constexpr int kMaxKrylov = 64;   // m_max limit (two tridiagonal rows per lane)
constexpr int kMaxDrives = 8;    // drive operators V_k
constexpr int kMaxSites = 30;    // spin chains: dim = 2^N < 2^31
constexpr int kMaxDiag = 32;     // DIA: stored diagonals over H0 and all V_k
constexpr int kSmallTaylorTerms = 18;

// Largest CTA (threads) of the kernels with a control warp (fixed point,
// complex64): 2 x block_size workers + 32, block_size <= 384.
#ifndef CFET_CTL_MAX_THREADS
#define CFET_CTL_MAX_THREADS 800
#endif

// ---------------------------------------------------------------- schemes
struct SchemeData {
  int id, order, s, M;
  double f[11][4];   // full table after rule (R1)
  double x[4], w[4];  // Gauss-Legendre points / weights on [0,1]
  double g[11][4];   // g_{i,m}
};
bool build_scheme(int id, SchemeData* out);
int default_scheme_for_order(int order);

// ---------------------------------------------------------------- device state
struct DevStatus {
  int status;          // cfet_status
  int max_k;
  int rec_overflow;
  unsigned tag_base;   // tags of the record exchange used so far (control-warp kernels)
  long long n_exp, n_sub, n_app;
  double max_err;
  long long rec_pos;   // next record slot
  long long forced_pos;  // next forced slot
  long long phase_ns[8];      // see cfet_stats.phase_ns (sum over CTAs)
  long long phase_max_ns[8];  // max over CTAs
};

// Spin chain operator family: H0 = XXZ chain, V_k = transverse fields.
struct OpSpin {
  int N;               // sites
  int lo_bits;         // L: diagonal table split
  double J2;           // 2 J  (matrix element of X X + Y Y between |01>, |10>)
  const double* dz_lo; // [2^L]        sum over bits [0, L)
  const double* dz_hi; // [2^(N-L+1)]  sum over bits [L-1, N)
  const double* xf;    // [nV * N] per-field per-site X coefficients
};

// Spin chain in the interaction picture of the diagonal of H0 (Secs. 9.3,
// 9.4): stage operator entries are the off-diagonal entries of H(t_m) times
// e^{i (d(x) - d(y)) t_m}, summed over the Gauss-Legendre nodes with g_{j,m}.
// They depend only on a few neighbouring spins, so each stage comes as a table
// of complex weights (host-computed): flip of site i, index i*10 + b*5 + n + 2
// (b = bit i of x, n = s_{i-1} + s_{i+1} over existing neighbours), then hop
// of bond (i, i+1), index 10 N + i*10 + b*5 + m + 2 (m = s_{i-1} - s_{i+2}).
constexpr int kIPWeightsPerSite = 10;
struct OpSpinIP {
  int N;
  int nw;              // complex weights per exponential: 10 N + 10 (N - 1)
  const double2* w;    // [nexp of the call][nw] (global exponential index)
};

// Pauli-sum family (FP64 kernel): the strings of all operators grouped by
// their X mask; string t of group g contributes
//   pc[t] (-1)^popc((y ^ gx[g]) & tz[t]) (i if tim[t]) v[y ^ gx[g]]
// with pc[t] = c_{top[t]} tc[t] for the stage scalars c (tc folds the sign of
// i^popc(x&z) into the coefficient, tim marks an odd popcount).
constexpr int kMaxPauliTerms = 4096;
struct OpPauli {
  int N;
  int ngroups;
  int nterms;
  const unsigned* gx;        // [ngroups]
  const int* gstart;         // [ngroups + 1]
  const unsigned* tz;        // [nterms]
  const int* top;            // [nterms]: 0 = H0, 1 + k = V_k
  const double* tc;          // [nterms]
  const unsigned char* tim;  // [nterms]
  const unsigned char* greal;  // [ngroups]: 1 when every string of the group has a real phase
  // Tabulated diagonal: the Z-only strings (group 0, X mask 0) summed per
  // operator for every index, dtab[j * 2^N + y] = sum over the strings of
  // operator dop[j] of tc (-1)^popc(y & z); the apply then starts at group g0.
  int g0;                    // 1 when group 0 is tabulated, else 0
  int nd;                    // operators with a table
  int dop[1 + kMaxDrives];
  const double* dtab;
};

// Banded family: all operators in DIA form, concatenated.
struct OpDia {
  int ndiag;
  const long long* off;  // [ndiag]
  const int* opidx;      // [ndiag]: 0 = H0, 1 + k = V_k
  const double* val;     // [ndiag * dim]
};

// General sparse family: every operator in compressed sparse row form,
// concatenated (Sec. 8: the stage operator sum_k c_k H_k is applied term by
// term with the stage scalars, never formed).  Row r of operator o holds the
// entries [rp[o * (dim + 1) + r], rp[o * (dim + 1) + r + 1]) of col / vr / vi.
struct OpCsr {
  int nops;              // 1 + nV
  const int* rp;         // [nops * (dim + 1)]
  const int* col;        // [nnz]
  const double* vr;      // [nnz] real parts
  const double* vi;      // [nnz] imaginary parts; NULL when every operator is real
};

// Fixed-point forms of the operator families (see kernels_fx.cu).
struct OpSpinFx {
  int N;
  int lo_bits;
  int E_dz;               // DZ tables hold dz * 2^-E_dz as int64, |DZ_lo + DZ_hi| < 2^61
  int uniform;            // every drive field has the same coefficient on all sites
  const long long* DZ_lo;
  const long long* DZ_hi;
  double maxdz;           // bound of |dz(x)| in real units
  double J2;              // 2 J
  double nbond, nsite;    // N - 1 and N as doubles (no conversion on the control path)
  const double* xf;       // [nV * N] per-field per-site X coefficients
};

struct OpDiaFx {
  int ndiag;
  int nops;               // 1 + nV
  const long long* off;   // [ndiag]
  const int* opidx;       // [ndiag], diagonals grouped by operator (non-decreasing)
  const long long* VAL;   // [ndiag * dim]: val * 2^-E_op[opidx[d]], |VAL| < 2^62
  int E_op[1 + kMaxDrives];
  double maxrow[1 + kMaxDrives];  // max over rows of sum_{d in op} |val_d[r]|
  int dfirst[1 + kMaxDrives];     // first diagonal of each operator
  int dcount[1 + kMaxDrives];     // number of diagonals of each operator
};

struct OpCsrFx {
  int nops;               // 1 + nV
  const int* rp;          // as OpCsr
  const int* col;
  const long long* VR;    // [nnz]: re * 2^-E_op[o]; per row sum |VR| + |VI| < 2^62
  const long long* VI;    // [nnz] or NULL (real operators)
  int E_op[1 + kMaxDrives];
  double maxrow[1 + kMaxDrives];  // max over rows of sum (|re| + |im|), real units
};

// Mixed-precision forms (see kernels_c64.cu): FP32 operator data.
struct OpSpinC {
  int N;
  int lo_bits;
  int uniform;            // every drive field has the same coefficient on all sites
  double J2;              // 2 J
  const float* dz_lo;     // [2^L]        FP32 copy of OpSpin::dz_lo
  const float* dz_hi;     // [2^(N-L+1)]  FP32 copy of OpSpin::dz_hi
  const double* xf;       // [nV * N] per-field per-site X coefficients (FP64)
};

struct OpDiaC {
  int ndiag;
  int nops;               // 1 + nV
  const long long* off;   // [ndiag], diagonals grouped by operator
  const float* val;       // [ndiag * dim], zero where the column is outside [0, dim)
  int dfirst[1 + kMaxDrives];
  int dcount[1 + kMaxDrives];
};

struct OpCsrC {
  int nops;
  const int* rp;
  const int* col;
  const float* vr;
  const float* vi;        // NULL for real operators
};

struct PropParams {
  int dim;
  int nV;
  double2* psi;
  double2* basis;        // m_max * dim; q_{i} lives at basis + (i-2)*dim, i >= 2
  const double* scal;    // [nexp * (1 + nV)]
  long long nexp;
  long long exp_base;    // global index of exponential 0 of this launch
  double tau, tol;
  int m_min, m_max, max_substeps;
  int tiled;             // spin chains: window-tiled apply (complex64 and fixed-point kernels)
  int reorth;            // FP64 kernel: full re-orthogonalisation of every Lanczos vector
  int small;             // fixed-point kernel, one CTA: the Krylov basis lives in shared memory
  // decisions (device arrays, nullable)
  const int* f_nsub; const int* f_k; const int* f_h;
  int* r_nsub; int* r_k; int* r_h; long long r_cap;
  // reductions and synchronisation
  double* partials;      // [2 * gridDim.x]
  unsigned* bar;         // [2]: arrival count, generation
  DevStatus* st;
  long long timeout_ns;
  // fixed-point path: Krylov vectors q_1 .. q_{m_max+1} as int64 (re, im)
  // pairs; q_i at qbasis + (i-1)*dim.  partials then hold 4 * gridDim.x.
  longlong2* qbasis;
  // mixed-precision path: complex64 Krylov vectors, q_i at qbasis32 + (i-1)*dim
  float2* qbasis32;
  // Chebyshev path: kChebRec doubles per exponential (global index) and the
  // concatenated expansion coefficients r_k
  const double* cheb;
  const double* cheb_coef;
  // interaction picture (propagate only): stage weights [nexp][ip_nw] of
  // OpSpinIP and the times {t0, t_end} of the picture changes; NULL otherwise
  const double2* ip_w;
  const double* ip_times;
  int ip_nw;
  // window-tiled complex64 apply: one TMA tensor map (128 bytes) per window
  // over the Krylov basis (device memory, 64-byte aligned)
  const unsigned char* tmaps;
};

// Chebyshev record of one stage exponential (host-computed, see chebyshev.cpp):
// 1/a, b/a, K, offset of r_0 in cheb_coef, sum_k |r_k|, cos(dt b), -sin(dt b),
// tail bound
constexpr int kChebRec = 8;
int cheb_kmax(double z);
int cheb_series(double z, double tol, std::vector<double>* r, double* tail);
void spin_h0_interval(int N, double J, double Delta, const double* h, double* lo, double* hi);
void xfield_interval(int N, const double* a, double* lo, double* hi);
void dia_interval(const int64_t* offsets, const double* values, int ndiag, int dim, double* lo, double* hi);
void csr_interval(const int64_t* row_ptr, const int32_t* col, const double* re, const double* im, int dim,
                  double* lo, double* hi);
void stage_interval(int nops, const double* op_lo, const double* op_hi, const double* s, double* lo, double* hi);
int launch_cheb_spin_fx(const PropParams& p, const OpSpinFx& op, int grid, int block, void* stream);
int launch_cheb_dia_fx(const PropParams& p, const OpDiaFx& op, int grid, int block, void* stream);
int launch_cheb_csr_fx(const PropParams& p, const OpCsrFx& op, int grid, int block, void* stream);
int max_coresident_blocks_cheb(int family, int block);
int cheb_threads(int workers);  // threads per CTA of the Chebyshev kernel for `workers` element threads

// Backward (adjoint) sweep of the fidelity gradient (see adjoint.cu).
constexpr int kAdjMaxK = 16;     // Krylov dimension limit of the adjoint sweep
constexpr int kAdjMaxNodes = 48; // Gauss-Legendre nodes of the stage integral

struct AdjParams {
  int dim;
  int m_min, m_max;
  int pad0;
  double tau, tol;
  double2* psi;            // in: state after exponential e_hi - 1; out: state before e_lo
  const double2* ckpt;     // nullable: stored forward state replacing psi on entry
  double2* lam;            // adjoint state, in / out
  const double2* phi;      // nullable (first launch): lam = phi, overlap <phi|psi>
  double2* Vp;             // Krylov vectors q_2 .. q_{m_max+1} of psi
  double2* Vl;             // Krylov vectors of lam
  const double* c0;        // per exponential (application order): H0 coefficient
  const double* c1;        //   V coefficient (amplitude x gamma)
  const double* gam;       //   d c1 / d amplitude
  const int* seg;          //   amplitude segment
  long long e_lo, e_hi;    // exponentials e_hi - 1 down to e_lo are undone
  int nq6, nq12, nq24, nq48;  // offsets of the 6-, 12-, 24-, 48-node rules in glx / glw
  int pad1;
  const double* glx;       // Gauss-Legendre nodes on [0, 1]
  const double* glw;
  double* grad;            // [2 nseg]: accumulated d<phi|psi(T)>/dA_k (re, im)
  double* out;             // [4]: re, im of the overlap (first launch), max drift, n_applies
  double* partials;        // [2 slots x 34 values x grid]
  unsigned* bar;
  DevStatus* st;
  long long timeout_ns;
};

// ---------------------------------------------------------------- launchers
// (defined in kernels.cu; return a cudaError_t as int)
int launch_propagate_spin(const PropParams& p, const OpSpin& op, int grid, int block, void* stream);
int launch_propagate_dia(const PropParams& p, const OpDia& op, int grid, int block, void* stream);
int launch_propagate_csr(const PropParams& p, const OpCsr& op, int grid, int block, void* stream);
int launch_propagate_spin_ip(const PropParams& p, const OpSpinIP& op, int grid, int block, void* stream);
int max_coresident_blocks_ip(int block, int nw);
int launch_propagate_pauli(const PropParams& p, const OpPauli& op, int grid, int block, void* stream);
int max_coresident_blocks_pauli(int block, int nterms);
int launch_pauli_diag_table(const OpPauli& op, int n0, double* dtab, void* stream);
int launch_apply_pauli(const OpPauli& op, int dim, const double* c, int nV, const double2* vin, double2* vout,
                       void* stream);
// psi[x] *= exp(i sign d(x) t[which]) with d the diagonal of the XXZ chain H0
int launch_phase_diag(double2* psi, const OpSpin& op, int dim, const double* t, int which, double sign, void* stream);
int launch_apply_spin(const OpSpin& op, int dim, const double* c, int nV, const double2* vin, double2* vout,
                      void* stream);
int launch_apply_dia(const OpDia& op, int dim, const double* c, int nV, const double2* vin, double2* vout,
                     void* stream);
int launch_apply_csr(const OpCsr& op, int dim, const double* c, int nV, const double2* vin, double2* vout,
                     void* stream);
int launch_spin_tables(int N, int L, double J, double Delta, const double* h, double* dz_lo, double* dz_hi,
                       void* stream);
int launch_propagate_spin_fx(const PropParams& p, const OpSpinFx& op, int grid, int block, void* stream);
int launch_propagate_dia_fx(const PropParams& p, const OpDiaFx& op, int grid, int block, void* stream);
int launch_propagate_csr_fx(const PropParams& p, const OpCsrFx& op, int grid, int block, void* stream);
int max_coresident_blocks_fx(int family, int block, bool tiled);
// One-CTA fixed-point launches with the Krylov basis in shared memory.
constexpr size_t kFxSmallSmemMax = 200 * 1024;
size_t fx_small_smem_bytes(int dim, int m_max);
int fx_small_prepare(size_t bytes);
int launch_propagate_spin_c64(const PropParams& p, const OpSpinC& op, int grid, int block, void* stream);
int launch_propagate_dia_c64(const PropParams& p, const OpDiaC& op, int grid, int block, void* stream);
int launch_propagate_csr_c64(const PropParams& p, const OpCsrC& op, int grid, int block, void* stream);
int max_coresident_blocks_c64(int family, int block, bool tiled);
// Chains of at least this many sites take the window-tiled apply
// (tiled_common.cuh) in the complex64 and fixed-point kernels, unless
// cfet_options.apply_form asks for one form.
constexpr int kC64TiledMinSites = 23;
constexpr int kC64TileBits = 12;    // tiles of 2^12 complex64 elements (32 KB)
constexpr int kFxTileBits = 11;    // fixed-point tiled apply: tiles of 2^11 int64 pairs
constexpr int kFxTiledMinSites = 23;
constexpr int kTiledMinSites = 13;  // tiles of up to 2^12 elements
constexpr int kTiledMaxSites = 30;  // four windows cover 32 sites at 2^11-element tiles
int launch_adjoint_spin(const AdjParams& p, const OpSpin& op, int grid, int block, void* stream);
int launch_wait_selftest(int which, unsigned long long* rec, unsigned* bar, int* status, long long timeout_ns);
constexpr int kDiffBlocks = 152;  // blocks (partials) of the difference norm
int launch_diff_norm2(const double2* a, const double2* b, int n, double* part, int nblk, void* stream);
int launch_copy_probe(void* a, void* b, long long n16, int reps, int grid, void* stream);
int max_coresident_blocks_adjoint(int block);
int max_coresident_blocks(int family, int block);  // per device, for the persistent kernel
size_t propagate_smem_bytes(int block);

enum Family { kFamilySpin = 1, kFamilyDia = 2, kFamilySpinIP = 3, kFamilyPauli = 4, kFamilyCsr = 5 };

}  // namespace cfet
