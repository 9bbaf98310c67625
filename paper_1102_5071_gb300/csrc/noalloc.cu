// Allocation-free stage exponential for small spin chains.
//
// Some callers cannot call cudaMalloc: code whose device memory is entirely
// owned by another allocator (a framework's caching pool, a fixed memory
// budget reserved up front), and latency-critical loops where the implicit
// device synchronisation of cudaMalloc/cudaFree is not acceptable.  For them
// cfet_expv_chain_static runs the same persistent Lanczos kernel as
// cfet_expv, but every piece of scratch memory it needs (Krylov basis,
// diagonal tables, stage scalars, reduction partials, barrier words, status)
// lives in one file-scope __device__ array of fixed size.  The caller passes
// only psi (in/out, device) and host-side parameters.
//
// The array is part of the loaded module: every GPU that loads this library
// holds it (kStaticBytes, about 2.1 MiB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "cfet_internal.h"

using namespace cfet;

namespace {

constexpr int kStaticMaxSites = 12;     // dim <= 4096
constexpr int kStaticMaxKrylov = 32;    // m_max <= 32
constexpr int kStaticBlock = 256;
constexpr int kStaticMaxDim = 1 << kStaticMaxSites;
constexpr int kStaticMaxGrid = kStaticMaxDim / kStaticBlock;  // one element per thread at most

constexpr size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// byte offsets of the regions inside the static array
constexpr size_t kOffBasis = 0;
constexpr size_t kOffDzLo = kOffBasis + align256(sizeof(double2) * kStaticMaxKrylov * kStaticMaxDim);
constexpr size_t kOffDzHi = kOffDzLo + align256(sizeof(double) * 1024);
constexpr size_t kOffH = kOffDzHi + align256(sizeof(double) * (1 << (kStaticMaxSites - 10 + 1)));
constexpr size_t kOffXf = kOffH + align256(sizeof(double) * kStaticMaxSites);
constexpr size_t kOffScal = kOffXf + align256(sizeof(double) * kStaticMaxSites);
constexpr size_t kOffPart = kOffScal + align256(sizeof(double) * 2);
constexpr size_t kOffBar = kOffPart + align256(sizeof(double) * 3 * kStaticMaxGrid);
constexpr size_t kOffSt = kOffBar + align256(sizeof(unsigned) * 2);
constexpr size_t kStaticBytes = kOffSt + align256(sizeof(DevStatus));

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct DeviceSetup {
  bool done = false;
  unsigned char* base = nullptr;  // device address of g_static_scratch
  int max_grid = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: resolve the device address of
// the static array (in host code its name is only a host-side stand-in) and
// the co-resident CTA limit of the persistent kernel.
cfet_status setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return CFET_ECUDA;
    }
    const int mg = max_coresident_blocks(kFamilySpin, kStaticBlock);
    if (mg < 1) return CFET_ECUDA;
    s.base = static_cast<unsigned char*>(ptr);
    s.max_grid = mg;
    s.done = true;
  }
  *out = &s;
  return CFET_OK;
}

}  // namespace

extern "C" cfet_status cfet_expv_chain_static(int32_t nsites, double J, double Delta, const double* h,
                                              const double* a, double c0, double c1, double tau, void* psi,
                                              double tol, int32_t m_max, void* stream, cfet_stats* stats) {
  if (nsites < 1 || nsites > kStaticMaxSites) return CFET_EINVAL;
  if (m_max < 1 || m_max > kStaticMaxKrylov) return CFET_EINVAL;
  if (!h || !a || !psi || (reinterpret_cast<uintptr_t>(psi) % 16) != 0) return CFET_EINVAL;
  if (!std::isfinite(J) || !std::isfinite(Delta) || !std::isfinite(c0) || !std::isfinite(c1) ||
      !std::isfinite(tau) || tau == 0.0 || !std::isfinite(tol))
    return CFET_EINVAL;
  for (int i = 0; i < nsites; ++i)
    if (!std::isfinite(h[i]) || !std::isfinite(a[i])) return CFET_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return CFET_ENODEV;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CFET_ECUDA;
  DeviceSetup* s = nullptr;
  cfet_status st = setup_device(dev, &s);
  if (st != CFET_OK) return st;

  const int N = nsites;
  const int L = N < 10 ? N : 10;
  const int dim = 1 << N;
  unsigned char* b = s->base;
  double2* basis = reinterpret_cast<double2*>(b + kOffBasis);
  double* dz_lo = reinterpret_cast<double*>(b + kOffDzLo);
  double* dz_hi = reinterpret_cast<double*>(b + kOffDzHi);
  double* d_h = reinterpret_cast<double*>(b + kOffH);
  double* d_xf = reinterpret_cast<double*>(b + kOffXf);
  double* d_scal = reinterpret_cast<double*>(b + kOffScal);
  double* d_part = reinterpret_cast<double*>(b + kOffPart);
  unsigned* d_bar = reinterpret_cast<unsigned*>(b + kOffBar);
  DevStatus* d_st = reinterpret_cast<DevStatus*>(b + kOffSt);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);

  const double scal[2] = {c0, c1};
  if (cudaMemcpyAsync(d_h, h, sizeof(double) * N, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
      cudaMemcpyAsync(d_xf, a, sizeof(double) * N, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
      cudaMemcpyAsync(d_scal, scal, sizeof(scal), cudaMemcpyHostToDevice, cs) != cudaSuccess ||
      cudaMemsetAsync(d_st, 0, sizeof(DevStatus), cs) != cudaSuccess ||
      cudaMemsetAsync(d_bar, 0, sizeof(unsigned) * 2, cs) != cudaSuccess)
    return CFET_ECUDA;
  if (launch_spin_tables(N, L, J, Delta, d_h, dz_lo, dz_hi, cs) != cudaSuccess) return CFET_ECUDA;

  OpSpin op{};
  op.N = N;
  op.lo_bits = L;
  op.J2 = 2.0 * J;
  op.dz_lo = dz_lo;
  op.dz_hi = dz_hi;
  op.xf = d_xf;
  PropParams p{};
  p.dim = dim;
  p.nV = 1;
  p.psi = static_cast<double2*>(psi);
  p.basis = basis;
  p.scal = d_scal;
  p.nexp = 1;
  p.exp_base = 0;
  p.tau = tau;
  p.tol = tol;
  p.m_min = m_max < 2 ? 1 : 2;
  p.m_max = m_max;
  p.max_substeps = 64;
  p.partials = d_part;
  p.bar = d_bar;
  p.st = d_st;
  p.timeout_ns = 2000000000LL;
  int grid = (dim + kStaticBlock - 1) / kStaticBlock;
  if (grid > s->max_grid) grid = s->max_grid;
  if (launch_propagate_spin(p, op, grid, kStaticBlock, cs) != cudaSuccess) return CFET_ECUDA;

  DevStatus hs;
  if (cudaMemcpyAsync(&hs, d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return CFET_ECUDA;
  if (stats) {
    stats->n_exp = hs.n_exp;
    stats->n_substeps = hs.n_sub;
    stats->n_applies = hs.n_app;
    stats->max_k = hs.max_k;
    stats->status = hs.status;
    stats->max_err_est = hs.max_err;
    for (int i = 0; i < 8; ++i) {
      stats->phase_ns[i] = hs.phase_ns[i];
      stats->phase_max_ns[i] = hs.phase_max_ns[i];
    }
  }
  return static_cast<cfet_status>(hs.status);
}
