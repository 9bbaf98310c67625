// Host side of the Chebyshev stage exponential (Sec. 8.1: the Chebyshev
// technique, which needs a-priori bounds on the eigenvalues of the stage
// operator).
//
//  * Spectral bounds: the Gershgorin interval [min_r (A_rr - R_r),
//    max_r (A_rr + R_r)] of each operator (H0 and every V_k), combined for a
//    stage operator sum_o s_o A_o by Weyl's inequality.  For the XXZ chain the
//    extremes over the 2^N rows are found exactly by a two-state dynamic
//    programme along the chain (the row value is a sum of site and bond terms).
//  * Expansion: exp(-i z x) = sum_k (2 - delta_k0) (-i)^k J_k(z) T_k(x) on
//    [-1, 1] (Jacobi-Anger); the Bessel values J_k(z), k = 0..n, come from
//    Miller's backward recurrence J_{k-1} = (2k / z) J_k - J_{k+1}, started
//    well above max(n, z) and normalised by J_0 + 2 sum_{k>=1} J_{2k} = 1.
//  * Truncation: the smallest K >= 0 with 2 sum_{k>K} |J_k(z)| <= tol (tail
//    summed up to kmax(z) = ceil(z + 16 z^(1/3) + 40), beyond which the
//    values are below 1e-30); tol <= 0 means 2^-52.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "cfet.h"
#include "cfet_internal.h"

namespace cfet {

int cheb_kmax(double z) {
  z = std::fabs(z);
  return (int)std::ceil(z + 16.0 * std::cbrt(z) + 40.0);
}

// J_0(z) .. J_n(z) for z > 0.
static void bessel_j_seq(double z, int n, std::vector<double>& J) {
  const int top = std::max(n, cheb_kmax(z)) + 30;
  std::vector<double> f((size_t)top + 2, 0.0);
  f[top] = 1e-280;
  for (int k = top; k >= 1; --k) {
    f[k - 1] = (2.0 * k / z) * f[k] - f[k + 1];
    if (std::fabs(f[k - 1]) > 1e250)
      for (int j = k - 1; j <= top; ++j) f[j] *= 1e-250;
  }
  double s = f[0];
  for (int k = 2; k <= top; k += 2) s += 2.0 * f[k];
  J.assign((size_t)n + 1, 0.0);
  for (int k = 0; k <= n; ++k) J[k] = f[k] / s;
}

int cheb_series(double z, double tol, std::vector<double>* r, double* tail_out) {
  const double eps = tol > 0.0 ? tol : std::ldexp(1.0, -52);
  if (z == 0.0) {
    if (r) r->assign(1, 1.0);
    if (tail_out) *tail_out = 0.0;
    return 0;
  }
  const int km = cheb_kmax(z);
  std::vector<double> J;
  bessel_j_seq(std::fabs(z), km, J);
  if (z < 0.0)
    for (int k = 1; k <= km; k += 2) J[k] = -J[k];  // J_k(-z) = (-1)^k J_k(z)
  // tail[K] = 2 sum_{k=K+1}^{km} |J_k|; the smallest K with tail <= eps
  std::vector<double> tail((size_t)km + 1, 0.0);
  double acc = 0.0;
  for (int k = km; k >= 0; --k) {
    tail[k] = 2.0 * acc;
    acc += std::fabs(J[k]);
  }
  int K = km;
  for (int k = 0; k <= km; ++k)
    if (tail[k] <= eps) {
      K = k;
      break;
    }
  if (r) {
    r->assign(J.begin(), J.begin() + K + 1);
    for (int k = 1; k <= K; ++k) (*r)[k] *= 2.0;
  }
  if (tail_out) *tail_out = tail[K];
  return K;
}

void spin_h0_interval(int N, double J, double Delta, const double* h, double* lo, double* hi) {
  // row value of site spins s_i = +-1: sum_i h_i s_i + sum_i J Delta s_i s_{i+1}
  // plus (upper end) or minus (lower end) 2|J| for every antiparallel bond
  const double JD = J * Delta, R = 2.0 * std::fabs(J);
  double up[2], dn[2];  // best value ending in s = +1 (index 0) / -1 (index 1)
  up[0] = h[0];
  up[1] = -h[0];
  dn[0] = h[0];
  dn[1] = -h[0];
  for (int i = 1; i < N; ++i) {
    double nu[2], nd[2];
    for (int b = 0; b < 2; ++b) {
      const double sb = b == 0 ? 1.0 : -1.0;
      double bu = -INFINITY, bd = INFINITY;
      for (int a = 0; a < 2; ++a) {
        const double sa = a == 0 ? 1.0 : -1.0;
        const double zz = JD * sa * sb;
        const double flip = (a != b) ? R : 0.0;
        bu = std::max(bu, up[a] + zz + flip);
        bd = std::min(bd, dn[a] + zz - flip);
      }
      nu[b] = bu + h[i] * sb;
      nd[b] = bd + h[i] * sb;
    }
    up[0] = nu[0];
    up[1] = nu[1];
    dn[0] = nd[0];
    dn[1] = nd[1];
  }
  *hi = std::max(up[0], up[1]);
  *lo = std::min(dn[0], dn[1]);
}

void xfield_interval(int N, const double* a, double* lo, double* hi) {
  double s = 0.0;
  for (int i = 0; i < N; ++i) s += std::fabs(a[i]);
  *lo = -s;
  *hi = s;
}

void dia_interval(const int64_t* offsets, const double* values, int ndiag, int dim, double* lo, double* hi) {
  std::vector<double> diag((size_t)dim, 0.0), R((size_t)dim, 0.0);
  for (int d = 0; d < ndiag; ++d)
    for (int r = 0; r < dim; ++r) {
      const int64_t c = (int64_t)r + offsets[d];
      const double v = values[(size_t)d * dim + r];
      if (offsets[d] == 0) diag[r] += v;
      else if (c >= 0 && c < dim) R[r] += std::fabs(v);
    }
  double l = INFINITY, u = -INFINITY;
  for (int r = 0; r < dim; ++r) {
    l = std::min(l, diag[r] - R[r]);
    u = std::max(u, diag[r] + R[r]);
  }
  *lo = l;
  *hi = u;
}

void csr_interval(const int64_t* row_ptr, const int32_t* col, const double* re, const double* im, int dim,
                  double* lo, double* hi) {
  double l = INFINITY, u = -INFINITY;
  for (int r = 0; r < dim; ++r) {
    double d = 0.0, R = 0.0;
    for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
      if (col[e] == r) d += re[e];
      else R += std::hypot(re[e], im ? im[e] : 0.0);
    }
    l = std::min(l, d - R);
    u = std::max(u, d + R);
  }
  if (dim < 1 || !(l <= u)) l = u = 0.0;
  *lo = l;
  *hi = u;
}

void stage_interval(int nops, const double* op_lo, const double* op_hi, const double* s, double* lo, double* hi) {
  double l = 0.0, u = 0.0;
  for (int o = 0; o < nops; ++o) {
    if (s[o] >= 0.0) {
      l += s[o] * op_lo[o];
      u += s[o] * op_hi[o];
    } else {
      l += s[o] * op_hi[o];
      u += s[o] * op_lo[o];
    }
  }
  *lo = l;
  *hi = u;
}

}  // namespace cfet

extern "C" cfet_status cfet_chebyshev_coefficients(double z, double tol, int32_t cap, double* r, int32_t* K,
                                                   double* tail) {
  if (!std::isfinite(z) || !std::isfinite(tol) || std::fabs(z) > 1e8) return CFET_EINVAL;
  std::vector<double> rv;
  double t = 0.0;
  const int k = cfet::cheb_series(z, tol, r ? &rv : nullptr, &t);
  if (K) *K = k;
  if (tail) *tail = t;
  if (r) {
    if (cap < k + 1) return CFET_EINVAL;
    std::copy(rv.begin(), rv.end(), r);
  }
  return CFET_OK;
}
