// Host eigendecomposition of a symmetric tridiagonal matrix (step 1 of Sec. 2.1 for the
// Q^1 operator H = h^-2 tridiag(-1, 2, -1) + diag f, which is tridiagonal already).
//
// Implicit symmetric QR steps with the Wilkinson shift on the unreduced trailing block,
// deflating off-diagonals below u (|a_i| + |a_{i+1}|) (Golub & Van Loan, Matrix
// Computations, Sec. 8.3); every Givens rotation is accumulated into the eigenvector
// matrix, so the columns are orthonormal to rounding.  At the axis lengths of a serving
// mix (n <= a few hundred) this costs well under a millisecond per axis on one host core,
// where a dense device eigensolver call costs several milliseconds and waits for all work
// on the device; plan builders on several host threads then run side by side with the
// GPU work of earlier requests.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace ts {

namespace {

// Z <- Z G^T on columns (k, k + 1): the inner loop of every rotation, where the time goes.
// Two builds of the same loop, chosen once at run time: 4-wide AVX2 where the host has it
// and 2-wide SSE2 otherwise.  Neither contracts to FMA, so both round alike.
using RotateFn = void (*)(int, double, double, double*, double*);

__attribute__((target("avx2"))) void rotate_avx2(int n, double c, double s, double* __restrict__ zk,
                                                 double* __restrict__ zk1) {
  for (int i = 0; i < n; ++i) {
    const double u = zk[i], v = zk1[i];
    zk[i] = c * u + s * v;
    zk1[i] = c * v - s * u;
  }
}

void rotate_plain(int n, double c, double s, double* __restrict__ zk, double* __restrict__ zk1) {
  for (int i = 0; i < n; ++i) {
    const double u = zk[i], v = zk1[i];
    zk[i] = c * u + s * v;
    zk1[i] = c * v - s * u;
  }
}

RotateFn pick_rotate() { return __builtin_cpu_supports("avx2") ? rotate_avx2 : rotate_plain; }

// One implicit QR step on the unreduced block [lo, hi] (b[lo..hi-1] nonzero).  The first
// rotation G acts on (lo, lo + 1) with (c, s) proportional to (a_lo - mu, b_lo); each later
// one on (k, k + 1) chases the bulge T[k+1][k-1] out of the band.  With
// G = [[c, s], [-s, c]] on rows/columns (k, k + 1) and T <- G T G^T:
//   a_k'     = c^2 p + 2 c s r + s^2 q,     a_{k+1}' = s^2 p - 2 c s r + c^2 q,
//   b_k'     = c s (q - p) + (c^2 - s^2) r, b_{k+1}' = c f, new bulge T[k+2][k] = s f,
// with p = a_k, q = a_{k+1}, r = b_k, f = b_{k+1}; Z <- Z G^T mixes columns k and k + 1.
void qr_step(int n, int lo, int hi, double* a, double* b, double* Z, RotateFn rotate) {
  const double d = 0.5 * (a[hi - 1] - a[hi]);
  const double e = b[hi - 1];
  const double den = d + std::copysign(std::hypot(d, e), d);
  const double mu = den != 0.0 ? a[hi] - e * e / den : a[hi] - std::fabs(e);
  double x = a[lo] - mu, z = b[lo];
  for (int k = lo; k < hi; ++k) {
    // |(x, z)|: the plain square root where x^2 + z^2 can neither overflow nor underflow
    // (hypot's rescaling costs more than the rest of the step), hypot outside that range
    const double m = std::fmax(std::fabs(x), std::fabs(z));
    const double rho = (m > 1e-150 && m < 1e150) ? std::sqrt(x * x + z * z) : std::hypot(x, z);
    double c = 1.0, s = 0.0;
    if (rho != 0.0) {
      const double inv = 1.0 / rho;
      c = x * inv;
      s = z * inv;
    }
    if (k > lo) b[k - 1] = rho;
    const double p = a[k], q = a[k + 1], r = b[k];
    const double cs = c * s, cc = c * c, ss = s * s;
    a[k] = cc * p + 2.0 * cs * r + ss * q;
    a[k + 1] = ss * p - 2.0 * cs * r + cc * q;
    b[k] = cs * (q - p) + (cc - ss) * r;
    if (k + 1 < hi) {
      const double f = b[k + 1];
      x = b[k];
      z = s * f;
      b[k + 1] = c * f;
    }
    rotate(n, c, s, Z + (size_t)k * n, Z + (size_t)(k + 1) * n);
  }
}

}  // namespace

bool tridiag_eig_host(int n, const double* diag, const double* offdiag, double* lam, double* Zout) {
  if (n <= 0) return true;
  static const RotateFn rotate = pick_rotate();
  std::vector<double> a(diag, diag + n), b(n > 1 ? n - 1 : 1, 0.0);
  for (int i = 0; i + 1 < n; ++i) b[i] = offdiag[i];
  std::vector<double> Z((size_t)n * n, 0.0);  // column-major
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  const double u = 0.5 * std::ldexp(1.0, -52);
  const long long max_steps = 30LL * n + 30;
  long long steps = 0;
  int hi = n - 1;
  while (hi > 0) {
    // deflate negligible couplings, then find the unreduced block ending at hi
    for (int i = 0; i < hi; ++i)
      if (std::fabs(b[i]) <= u * (std::fabs(a[i]) + std::fabs(a[i + 1]))) b[i] = 0.0;
    while (hi > 0 && b[hi - 1] == 0.0) --hi;
    if (hi == 0) break;
    int lo = hi - 1;
    while (lo > 0 && b[lo - 1] != 0.0) --lo;
    if (++steps > max_steps) return false;
    qr_step(n, lo, hi, a.data(), b.data(), Z.data(), rotate);
  }
  // ascending order, columns permuted alike
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return a[x] < a[y]; });
  for (int j = 0; j < n; ++j) {
    lam[j] = a[perm[j]];
    std::copy(Z.begin() + (size_t)perm[j] * n, Z.begin() + (size_t)perm[j] * n + n, Zout + (size_t)j * n);
  }
  return true;
}

}  // namespace ts

extern "C" ts_status ts_tridiag_eig(int n, const double* diag, const double* offdiag, double* lambda_host,
                                    double* Z_host) {
  ts::clear_error();
  if (n < 1 || !diag || (n > 1 && !offdiag) || !lambda_host || !Z_host) {
    ts::set_error("ts_tridiag_eig: n >= 1 and non-NULL arrays required");
    return TS_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(diag[i]) || (i + 1 < n && !std::isfinite(offdiag[i]))) {
      ts::set_error("ts_tridiag_eig: non-finite entry at %d", i);
      return TS_ERR_INVALID_ARG;
    }
  if (!ts::tridiag_eig_host(n, diag, offdiag, lambda_host, Z_host)) {
    ts::set_error("ts_tridiag_eig: no convergence within 30 n QR steps");
    return TS_ERR_NOT_CONVERGED;
  }
  return TS_OK;
}
