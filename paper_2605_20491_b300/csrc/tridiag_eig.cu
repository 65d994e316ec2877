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

// The QR iteration above on the whole matrix.
bool tridiag_qr(int n, const double* diag, const double* offdiag, double* lam, double* Zout) {
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

// A persymmetric matrix (a_i = a_{n-1-i}, b_i = b_{n-2-i}: a potential symmetric about the
// middle of a uniform grid, as x^2 on [-L, L]) commutes with the exchange J, so its
// eigenvectors are even or odd under J and it splits into two tridiagonal problems of half
// the size; the accumulated rotations, O(n^3), then cost a quarter.  With m = n / 2 and the
// entries of the first half:
//   n = 2m:     even: a_{m-1} + b_{m-1} in the last diagonal entry, v = [u; J u] / sqrt 2;
//               odd:  a_{m-1} - b_{m-1},                             v = [u; -J u] / sqrt 2;
//   n = 2m + 1: even: size m + 1 with the middle entry a_m coupled by sqrt 2 b_{m-1}
//               (unknown y_m = v_m / sqrt 2), v = [y_0 .. y_{m-1}, sqrt 2 y_m, mirror] / sqrt 2;
//               odd:  size m (v_m = 0), v = [u; 0; -J u] / sqrt 2.
// Node grids computed in floating point are symmetric only to rounding, so the test allows
// 16 ulp of the matrix's scale and the halves are formed from the mirrored pairs' means:
// the decomposition is that of a matrix within that distance of the input, the order of
// the QR iteration's own backward error.  Even and odd vectors are orthogonal exactly.
bool split_persymmetric(int n, const double* a, const double* b, double* lam, double* Zout) {
  double amax = 0.0, bmax = 0.0;
  for (int i = 0; i < n; ++i) amax = std::fmax(amax, std::fabs(a[i]));
  for (int i = 0; i + 1 < n; ++i) bmax = std::fmax(bmax, std::fabs(b[i]));
  const double tol = 16.0 * std::ldexp(1.0, -52) * (amax + 2.0 * bmax);
  for (int i = 0; i < n / 2; ++i)
    if (std::fabs(a[i] - a[n - 1 - i]) > tol) return false;
  for (int i = 0; i + 1 < n - 1 - i; ++i)
    if (std::fabs(b[i] - b[n - 2 - i]) > tol) return false;
  const int m = n / 2;
  const bool odd_n = n & 1;
  const int ne = odd_n ? m + 1 : m, no = m;
  std::vector<double> ea(ne), eb(ne), oa(no), ob(no > 1 ? no : 1);
  for (int i = 0; i < m; ++i) ea[i] = oa[i] = 0.5 * (a[i] + a[n - 1 - i]);
  for (int i = 0; i + 1 < m; ++i) eb[i] = ob[i] = 0.5 * (b[i] + b[n - 2 - i]);
  const double sq2 = std::sqrt(2.0), is2 = 1.0 / sq2;
  if (odd_n) {
    ea[m] = a[m];
    eb[m - 1] = sq2 * 0.5 * (b[m - 1] + b[m]);
  } else {
    ea[m - 1] += b[m - 1];
    oa[m - 1] -= b[m - 1];
  }
  std::vector<double> el(ne), ol(no), EZ((size_t)ne * ne), OZ((size_t)no * no);
  if (!tridiag_qr(ne, ea.data(), eb.data(), el.data(), EZ.data())) return false;
  if (!tridiag_qr(no, oa.data(), ob.data(), ol.data(), OZ.data())) return false;
  // merge the two ascending spectra; column j of Zout is the eigenvector of lam[j]
  int ie = 0, io = 0;
  for (int j = 0; j < n; ++j) {
    double* z = Zout + (size_t)j * n;
    if (io >= no || (ie < ne && el[ie] <= ol[io])) {
      const double* u = EZ.data() + (size_t)ie * ne;
      for (int i = 0; i < m; ++i) z[i] = z[n - 1 - i] = u[i] * is2;
      if (odd_n) z[m] = u[m];  // sqrt 2 y_m / sqrt 2
      lam[j] = el[ie++];
    } else {
      const double* u = OZ.data() + (size_t)io * no;
      for (int i = 0; i < m; ++i) {
        z[i] = u[i] * is2;
        z[n - 1 - i] = -u[i] * is2;
      }
      if (odd_n) z[m] = 0.0;
      lam[j] = ol[io++];
    }
  }
  return true;
}

}  // namespace

bool tridiag_eig_host(int n, const double* diag, const double* offdiag, double* lam, double* Zout) {
  if (n >= 16 && split_persymmetric(n, diag, offdiag, lam, Zout)) return true;
  return tridiag_qr(n, diag, offdiag, lam, Zout);
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
