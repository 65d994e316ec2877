// One axis of the Q^k spectral element discretisation (Sec. 2, eqs. general_system and
// eigen_decomp): Gauss-Lobatto-Legendre (GLL) nodes and weights, the element stiffness,
// and the assembled interior stiffness and lumped mass.  Host code, run at plan creation.
//
// [-L, L] is cut into c = (n + 1) / k elements of width h_e = 2L / c carrying the k + 1
// GLL points of degree k; neighbours share their end points, and the n = c k - 1
// interior nodes carry the unknowns (homogeneous Dirichlet).  Every integral uses the
// (k + 1)-point GLL rule, so the mass matrix is diagonal and the stiffness is
//     Stiff_ij = sum_e (2 / h_e) sum_q w_q l_i'(xi_q) l_j'(xi_q).
// For k = 1 this is h^-1 tridiag(-1, 2, -1) with M = h I.
#include <cmath>
#include <vector>

#include "sem_axis.cuh"

namespace ts {
namespace {

// P_k(x) and P_{k-1}(x) by the three-term recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}.
void legendre_pair(int k, double x, double* pk, double* pkm1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (k == 0) {
    *pk = 1.0;
    *pkm1 = 0.0;
    return;
  }
  for (int j = 1; j < k; ++j) {
    const double c = ((2.0 * j + 1.0) * x * b - j * a) / (j + 1.0);
    a = b;
    b = c;
  }
  *pk = b;
  *pkm1 = a;
}

}  // namespace

// GLL points of degree k, ascending, and their weights.  The interior points are the roots
// of P_k'; since (1 - x^2) P_k' = k (P_{k-1} - x P_k) and, by Legendre's equation,
// d/dx [(1 - x^2) P_k'] = -k (k+1) P_k, they are the roots of r = P_{k-1} - x P_k with
// r' = -(k+1) P_k, found by Newton's method from the Chebyshev-Gauss-Lobatto points
// cos(pi j / k).  Weights w_j = 2 / (k (k+1) P_k(xi_j)^2).
void gll_rule(int k, std::vector<double>* xi, std::vector<double>* w) {
  xi->assign(k + 1, 0.0);
  w->assign(k + 1, 0.0);
  for (int j = 0; j <= k; ++j) {
    double x = -std::cos(M_PI * j / k);
    if (j > 0 && j < k) {
      for (int it = 0; it < 100; ++it) {
        double pk, pkm1;
        legendre_pair(k, x, &pk, &pkm1);
        const double dx = (pkm1 - x * pk) / ((k + 1.0) * pk);
        x += dx;
        if (std::fabs(dx) < 1e-16) break;
      }
    }
    (*xi)[j] = x;
  }
  (*xi)[0] = -1.0;
  (*xi)[k] = 1.0;
  if (k % 2 == 0) (*xi)[k / 2] = 0.0;
  for (int j = 0; j <= k; ++j)  // symmetric about 0
    if (j < k - j) {
      const double s = 0.5 * ((*xi)[k - j] - (*xi)[j]);
      (*xi)[j] = -s;
      (*xi)[k - j] = s;
    }
  for (int j = 0; j <= k; ++j) {
    double pk, pkm1;
    legendre_pair(k, (*xi)[j], &pk, &pkm1);
    (*w)[j] = 2.0 / (k * (k + 1.0) * pk * pk);
  }
}

// D[q][j] = l_j'(xi_q) in barycentric form (Berrut & Trefethen, SIAM Review 46, 2004):
// with beta_j = 1 / prod_{m != j} (xi_j - xi_m),  D[q][j] = (beta_j / beta_q) / (xi_q - xi_j)
// for q != j, and the diagonal makes every row sum to zero (the derivative of a constant).
void gll_diff_matrix(const std::vector<double>& xi, std::vector<double>* D) {
  const int m = (int)xi.size();
  std::vector<double> beta(m, 1.0);
  for (int j = 0; j < m; ++j)
    for (int q = 0; q < m; ++q)
      if (q != j) beta[j] /= (xi[j] - xi[q]);
  D->assign((size_t)m * m, 0.0);
  for (int q = 0; q < m; ++q) {
    double diag = 0.0;
    for (int j = 0; j < m; ++j) {
      if (j == q) continue;
      const double v = (beta[j] / beta[q]) / (xi[q] - xi[j]);
      (*D)[(size_t)q * m + j] = v;
      diag -= v;
    }
    (*D)[(size_t)q * m + q] = diag;
  }
}

ts_status sem_axis_build(int n, double L, int k, SemAxis* out) {
  if (k < 1 || (n + 1) % k != 0) {
    set_error("Q^%d needs n + 1 to be a multiple of %d (n = %d)", k, k, n);
    return TS_ERR_INVALID_ARG;
  }
  const int c = (n + 1) / k;
  const double he = 2.0 * L / c;
  std::vector<double> xi, w, D;
  gll_rule(k, &xi, &w);
  gll_diff_matrix(xi, &D);
  const int m = k + 1;
  // element stiffness Se = (2 / h_e) D^T diag(w) D, symmetric by construction
  std::vector<double> Se((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = i; j < m; ++j) {
      double s = 0.0;
      for (int q = 0; q < m; ++q) s += w[q] * D[(size_t)q * m + i] * D[(size_t)q * m + j];
      Se[(size_t)i * m + j] = Se[(size_t)j * m + i] = 2.0 / he * s;
    }
  const int G = c * k + 1;  // all nodes, boundary included
  std::vector<double> Sg((size_t)G * G, 0.0), mg(G, 0.0), xg(G, 0.0);
  for (int e = 0; e < c; ++e)
    for (int a = 0; a < m; ++a) {
      const int ga = e * k + a;
      mg[ga] += 0.5 * he * w[a];
      xg[ga] = -L + e * he + 0.5 * (xi[a] + 1.0) * he;
      for (int b = 0; b < m; ++b) Sg[(size_t)ga * G + e * k + b] += Se[(size_t)a * m + b];
    }
  out->n = n;
  out->k = k;
  out->x.assign(xg.begin() + 1, xg.end() - 1);
  out->m.assign(mg.begin() + 1, mg.end() - 1);
  out->stiff.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out->stiff[(size_t)i * n + j] = Sg[(size_t)(i + 1) * G + (j + 1)];
  return TS_OK;
}

// ---------------------------------------------------------------- Hermite functions ------

// Eigenvalues of the symmetric tridiagonal Jacobi matrix of the Hermite functions
// (J_kk = 0, J_{k,k+1} = sqrt(k/2)): the Gauss-Hermite nodes (Golub-Welsch), found by
// bisection on the Sturm-sequence count (Golub & Van Loan, Matrix Computations, Sec. 8.4):
// the number of eigenvalues below t is the number of negative terms of
// q_1 = -t, q_k = -t - b_{k-1}^2 / q_{k-1}.
void hermite_nodes(int n, double* x) {
  auto count_below = [n](double t) {
    int c = 0;
    double q = 1.0;
    for (int k = 0; k < n; ++k) {
      const double b2 = k == 0 ? 0.0 : 0.5 * k;  // b_k^2 = k / 2
      q = -t - (k == 0 ? 0.0 : b2 / q);
      if (q == 0.0) q = -1e-300;
      c += q < 0.0;
    }
    return c;
  };
  const double R = std::sqrt(2.0 * n + 1.0) + 1.0;  // Gershgorin-type bound on |x|
  for (int j = 0; j < n; ++j) {
    double lo = -R, hi = R;  // count_below(lo) <= j < count_below(hi)
    for (int it = 0; it < 200 && hi - lo > 4e-16 * (std::fabs(lo) + std::fabs(hi)) + 1e-300; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (count_below(mid) > j)
        hi = mid;
      else
        lo = mid;
    }
    x[j] = 0.5 * (lo + hi);
  }
}

ts_status hermite_axis_build(int n, HermiteAxis* out) {
  if (n < 1 || n > HERMITE_MAX_N) {
    set_error("Hermite axis: n = %d out of range [1, %d]", n, HERMITE_MAX_N);
    return TS_ERR_INVALID_ARG;
  }
  out->n = n;
  out->x.resize(n);
  hermite_nodes(n, out->x.data());
  // log |psi_{n-1}(x_j)| and its sign: psi_m = p_m e^{-x^2/2} with the normalised recurrence
  // p_0 = pi^{-1/4}, p_1 = sqrt(2) x p_0, p_{m+1} = sqrt(2/(m+1)) x p_m - sqrt(m/(m+1)) p_{m-1},
  // rescaled whenever |p| exceeds 1e100, so that neither p nor e^{-x^2/2} (which underflows
  // for |x| > ~38, i.e. from n ~ 745 in the plain recurrence) leaves the FP64 range.
  std::vector<double> sg(n);
  out->log_w.resize(n);
  for (int j = 0; j < n; ++j) {
    const double xj = out->x[j];
    double p0 = std::pow(M_PI, -0.25), p1 = std::sqrt(2.0) * xj * p0, lg = 0.0;
    if (n == 1) p1 = p0;
    for (int m = 1; m < n - 1; ++m) {
      const double p2 = std::sqrt(2.0 / (m + 1)) * xj * p1 - std::sqrt(m / (m + 1.0)) * p0;
      p0 = p1;
      p1 = p2;
      if (std::fabs(p1) > 1e100) {
        p0 *= 1e-100;
        p1 *= 1e-100;
        lg += 100.0 * std::log(10.0);
      }
    }
    const double log_psi = std::log(std::fabs(p1)) + lg - 0.5 * xj * xj;
    sg[j] = p1 < 0.0 ? -1.0 : 1.0;
    out->log_w[j] = -std::log((double)n) - 2.0 * log_psi;  // W_j = 1 / (n psi_{n-1}(x_j)^2)
  }
  // the skew B_ij = s_i s_j / (x_i - x_j) with W^{1/2} D W^{-1/2} = B, and -B^2
  std::vector<double> B((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (i != j) B[(size_t)i * n + j] = sg[i] * sg[j] / (out->x[i] - out->x[j]);
  out->hs0.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      double acc = 0.0;
      for (int q = 0; q < n; ++q) acc -= B[(size_t)i * n + q] * B[(size_t)q * n + j];
      out->hs0[(size_t)i * n + j] = out->hs0[(size_t)j * n + i] = acc;
    }
  return TS_OK;
}

ts_status grid_nodes_host(int n, double L, int order, double* x, double* m) {
  if (order == ORDER_HERMITE) {
    if (n < 1 || n > HERMITE_MAX_N) {
      set_error("Hermite axis: n = %d out of range [1, %d]", n, HERMITE_MAX_N);
      return TS_ERR_INVALID_ARG;
    }
    hermite_nodes(n, x);
    if (m) {
      HermiteAxis ax;
      TS_TRY(hermite_axis_build(n, &ax));
      for (int i = 0; i < n; ++i) m[i] = std::exp(ax.log_w[i]);
    }
    return TS_OK;
  }
  if (order < 2) {
    const double h = 2.0 * L / (n + 1);
    for (int i = 0; i < n; ++i) {
      x[i] = -L + (i + 1) * h;
      if (m) m[i] = h;
    }
    return TS_OK;
  }
  const int k = order;
  if ((n + 1) % k != 0) {
    set_error("Q^%d needs n + 1 to be a multiple of %d (n = %d)", k, k, n);
    return TS_ERR_INVALID_ARG;
  }
  const int c = (n + 1) / k;
  const double he = 2.0 * L / c;
  std::vector<double> xi, w;
  gll_rule(k, &xi, &w);
  // interior node i is global node g = i + 1 = e k + a (a = 0 only for shared element ends)
  for (int i = 0; i < n; ++i) {
    const int g = i + 1, e = g / k, a = g % k;
    x[i] = -L + e * he + 0.5 * (xi[a] + 1.0) * he;
    if (m) m[i] = a == 0 ? 0.5 * he * (w[0] + w[k]) : 0.5 * he * w[a];
  }
  return TS_OK;
}

}  // namespace ts
