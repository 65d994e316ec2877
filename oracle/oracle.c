/*
 * oracle.c -- plain, slow, FP64 CPU reference of the tensor-product solver for
 * the Schroedinger operator -Delta + V1 (+ V2) on [-L_1,L_1] x ... x [-L_d,L_d]
 * with homogeneous Dirichlet conditions, Q^1 spectral elements (= second-order
 * central differences).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle of the library:
 * only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or helper with the CUDA library
 * and never calls it.  Every loop below is the plain definition of what the paper
 * computes; there is no blocking, fusion or reordering beyond it.
 *
 * Array convention (Sec. 2.1, eq. general_system): a d-dimensional grid function X of size
 * n_1 x ... x n_d is stored as vec(X), axis 1 fastest:
 *     linear index = i_1 + n_1*(i_2 + n_2*(i_3 + ...)),  0 <= i_k < n_k.
 * Complex arrays are interleaved (re, im) pairs of doubles.
 *
 * Functions and the passage each one follows:
 *   or_grid            -- grid nodes x_{k,i} = -L_k + i h_k, h_k = 2L_k/(n_k+1)   (Sec. 2.1)
 *   or_operator_1d     -- H_k = K_k + F_k, K_k = h^-2 tridiag(-1,2,-1) (Q^1, lumped
 *                         mass M = hI, Stiff = h^-1 tridiag), F_k = diag f_k(x_i)
 *                         (Sec. 2.1, eqs. general_system, tensor_system, eigen_decomp)
 *   or_jacobi_eigh     -- cyclic-by-row Jacobi eigensolver (Golub & Van Loan,
 *                         Matrix Computations, Sec. 8.5) for step 1 of Sec. 2.1
 *   or_mode_forward    -- coefficient_j = sum_i S[i][j] x_i along one axis (step 2)
 *   or_mode_backward   -- x_i = sum_j S[i][j] c_j along one axis             (step 4)
 *   or_apply_inverse   -- 4-step direct solve of (-Delta+V1+sigma) u = b     (Sec. 2.1, steps 1-4)
 *   or_apply_exp       -- exact propagator T (e^{-i Lambda tau} . T^{-1} psi) (Sec. 2.1; eq. exact_prop)
 *   or_dense_operator  -- the Kronecker-sum matrix of eq. general_system written out entry by entry
 *   or_lu_solve        -- LU with partial pivoting (textbook), for the dense check
 *   or_dense_exp       -- e^{-i tau H} psi from a Jacobi eigendecomposition of dense H
 *   or_stencil         -- (-Delta_h + V1 + V2 + sigma) x by the 2d+1 point stencil (eq. general_system)
 *   or_pcg             -- preconditioned CG with P = (-Delta+V1+sigma_P)^{-1}      (Sec. 3.2)
 *   or_inverse_iteration -- shifted inverse iteration, PCG inner solves        (Sec. 4.1, 5.3.1)
 *   or_strang          -- e^{-iV2 dt/2} e^{-iA dt} e^{-iV2 dt/2}, A = -Delta+V1  (Sec. 5.1, Remark cost_naive_merged)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 12

/* ------------------------------------------------------------------ grid --- */

/* x[i-1] = -L + i*h, i = 1..n, h = 2L/(n+1): the n interior nodes of n+1 cells. */
void or_grid(int n, double L, double* x) {
  double h = 2.0 * L / (n + 1);
  for (int i = 1; i <= n; ++i) x[i - 1] = -L + i * h;
}

/* ------------------------------------------------------- 1D operator ------ */

/* H = h^-2 tridiag(-1, 2, -1) + diag(f), dense, row-major n x n. */
void or_operator_1d(int n, double L, const double* f, double* H) {
  double h = 2.0 * L / (n + 1);
  double ih2 = 1.0 / (h * h);
  for (int i = 0; i < n * n; ++i) H[i] = 0.0;
  for (int i = 0; i < n; ++i) {
    H[i * n + i] = 2.0 * ih2 + f[i];
    if (i > 0) H[i * n + i - 1] = -ih2;
    if (i + 1 < n) H[i * n + i + 1] = -ih2;
  }
}

/* ------------------------------------------------ Jacobi eigensolver ------ */

/*
 * Cyclic-by-row Jacobi for a symmetric matrix A (row-major n x n, not modified).
 * On return lam[0..n-1] holds the eigenvalues in ascending order and Q (row-major)
 * holds the matching orthonormal eigenvectors as columns: A = Q diag(lam) Q^T.
 * A rotation is skipped when |a_pq| <= 1e-15 * ||A||_F (scaled below the rounding
 * level); sweeps stop when a sweep performs no rotation.  Returns the number of
 * sweeps, or -1 if 100 sweeps did not converge.
 */
int or_jacobi_eigh(int n, const double* Ain, double* lam, double* Q) {
  double* A = (double*)malloc(sizeof(double) * n * n);
  memcpy(A, Ain, sizeof(double) * n * n);
  for (int i = 0; i < n * n; ++i) Q[i] = 0.0;
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  double fro = 0.0;
  for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
  fro = sqrt(fro);
  double thresh = 1e-15 * fro;
  int sweep;
  for (sweep = 1; sweep <= 100; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (fabs(apq) <= thresh) continue;
        rotated = 1;
        /* Symmetric Schur decomposition of the 2x2 block (GVL Alg. 8.5.1). */
        double app = A[p * n + p], aqq = A[q * n + q];
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        /* A <- J^T A J with J = rotation in the (p,q) plane. */
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        A[p * n + q] = 0.0;
        A[q * n + p] = 0.0;
        /* Q <- Q J */
        for (int k = 0; k < n; ++k) {
          double qkp = Q[k * n + p], qkq = Q[k * n + q];
          Q[k * n + p] = c * qkp - s * qkq;
          Q[k * n + q] = s * qkp + c * qkq;
        }
      }
    }
    if (!rotated) break;
  }
  /* Sort ascending (selection sort on the diagonal; columns of Q follow). */
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
  for (int i = 0; i < n; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (lam[j] < lam[m]) m = j;
    if (m != i) {
      double tl = lam[i]; lam[i] = lam[m]; lam[m] = tl;
      for (int k = 0; k < n; ++k) {
        double tq = Q[k * n + i]; Q[k * n + i] = Q[k * n + m]; Q[k * n + m] = tq;
      }
    }
  }
  free(A);
  return sweep > 100 ? -1 : sweep;
}

/* --------------------------------------------------- mode products ------- */

static long or_total(int d, const int* n) {
  long N = 1;
  for (int k = 0; k < d; ++k) N *= n[k];
  return N;
}

/*
 * Forward transform along axis k (step 2 of Sec. 2.1 for one axis):
 *     Y[.., j, ..] = sum_i S[i][j] X[.., i, ..]     (S^T applied to every axis-k fiber)
 * S is row-major n_k x n_k.  ncomp = 1 (real) or 2 (complex interleaved; S is real,
 * so the real and imaginary parts transform independently).  X and Y must differ.
 */
void or_mode_forward(int d, const int* n, int k, const double* S, int ncomp,
                     const double* X, double* Y) {
  long lo = 1, hi = 1;
  for (int j = 0; j < k; ++j) lo *= n[j];
  for (int j = k + 1; j < d; ++j) hi *= n[j];
  int nk = n[k];
#pragma omp parallel for collapse(2) schedule(static)
  for (long h = 0; h < hi; ++h)
    for (long l = 0; l < lo; ++l)
      for (int c = 0; c < ncomp; ++c)
        for (int j = 0; j < nk; ++j) {
          double acc = 0.0;
          for (int i = 0; i < nk; ++i)
            acc += S[(long)i * nk + j] * X[(l + lo * (i + (long)nk * h)) * ncomp + c];
          Y[(l + lo * (j + (long)nk * h)) * ncomp + c] = acc;
        }
}

/* Backward transform along axis k (step 4):  Y[.., i, ..] = sum_j S[i][j] X[.., j, ..]. */
void or_mode_backward(int d, const int* n, int k, const double* S, int ncomp,
                      const double* X, double* Y) {
  long lo = 1, hi = 1;
  for (int j = 0; j < k; ++j) lo *= n[j];
  for (int j = k + 1; j < d; ++j) hi *= n[j];
  int nk = n[k];
#pragma omp parallel for collapse(2) schedule(static)
  for (long h = 0; h < hi; ++h)
    for (long l = 0; l < lo; ++l)
      for (int c = 0; c < ncomp; ++c)
        for (int i = 0; i < nk; ++i) {
          double acc = 0.0;
          for (int j = 0; j < nk; ++j)
            acc += S[(long)i * nk + j] * X[(l + lo * (j + (long)nk * h)) * ncomp + c];
          Y[(l + lo * (i + (long)nk * h)) * ncomp + c] = acc;
        }
}

/*
 * Timing sample of the two transforms above (real data): the same loops restricted to the
 * axis-k fibers with flat index f = l + lo * h in [f0, f1) (0 <= f0 <= f1 <= lo * hi);
 * backward = 0 gives or_mode_forward's sum over S[i][j] x_i, 1 gives or_mode_backward's
 * sum over S[i][j] x_j.  Outputs of other fibers are left as they are.  Used to time the
 * oracle on a bounded part of a grid too large to transform whole within a time budget.
 */
void or_mode_fibers(int d, const int* n, int k, const double* S, int backward, const double* X,
                    double* Y, long f0, long f1) {
  long lo = 1;
  for (int j = 0; j < k; ++j) lo *= n[j];
  int nk = n[k];
#pragma omp parallel for schedule(static)
  for (long f = f0; f < f1; ++f) {
    const long l = f % lo, h = f / lo;
    for (int o = 0; o < nk; ++o) {
      double acc = 0.0;
      for (int i = 0; i < nk; ++i) {
        const double s = backward ? S[(long)o * nk + i] : S[(long)i * nk + o];
        acc += s * X[l + lo * (i + (long)nk * h)];
      }
      Y[l + lo * (o + (long)nk * h)] = acc;
    }
  }
}

/* Sum of the per-axis eigenvalues at the multi-index of linear index idx. */
static double or_lambda_sum(int d, const int* n, const double* const* lam, long idx) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    s += lam[k][idx % n[k]];
    idx /= n[k];
  }
  return s;
}

/* ------------------------------------------------------ direct apply ------ */

/*
 * u = (-Delta_h + V1 + sigma)^{-1} b by steps 2-4 of Sec. 2.1, given the per-axis
 * eigendecompositions H_k = S_k diag(lam_k) S_k^T (step 1).  Q^1 has lumped mass
 * M = hI, so T_k = S_k is orthogonal and T_k^{-1} = S_k^T.  b and u may alias.
 */
void or_apply_inverse(int d, const int* n, const double* const* S, const double* const* lam,
                      double sigma, const double* b, double* u) {
  long N = or_total(d, n);
  double* t0 = (double*)malloc(sizeof(double) * N);
  double* t1 = (double*)malloc(sizeof(double) * N);
  memcpy(t0, b, sizeof(double) * N);
  for (int k = 0; k < d; ++k) {            /* step 2: T^{-1} b */
    or_mode_forward(d, n, k, S[k], 1, t0, t1);
    double* t = t0; t0 = t1; t1 = t;
  }
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx)       /* step 3: divide by sum of eigenvalues */
    t0[idx] = t0[idx] / (or_lambda_sum(d, n, lam, idx) + sigma);
  for (int k = 0; k < d; ++k) {            /* step 4: T (.) */
    or_mode_backward(d, n, k, S[k], 1, t0, t1);
    double* t = t0; t0 = t1; t1 = t;
  }
  memcpy(u, t0, sizeof(double) * N);
  free(t0);
  free(t1);
}

/*
 * psi_out = e^{-i tau (-Delta_h + V1)} psi_in  (exact propagator, eq. exact_prop):
 * forward transform, multiply coefficient idx by e^{-i tau Lambda_idx} with
 * Lambda_idx the sum of per-axis eigenvalues, backward transform.  Complex
 * interleaved; in and out may alias.
 */
void or_apply_exp(int d, const int* n, const double* const* S, const double* const* lam,
                  double tau, const double* psi_in, double* psi_out) {
  long N = or_total(d, n);
  double* t0 = (double*)malloc(sizeof(double) * 2 * N);
  double* t1 = (double*)malloc(sizeof(double) * 2 * N);
  memcpy(t0, psi_in, sizeof(double) * 2 * N);
  for (int k = 0; k < d; ++k) {
    or_mode_forward(d, n, k, S[k], 2, t0, t1);
    double* t = t0; t0 = t1; t1 = t;
  }
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx) {
    double th = tau * or_lambda_sum(d, n, lam, idx);
    double c = cos(th), s = sin(th);
    double re = t0[2 * idx], im = t0[2 * idx + 1];
    /* (re + i im)(cos th - i sin th) */
    t0[2 * idx] = re * c + im * s;
    t0[2 * idx + 1] = im * c - re * s;
  }
  for (int k = 0; k < d; ++k) {
    or_mode_backward(d, n, k, S[k], 2, t0, t1);
    double* t = t0; t0 = t1; t1 = t;
  }
  memcpy(psi_out, t0, sizeof(double) * 2 * N);
  free(t0);
  free(t1);
}

/* ---------------------------------------------------- dense checks ------- */

/*
 * Dense N x N matrix of eq. general_system for the separable part plus diag(V2) + sigma I:
 *   A = sum_k I x .. x H_k x .. x I + diag(V2) + sigma I,
 * written entry by entry: A[p][q] = sum_k H_k[p_k][q_k] prod_{j != k} delta(p_j, q_j)
 * (+ V2[p] + sigma if p == q).  H[k] are the dense 1D operators (row-major); V2 may be NULL.
 */
void or_dense_operator(int d, const int* n, const double* const* H, const double* V2,
                       double sigma, double* A) {
  long N = or_total(d, n);
  for (long p = 0; p < N; ++p)
    for (long q = 0; q < N; ++q) {
      int pi[OR_MAXD], qi[OR_MAXD];
      long pp = p, qq = q;
      for (int k = 0; k < d; ++k) {
        pi[k] = (int)(pp % n[k]); pp /= n[k];
        qi[k] = (int)(qq % n[k]); qq /= n[k];
      }
      double a = 0.0;
      for (int k = 0; k < d; ++k) {
        int others_equal = 1;
        for (int j = 0; j < d; ++j)
          if (j != k && pi[j] != qi[j]) others_equal = 0;
        if (others_equal) a += H[k][(long)pi[k] * n[k] + qi[k]];
      }
      if (p == q) a += sigma + (V2 ? V2[p] : 0.0);
      A[p * N + q] = a;
    }
}

/* Solve A x = b (A row-major N x N, not modified) by LU with partial pivoting.
 * Returns 0, or -1 on an exactly singular pivot. */
int or_lu_solve(long N, const double* Ain, const double* b, double* x) {
  double* A = (double*)malloc(sizeof(double) * N * N);
  memcpy(A, Ain, sizeof(double) * N * N);
  memcpy(x, b, sizeof(double) * N);
  for (long k = 0; k < N; ++k) {
    long piv = k;
    for (long i = k + 1; i < N; ++i)
      if (fabs(A[i * N + k]) > fabs(A[piv * N + k])) piv = i;
    if (A[piv * N + k] == 0.0) { free(A); return -1; }
    if (piv != k) {
      for (long j = 0; j < N; ++j) {
        double t = A[k * N + j]; A[k * N + j] = A[piv * N + j]; A[piv * N + j] = t;
      }
      double t = x[k]; x[k] = x[piv]; x[piv] = t;
    }
    for (long i = k + 1; i < N; ++i) {
      double m = A[i * N + k] / A[k * N + k];
      A[i * N + k] = m;
      for (long j = k + 1; j < N; ++j) A[i * N + j] -= m * A[k * N + j];
      x[i] -= m * x[k];
    }
  }
  for (long i = N - 1; i >= 0; --i) {
    double s = x[i];
    for (long j = i + 1; j < N; ++j) s -= A[i * N + j] * x[j];
    x[i] = s / A[i * N + i];
  }
  free(A);
  return 0;
}

/* psi_out = sum_j e^{-i tau mu_j} v_j (v_j^T psi_in) from the Jacobi eigendecomposition
 * H = V diag(mu) V^T of a dense symmetric H (row-major N x N).  Complex interleaved. */
int or_dense_exp(int N, const double* H, double tau, const double* psi_in, double* psi_out) {
  double* mu = (double*)malloc(sizeof(double) * N);
  double* V = (double*)malloc(sizeof(double) * (long)N * N);
  int sw = or_jacobi_eigh(N, H, mu, V);
  for (long i = 0; i < 2L * N; ++i) psi_out[i] = 0.0;
  for (int j = 0; j < N; ++j) {
    double cre = 0.0, cim = 0.0;
    for (int i = 0; i < N; ++i) {
      cre += V[(long)i * N + j] * psi_in[2 * i];
      cim += V[(long)i * N + j] * psi_in[2 * i + 1];
    }
    double c = cos(tau * mu[j]), s = sin(tau * mu[j]);
    double pre = cre * c + cim * s, pim = cim * c - cre * s;
    for (int i = 0; i < N; ++i) {
      psi_out[2 * i] += V[(long)i * N + j] * pre;
      psi_out[2 * i + 1] += V[(long)i * N + j] * pim;
    }
  }
  free(mu);
  free(V);
  return sw;
}

/* ------------------------------------------------------- stencil ---------- */

/*
 * y = (-Delta_h + V1 + V2 + sigma) x with the 2d+1 point stencil of eq. general_system:
 *   y_idx = sum_k h_k^-2 (2 x_idx - x_{idx-e_k} - x_{idx+e_k})
 *         + (sum_k f_k(x_{k,i_k}) + V2_idx + sigma) x_idx,
 * neighbours outside the grid are zero (homogeneous Dirichlet).  f[k] are the sampled
 * per-axis potentials; V2 may be NULL.
 */
void or_stencil(int d, const int* n, const double* L, const double* const* f, const double* V2,
                double sigma, const double* x, double* y) {
  long N = or_total(d, n);
  double ih2[OR_MAXD];
  long stride[OR_MAXD];
  long st = 1;
  for (int k = 0; k < d; ++k) {
    double h = 2.0 * L[k] / (n[k] + 1);
    ih2[k] = 1.0 / (h * h);
    stride[k] = st;
    st *= n[k];
  }
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < N; ++idx) {
    long r = idx;
    double acc = 0.0, v = sigma + (V2 ? V2[idx] : 0.0);
    for (int k = 0; k < d; ++k) {
      int i = (int)(r % n[k]);
      r /= n[k];
      double left = i > 0 ? x[idx - stride[k]] : 0.0;
      double right = i + 1 < n[k] ? x[idx + stride[k]] : 0.0;
      acc += ih2[k] * (2.0 * x[idx] - left - right);
      v += f[k][i];
    }
    y[idx] = acc + v * x[idx];
  }
}

static double or_dot(long N, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long i = 0; i < N; ++i) s += a[i] * b[i];
  return s;
}

/* ---------------------------------------------------------- PCG ----------- */

/*
 * Preconditioned conjugate gradient (Sec. 3.2) for
 *     (-Delta_h + V1 + V2 + sigma) x = b,
 * preconditioner P = (-Delta_h + V1 + sigma_P)^{-1} applied by or_apply_inverse with
 * the plan tables (S, lam).  x holds the initial guess on entry and the iterate on
 * exit.  Stops when the recurrence residual satisfies ||r||_2/||b||_2 < tol, or
 * after maxit iterations.  Returns the iteration count (negative when maxit was hit);
 * *relres_out receives the true relative residual ||b - A x||/||b|| at exit.
 */
int or_pcg(int d, const int* n, const double* L, const double* const* f,
           const double* const* S, const double* const* lam, const double* V2, double sigma,
           double sigma_P, const double* b, double* x, double tol, int maxit,
           double* relres_out) {
  long N = or_total(d, n);
  double* r = (double*)malloc(sizeof(double) * N);
  double* z = (double*)malloc(sizeof(double) * N);
  double* p = (double*)malloc(sizeof(double) * N);
  double* q = (double*)malloc(sizeof(double) * N);
  or_stencil(d, n, L, f, V2, sigma, x, q);
  for (long i = 0; i < N; ++i) r[i] = b[i] - q[i];
  double bnorm = sqrt(or_dot(N, b, b));
  if (bnorm == 0.0) bnorm = 1.0;
  int it = 0, converged = 0;
  if (sqrt(or_dot(N, r, r)) / bnorm < tol) converged = 1;
  double rz = 0.0;
  if (!converged) {
    or_apply_inverse(d, n, S, lam, sigma_P, r, z);
    memcpy(p, z, sizeof(double) * N);
    rz = or_dot(N, r, z);
  }
  while (!converged && it < maxit) {
    or_stencil(d, n, L, f, V2, sigma, p, q);
    double alpha = rz / or_dot(N, p, q);
    for (long i = 0; i < N; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    ++it;
    if (sqrt(or_dot(N, r, r)) / bnorm < tol) { converged = 1; break; }
    or_apply_inverse(d, n, S, lam, sigma_P, r, z);
    double rz_new = or_dot(N, r, z);
    double beta = rz_new / rz;
    rz = rz_new;
    for (long i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
  }
  or_stencil(d, n, L, f, V2, sigma, x, q);
  double rr = 0.0;
  for (long i = 0; i < N; ++i) rr += (b[i] - q[i]) * (b[i] - q[i]);
  if (relres_out) *relres_out = sqrt(rr) / bnorm;
  free(r); free(z); free(p); free(q);
  return converged ? it : -it - 1;
}

/* ------------------------------------------------ inverse iteration ------ */

/*
 * Shifted inverse iteration (Sec. 4.1, Sec. 5.3.1) for the smallest eigenpair of
 * H = -Delta_h + V1 + V2, shift s:
 *   u_0 = tensor product of the per-axis ground eigenvectors (column 0 of each S_k),
 *   lambda_0 = (u_0, H u_0);
 *   repeat: solve (H - s) w = u_k by PCG (P = (-Delta_h + V1 - s)^{-1}, tolerance
 *           pcg_tol, initial guess u_k / (lambda_k - s)); u_{k+1} = w/||w||;
 *           lambda_{k+1} = (u_{k+1}, H u_{k+1});
 *   until |lambda_{k+1} - lambda_k| / |lambda_{k+1}| < tol_lambda.
 * The sign of u is fixed so that sum(u) > 0.  u receives the eigenvector; returns the
 * outer iteration count (negative if maxit was hit); *lambda_out the eigenvalue and
 * *pcg_total the sum of PCG iterations.
 */
int or_inverse_iteration(int d, const int* n, const double* L, const double* const* f,
                         const double* const* S, const double* const* lam, const double* V2,
                         double shift, double tol_lambda, int maxit, double pcg_tol,
                         int pcg_maxit, double* u, double* lambda_out, long* pcg_total) {
  long N = or_total(d, n);
  double* w = (double*)malloc(sizeof(double) * N);
  double* Hu = (double*)malloc(sizeof(double) * N);
  for (long idx = 0; idx < N; ++idx) {
    long r = idx;
    double v = 1.0;
    for (int k = 0; k < d; ++k) {
      int i = (int)(r % n[k]);
      r /= n[k];
      v *= S[k][(long)i * n[k] + 0];
    }
    u[idx] = v;
  }
  double nu = sqrt(or_dot(N, u, u));
  for (long i = 0; i < N; ++i) u[i] /= nu;
  or_stencil(d, n, L, f, V2, 0.0, u, Hu);
  double lambda = or_dot(N, u, Hu);
  long total = 0;
  int it = 0, converged = 0;
  while (it < maxit) {
    for (long i = 0; i < N; ++i) w[i] = u[i] / (lambda - shift);
    double rel;
    int pit = or_pcg(d, n, L, f, S, lam, V2, -shift, -shift, u, w, pcg_tol, pcg_maxit, &rel);
    total += pit >= 0 ? pit : -pit - 1;
    double nw = sqrt(or_dot(N, w, w));
    for (long i = 0; i < N; ++i) u[i] = w[i] / nw;
    or_stencil(d, n, L, f, V2, 0.0, u, Hu);
    double lambda_new = or_dot(N, u, Hu);
    ++it;
    double change = fabs(lambda_new - lambda) / fabs(lambda_new);
    lambda = lambda_new;
    if (change < tol_lambda) { converged = 1; break; }
  }
  double su = 0.0;
  for (long i = 0; i < N; ++i) su += u[i];
  if (su < 0.0)
    for (long i = 0; i < N; ++i) u[i] = -u[i];
  if (lambda_out) *lambda_out = lambda;
  if (pcg_total) *pcg_total = total;
  free(w);
  free(Hu);
  return converged ? it : -it;
}

/* ------------------------------------------------------------ Strang ------ */

/*
 * nsteps Strang steps (Sec. 5.1 and Remark cost_naive_merged, M = 1), A = -Delta_h + V1, B = V2:
 *     psi <- e^{-i V2 dt/2} . ( e^{-i A dt} ( e^{-i V2 dt/2} . psi ) ),
 * with e^{-iA dt} the exact propagator or_apply_exp.  The two half-steps of adjacent
 * steps are NOT merged here.  psi is complex interleaved, updated in place.
 */
void or_strang(int d, const int* n, const double* const* S, const double* const* lam,
               const double* V2, double dt, int nsteps, double* psi) {
  long N = or_total(d, n);
  for (int s = 0; s < nsteps; ++s) {
    for (int half = 0; half < 2; ++half) {
      if (half == 1) or_apply_exp(d, n, S, lam, dt, psi, psi);
#pragma omp parallel for schedule(static)
      for (long i = 0; i < N; ++i) {
        double th = 0.5 * dt * V2[i];
        double c = cos(th), sn = sin(th);
        double re = psi[2 * i], im = psi[2 * i + 1];
        psi[2 * i] = re * c + im * sn;
        psi[2 * i + 1] = im * c - re * sn;
      }
    }
  }
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops that follow (timing on one core or on all of them). */
void or_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}
