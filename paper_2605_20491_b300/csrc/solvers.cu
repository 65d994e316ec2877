// Iterative drivers built on the tensor-product apply:
//   pcg_impl              -- PCG with P = (-Delta+V1+sigma_P)^{-1}            (Sec. 3.2)
//   inverse_iteration_impl -- shifted inverse iteration, warm-started PCG      (Sec. 4.1, 5.3.1)
//   split_step_impl       -- Strang e^{-iV2 dt/2} e^{-iA dt} e^{-iV2 dt/2}, A = -Delta+V1
//                            with adjacent half steps merged                  (Sec. 5.1)
// Every vector update and inner product is FP64 on the device; scalars live in device
// memory and only the residual norm / eigenvalue crosses to the host once per iteration
// for the stopping test.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "mixed.cuh"
#include "pointwise.cuh"
#include "small_n.cuh"
#include "solvers.cuh"

namespace ts {

namespace {

struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (void* p : ptrs) scratch_free(p, s);
  }
  ts_status get(double** out, size_t count) {
    void* p = nullptr;
    TS_TRY(scratch_alloc(&p, sizeof(double) * count, s));
    ptrs.push_back(p);
    *out = (double*)p;
    return TS_OK;
  }
};

ts_status read_scalars(const double* dev, double* host, int count, cudaStream_t s) {
  TS_CHECK_CUDA(cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  TS_CHECK_CUDA(cudaStreamSynchronize(s));
  return TS_OK;
}

// Pinned two-slot mailbox for the PCG stopping test: iteration k copies its r.r into slot
// k % 2 and records an event, and the host reads slot (k - 1) % 2 while iteration k runs.
// One per host thread and device, kept for the thread's lifetime: a pinned allocation and
// its release cost about a millisecond, once per PCG solve otherwise (inverse iteration
// runs one solve per outer step).
struct RrMailbox {
  int device = -1;
  double* host = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~RrMailbox() { release(); }
  void release() {
    if (host) cudaFreeHost(host);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    host = nullptr;
    ev[0] = ev[1] = nullptr;
    device = -1;
  }
  ts_status init() {
    int dev = 0;
    TS_CHECK_CUDA(cudaGetDevice(&dev));
    if (host && device == dev) return TS_OK;
    release();
    TS_CHECK_CUDA(cudaMallocHost(&host, 2 * sizeof(double)));
    for (cudaEvent_t& e : ev) TS_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    device = dev;
    return TS_OK;
  }
  ts_status post(const double* dev, int k, cudaStream_t s) {
    TS_CHECK_CUDA(cudaMemcpyAsync(host + (k & 1), dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    TS_CHECK_CUDA(cudaEventRecord(ev[k & 1], s));
    return TS_OK;
  }
  ts_status take(int k, double* out) {
    TS_CHECK_CUDA(cudaEventSynchronize(ev[k & 1]));
    *out = host[k & 1];
    return TS_OK;
  }
};

}  // namespace

ts_status pcg_impl(const ts_plan* p, double sigma, double sigma_P, const double* V2, const double* b, double* x,
                   double tol, int maxit, ts_precision prec, int* iters_out, double* relres_out, cudaStream_t s) {
  const long long N = p->N;
  Scratch sc_mem(s);
  double *r, *z, *pv, *q, *partial, *sc, *qtab, *opart;
  TS_TRY(sc_mem.get(&r, N));
  TS_TRY(sc_mem.get(&z, N));
  TS_TRY(sc_mem.get(&pv, N));
  TS_TRY(sc_mem.get(&q, N));
  TS_TRY(sc_mem.get(&partial, 2 * RED_BLOCKS));
  TS_TRY(sc_mem.get(&sc, 16));
  // On grids with one spacing (d = 3) the operator apply q = A p runs in exact fixed point
  // (Laplacian and sigma + V1 folded into an integer sum, V2 p in FP64); its scale is the
  // largest exponent of p, which the update of p reports into sc[15]'s int slot.
  FixedOperator fo;
  int* emax = reinterpret_cast<int*>(sc + 15);
  if (qtable_count(p) > 0) {
    TS_TRY(sc_mem.get(&qtab, (size_t)qtable_count(p)));
    TS_TRY(fixed_operator_prepare(p, sigma, reinterpret_cast<long long*>(qtab), &fo, s));
    if (fo.ok) TS_TRY(sc_mem.get(&opart, 2 * (size_t)fo.blocks));
  }
  auto apply_A = [&](double* out2) -> ts_status {  // q = A p; out2[0] = p.q
    if (fo.ok) return operator_apply_fixed(p, fo, V2, pv, q, emax, opart, out2, s);
    return stencil_apply(p, V2, sigma, pv, q, partial, out2, s);
  };
  auto residual = [&](double* out2) -> ts_status {  // r = b - A x; out2[0] = r.r, out2[1] = b.b
    if (fo.ok) return residual_fixed(p, fo, V2, x, b, r, emax, opart, partial, out2, s);
    return stencil_residual(p, V2, sigma, x, b, r, partial, out2, s);
  };
  double h[2];
  TS_TRY(residual(sc + 0));
  TS_TRY(read_scalars(sc, h, 2, s));
  double bnorm = std::sqrt(h[1]);
  if (bnorm == 0.0) bnorm = 1.0;
  int it = 0;
  bool converged = std::sqrt(h[0]) / bnorm < tol;
  if (!converged) {
    TS_TRY(apply_inverse_impl(p, sigma_P, r, z, prec, s));           // z = P r
    TS_TRY(dot2(N, r, z, nullptr, nullptr, partial, sc + 2, s));     // sc[2] = r.z
    TS_TRY(pcg_update_p(nullptr, nullptr, nullptr, 1, pv, z, N, s, fo.ok ? emax : nullptr));  // p = z
  }
  // The stopping test lags one iteration: iteration k posts its r.r, and the host reads
  // iteration k - 1's while the GPU runs iteration k, so the GPU never waits for the host.
  // The solve therefore stops one iteration after the first one below tol (a smaller
  // residual, reported with its own iteration count).
  thread_local RrMailbox mb;
  if (!converged) TS_TRY(mb.init());
  double rr_last = 0.0, rr_prev = 0.0;  // the two most recent tested r.r
  auto check = [&](int k, bool* stop) -> ts_status {
    double rr = 0.0;
    TS_TRY(mb.take(k, &rr));
    if (!std::isfinite(rr)) {
      set_error("PCG breakdown: non-finite residual at iteration %d", k);
      if (iters_out) *iters_out = it;
      return TS_ERR_NOT_CONVERGED;
    }
    rr_prev = rr_last;
    rr_last = rr;
    *stop = std::sqrt(rr) / bnorm < tol;
    return TS_OK;
  };
  int last_checked = 0;
  while (!converged && it < maxit) {
    TS_TRY(apply_A(sc + 4));                                                            // q = A p; sc[4] = p.q
    TS_TRY(pcg_update_xr(sc + 2, sc + 4, sc + 6, x, r, pv, q, N, partial, sc + 8, s));  // sc[6] = alpha, sc[8] = r.r
    ++it;
    TS_TRY(mb.post(sc + 8, it, s));
    // the first iteration is tested at once (an exact preconditioner converges in one),
    // later ones one iteration behind
    const int ck = it == 1 ? 1 : it - 1;
    if (ck > last_checked) {
      bool stop = false;
      TS_TRY(check(ck, &stop));
      last_checked = ck;
      if (stop) {  // iteration ck converged: stop with iterate it (ck or ck + 1)
        converged = true;
        break;
      }
      // When the contraction of the last two tested residuals predicts that iteration it
      // already meets tol, test it now instead of running one more iteration behind it.
      if (ck < it && rr_prev > 0.0) {
        const double predicted = rr_last * (rr_last / rr_prev);
        if (std::sqrt(predicted) / bnorm < tol) {
          TS_TRY(check(it, &stop));
          last_checked = it;
          if (stop) {
            converged = true;
            break;
          }
        }
      }
    }
    if (it == maxit) break;
    TS_TRY(apply_inverse_impl(p, sigma_P, r, z, prec, s));          // z = P r
    TS_TRY(dot2(N, r, z, z, q, partial, sc + 10, s));               // sc[10] = r.z, sc[11] = z.q
    TS_TRY(pcg_update_p(sc + 6, sc + 11, sc + 2, 0, pv, z, N, s, fo.ok ? emax : nullptr));  // p = z + beta p
    TS_TRY(copy_scalar(sc + 10, sc + 2, s));
  }
  if (!converged && it > last_checked) {  // the last iteration's own test
    bool stop = false;
    TS_TRY(check(it, &stop));
    converged = stop;
  }
  // true residual at exit
  TS_TRY(residual(sc + 12));
  TS_TRY(read_scalars(sc + 12, h, 1, s));
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = std::sqrt(h[0]) / bnorm;
  if (!converged) {
    set_error("PCG did not reach tol %.3e in %d iterations", tol, maxit);
    return TS_ERR_NOT_CONVERGED;
  }
  return TS_OK;
}

ts_status inverse_iteration_impl(const ts_plan* p, double shift, const double* V2, double* u, int init_from_plan,
                                 double tol_lambda, int maxit, double pcg_tol, int pcg_maxit, ts_precision prec,
                                 double* lambda_out, int* outer_out, long long* pcg_out, cudaStream_t s) {
  const long long N = p->N;
  Scratch sc_mem(s);
  double *w, *Hu, *partial, *sc;
  TS_TRY(sc_mem.get(&w, N));
  TS_TRY(sc_mem.get(&Hu, N));
  TS_TRY(sc_mem.get(&partial, 2 * RED_BLOCKS));
  TS_TRY(sc_mem.get(&sc, 8));
  // H u for the Rayleigh quotient, in exact fixed point where the form applies (its
  // exponent pass in sc[7]'s int slot), else by the FP64 stencil; out[0] = (u, H u)
  FixedOperator fo0;
  double* opart0 = nullptr;
  int* emax0 = reinterpret_cast<int*>(sc + 7);
  if (qtable_count(p) > 0) {
    double* qt = nullptr;
    TS_TRY(sc_mem.get(&qt, (size_t)qtable_count(p)));
    TS_TRY(fixed_operator_prepare(p, 0.0, reinterpret_cast<long long*>(qt), &fo0, s));
    if (fo0.ok) TS_TRY(sc_mem.get(&opart0, 2 * (size_t)fo0.blocks));
  }
  auto apply_H = [&](double* out) -> ts_status {
    if (!fo0.ok) return stencil_apply(p, V2, 0.0, u, Hu, partial, out, s);
    TS_TRY(max_exponent(u, N, emax0, s));
    return operator_apply_fixed(p, fo0, V2, u, Hu, emax0, opart0, out, s);
  };
  if (init_from_plan) TS_TRY(tensor_ground(p, u, s));
  // u <- u / ||u||; lambda = (u, H u)
  TS_TRY(dot2(N, u, u, nullptr, nullptr, partial, sc, s));
  TS_TRY(scale_by_device_ratio(N, sc, nullptr, u, u, s));
  TS_TRY(apply_H(sc + 2));
  double h[2];
  TS_TRY(read_scalars(sc + 2, h, 1, s));
  double lambda = h[0];
  long long pcg_total = 0;
  int it = 0;
  bool converged = false;
  ts_status st = TS_OK;
  while (it < maxit) {
    double den = lambda - shift;
    if (!(den > 0.0)) {
      set_error("inverse iteration: Rayleigh quotient %.6e is not above the shift %.6e", lambda, shift);
      return TS_ERR_INVALID_ARG;
    }
    TS_TRY(axpby(N, 1.0 / den, u, 0.0, w, s));  // warm start w0 = u / (lambda - s)
    int pit = 0;
    st = pcg_impl(p, -shift, -shift, V2, u, w, pcg_tol, pcg_maxit, prec, &pit, nullptr, s);
    pcg_total += pit;
    if (st != TS_OK && st != TS_ERR_NOT_CONVERGED) return st;
    TS_TRY(dot2(N, w, w, nullptr, nullptr, partial, sc, s));
    TS_TRY(scale_by_device_ratio(N, sc, nullptr, w, u, s));  // u = w / ||w||
    TS_TRY(apply_H(sc + 2));
    TS_TRY(read_scalars(sc + 2, h, 1, s));
    ++it;
    double change = std::fabs(h[0] - lambda) / std::fabs(h[0]);
    lambda = h[0];
    if (change < tol_lambda) {
      converged = true;
      break;
    }
  }
  // sign: sum(u) > 0
  TS_TRY(dot2(N, u, nullptr, nullptr, nullptr, partial, sc + 4, s));
  TS_TRY(read_scalars(sc + 4, h, 1, s));
  if (h[0] < 0.0) TS_TRY(axpby(N, -1.0, u, 0.0, u, s));
  if (lambda_out) *lambda_out = lambda;
  if (outer_out) *outer_out = it;
  if (pcg_out) *pcg_out = pcg_total;
  TS_CHECK_CUDA(cudaStreamSynchronize(s));
  if (!converged) {
    set_error("inverse iteration did not reach |dlambda|/|lambda| < %.3e in %d iterations", tol_lambda, maxit);
    return TS_ERR_NOT_CONVERGED;
  }
  return TS_OK;
}

ts_status pcg_solve(const ts_plan* p, double sigma, double sigma_P, const double* V2, const double* b, double* x,
                    double tol, int maxit, ts_precision prec, int* iters_out, double* relres_out, cudaStream_t s) {
  if (!p->sym) return pcg_impl(p, sigma, sigma_P, V2, b, x, tol, maxit, prec, iters_out, relres_out, s);
  // (M^{1/2} A M^{-1/2}) (M^{1/2} x) = M^{1/2} b; V2, V1 and sigma are diagonal and commute with M
  Scratch sc_mem(s);
  double* bt = nullptr;
  TS_TRY(sc_mem.get(&bt, p->N));
  TS_TRY(scale_separable(p, false, b, bt, s));
  TS_TRY(scale_separable(p, false, x, x, s));
  const ts_status st = pcg_impl(p->sym, sigma, sigma_P, V2, bt, x, tol, maxit, prec, iters_out, relres_out, s);
  const ts_status st2 = scale_separable(p, true, x, x, s);  // the iterate, also when not converged
  return st != TS_OK ? st : st2;
}

ts_status inverse_iteration_solve(const ts_plan* p, double shift, const double* V2, double* u, int init_from_plan,
                                  double tol_lambda, int maxit, double pcg_tol, int pcg_maxit, ts_precision prec,
                                  double* lambda_out, int* outer_out, long long* pcg_out, cudaStream_t s) {
  if (!p->sym)
    return inverse_iteration_impl(p, shift, V2, u, init_from_plan, tol_lambda, maxit, pcg_tol, pcg_maxit, prec,
                                  lambda_out, outer_out, pcg_out, s);
  if (!init_from_plan) TS_TRY(scale_separable(p, false, u, u, s));
  const ts_status st = inverse_iteration_impl(p->sym, shift, V2, u, init_from_plan, tol_lambda, maxit, pcg_tol,
                                              pcg_maxit, prec, lambda_out, outer_out, pcg_out, s);
  const ts_status st2 = scale_separable(p, true, u, u, s);
  if (st2 == TS_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("stream synchronisation failed");
    return TS_ERR_CUDA;
  }
  return st != TS_OK ? st : st2;
}

namespace {

// Gauss-Legendre rule of M points mapped onto [0, 1]: nodes c ascending, weights summing to
// 1 (the normalised weights of Sec. 5.1).  Roots of P_M by Newton's method from the
// asymptotic guesses cos(pi (j + 3/4) / (M + 1/2)), with P_M' = M (x P_M - P_{M-1}) / (x^2 - 1);
// the weight of root x on [-1, 1] is 2 / ((1 - x^2) P_M'(x)^2).
void gauss_legendre_01(int M, std::vector<double>* c, std::vector<double>* w) {
  c->assign(M, 0.0);
  w->assign(M, 0.0);
  for (int j = 0; j < M; ++j) {
    double x = std::cos(M_PI * (j + 0.75) / (M + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;  // P_0, P_1 -> P_{M-1}, P_M
      for (int q = 1; q < M; ++q) {
        const double p2 = ((2.0 * q + 1.0) * x * p1 - q * p0) / (q + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = M * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    // j = 0 is the largest root: store ascending on [0, 1]
    (*c)[M - 1 - j] = 0.5 * (x + 1.0);
    (*w)[M - 1 - j] = 1.0 / ((1.0 - x * x) * dp * dp);
  }
}

struct SplitOp {
  bool a;    // true: e^{-i t A} (exact propagator), false: e^{-i t B} (pointwise)
  double t;
};

// Appends an operation, merging it into the previous one of the same kind (A with A: the
// propagator's group property; B with B: both diagonal).
void push_op(std::vector<SplitOp>& v, bool a, double t) {
  if (!v.empty() && v.back().a == a)
    v.back().t += t;
  else
    v.push_back({a, t});
}

// One step of size h of the scheme's base method: M = 1, Strang B(h/2) A(h) B(h/2); M >= 2,
// approximated qHOP in its merged form (Remark cost_naive_merged):
// A(c_1 h) B(w_1 h) A((c_2 - c_1) h) ... B(w_M h) A((1 - c_M) h), in the order of application.
void push_base_step(std::vector<SplitOp>& v, int M, const std::vector<double>& c, const std::vector<double>& w,
                    double h) {
  if (M == 1) {
    push_op(v, false, 0.5 * h);
    push_op(v, true, h);
    push_op(v, false, 0.5 * h);
    return;
  }
  double prev = 0.0;
  for (int k = 0; k < M; ++k) {
    push_op(v, true, (c[k] - prev) * h);
    push_op(v, false, w[k] * h);
    prev = c[k];
  }
  push_op(v, true, (1.0 - prev) * h);
}

}  // namespace

ts_status propagate_impl(const ts_plan* p, ts_scheme scheme, int M, double dt, int nsteps, const double* VB,
                         void* psi, ts_dtype dtype, ts_precision prec, int* a_props, cudaStream_t s) {
  if (a_props) *a_props = 0;
  if (nsteps <= 0) return TS_OK;
  const long long N = p->N;
  if (prec == TS_FP64 && dtype == TS_C64) {  // FP64 arithmetic on complex64 data
    Scratch sc_mem(s);
    double* wbuf;
    TS_TRY(sc_mem.get(&wbuf, 2 * N));
    TS_TRY(convert_c64_to_c128(N, (const float*)psi, wbuf, s));
    TS_TRY(propagate_impl(p, scheme, M, dt, nsteps, VB, wbuf, TS_C128, prec, a_props, s));
    return convert_c128_to_c64(N, wbuf, (float*)psi, s);
  }
  const int Mb = scheme == TS_STRANG ? 1 : M;
  std::vector<double> c, w;
  if (Mb > 1) gauss_legendre_01(Mb, &c, &w);
  // Yoshida's fourth-order composition (eq. yoshida): g1 + g2 + g1 = 1, 2 g1^3 + g2^3 = 0
  const double g1 = 1.0 / (2.0 - std::cbrt(2.0)), g2 = -std::cbrt(2.0) / (2.0 - std::cbrt(2.0));
  std::vector<SplitOp> ops;
  for (int k = 0; k < nsteps; ++k) {
    if (scheme == TS_MAGNUS2) {
      push_base_step(ops, Mb, c, w, g1 * dt);
      push_base_step(ops, Mb, c, w, g2 * dt);
      push_base_step(ops, Mb, c, w, g1 * dt);
    } else {
      push_base_step(ops, Mb, c, w, dt);
    }
  }
  int na = 0;
  for (const SplitOp& op : ops) {
    if (op.a) {
      TS_TRY(apply_exp_impl(p, op.t, psi, psi, dtype, prec, s));
      ++na;
    } else if (dtype == TS_C128) {
      TS_TRY(phase_v2_c128(N, VB, op.t, (double*)psi, s));
    } else {
      TS_TRY(phase_v2_c64(N, VB, op.t, (float*)psi, s));
    }
  }
  if (a_props) *a_props = na;
  return TS_OK;
}

// Multi-level shifted inverse iteration (Sec. 5.3.1): inverse iteration on plans[0] from the
// tensor product of its per-axis ground states, then on each finer plan from the previous
// level's eigenvector carried over by tensor-product linear interpolation.  u receives the
// finest level's eigenvector; outer[l] and pcg[l] the per-level iteration counts.
ts_status inverse_iteration_multilevel_impl(const ts_plan* const* plans, const double* const* V2, int levels,
                                            double shift, double* u, double tol_lambda, int maxit, double pcg_tol,
                                            int pcg_maxit, ts_precision prec, double* lambda_out, int* outer,
                                            long long* pcg, cudaStream_t s) {
  Scratch sc_mem(s);
  double* prev = nullptr;
  const ts_plan* prev_plan = nullptr;
  double lambda = 0.0;
  for (int l = 0; l < levels; ++l) {
    const ts_plan* p = plans[l];
    double* ul = u;
    if (l + 1 < levels) TS_TRY(sc_mem.get(&ul, p->N));
    if (l > 0) TS_TRY(interpolate(prev_plan, prev, p, ul, s));
    int it = 0;
    long long pit = 0;
    const ts_status st = inverse_iteration_solve(p, shift, V2 ? V2[l] : nullptr, ul, l == 0, tol_lambda, maxit,
                                                 pcg_tol, pcg_maxit, prec, &lambda, &it, &pit, s);
    if (outer) outer[l] = it;
    if (pcg) pcg[l] = pit;
    if (st != TS_OK && !(st == TS_ERR_NOT_CONVERGED && l + 1 < levels)) {
      if (lambda_out) *lambda_out = lambda;
      return st;
    }
    prev = ul;
    prev_plan = p;
  }
  if (lambda_out) *lambda_out = lambda;
  return TS_OK;
}

ts_status plan_create(const ts_plan_desc* desc, unsigned mask, cudaStream_t s, ts_plan** out);
void plan_free(ts_plan* p);

// The GPE ground state by Riemannian gradient flows on the L2 sphere (Sec. 4.2-4.3):
//   u <- (u - tau grad) / ||u - tau grad||,  grad = G H_u u - [(u, G H_u u) / (u, G u)] G u,
// H_u = -Delta + V1 + V2 + beta u^2, inner products weighted by the quadrature (W = prod M_k).
// Modified H^1 flow: G = (-Delta + alpha)^{-1}, two direct solves per step on a plan of the
// same grid with f = 0 (split precisions: two refinements with the FP64 residual).  a_u flow:
// G = H_u^{-1}, so G H_u u = u and G u is one PCG solve with the plan's (-Delta + V1)^{-1}
// as preconditioner, warm-started from the previous step's solution.
ts_status gpe_ground_state_impl(const ts_plan* p, const double* V2, double beta, ts_gpe_flow flow, double alpha,
                                double tau, double* u, double tol_energy, double tol_residual, int maxit,
                                ts_precision prec, double pcg_tol, double* energy_out, double* lambda_out,
                                double* residual_out, int* iters_out, long long* solves_out, cudaStream_t s) {
  const long long N = p->N;
  Scratch sc_mem(s);
  double *r, *w1, *w2, *veff, *partial, *sc;
  TS_TRY(sc_mem.get(&r, N));
  TS_TRY(sc_mem.get(&w1, N));
  TS_TRY(sc_mem.get(&w2, N));
  TS_TRY(sc_mem.get(&veff, N));
  TS_TRY(sc_mem.get(&partial, 2 * RED_BLOCKS));
  TS_TRY(sc_mem.get(&sc, 8));
  ts_plan* p0 = nullptr;  // -Delta alone on the same grid (modified H^1 flow)
  struct Owner {  // the internal plan outlives every kernel that reads its tables
    ts_plan* q;
    cudaStream_t s;
    ~Owner() {
      if (!q) return;
      cudaStreamSynchronize(s);
      plan_free(q);
    }
  } own{nullptr, s};
  if (flow == TS_GPE_H1) {
    std::vector<std::vector<double>> zeros(p->d);
    std::vector<const double*> fz(p->d);
    for (int k = 0; k < p->d; ++k) {
      zeros[k].assign(p->n[k], 0.0);
      fz[k] = zeros[k].data();
    }
    ts_plan_desc desc{};
    desc.d = p->d;
    desc.n = p->n;
    desc.L = p->L;
    desc.f = fz.data();
    desc.bc = 0;
    desc.order = p->order;
    TS_TRY(plan_create(&desc, p->precision_mask, s, &p0));
    own.q = p0;
  }
  // A split-precision G carries two FP64-residual refinements: the flow's fixed point moves
  // by about G's error over the spectral gap, and one refinement (~1e-10 for BF16X3)
  // leaves the Euler-Lagrange residual near 1e-8.
  const ts_precision sched[3] = {prec, prec, prec};
  auto applyG = [&](const double* in, double* out) -> ts_status {
    if (prec == TS_FP64) return apply_inverse_impl(p0, alpha, in, out, prec, s);
    return mixed_solve_schedule(p0, sched, 3, alpha, in, out, s);
  };
  // u <- u / ||u||
  TS_TRY(wdot2(p, u, u, nullptr, nullptr, partial, sc, s));
  TS_TRY(scale_by_device_ratio(N, sc, nullptr, u, u, s));
  TS_CHECK_CUDA(cudaMemsetAsync(w2, 0, sizeof(double) * N, s));
  double E_prev = 0.0, E = 0.0, lam = 0.0, res = 0.0;
  long long solves = 0;
  int it = 0;
  bool converged = false;
  for (;; ++it) {
    // H_u u, then E = 1/2 (u, H_u u) - beta/4 (u^2, u^2), lambda = (u, H_u u) and, when asked
    // for, the Euler-Lagrange residual ||H_u u - lambda u|| / lambda
    TS_TRY(gpe_veff(N, V2, beta, u, veff, s));
    TS_TRY(stencil_apply(p, veff, 0.0, u, r, partial, nullptr, s));
    TS_TRY(wdot_energy(p, u, r, partial, sc, s));
    double h[2];
    TS_TRY(read_scalars(sc, h, 2, s));
    lam = h[0];
    E = 0.5 * h[0] - 0.25 * beta * h[1];
    if (tol_residual > 0.0 || residual_out) {
      TS_TRY(wdot_residual(p, u, r, lam, partial, sc, s));
      TS_TRY(read_scalars(sc, h, 1, s));
      res = std::sqrt(std::max(h[0], 0.0)) / std::fabs(lam);
    }
    converged = (tol_energy > 0.0 || tol_residual > 0.0) &&
                (tol_energy <= 0.0 || (it > 0 && std::fabs(E - E_prev) < tol_energy * std::fabs(E))) &&
                (tol_residual <= 0.0 || res < tol_residual);
    if (converged || it == maxit) break;
    E_prev = E;
    const double* g1;
    if (flow == TS_GPE_H1) {
      TS_TRY(applyG(r, w1));
      TS_TRY(applyG(u, w2));
      solves += 2;
      g1 = w1;
    } else {
      int pit = 0;
      const ts_status st = pcg_solve(p, 0.0, 0.0, veff, u, w2, pcg_tol, 10000, prec, &pit, nullptr, s);
      if (st != TS_OK && st != TS_ERR_NOT_CONVERGED) return st;
      solves += pit;
      g1 = u;  // G H_u u = u
    }
    TS_TRY(wdot2(p, u, g1, u, w2, partial, sc, s));
    TS_TRY(read_scalars(sc, h, 2, s));
    const double gamma = h[0] / h[1];
    // u <- u - tau (g1 - gamma w2), then normalise
    if (g1 == u) {
      TS_TRY(axpy2(N, u, -tau, u, tau * gamma, w2, s));
    } else {
      TS_TRY(axpy2(N, u, -tau, g1, tau * gamma, w2, s));
    }
    TS_TRY(wdot2(p, u, u, nullptr, nullptr, partial, sc, s));
    TS_TRY(scale_by_device_ratio(N, sc, nullptr, u, u, s));
  }
  if (energy_out) *energy_out = E;
  if (lambda_out) *lambda_out = lam;
  if (residual_out) *residual_out = res;
  if (iters_out) *iters_out = it;
  if (solves_out) *solves_out = solves;
  if (!converged) {
    set_error("GPE flow: no convergence in %d iterations (|dE|/E = %.3e, residual %.3e)", maxit,
              std::fabs(E - E_prev) / std::fabs(E), res);
    return TS_ERR_NOT_CONVERGED;
  }
  return TS_OK;
}

ts_status split_step_impl(const ts_plan* p, double dt, int nsteps, const double* V2, void* psi, ts_dtype dtype,
                          ts_precision prec, cudaStream_t s) {
  if (nsteps <= 0) return TS_OK;
  const long long N = p->N;
  if (prec == TS_FP32) {
    if (dtype != TS_C64) {
      set_error("TS_FP32 split steps work on complex64 data");
      return TS_ERR_UNSUPPORTED;
    }
    return small_n_propagate(p, dt, (const float2*)psi, (float2*)psi, V2, dt, nsteps, s);
  }
  if (prec == TS_BF16X6 && dtype == TS_C64 && small_tc_applicable(p))
    return small_n_propagate(p, dt, (const float2*)psi, (float2*)psi, V2, dt, nsteps, s, true);
  if (prec == TS_FP64 && dtype == TS_C64) {
    // FP64 arithmetic on complex64 data: widen once, run in complex128, narrow once.
    Scratch sc_mem(s);
    double* w;
    TS_TRY(sc_mem.get(&w, 2 * N));
    TS_TRY(convert_c64_to_c128(N, (const float*)psi, w, s));
    TS_TRY(split_step_impl(p, dt, nsteps, V2, w, TS_C128, prec, s));
    TS_TRY(convert_c128_to_c64(N, w, (float*)psi, s));
    return TS_OK;
  }
  auto phase = [&](double theta) -> ts_status {
    if (dtype == TS_C128) return phase_v2_c128(N, V2, theta, (double*)psi, s);
    return phase_v2_c64(N, V2, theta, (float*)psi, s);
  };
  TS_TRY(phase(0.5 * dt));
  for (int k = 0; k < nsteps; ++k) {
    TS_TRY(apply_exp_impl(p, dt, psi, psi, dtype, prec, s));
    TS_TRY(phase(k == nsteps - 1 ? 0.5 * dt : dt));  // merged half steps between steps
  }
  return TS_OK;
}

}  // namespace ts
