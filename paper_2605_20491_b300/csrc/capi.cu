// extern "C" entry points of include/tschrod.h: argument validation, device selection
// and error reporting around the drivers.
#include <cstdarg>
#include <cstring>

#include <vector>

#include "common.cuh"
#include "mixed.cuh"
#include "pointwise.cuh"
#include "sem_axis.cuh"
#include "small_n.cuh"
#include "solvers.cuh"

namespace ts {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

void plan_free(ts_plan* p);
ts_status plan_create(const ts_plan_desc* desc, unsigned mask, cudaStream_t s, ts_plan** out);

namespace {

// Makes the plan's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

ts_status check_prec(const ts_plan* p, ts_precision prec) {
  if ((int)prec < 0 || (int)prec >= NPREC || (int)prec == 3 || (int)prec == 4) {
    set_error("invalid precision %d", (int)prec);
    return TS_ERR_INVALID_ARG;
  }
  if (prec == TS_FP64) return TS_OK;
  if (!(p->precision_mask & (1u << prec))) {
    set_error("precision %d was not requested in the plan's precision_mask", (int)prec);
    return TS_ERR_UNSUPPORTED;
  }
  return TS_OK;
}

}  // namespace
}  // namespace ts

using namespace ts;

#define TS_API_BEGIN(plan)                                       \
  clear_error();                                                 \
  if (!(plan)) {                                                 \
    set_error("plan is NULL");                                   \
    return TS_ERR_INVALID_ARG;                                   \
  }                                                              \
  DeviceGuard _guard((plan)->device);                            \
  if (!_guard.ok) {                                              \
    set_error("cannot select device %d", (plan)->device);        \
    return TS_ERR_CUDA;                                          \
  }

extern "C" {

const char* ts_last_error(void) { return g_err; }

const char* ts_version(void) {
  return "tschrod 0.1 (sm_103a; FP64 SIMT, bf16 split tcgen05, small-n fused kernels)";
}

ts_status ts_plan_create(const ts_plan_desc* desc, unsigned precision_mask, void* stream, ts_plan** out) {
  clear_error();
  if (!out) {
    set_error("out is NULL");
    return TS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  TS_REQUIRE(desc, "desc is NULL");
  TS_REQUIRE(desc->d >= 1 && desc->d <= TS_MAX_DIM, "d = %d out of range [1, %d]", desc->d, TS_MAX_DIM);
  TS_REQUIRE(desc->n && desc->L && desc->f, "desc->n, desc->L and desc->f must be non-NULL");
  TS_REQUIRE(desc->bc == 0, "only homogeneous Dirichlet (bc = 0) is supported");
  TS_REQUIRE(precision_mask < (1u << NPREC) && !(precision_mask & 0x18u),
             "precision_mask 0x%x has unknown bits (3 and 4 are not assigned)", precision_mask);
  long long N = 1;
  for (int k = 0; k < desc->d; ++k) {
    TS_REQUIRE(desc->n[k] >= 1 && desc->n[k] <= 4096, "n[%d] = %d out of range [1, 4096]", k, desc->n[k]);
    TS_REQUIRE(desc->L[k] > 0.0, "L[%d] must be positive", k);
    TS_REQUIRE(desc->f[k], "f[%d] is NULL", k);
    TS_REQUIRE(desc->order >= -1 && desc->order <= 32, "order = %d out of range [-1, 32]", desc->order);
    TS_REQUIRE(desc->order < 2 || (desc->n[k] + 1) % desc->order == 0,
               "Q^%d: n[%d] + 1 = %d is not a multiple of %d", desc->order, k, desc->n[k] + 1, desc->order);
    TS_REQUIRE(desc->order != -1 || desc->n[k] <= 2048, "Hermite axis %d: n = %d above 2048", k, desc->n[k]);
    N *= desc->n[k];
    TS_REQUIRE(N <= (1LL << 40), "grid too large");
  }
  return plan_create(desc, precision_mask, (cudaStream_t)stream, out);
}

ts_status ts_plan_destroy(ts_plan* plan) {
  clear_error();
  if (!plan) return TS_OK;
  DeviceGuard g(plan->device);
  plan_free(plan);
  return TS_OK;
}

ts_status ts_grid_nodes(int n, double L, int order, double* x, double* m) {
  clear_error();
  TS_REQUIRE(x, "x is NULL");
  TS_REQUIRE(n >= 1 && n <= 4096, "n = %d out of range [1, 4096]", n);
  TS_REQUIRE(L > 0.0, "L must be positive");
  TS_REQUIRE(order >= -1 && order <= 32, "order = %d out of range [-1, 32]", order);
  return grid_nodes_host(n, L, order, x, m);
}

ts_status ts_plan_eigs(const ts_plan* plan, int axis, double* lambda_host) {
  clear_error();
  TS_REQUIRE(plan && lambda_host, "NULL argument");
  TS_REQUIRE(axis >= 0 && axis < plan->d, "axis %d out of range", axis);
  std::memcpy(lambda_host, plan->axis[axis]->lam_host.data(), sizeof(double) * plan->n[axis]);
  return TS_OK;
}

ts_status ts_plan_eigvecs(const ts_plan* plan, int axis, double* S_host) {
  clear_error();
  TS_REQUIRE(plan && S_host, "NULL argument");
  TS_REQUIRE(axis >= 0 && axis < plan->d, "axis %d out of range", axis);
  std::memcpy(S_host, plan->axis[axis]->S_host.data(), sizeof(double) * plan->n[axis] * plan->n[axis]);
  return TS_OK;
}

ts_status ts_plan_shape(const ts_plan* plan, int* d, int* n, long long* N) {
  clear_error();
  TS_REQUIRE(plan, "plan is NULL");
  if (d) *d = plan->d;
  if (n)
    for (int k = 0; k < plan->d; ++k) n[k] = plan->n[k];
  if (N) *N = plan->N;
  return TS_OK;
}

ts_status ts_plan_bytes(const ts_plan* plan, long long* bytes) {
  clear_error();
  TS_REQUIRE(plan && bytes, "NULL argument");
  *bytes = plan->bytes;
  return TS_OK;
}

ts_status ts_apply_inverse(const ts_plan* plan, double sigma, const double* b, double* u, ts_precision prec,
                           void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(b && u, "b and u must be non-NULL");
  TS_TRY(check_prec(plan, prec));
  return apply_inverse_impl(plan, sigma, b, u, prec, (cudaStream_t)stream);
}

ts_status ts_solve_refined(const ts_plan* plan, double sigma, const double* b, double* u, ts_precision prec,
                           int refinements, void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(b && u && b != u, "b and u must be non-NULL and distinct");
  TS_REQUIRE(refinements >= 0 && refinements <= 16, "refinements must be in [0, 16]");
  TS_TRY(check_prec(plan, prec));
  if (prec == TS_FP64) return apply_inverse_impl(plan, sigma, b, u, prec, (cudaStream_t)stream);
  return mixed_refine(plan, prec, sigma, b, u, refinements, (cudaStream_t)stream);
}

ts_status ts_solve_schedule(const ts_plan* plan, double sigma, const double* b, double* u,
                            const ts_precision* schedule, int count, void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(b && u && b != u, "b and u must be non-NULL and distinct");
  TS_REQUIRE(schedule, "schedule is NULL");
  TS_REQUIRE(count >= 1 && count <= 17, "count must be in [1, 17]");
  for (int k = 0; k < count; ++k) {
    TS_TRY(check_prec(plan, schedule[k]));
    TS_REQUIRE(schedule[k] != TS_FP64 && schedule[k] != TS_FP32, "schedule[%d]: split precisions only", k);
  }
  return mixed_solve_schedule(plan, schedule, count, sigma, b, u, (cudaStream_t)stream);
}

ts_status ts_apply_exp(const ts_plan* plan, double tau, const void* psi_in, void* psi_out, ts_dtype dtype,
                       ts_precision prec, void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(psi_in && psi_out, "psi_in and psi_out must be non-NULL");
  TS_REQUIRE(dtype == TS_C128 || dtype == TS_C64, "dtype must be TS_C128 or TS_C64");
  TS_TRY(check_prec(plan, prec));
  return apply_exp_impl(plan, tau, psi_in, psi_out, dtype, prec, (cudaStream_t)stream);
}

ts_status ts_apply_batch(const ts_batch_item* items, int count, void* stream) {
  clear_error();
  TS_REQUIRE(count >= 0, "count must be >= 0");
  TS_REQUIRE(items || count == 0, "items is NULL");
  if (count == 0) return TS_OK;
  std::vector<BatchApply> q(count);
  int device = -1;
  for (int i = 0; i < count; ++i) {
    const ts_batch_item& it = items[i];
    TS_REQUIRE(it.plan, "items[%d].plan is NULL", i);
    TS_REQUIRE(it.in && it.out, "items[%d]: in and out must be non-NULL", i);
    TS_REQUIRE(it.dtype == TS_R64 || it.dtype == TS_C128 || it.dtype == TS_C64, "items[%d]: bad dtype", i);
    TS_REQUIRE(bf16_planes(it.prec) > 0, "items[%d]: split precisions only", i);
    TS_TRY(check_prec(it.plan, it.prec));
    TS_REQUIRE(device < 0 || it.plan->device == device, "items[%d]: all plans must be on one device", i);
    device = it.plan->device;
    q[i] = BatchApply{it.plan, it.prec, it.dtype == TS_R64 ? MixedOp::Inverse : MixedOp::Exp, it.param, it.in,
                      it.out, it.dtype};
  }
  DeviceGuard g(device);
  if (!g.ok) {
    set_error("cannot select device %d", device);
    return TS_ERR_CUDA;
  }
  return mixed_apply_batch(q.data(), count, (cudaStream_t)stream);
}

ts_status ts_apply_operator(const ts_plan* plan, double sigma, const double* V2, const double* x, double* y,
                            void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(x && y && x != y, "x and y must be non-NULL and distinct");
  return operator_apply(plan, V2, sigma, x, y, (cudaStream_t)stream);
}

ts_status ts_pcg(const ts_plan* plan, double sigma, double sigma_P, const double* V2, const double* b, double* x,
                 double tol, int maxit, ts_precision precond, int* iters, double* relres, void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(b && x && b != x, "b and x must be non-NULL and distinct");
  TS_REQUIRE(tol > 0.0 && maxit >= 0, "tol must be > 0 and maxit >= 0");
  TS_TRY(check_prec(plan, precond));
  return pcg_solve(plan, sigma, sigma_P, V2, b, x, tol, maxit, precond, iters, relres, (cudaStream_t)stream);
}

ts_status ts_inverse_iteration(const ts_plan* plan, double shift, const double* V2, double* u, int init_from_plan,
                               double tol_lambda, int maxit, double pcg_tol, int pcg_maxit, ts_precision precond,
                               double* lambda, int* outer_iters, long long* pcg_iters, void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(u, "u must be non-NULL");
  TS_REQUIRE(tol_lambda > 0.0 && pcg_tol > 0.0 && maxit >= 1 && pcg_maxit >= 1, "bad tolerances or caps");
  TS_TRY(check_prec(plan, precond));
  return inverse_iteration_solve(plan, shift, V2, u, init_from_plan, tol_lambda, maxit, pcg_tol, pcg_maxit, precond,
                                lambda, outer_iters, pcg_iters, (cudaStream_t)stream);
}

ts_status ts_tc_config_set(int complex_data, int n, int bk, int bn_cap, int cluster) {
  clear_error();
  return tc_config_set(complex_data, n, bk, bn_cap, cluster);
}

ts_status ts_selftest_wait_timeout(long long cycles, void* stream) {
  clear_error();
  TS_REQUIRE(cycles > 0 && cycles <= 4000000000LL, "cycles must be in (0, 4e9]");
  return wait_selftest(cycles, (cudaStream_t)stream);
}

ts_status ts_device_status(void* stream) {
  clear_error();
  int flag = 0;
  TS_TRY(mixed_error_flag(&flag, true, (cudaStream_t)stream));
  if (flag == 0) TS_TRY(small_n_error_flag(&flag, true, (cudaStream_t)stream));
  if (flag != 0) {
    set_error("a bounded device-side wait ran out (code %d)", flag);
    return TS_ERR_TIMEOUT;
  }
  return TS_OK;
}

ts_status ts_split_step(const ts_plan* plan, double dt, int nsteps, const double* V2, void* psi, ts_dtype dtype,
                        ts_precision prec, void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(V2 && psi, "V2 and psi must be non-NULL");
  TS_REQUIRE(dtype == TS_C128 || dtype == TS_C64, "dtype must be TS_C128 or TS_C64");
  TS_REQUIRE(nsteps >= 0, "nsteps must be >= 0");
  TS_TRY(check_prec(plan, prec));
  return split_step_impl(plan, dt, nsteps, V2, psi, dtype, prec, (cudaStream_t)stream);
}

ts_status ts_propagate(const ts_plan* plan, ts_scheme scheme, int M, double dt, int nsteps, const double* VB,
                       void* psi, ts_dtype dtype, ts_precision prec, int* a_propagations, void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(VB && psi, "VB and psi must be non-NULL");
  TS_REQUIRE(scheme == TS_STRANG || scheme == TS_QHOP || scheme == TS_MAGNUS2, "unknown scheme %d", (int)scheme);
  TS_REQUIRE(M >= 1 && M <= 64, "M = %d out of range [1, 64]", M);
  TS_REQUIRE(dtype == TS_C128 || dtype == TS_C64, "dtype must be TS_C128 or TS_C64");
  TS_REQUIRE(nsteps >= 0, "nsteps must be >= 0");
  TS_TRY(check_prec(plan, prec));
  return propagate_impl(plan, scheme, M, dt, nsteps, VB, psi, dtype, prec, a_propagations, (cudaStream_t)stream);
}

ts_status ts_gpe_ground_state(const ts_plan* plan, const double* V2, double beta, ts_gpe_flow flow, double alpha,
                              double tau, double* u, double tol_energy, double tol_residual, int maxit,
                              ts_precision prec, double pcg_tol, double* energy, double* lambda, double* residual,
                              int* iters, long long* solves, void* stream) {
  TS_API_BEGIN(plan);
  TS_REQUIRE(u, "u must be non-NULL");
  TS_REQUIRE(flow == TS_GPE_H1 || flow == TS_GPE_AU, "unknown flow %d", (int)flow);
  TS_REQUIRE(beta >= 0.0 && tau > 0.0 && maxit >= 0, "need beta >= 0, tau > 0, maxit >= 0");
  TS_REQUIRE(flow != TS_GPE_H1 || alpha > 0.0, "the modified H^1 flow needs alpha > 0");
  TS_REQUIRE(flow != TS_GPE_AU || pcg_tol > 0.0, "the a_u flow needs pcg_tol > 0");
  TS_TRY(check_prec(plan, prec));
  return gpe_ground_state_impl(plan, V2, beta, flow, alpha, tau, u, tol_energy, tol_residual, maxit, prec, pcg_tol,
                               energy, lambda, residual, iters, solves, (cudaStream_t)stream);
}

ts_status ts_interpolate(const ts_plan* coarse, const double* uc, const ts_plan* fine, double* uf, void* stream) {
  TS_API_BEGIN(fine);
  TS_REQUIRE(coarse && uc && uf && uc != uf, "coarse, uc, uf must be non-NULL and uc != uf");
  TS_REQUIRE(coarse->device == fine->device, "both plans must be on one device");
  return interpolate(coarse, uc, fine, uf, (cudaStream_t)stream);
}

ts_status ts_inverse_iteration_multilevel(const ts_plan* const* plans, const double* const* V2, int levels,
                                          double shift, double* u, double tol_lambda, int maxit, double pcg_tol,
                                          int pcg_maxit, ts_precision precond, double* lambda, int* outer,
                                          long long* pcg, void* stream) {
  clear_error();
  TS_REQUIRE(plans && levels >= 1 && u, "need plans, levels >= 1 and u");
  for (int l = 0; l < levels; ++l) {
    TS_REQUIRE(plans[l], "plans[%d] is NULL", l);
    TS_REQUIRE(plans[l]->device == plans[0]->device && plans[l]->d == plans[0]->d,
               "all levels must share the device and the dimension");
    TS_TRY(check_prec(plans[l], precond));
  }
  TS_REQUIRE(maxit >= 1 && pcg_maxit >= 1, "maxit and pcg_maxit must be >= 1");
  DeviceGuard g(plans[0]->device);
  if (!g.ok) {
    set_error("cannot select device %d", plans[0]->device);
    return TS_ERR_CUDA;
  }
  return inverse_iteration_multilevel_impl(plans, V2, levels, shift, u, tol_lambda, maxit, pcg_tol, pcg_maxit, precond,
                                           lambda, outer, pcg, (cudaStream_t)stream);
}

}  // extern "C"
