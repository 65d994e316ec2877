// Iterative drivers: see solvers.cu.
#pragma once
#include "common.cuh"

namespace ts {

ts_status pcg_impl(const ts_plan* p, double sigma, double sigma_P, const double* V2, const double* b, double* x,
                   double tol, int maxit, ts_precision prec, int* iters_out, double* relres_out, cudaStream_t s);
ts_status inverse_iteration_impl(const ts_plan* p, double shift, const double* V2, double* u, int init_from_plan,
                                 double tol_lambda, int maxit, double pcg_tol, int pcg_maxit, ts_precision prec,
                                 double* lambda_out, int* outer_out, long long* pcg_out, cudaStream_t s);
// The entry points of ts_pcg and ts_inverse_iteration: the *_impl drivers above run on the
// plan's symmetric frame, which for Q^k (k >= 2) is the twin p->sym with unknowns M^{1/2} x
// (self-adjoint operator and preconditioner in the plain inner product); these convert the
// caller's vectors into it and back.  For Q^1 they call the drivers directly.
ts_status pcg_solve(const ts_plan* p, double sigma, double sigma_P, const double* V2, const double* b, double* x,
                    double tol, int maxit, ts_precision prec, int* iters_out, double* relres_out, cudaStream_t s);
ts_status inverse_iteration_solve(const ts_plan* p, double shift, const double* V2, double* u, int init_from_plan,
                                  double tol_lambda, int maxit, double pcg_tol, int pcg_maxit, ts_precision prec,
                                  double* lambda_out, int* outer_out, long long* pcg_out, cudaStream_t s);
// The splitting schemes of Sec. 5.1 for i dpsi/dt = (A + B) psi, A = the plan's operator
// (exact propagator), B = diag(VB): Strang, approximated qHOP with M Gauss-Legendre nodes,
// approximated Magnus-2 (Yoshida composition), all with adjacent propagations merged.
ts_status propagate_impl(const ts_plan* p, ts_scheme scheme, int M, double dt, int nsteps, const double* VB,
                         void* psi, ts_dtype dtype, ts_precision prec, int* a_props, cudaStream_t s);
ts_status inverse_iteration_multilevel_impl(const ts_plan* const* plans, const double* const* V2, int levels,
                                            double shift, double* u, double tol_lambda, int maxit, double pcg_tol,
                                            int pcg_maxit, ts_precision prec, double* lambda_out, int* outer,
                                            long long* pcg, cudaStream_t s);
ts_status gpe_ground_state_impl(const ts_plan* p, const double* V2, double beta, ts_gpe_flow flow, double alpha,
                                double tau, double* u, double tol_energy, double tol_residual, int maxit,
                                ts_precision prec, double pcg_tol, double* energy_out, double* lambda_out,
                                double* residual_out, int* iters_out, long long* solves_out, cudaStream_t s);
ts_status split_step_impl(const ts_plan* p, double dt, int nsteps, const double* V2, void* psi, ts_dtype dtype,
                          ts_precision prec, cudaStream_t s);

}  // namespace ts
