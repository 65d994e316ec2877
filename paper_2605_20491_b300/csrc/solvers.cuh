// Iterative drivers: see solvers.cu.
#pragma once
#include "common.cuh"

namespace ts {

ts_status pcg_impl(const ts_plan* p, double sigma, double sigma_P, const double* V2, const double* b, double* x,
                   double tol, int maxit, ts_precision prec, int* iters_out, double* relres_out, cudaStream_t s);
ts_status inverse_iteration_impl(const ts_plan* p, double shift, const double* V2, double* u, int init_from_plan,
                                 double tol_lambda, int maxit, double pcg_tol, int pcg_maxit, ts_precision prec,
                                 double* lambda_out, int* outer_out, long long* pcg_out, cudaStream_t s);
ts_status split_step_impl(const ts_plan* p, double dt, int nsteps, const double* V2, void* psi, ts_dtype dtype,
                          ts_precision prec, cudaStream_t s);

}  // namespace ts
