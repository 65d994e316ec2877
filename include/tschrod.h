/*
 * tschrod.h -- C ABI of the B300 (sm_103a) tensor-product solver for the
 * Schroedinger operator  H = -Delta + V1 (+ V2)  on the box [-L_1,L_1] x ... x [-L_d,L_d]
 * with homogeneous Dirichlet conditions, discretised by Q^1 spectral elements
 * (second-order central differences), with a separable potential
 *     V1(x) = f_1(x_1) + ... + f_d(x_d).
 *
 * Method (Sec. 2.1, eqs. general_system, tensor_system, eigen_decomp): per axis k the
 * 1D operator H_k = h_k^-2 tridiag(-1,2,-1) + diag f_k(x_{k,i}) is eigendecomposed once,
 * H_k = S_k diag(lambda_k) S_k^T (plan creation; S_k orthogonal because the Q^1 mass
 * matrix is h I).  Every apply then runs d mode-k contractions with S_k^T (forward
 * transform), a pointwise scale of coefficient (i_1..i_d) by a function of
 * Lambda = lambda_1[i_1] + ... + lambda_d[i_d], and d mode-k contractions with S_k
 * (backward transform).
 *
 * Conventions shared by every entry point:
 *   - Grid: axis k has n_k interior nodes x_{k,i} = -L_k + i h_k, i = 1..n_k,
 *     h_k = 2 L_k / (n_k + 1).
 *   - Layout: a grid function is the vector vec(U) with axis 1 fastest, i.e. element
 *     (i_1, ..., i_d) (0-based) sits at i_1 + n_1 (i_2 + n_2 (i_3 + ...)).
 *     N = n_1 n_2 ... n_d.  Complex data are interleaved (re, im) pairs:
 *     TS_C128 = 2 doubles per element, TS_C64 = 2 floats per element.
 *   - Every array argument is caller-owned DEVICE memory on the plan's device unless
 *     stated otherwise, aligned to at least 16 bytes.  The library never frees it.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls enqueue
 *     their work on it and return without waiting, except those that return host
 *     scalars (iterations, residuals, eigenvalues), which synchronise that stream.
 *   - Scratch memory (a few N-sized buffers) comes from the stream-ordered CUDA memory
 *     pool of the plan's device (cudaMallocAsync / cudaFreeAsync on `stream`).
 *   - A plan is immutable once created; several host threads may use one plan at once
 *     on different streams.
 *   - Errors are returned as a ts_status, never by aborting; ts_last_error() gives a
 *     thread-local message for the last failing call of the calling thread.
 */
#ifndef TSCHROD_H
#define TSCHROD_H

#ifdef __cplusplus
extern "C" {
#endif

#define TS_MAX_DIM 12

typedef enum {
  TS_OK = 0,
  TS_ERR_INVALID_ARG = 1,   /* a pointer, size or enum is out of range                */
  TS_ERR_NO_MEMORY = 2,     /* a device allocation failed                             */
  TS_ERR_CUDA = 3,          /* a CUDA runtime/library call failed                     */
  TS_ERR_NOT_CONVERGED = 4, /* an iteration hit its cap; the best iterate is written  */
  TS_ERR_UNSUPPORTED = 5,   /* valid request that this build/plan cannot serve        */
  TS_ERR_TIMEOUT = 6        /* a bounded device-side wait ran out                     */
} ts_status;

/* Arithmetic of the mode-k contractions (the eigendecompositions, the eigenvalue sums,
 * PCG scalars and inner products are always FP64). */
typedef enum {
  TS_FP64 = 0,   /* plain FP64 (FFMA64) contractions                                      */
  TS_BF16X3 = 1, /* 2-term bf16 splits of data and S_k, 3 products, FP32 accumulate (tcgen05) */
  TS_BF16X6 = 2, /* 3-term bf16 splits, 6 products, FP32 accumulate (tcgen05)              */
  /* values 3 and 4 are not assigned (precision_mask bits 3 and 4 are refused): with one
     FP32 accumulator the tensor-core passes lose about 1e-5 at n = 512 to the truncating
     accumulation whatever the split format, so tf32 or scaled fp16 splits would not give a
     cheaper refinement schedule than the bf16 ones */
  TS_FP32 = 5,   /* plain FP32 (FFMA) fused small-n kernels: complex64 propagation with
                    every n_k in {8, 16, 24, 32} (the paper's FP32 variant)              */
  TS_BF16X1 = 6  /* one bf16 plane, one product, FP32 accumulate (tcgen05): a cheap,
                    coarse inverse (relative error ~1e-2) for the late refinements      */
} ts_precision;

typedef enum { TS_R64 = 0, TS_C128 = 1, TS_C64 = 2 } ts_dtype;

typedef struct ts_plan ts_plan;

/* Problem description.  All pointers are HOST memory, read during ts_plan_create only. */
typedef struct {
  int d;                   /* dimension, 1 <= d <= TS_MAX_DIM                          */
  const int* n;            /* n[k] interior nodes on axis k, 1 <= n[k] <= 4096          */
  const double* L;         /* L[k] > 0: axis k spans [-L[k], L[k]]                     */
  const double* const* f;  /* f[k][i] = f_k(x_{k,i}), i = 0..n[k]-1, at the interior nodes
                              of axis k (ts_grid_nodes) (V1 samples)                     */
  int bc;                  /* boundary condition: 0 = homogeneous Dirichlet (only one) */
  int order;               /* the k of Q^k (Sec. 2): 0 or 1 = Q^1, the second-order
                              finite-difference scheme on the uniform nodes
                              x_i = -L + (i+1) h, h = 2L/(n+1); 2..32 = Q^k spectral
                              elements with GLL quadrature, (n[k] + 1) / order elements
                              per axis ((n[k] + 1) % order == 0 on every axis);
                              -1 = the Hermite spectral method on R (Appendix app:hermite):
                              n[k] <= 2048 Gauss-Hermite nodes, L[k] unused (must be > 0),
                              the operator dense per axis; no interpolation               */
} ts_plan_desc;

/*
 * Nodes of one axis (Sec. 2): for order 0 or 1 the uniform x_i = -L + (i+1) h,
 * h = 2L/(n+1); for order k >= 2 the Gauss-Lobatto-Legendre points of degree k mapped onto
 * the c = (n+1)/k equal elements of [-L, L], end points shared, the two boundary nodes
 * dropped; for order -1 the n Gauss-Hermite nodes (eigenvalues of the Jacobi matrix with
 * off-diagonal sqrt(k/2), by Sturm bisection).  x (n doubles, HOST) receives the
 * coordinates; m (n doubles, HOST, may be NULL) the quadrature weights: the lumped mass,
 * i.e. the diagonal of the GLL mass matrix M (h for order 1), or for order -1 the Gauss
 * weights of Hermite functions 1/(n psi_{n-1}(x_j)^2).  Needs no GPU.  TS_ERR_INVALID_ARG if
 * n < 1, L <= 0, order outside [-1, 32], (n+1) % order != 0, or order -1 with n > 2048.
 */
ts_status ts_grid_nodes(int n, double L, int order, double* x, double* m);

/*
 * Step 1 of Sec. 2.1 (eq. eigen_decomp) for a symmetric tridiagonal matrix, such as the Q^1
 * operator h^-2 tridiag(-1, 2, -1) + diag f: T = Z diag(lambda) Z^T by implicit symmetric
 * QR steps with the Wilkinson shift on the host, every rotation accumulated into Z (Golub &
 * Van Loan, Sec. 8.3).  diag (n doubles), offdiag (n - 1 doubles; may be NULL for n = 1),
 * lambda_host (n doubles, receives the eigenvalues ascending) and Z_host (n x n doubles,
 * column-major: Z_host[i + n j] is component i of the unit eigenvector for lambda_j) are
 * HOST arrays owned by the caller.  ts_plan_create uses it for Q^1 axes with n <= 192.
 * Needs no GPU.  TS_ERR_INVALID_ARG for n < 1, NULL arrays or non-finite entries;
 * TS_ERR_NOT_CONVERGED after 30 n + 30 QR steps.
 */
ts_status ts_tridiag_eig(int n, const double* diag, const double* offdiag, double* lambda_host, double* Z_host);

/*
 * Step 1 of Sec. 2.1 (eq. eigen_decomp): for every axis assemble H_k = M_k^{-1} Stiff_k + F_k
 * (Q^1: h_k^-2 tridiag(-1,2,-1) + diag f_k), eigendecompose the symmetric
 * M_k^{-1/2} Stiff_k M_k^{-1/2} + F_k = Q_k Lambda_k Q_k^T in FP64 (Q^1 axes with n <= 192:
 * ts_tridiag_eig on the host; otherwise a dense solver on the GPU) (axes with
 * identical (n, L, f, order) share one decomposition) and keep T_k^{-1} = Q_k^T M_k^{1/2},
 * T_k = M_k^{-1/2} Q_k, lambda_k and, for every precision bit set in precision_mask
 * (bit p = 1u << ts_precision p; TS_FP64 is always built), their split low-precision
 * copies resident on the current device.  For Q^1, M_k = h_k I and T_k = Q_k is
 * orthogonal.  For Q^k, k >= 2, the plan also keeps the orthogonal Q_k and the banded
 * M^{-1} Stiff and M^{-1/2} Stiff M^{-1/2} that PCG and inverse iteration use.  The work
 * runs on `stream` and is complete when the call returns.  *out receives the plan; on
 * error it is set to NULL.
 */
ts_status ts_plan_create(const ts_plan_desc* desc, unsigned precision_mask, void* stream,
                         ts_plan** out);

/* Releases the plan.  NULL is accepted.  No call may be using the plan, and every kernel
 * enqueued with it must have completed (synchronise the streams that used it first): its
 * tables go back to the library's device pool, reusable at once, without a device-wide
 * synchronisation.  Tables shared with other plans stay until the last of them is gone. */
ts_status ts_plan_destroy(ts_plan* plan);

/* Copies lambda_axis (ascending, n[axis] doubles) into HOST memory lambda_host. */
ts_status ts_plan_eigs(const ts_plan* plan, int axis, double* lambda_host);

/* Copies T_axis (row-major n x n, column j = eigenvector of H_axis for lambda_j; for
 * Q^1 the orthonormal S_axis, for Q^k T = M^{-1/2} Q, M-orthonormal columns) into HOST
 * memory. */
ts_status ts_plan_eigvecs(const ts_plan* plan, int axis, double* S_host);

/* Plan geometry: *d, n[0..d-1] (n may be NULL) and *N (may be NULL). */
ts_status ts_plan_shape(const ts_plan* plan, int* d, int* n, long long* N);

/* Bytes of device memory the plan's tables hold. */
ts_status ts_plan_bytes(const ts_plan* plan, long long* bytes);

/*
 * u = (-Delta_h + V1 + sigma)^{-1} b   (steps 2-4 of Sec. 2.1; direct solve).
 * b, u: N doubles (real, FP64).  b and u may alias.  sigma must keep the operator
 * nonsingular (sigma != -lambda_min sum); the call does not check definiteness.
 * prec selects the contraction arithmetic (TS_FP64, TS_BF16X3, TS_BF16X6); a split
 * precision needs its bit in the plan's precision_mask (any n_k: its bf16 planes store each
 * pass's contracted axis in rows padded to a multiple of 8 elements).
 */
ts_status ts_apply_inverse(const ts_plan* plan, double sigma, const double* b, double* u,
                           ts_precision prec, void* stream);

/*
 * ts_apply_inverse without any device allocation (the paper has no counterpart: this is
 * a library service).  For callers that must not allocate device memory while they run,
 * e.g. an application that gives the whole device to its own allocator at start-up, or
 * a latency-critical loop that cannot pay for cudaMalloc/cudaFree (cudaFree synchronises
 * the device) or for growing a memory pool.  Same arguments and result as
 * ts_apply_inverse (prec TS_FP64, TS_BF16X1, TS_BF16X3 or TS_BF16X6, checked as there;
 * b and u may alias); the two intermediate buffers come from a fixed 32 MiB array inside
 * the library, which every GPU that loads the library holds until the process exits.
 * Limit: two buffers of N doubles (TS_FP64) or of the bf16 planes of the widest pass
 * (2, 4 or 6 bytes per value for TS_BF16X1 / X3 / X6, each pass's contracted axis padded to
 * a multiple of 8) must fit in 32 MiB: N <= 2,097,152 (FP64), 8,388,608 (BF16X1), 4,194,304
 * (BF16X3) or 2,796,202 (BF16X6) when every n_k is a multiple of 8, less otherwise; a plan
 * above it returns TS_ERR_INVALID_ARG with its own requirement in the message.  Set-up: the
 * first call in each CUDA context of a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for that context; a device whose context has been
 * replaced (e.g. after cudaDeviceReset) is looked up again.  All calls share the array
 * and it keeps the last call's contents (nothing needs to start at zero); calls that
 * overlap on the GPU (other streams or threads) race on it, so serialise them.
 */
ts_status ts_apply_inverse_noalloc(const ts_plan* plan, double sigma, const double* b, double* u,
                                   ts_precision prec, void* stream);

/*
 * The direct solve of ts_apply_inverse carried to FP64 accuracy by mixed-precision
 * iterative refinement (the split-precision inverse as preconditioner of the Richardson
 * iteration, a special case of Sec. 3.2's PCG with V2 = 0):
 *     u_0 = P b,   u_{k+1} = u_k + P (b - (-Delta_h + V1 + sigma) u_k),  k < refinements,
 * P = (-Delta_h + V1 + sigma)^{-1} applied in precision prec, residuals in FP64 by the
 * stencil of eq. general_system.  Each refinement multiplies the error by about the
 * relative error of one split-precision apply (~1e-5 for TS_BF16X3), so two refinements
 * reach FP64 rounding.  No host synchronisation.  b, u: N doubles, must not alias.
 * prec = TS_FP64 performs the plain FP64 apply (refinements ignored).
 */
/*
 * The same refinement with a precision per apply (no counterpart in the paper): schedule[0]
 * is the precision of u_0 = P b, schedule[k] that of refinement k (count = 1 + the number of
 * refinements, 1..17; split precisions only, each in the plan's mask).  The error after
 * the schedule is about the product of the applies' relative errors, so the late
 * refinements can use a coarser, cheaper inverse: {TS_BF16X3, TS_BF16X3, TS_BF16X1} takes
 * ~1.6e-5 -> ~2.5e-10 -> ~1e-12 at a third of the tensor work for the last apply.
 */
ts_status ts_solve_schedule(const ts_plan* plan, double sigma, const double* b, double* u,
                            const ts_precision* schedule, int count, void* stream);

ts_status ts_solve_refined(const ts_plan* plan, double sigma, const double* b, double* u,
                           ts_precision prec, int refinements, void* stream);

/*
 * psi_out = e^{-i tau (-Delta_h + V1)} psi_in   (exact propagator, eq. exact_prop):
 * forward transform, multiply coefficient (i_1..i_d) by e^{-i tau Lambda}, backward
 * transform.  dtype TS_C128 (2N doubles) or TS_C64 (2N floats); psi_in and psi_out may
 * alias.  prec as for ts_apply_inverse (TS_C64 data with TS_FP64 arithmetic is allowed).
 * TS_FP32 (complex64 only, every n_k in {8, 16, 24, 32}) applies the factored form
 * e^{-i tau A} = (x)_k E_k, E_k = T_k diag(e^{-i tau lambda_k}) T_k^{-1}, a few axes per
 * pass through HBM on the FFMA pipes.  TS_BF16X6 on TS_C64 data with d >= 2 and every n_k
 * in {8, 16, 24} takes the same factored form: pairs of 16- or 24-point axes on the tensor
 * cores (the real 2n x 2n embedding of E_k, three bf16 planes, six products, two axes per
 * pass), 8-point axes on the FP32 kernels (at least BF16X6's accuracy); other shapes and
 * dtypes use the transform-scale-transform passes.  The factored forms need no extra device memory
 * beyond d small E_k tables (and an FP32 copy of V2 in the split steps).
 */
ts_status ts_apply_exp(const ts_plan* plan, double tau, const void* psi_in, void* psi_out,
                       ts_dtype dtype, ts_precision prec, void* stream);

/*
 * Many independent applies in one call (no counterpart in the paper; the serving
 * subsystem's batched launch): items[q] asks for ts_apply_inverse (dtype TS_R64, param =
 * sigma) or ts_apply_exp (dtype TS_C128 / TS_C64, param = tau) of its own plan, input and
 * output, in a split precision (TS_BF16X1 / TS_BF16X3 / TS_BF16X6, in the plan's mask).
 * Instead of 2d + 1 launches per item, every stage of all items runs in one launch:
 * one input split over all items, then for each pass s one tensor-core launch per group
 * of items with the same precision and data kind, walking the tiles of all of them (a
 * work list of up to 40 (item, pass) entries per launch).  Results equal the per-item
 * calls bit for bit.  Items must not share outputs; inputs are not modified.
 */
typedef struct {
  const ts_plan* plan;
  ts_dtype dtype;      /* TS_R64: inverse; TS_C128 / TS_C64: exp                         */
  ts_precision prec;   /* split precision                                                 */
  double param;        /* sigma (inverse) or tau (exp)                                    */
  const void* in;      /* device input (N doubles, or N complex values of dtype)          */
  void* out;           /* device output, same layout                                      */
} ts_batch_item;
ts_status ts_apply_batch(const ts_batch_item* items, int count, void* stream);

/*
 * y = (-Delta_h + V1 + V2 + sigma) x (eq. general_system, zero Dirichlet ghosts).
 * V2: N doubles or NULL.  x, y: N doubles, must not alias.  Q^1: the 2d+1 point stencil;
 * for d = 3 with one spacing h on all axes (and sigma + V1 not too large against h^-2)
 * the Laplacian and sigma + V1 are summed exactly in 64-bit fixed point scaled by the
 * largest exponent of x (V2 x in FP64); otherwise in FP64.  Q^k, k >= 2: the per-axis
 * banded product with K_k = M_k^{-1} Stiff_k (bandwidth 2k + 1) in FP64.
 */
ts_status ts_apply_operator(const ts_plan* plan, double sigma, const double* V2,
                            const double* x, double* y, void* stream);

/*
 * Preconditioned CG (Sec. 3.2) for (-Delta_h + V1 + V2 + sigma) x = b with the
 * preconditioner P = (-Delta_h + V1 + sigma_P)^{-1} applied in precision `precond`.
 * The recurrence uses the flexible (Polak-Ribiere) beta = -alpha (z_{k+1}, q_k)/(z_k, r_k),
 * which equals the standard beta when P is applied exactly.  All inner products and
 * vector updates are FP64 with deterministic reductions.
 * x: in = initial guess, out = iterate.  Stops when ||r_k||_2 / ||b||_2 < tol on the
 * recurrence residual, or after maxit iterations (then TS_ERR_NOT_CONVERGED, x holds
 * the last iterate).  *iters (may be NULL) = iterations taken; *relres (may be NULL) =
 * TRUE relative residual ||b - A x|| / ||b|| recomputed at exit.  Synchronises stream.
 * Every product A x (the iteration's and the residuals at entry and exit) is formed as
 * ts_apply_operator forms it, in exact fixed point where that form applies.
 * Q^k, k >= 2: A and P are self-adjoint in the M-inner product <u, v>_M = sum M u v
 * (M = prod_k M_k, the lumped mass), not in the plain one; the iteration runs in
 * x~ = M^{1/2} x on the symmetric M^{1/2} A M^{-1/2}, so every inner product and norm
 * above is the M-weighted one (for Q^1, M = prod h_k I and the two coincide).
 */
ts_status ts_pcg(const ts_plan* plan, double sigma, double sigma_P, const double* V2,
                 const double* b, double* x, double tol, int maxit, ts_precision precond,
                 int* iters, double* relres, void* stream);

/*
 * Shifted inverse iteration (Sec. 4.1, Sec. 5.3.1) for the smallest eigenpair of
 * H = -Delta_h + V1 + V2 with shift s (H - s must be positive definite):
 *   u_0 = product of the per-axis ground eigenvectors (if init_from_plan != 0, else
 *         the caller's u), lambda_0 = (u_0, H u_0);
 *   repeat  solve (H - s) w = u_k by ts_pcg (sigma = sigma_P = -s, tolerance pcg_tol,
 *           warm start w_0 = u_k / (lambda_k - s));  u_{k+1} = w / ||w||;
 *           lambda_{k+1} = (u_{k+1}, H u_{k+1})
 *   until |lambda_{k+1} - lambda_k| / |lambda_{k+1}| < tol_lambda or maxit.
 * u: N doubles (in/out).  The sign is fixed so that sum(u) > 0.  *lambda, *outer_iters,
 * *pcg_iters may be NULL.  Synchronises stream.  Q^k, k >= 2: inner products and norms
 * are M-weighted as in ts_pcg, so the returned u has ||u||_M = 1.
 */
ts_status ts_inverse_iteration(const ts_plan* plan, double shift, const double* V2, double* u,
                               int init_from_plan, double tol_lambda, int maxit, double pcg_tol,
                               int pcg_maxit, ts_precision precond, double* lambda,
                               int* outer_iters, long long* pcg_iters, void* stream);

/*
 * uf = tensor-product linear interpolation of uc from the grid of plan `coarse` to the grid
 * of plan `fine` (Sec. 5.3.1): the same d and the same L per axis, any n and order on
 * either side; per axis each fine node takes the linear interpolant between its two
 * neighbouring coarse nodes, the walls x = -L, L carrying the Dirichlet zero.  uc, uf:
 * device arrays of the two grids' N doubles, must not alias.  Synchronises stream.
 */
ts_status ts_interpolate(const ts_plan* coarse, const double* uc, const ts_plan* fine, double* uf, void* stream);

/*
 * Multi-level shifted inverse iteration (Sec. 5.3.1, Table multilevel): ts_inverse_iteration
 * on plans[0] from the tensor product of its per-axis ground states, then on plans[1], ...
 * each from the previous level's eigenvector interpolated by ts_interpolate.  V2[l]: the
 * non-separable potential sampled on level l's grid (V2 itself or V2[l] may be NULL).
 * shift, tolerances and precond as in ts_inverse_iteration, the same for every level.
 * u: the finest grid's N doubles (out).  outer[l], pcg[l] (levels entries each, may be
 * NULL): the per-level outer and total PCG iterations.  Synchronises stream.
 */
ts_status ts_inverse_iteration_multilevel(const ts_plan* const* plans, const double* const* V2, int levels,
                                          double shift, double* u, double tol_lambda, int maxit, double pcg_tol,
                                          int pcg_maxit, ts_precision precond, double* lambda, int* outer,
                                          long long* pcg, void* stream);

/* Riemannian gradient flows of Sec. 4.2 (ts_gpe_ground_state). */
typedef enum {
  TS_GPE_H1 = 0,  /* modified H^1 flow, metric (grad w, grad z) + alpha (w, z) (eq. h1_metric)   */
  TS_GPE_AU = 1   /* a_u flow, metric (grad w, grad z) + (w, V z) + beta (w, u^2 z) (eq. au_metric) */
} ts_gpe_flow;

/*
 * Ground state of the Gross-Pitaevskii eigenproblem -Delta u + V u + beta u^3 = lambda u,
 * ||u||_L2 = 1 (eq. gpe), V = V1 + V2 (V1: the plan's separable potential; V2: N doubles on
 * the device or NULL), by the Riemannian gradient flow (eq. riemannian_update)
 *     u <- (u - tau grad) / ||u - tau grad||,  grad = G H_u u - [(u, G H_u u)/(u, G u)] G u,
 * H_u = -Delta + V + beta u^2, with L2 inner products by the grid's quadrature (h_k per axis
 * for Q^1, the GLL masses for Q^k).  TS_GPE_H1: G = (-Delta + alpha)^{-1}, two direct solves
 * per step on a plan of the same grid without potential (prec: TS_FP64, or a split
 * precision with two FP64-residual refinements).  TS_GPE_AU: G = H_u^{-1}, one PCG solve per
 * step with preconditioner (-Delta + V1)^{-1} in precision prec to relative residual
 * pcg_tol, warm-started.  u: N doubles, in = initial guess (normalised first), out = the
 * last iterate.  Stops when every criterion with a positive tolerance holds:
 * |E_k - E_{k-1}| < tol_energy |E_k| (E: the energy of eq. gpe_energy; E converges as the
 * square of the error of u) and ||H_u u - lambda u||_L2 / lambda < tol_residual (eq. gpe; this
 * one bounds the error of u and lambda); with neither positive, or after maxit steps:
 * TS_ERR_NOT_CONVERGED, outputs still written.  *energy, *lambda = (u, H_u u), *residual,
 * *iters, *solves (direct solves, or PCG iterations) may be NULL.  Synchronises stream.
 */
ts_status ts_gpe_ground_state(const ts_plan* plan, const double* V2, double beta, ts_gpe_flow flow, double alpha,
                              double tau, double* u, double tol_energy, double tol_residual, int maxit,
                              ts_precision prec, double pcg_tol, double* energy, double* lambda, double* residual,
                              int* iters, long long* solves, void* stream);

/* Splitting schemes of Sec. 5.1 (ts_propagate). */
typedef enum {
  TS_STRANG = 0,   /* e^{-i B dt/2} e^{-i A dt} e^{-i B dt/2} (M is ignored)                 */
  TS_QHOP = 1,     /* approximated qHOP, eq. qhop_product: e^{-iA dt} prod_k e^{-i w_k dt H_I(s_k)},
                      H_I(s) = e^{iAs} B e^{-iAs}, M Gauss-Legendre nodes s_k in [0, dt] with
                      weights w_k (sum 1); M = 1 runs the Strang step                       */
  TS_MAGNUS2 = 2   /* approximated Magnus-2, eq. yoshida: P(g1 dt) P(g2 dt) P(g1 dt) with P the
                      TS_QHOP step (M = 1: plain Yoshida over Strang),
                      g1 = 1/(2 - 2^{1/3}), g2 = -2^{1/3}/(2 - 2^{1/3})                       */
} ts_scheme;

/*
 * nsteps steps of size dt of `scheme` for i dpsi/dt = (A + B) psi with A = -Delta_h + V1
 * (the plan's operator, applied by the exact propagator of Sec. 2.1) and B = diag(VB)
 * (VB: N doubles on the device, e.g. V2, or V1 + V2 for a plan built with f = 0).
 * Adjacent factors are merged as in Remark cost_naive_merged (A with A by the group
 * property, B with B), also across steps and Yoshida sub-steps: qHOP costs about M
 * A-propagations per step, Magnus-2 about 3M (3 for M = 1).  psi: TS_C128 or TS_C64, in
 * place; prec: the propagator's precision (TS_FP32: fused small-n kernels, complex64).
 * 1 <= M <= 64.  *a_propagations (may be NULL) = A-propagations applied.
 */
ts_status ts_propagate(const ts_plan* plan, ts_scheme scheme, int M, double dt, int nsteps, const double* VB,
                       void* psi, ts_dtype dtype, ts_precision prec, int* a_propagations, void* stream);

/*
 * nsteps Strang steps (Sec. 5.1, Remark cost_naive_merged with M = 1) of
 * i d psi/dt = (A + B) psi, A = -Delta_h + V1 (exact propagator), B = diag(V2):
 *     psi <- e^{-i V2 dt/2} e^{-i A dt} e^{-i V2 dt/2} psi.
 * The half steps of adjacent steps are merged into one e^{-i V2 dt} factor.
 * V2: N doubles (device).  psi: TS_C128 or TS_C64, updated in place.  prec as for
 * ts_apply_exp; on the factored small-n forms (TS_FP32, and TS_BF16X6 on TS_C64 with every
 * n_k in {8, 16, 24}) the potential phases are applied inside the passes: the merged
 * e^{-i V2 dt} (e^{-i V2 dt/2} in the first step) as each step's first pass loads psi,
 * the closing e^{-i V2 dt/2} as the last step's last pass stores it.  A step then costs
 * ceil(d / 2) or ceil(d / 3) passes over psi.
 */
ts_status ts_split_step(const ts_plan* plan, double dt, int nsteps, const double* V2, void* psi,
                        ts_dtype dtype, ts_precision prec, void* stream);

/*
 * Tile configuration of the split-precision tensor-core contraction (no counterpart in
 * the paper; set by the autotuner).  For real (complex_data = 0) or complex data and a
 * contracted axis of length n (n = 0: the default for all lengths): K chunk bk (64 =
 * 128-byte swizzled rows, 32 = 64-byte), the cap bn_cap (multiple of 16, <= 256) on the
 * N tile, and `cluster`: 1 = single CTAs, each staging its whole S_k tile; TS_TC_PAIR =
 * CTA pairs that share each tensor-core instruction (tcgen05 cta_group::2: 256-row units,
 * each CTA staging its own 128 rows and half of the S_k tile; the built-in choice for real
 * data on axes of 256 points or more).  Every other cluster value returns
 * TS_ERR_INVALID_ARG: no tile is ever shared by a multicast load.  bk = bn_cap = cluster = 0
 * forgets the entry for (complex_data, n), restoring the built-in choice.  Process-wide;
 * takes effect for calls issued afterwards.
 */
#define TS_TC_PAIR (-2)
ts_status ts_tc_config_set(int complex_data, int n, int bk, int bn_cap, int cluster);

/* ------------------------------------------------------------------ serving ----- */
/*
 * Continuous-batching request server (no counterpart in the paper; it serves the paper's
 * three operations to many independent callers).  A scheduler thread admits queued
 * requests while fewer than max_inflight are on the GPU and their scratch fits
 * memory_budget_bytes.  Planner threads look each grid's plan up in a cache keyed by
 * (n_k, L_k, f_k) ahead of admission (building it on a miss, on top of the process-wide
 * per-axis eigendecomposition cache).  The scheduler captures every round of admitted
 * inverse / exp requests into
 * one CUDA graph with one stream per request (their kernels overlap), and runs PCG
 * requests (which read one scalar back per iteration) on pooled host threads with their
 * own streams.  Results are bitwise the same alone and in a mix.  in / out / V2 are
 * caller-owned device arrays that must stay valid until ts_server_wait returns.
 */
typedef enum { TS_REQ_INVERSE = 0, TS_REQ_EXP = 1, TS_REQ_PCG = 2 } ts_request_kind;

typedef struct {
  int kind;            /* ts_request_kind                                                 */
  ts_plan_desc grid;   /* grid and V1 samples (host memory, copied at submit)             */
  double sigma;        /* inverse: shift; PCG: shift of the system and of P (sigma_P)     */
  double tau;          /* exp: time                                                       */
  const double* V2;    /* PCG: N doubles on the device, or NULL                           */
  double tol;          /* PCG: relative residual tolerance                                */
  int maxit;           /* PCG: iteration cap                                              */
  const void* in;      /* device: b (inverse, PCG) or psi_in (exp)                        */
  void* out;           /* device: u, x (PCG; initial guess on entry) or psi_out           */
  ts_dtype dtype;      /* TS_R64 for inverse / PCG; TS_C128 or TS_C64 for exp             */
  ts_precision prec;   /* contraction precision (PCG: of the preconditioner)              */
} ts_request;

#define TS_SERVER_MAX_INFLIGHT 1024
typedef struct {
  long long memory_budget_bytes; /* scratch budget (<= 0: half the free device memory)   */
  int max_inflight;              /* requests on the GPU at once (<= 0: 8); each is one
                                    stream and one pooled PCG thread, so values above
                                    TS_SERVER_MAX_INFLIGHT are refused with
                                    TS_ERR_INVALID_ARG before any CUDA call             */
  int max_batch;                 /* requests per captured graph (<= 0: max_inflight)     */
  int plan_cache_entries;        /* cached plans (<= 0: 1024)                            */
  int planner_threads;           /* host threads building plans ahead of admission
                                    (<= 0: 4; above 64: 64); each build eigendecomposes the new axes on
                                    the host, so more threads help while host cores are
                                    free and hurt once they compete with the scheduler
                                    and the PCG threads                                 */
} ts_server_config;

typedef struct {
  long long completed;
  double p50_ms, p99_ms, max_ms;   /* latency from submit to completion                 */
  double makespan_ms;              /* first submit to last completion                   */
  double gdofs;                    /* sum of N over completed requests / makespan       */
  long long plan_hits, plan_misses;
  long long batches, graph_requests;
  long long peak_scratch_bytes;
} ts_serving_stats;

typedef struct ts_server ts_server;

/* Start a server on the current device. */
ts_status ts_server_create(const ts_server_config* cfg, ts_server** out);
/* Queue a request; *ticket identifies it.  Non-blocking. */
ts_status ts_server_submit(ts_server* server, const ts_request* req, long long* ticket);
/* Block until the request finishes; *result = its status (the message is in
 * ts_last_error), *latency_ms, *iterations (PCG).  Each ticket may be waited once. */
ts_status ts_server_wait(ts_server* server, long long ticket, ts_status* result, double* latency_ms,
                         int* iterations);
/* Block until every submitted request has finished. */
ts_status ts_server_drain(ts_server* server);
/* Latency percentiles, throughput, plan-cache and batching counters since the last reset. */
ts_status ts_server_stats(ts_server* server, ts_serving_stats* stats);
ts_status ts_server_reset_stats(ts_server* server);
/* Finish all queued work, then free the server, its streams and its cached plans. */
ts_status ts_server_destroy(ts_server* server);

/*
 * Autotuner of the split-precision contraction (no counterpart in the paper).  For every
 * distinct axis length n of the plan and the data kind (dtype TS_R64: real data of
 * ts_apply_inverse; TS_C128: complex data of ts_apply_exp) it times the tile
 * configurations (K chunk 64 / 32, N-tile cap 256 / 128 / 64, cluster 1 / TS_TC_PAIR) on
 * whole applies with CUDA events on `stream`, keeps the fastest with ts_tc_config_set, and appends it to the text
 * file cache_path (NULL or "" = no file).  Entries already in the file are applied without
 * timing.  *tuned (may be NULL) = number of axis lengths searched.  Synchronises stream.
 */
ts_status ts_autotune(const ts_plan* plan, ts_dtype dtype, ts_precision prec, const char* cache_path,
                      int* tuned, void* stream);

/*
 * Runtime instrumentation (no counterpart in the paper).
 * ts_launch_count: number of CUDA kernels the library has launched in this process.
 * ts_profile_begin: start recording a CUDA event pair around every launch of the
 *   contraction kernels (on the launching stream); clears earlier records.
 * ts_profile_end: stop recording and sum the records of one kernel kind
 *   (0 = split-precision tensor-core pass writing 2 or 3 bf16 planes, 1 = FP64 pass,
 *   2 = small-n fused pass, 3 = refinement residual with the exact fixed-point Laplacian,
 *   4 = tensor-core pass writing one bf16 plane, 5 = tensor-core pass writing the FP64 or
 *   complex result (the last pass of an apply, any plane count), 6 = work-list tensor-core
 *   pass of a batched apply; launches captured into a CUDA graph are not recorded):
 *   launches, total device time in ms, algorithmic FLOPs and algorithmic HBM bytes.
 *   Synchronises on the recorded events.  Any pointer may be NULL.
 */
long long ts_launch_count(void);
ts_status ts_profile_begin(void);
ts_status ts_profile_end(int kind, long long* launches, double* total_ms, double* flops, double* bytes);

/*
 * Device-side failure check (no counterpart in the paper).  The tensor-core kernels never
 * wait without a bound: a wait that runs out (about 2 s) sets a device flag and the kernel
 * returns.  This call synchronises `stream`, returns TS_ERR_TIMEOUT if the flag was set
 * since the previous call (and clears it), else TS_OK.
 */
ts_status ts_device_status(void* stream);

/*
 * Self-test of the failure path above (no counterpart in the paper): launches one thread
 * that waits, with the same bounded wait as the tensor-core kernels, on a barrier that
 * nothing arrives on.  After `cycles` clock cycles (0 < cycles <= 4e9) the wait gives up,
 * sets the device flag and the kernel returns; the next ts_device_status reports
 * TS_ERR_TIMEOUT and the context stays usable.
 */
ts_status ts_selftest_wait_timeout(long long cycles, void* stream);

/* Thread-local message of the calling thread's last failing call ("" if none). */
const char* ts_last_error(void);

/* Library build string (compile flags, architecture). */
const char* ts_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TSCHROD_H */
