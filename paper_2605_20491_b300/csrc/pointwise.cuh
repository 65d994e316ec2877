// Declarations of the pointwise / reduction kernels in pointwise.cu.
#pragma once
#include "common.cuh"

namespace ts {

// Fixed reduction grid: 148 SMs x 4 CTAs of 256 threads.  Partial buffers hold
// 2 doubles per CTA.
constexpr int RED_BLOCKS = 148 * 4;
int red_blocks();

// y = (A + V2 + sigma) x; if out2 != NULL, out2[0] = x.y (partials in `partial`).
ts_status stencil_apply(const ts_plan* p, const double* V2, double sigma, const double* x, double* y,
                        double* partial, double* out2, cudaStream_t s);
// r = b - (A + V2 + sigma) x; out2[0] = r.r, out2[1] = b.b.
ts_status stencil_residual(const ts_plan* p, const double* V2, double sigma, const double* x, const double* b,
                           double* r, double* partial, double* out2, cudaStream_t s);
// planes (np bf16 planes of N values) = split(b - (A + V2 + sigma) x); partial sums only.
ts_status stencil_residual_split(const ts_plan* p, const double* V2, double sigma, const double* x,
                                 const double* b, __nv_bfloat16* planes, int np, double* partial, cudaStream_t s);
// Q^k plans (k >= 2): the three functions above evaluate the banded operator
// sum_k K_k + V1 + V2 + sigma of the plan's frame instead of the stencil.
// y = x * prod_k M_k^{1/2} (inverse: M_k^{-1/2}) for a Q^k plan; x and y may alias.
ts_status scale_separable(const ts_plan* p, bool inverse, const double* x, double* y, cudaStream_t s);
// Weighted inner products of the L2 quadrature (W = prod_k M_k: GLL masses for Q^k, h_k for
// Q^1): out2[0] = sum W a b, out2[1] = sum W c d (c, d may be NULL -> 0).
ts_status wdot2(const ts_plan* p, const double* a, const double* b, const double* c, const double* d,
                double* partial, double* out2, cudaStream_t s);
// out2[0] = sum W u Hu, out2[1] = sum W u^4.
ts_status wdot_energy(const ts_plan* p, const double* u, const double* Hu, double* partial, double* out2,
                      cudaStream_t s);
// uf (fine grid pf) = tensor-product linear interpolation of uc (coarse grid pc, same d and
// box), the walls carrying the Dirichlet zero.  Synchronises s.
ts_status interpolate(const ts_plan* pc, const double* uc, const ts_plan* pf, double* uf, cudaStream_t s);
// out2[0] = sum W (Hu - lambda u)^2.
ts_status wdot_residual(const ts_plan* p, const double* u, const double* Hu, double lambda, double* partial,
                        double* out2, cudaStream_t s);
// veff = V2 + beta u^2 (V2 may be NULL).
ts_status gpe_veff(long long N, const double* V2, double beta, const double* u, double* veff, cudaStream_t s);
// u += a x + b y.
ts_status axpy2(long long N, double* u, double a, const double* x, double b, const double* y, cudaStream_t s);
// True when every axis has the same grid spacing h (never for Q^k, k >= 2).
bool isotropic_h(const ts_plan* p);
// As stencil_residual_split without V2, for isotropic grids: the Laplacian part in exact
// 64-bit fixed point, scaled by *emax_dev, which must hold the largest biased exponent of
// the values of x (a larger value is safe and costs precision; a smaller one overflows).
// qtab (may be NULL): qtable_count(p) int64 of device scratch; when given (d = 3), the
// diagonal (sigma + V1) x is folded into the exact fixed-point sum too, leaving one FP64
// instruction per point, unless sigma + V1 is too large against h^-2 for 53 bits of headroom.
ts_status residual_split_fixed(const ts_plan* p, double sigma, const double* x, const double* b,
                               __nv_bfloat16* planes, int np, const int* emax_dev, long long* qtab, cudaStream_t s);
int qtable_count(const ts_plan* p);

// The operator apply of PCG in exact fixed point (d = 3, one spacing): y = A x with the
// Laplacian and sigma + V1 folded into the integer sum and V2 x in FP64, plus x.y into
// out2[0] (fixed-order reduction over `blocks` partials; partial holds 2 * blocks doubles).
// *emax_dev must hold the largest biased exponent of x.  fixed_operator_prepare fills the
// Q tables for sigma (qtab: qtable_count(p) int64) and leaves ok = false when the form does
// not apply (then use stencil_apply).
// y = A x for any plan: the exact fixed-point form where it applies (a max-exponent pass
// over x first), else the FP64 stencil.
ts_status operator_apply(const ts_plan* p, const double* V2, double sigma, const double* x, double* y,
                         cudaStream_t s);
struct FixedOperator {
  bool ok = false;
  int H = 0, F = 0;
  double sigma = 0.0;
  const long long* qtab = nullptr;
  long long blocks = 0;
};
ts_status fixed_operator_prepare(const ts_plan* p, double sigma, long long* qtab, FixedOperator* fo, cudaStream_t s);
ts_status operator_apply_fixed(const ts_plan* p, const FixedOperator& fo, const double* V2, const double* x, double* y,
                               const int* emax_dev, double* partial, double* out2, cudaStream_t s);
// *emax = the largest biased exponent over x (reset first).
ts_status max_exponent(const double* x, long long N, int* emax, cudaStream_t s);
// r = b - A x through the fixed-point operator (its exponent pass included), with
// out2[0] = r.r and out2[1] = b.b; opart holds 2 * fo.blocks doubles, partial
// 2 * RED_BLOCKS.  The same quantities as stencil_residual, with A x exact.
ts_status residual_fixed(const ts_plan* p, const FixedOperator& fo, const double* V2, const double* x,
                         const double* b, double* r, int* emax, double* opart, double* partial, double* out2,
                         cudaStream_t s);
// out2[0] = a.b (b == NULL: sum of a), out2[1] = c.d (c, d may be NULL).
ts_status dot2(long long N, const double* a, const double* b, const double* c, const double* d, double* partial,
               double* out2, cudaStream_t s);
// alpha = rz/pq (-> *alpha_out); x += alpha p; r -= alpha q; out2[0] = r.r.
ts_status pcg_update_xr(const double* rz, const double* pq, double* alpha_out, double* x, double* r,
                        const double* p, const double* q, long long N, double* partial, double* out2,
                        cudaStream_t s);
// p = z + beta p, beta = -alpha zq / rz_old (first: p = z).
ts_status pcg_update_p(const double* alpha, const double* zq, const double* rz_old, int first, double* p,
                       const double* z, long long N, cudaStream_t s, int* emax_out = nullptr);
ts_status copy_scalar(const double* src, double* dst, cudaStream_t s);
// u = tensor product of the per-axis ground eigenvectors (column 0 of each S_k).
ts_status tensor_ground(const ts_plan* p, double* u, cudaStream_t s);
// y = a x + b y (x may alias y).
ts_status axpby(long long N, double a, const double* x, double b, double* y, cudaStream_t s);
// y = x * num/den (den != NULL) or y = x / sqrt(num) (den == NULL); num, den device scalars.
ts_status scale_by_device_ratio(long long N, const double* num, const double* den, const double* x, double* y,
                                cudaStream_t s);

}  // namespace ts
