// Split-precision (tensor-core) apply: see mixed.cu.
#pragma once
#include "common.cuh"

namespace ts {

enum class MixedOp { Inverse = 0, Exp = 1 };

// Number of bf16 planes per value for a split precision (0 if not a bf16 split).
int bf16_planes(ts_precision prec);
// Elements of one bf16 plane of the split-precision passes: the grid with the contracted
// (fastest) axis of each pass padded to a multiple of 8, maximised over the passes.
long long mixed_plane_elems(const ts_plan* p);

// Mixed-precision apply: op Inverse (real FP64 in/out, param = sigma) or Exp (complex
// in/out of dtype dt, param = tau).
ts_status mixed_apply(const ts_plan* p, ts_precision prec, MixedOp op, double param, const void* in, void* out,
                      ts_dtype dt, cudaStream_t s);

// Many independent split-precision applies; every stage of all of them runs in one launch
// (work-list tensor-core passes).
struct BatchApply {
  const ts_plan* p;
  ts_precision prec;
  MixedOp op;
  double param;  // sigma (Inverse) or tau (Exp)
  const void* in;
  void* out;
  ts_dtype dt;
};
ts_status mixed_apply_batch(const BatchApply* q, int count, cudaStream_t s);

// Split-precision inverse apply with caller-provided plane buffers w0, w1 of
// bf16_planes(prec) * mixed_plane_elems(p) bf16 each (no allocation).
ts_status mixed_inverse_buffers(const ts_plan* p, ts_precision prec, double sigma, const double* b, double* u,
                                __nv_bfloat16* w0, __nv_bfloat16* w1, cudaStream_t s);

// Mixed-precision iterative refinement of the direct solve: u_0 = P b,
// u_{k+1} = u_k + P (b - A u_k), P the split-precision inverse, residuals in FP64.
ts_status mixed_refine(const ts_plan* p, ts_precision prec, double sigma, const double* b, double* u,
                       int refinements, cudaStream_t s);
// The same with a precision per apply: sched[0] for u_0, sched[k] for refinement k.
ts_status mixed_solve_schedule(const ts_plan* p, const ts_precision* sched, int count, double sigma,
                               const double* b, double* u, cudaStream_t s);

// Reads (and optionally clears) the flag that bounded device-side waits of the
// tensor-core kernels set when they time out.  Synchronises s.
ts_status mixed_error_flag(int* host_flag, bool reset, cudaStream_t s);

// Opt every tensor-core kernel instantiation into its shared-memory size (call before
// capturing launches into a graph).
ts_status tc_prepare_kernels();

// Tile configuration of the tensor-core pass for data of the given kind and contracted
// extent n (n = 0: default for every n): K chunk bk (64 or 32), N-tile cap bn_cap and the
// cluster size sharing each B tile by multicast (1, 2, 4).
ts_status tc_config_set(int complex_data, int n, int bk, int bn_cap, int cluster);

// Self-test of the bounded device wait: a kernel waits `cycles` clocks on a barrier that
// nothing arrives on, then records a timeout in the device flag and returns.
ts_status wait_selftest(long long cycles, cudaStream_t s);

// Build the split planes of S_k^T and S_k for precision `prec` (plan creation).
ts_status build_split_tables(ts_plan* p, ts_precision prec, cudaStream_t s);

}  // namespace ts
