// FP32 fused multi-mode path for small axis lengths (complex64): see small_n.cu.
#pragma once
#include "common.cuh"

namespace ts {

// True when the tensor-core small-n pass serves the plan's complex64 propagation in
// TS_BF16X6: d >= 2 axes, each of length 8, 16 or 24.  Groups of two equal axes of 16 or 24
// whose tile dimension divides by 16 take the tensor-core kernel; the others, and every
// group of 8-point axes, take the FP32 FFMA kernels (at least as accurate; on 8-point axes
// also the faster: a three-axis tensor-core form was latency-bound, 3.7 against 2.8 ms per
// 9D Strang step).
bool small_tc_applicable(const ts_plan* p);
// True when every n_k is one of the lengths the fused kernel is instantiated for.
bool small_n_supported(const ts_plan* p);
// FP32 copies of S_k and S_k^T (plan creation, precision TS_FP32).
ts_status build_small_tables(ts_plan* p, cudaStream_t s);
// out = e^{-i tau (-Delta+V1)} in (V2 == NULL, nsteps = 1), or nsteps Strang steps of
// length dt (V2 != NULL; tau must equal dt) from in to out (in may equal out).
// tensor = true: groups of two 16- or 24-point axes run on the tensor cores (bf16x6
// products, FP32 accumulation: precision TS_BF16X6), the others on the FP32 kernels.
ts_status small_n_propagate(const ts_plan* p, double tau, const float2* in, float2* out, const double* V2, double dt,
                            int nsteps, cudaStream_t s, bool tensor = false);
// Reads (and optionally clears) the flag set when a bounded wait of the tensor-core small-n
// pass runs out.  Synchronises s.
ts_status small_n_error_flag(int* host_flag, bool reset, cudaStream_t s);

}  // namespace ts
