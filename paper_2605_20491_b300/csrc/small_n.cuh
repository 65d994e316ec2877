// FP32 fused multi-mode path for small axis lengths (complex64): see small_n.cu.
#pragma once
#include "common.cuh"

namespace ts {

// True when every n_k is one of the lengths the fused kernel is instantiated for.
bool small_n_supported(const ts_plan* p);
// FP32 copies of S_k and S_k^T (plan creation, precision TS_FP32).
ts_status build_small_tables(ts_plan* p, cudaStream_t s);
// out = e^{-i tau (-Delta+V1)} in (V2 == NULL, nsteps = 1), or nsteps Strang steps of
// length dt (V2 != NULL; tau must equal dt) from in to out (in may equal out).
ts_status small_n_propagate(const ts_plan* p, double tau, const float2* in, float2* out, const double* V2, double dt,
                            int nsteps, cudaStream_t s);

}  // namespace ts
