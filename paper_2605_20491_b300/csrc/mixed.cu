// Split-precision apply on the tensor cores (placeholder until the tcgen05 path lands).
#include "mixed.cuh"

namespace ts {

int bf16_planes(ts_precision prec) {
  if (prec == TS_BF16X3) return 2;
  if (prec == TS_BF16X6) return 3;
  return 0;
}

ts_status build_split_tables(ts_plan*, ts_precision prec, cudaStream_t) {
  set_error("precision %d is not available in this build", (int)prec);
  return TS_ERR_UNSUPPORTED;
}

ts_status mixed_apply(const ts_plan*, ts_precision prec, MixedOp, double, const void*, void*, ts_dtype,
                      cudaStream_t) {
  set_error("precision %d is not available in this build", (int)prec);
  return TS_ERR_UNSUPPORTED;
}

}  // namespace ts
