// Stage kernels of the ES-BGK library with f stored as __nv_bfloat16 whose moment sums
// follow the run-time parameter (compensated sums requested).
#include "kernels_impl.cuh"

namespace esbgk {
StageFnT stage_fn_runtime_sums(const __nv_bfloat16*, int m, int var) {
  return Launch<__nv_bfloat16>::stage_fn_sums<kSumsRunTime>(m, var);
}
BatchFnT batch_fn_runtime_sums(const __nv_bfloat16*, int m, int var) {
  return Launch<__nv_bfloat16>::batch_fn_sums<kSumsRunTime>(m, var);
}
}  // namespace esbgk
