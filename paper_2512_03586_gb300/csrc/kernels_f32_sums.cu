// Stage kernels of the ES-BGK library with f stored as float whose moment sums
// follow the run-time parameter (compensated sums requested).
#include "kernels_impl.cuh"

namespace esbgk {
StageFnT stage_fn_runtime_sums(const float*, int m, int var) {
  return Launch<float>::stage_fn_sums<kSumsRunTime>(m, var);
}
BatchFnT batch_fn_runtime_sums(const float*, int m, int var) {
  return Launch<float>::batch_fn_sums<kSumsRunTime>(m, var);
}
}  // namespace esbgk
