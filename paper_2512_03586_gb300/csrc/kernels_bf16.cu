// Kernels of the ES-BGK library with f stored as __nv_bfloat16.
#include "kernels_impl.cuh"

namespace esbgk {
ESBGK_INSTANTIATE(__nv_bfloat16, kLaunchBF16)
}  // namespace esbgk
