// Kernels of the ES-BGK library with f stored as float.
#include "kernels_impl.cuh"

namespace esbgk {
ESBGK_INSTANTIATE(float, kLaunchF32)
}  // namespace esbgk
