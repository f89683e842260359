// Kernels of the ES-BGK library with f stored as double.
#include "kernels_impl.cuh"

namespace esbgk {
ESBGK_INSTANTIATE(double, kLaunchF64)
}  // namespace esbgk
