// Instantiation of the persistent imaging kernel (batching pattern) for a 64x64 grid.
#include "moff_image_kernels.cuh"

namespace moff {
MOFF_DEFINE_PERSIST_N(64)
}  // namespace moff
