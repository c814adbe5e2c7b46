// Instantiation of the persistent imaging kernel (batching pattern) for a 32x32 grid.
#include "moff_image_kernels.cuh"

namespace moff {
MOFF_DEFINE_PERSIST_N(32)
}  // namespace moff
