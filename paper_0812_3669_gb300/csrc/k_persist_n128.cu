// Instantiation of the persistent imaging kernel (batching pattern) for a 128x128 grid.
#include "moff_image_kernels.cuh"

namespace moff {
MOFF_DEFINE_PERSIST_N(128)
}  // namespace moff
