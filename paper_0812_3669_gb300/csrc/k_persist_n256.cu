// Instantiation of the persistent imaging kernel (batching pattern) for a 256x256 grid.
#include "moff_image_kernels.cuh"

namespace moff {
MOFF_DEFINE_PERSIST_N(256)
}  // namespace moff
