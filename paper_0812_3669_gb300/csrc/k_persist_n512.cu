// Instantiation of the persistent imaging kernel (batching pattern) for a 512x512 grid.
#include "moff_image_kernels.cuh"

namespace moff {
MOFF_DEFINE_PERSIST_N(512)
}  // namespace moff
