// Instantiation of the imaging kernels for a 32x32 grid (one unit per size so
// the sizes compile in parallel).
#include "moff_image_kernels.cuh"

namespace moff {
MOFF_DEFINE_N(32)
}  // namespace moff
