// Instantiation of the imaging kernels for a 128x128 grid (one unit per size so
// the sizes compile in parallel).
#include "moff_image_kernels.cuh"

namespace moff {
MOFF_DEFINE_N(128)
}  // namespace moff
