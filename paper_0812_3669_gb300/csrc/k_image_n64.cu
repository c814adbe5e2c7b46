// Instantiation of the imaging kernels for a 64x64 grid (one unit per size so
// the sizes compile in parallel).
#include "moff_image_kernels.cuh"

namespace moff {
MOFF_DEFINE_N(64)
}  // namespace moff
