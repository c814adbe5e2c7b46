// Instantiation of the gridding kernel with the tensor-core row transform for a
// 256x256 grid (one unit per size so the sizes compile in parallel).
#include "moff_image_kernels.cuh"

namespace moff {
namespace {

template <int P, int TB, int CPL>
cudaError_t launch_t(const GridArgs &a, int n_stripes, size_t smem, cudaStream_t st) {
    // 2 x 2 cell blocks need an even stripe height
    if constexpr (CPL == 4 && GridShape<256, P, TB, false>::ROWS % 2 != 0) {
        return cudaErrorInvalidValue;
    } else {
        auto k = k_grid_rows_dft<256, P, TB, CPL>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<dim3(n_stripes, a.nc), kBlock, smem, st>>>(a);
        return cudaGetLastError();
    }
}

template <int P, int CPL>
cudaError_t launch_c(int TB, const GridArgs &a, int n_stripes, size_t smem, cudaStream_t st) {
    switch (TB) {
        case 1: return launch_t<P, 1, CPL>(a, n_stripes, smem, st);
        case 2: return launch_t<P, 2, CPL>(a, n_stripes, smem, st);
        case 4: return launch_t<P, 4, CPL>(a, n_stripes, smem, st);
        case 8: return launch_t<P, 8, CPL>(a, n_stripes, smem, st);
    }
    return cudaErrorInvalidValue;
}

template <int P>
cudaError_t launch_p(int TB, int CPL, const GridArgs &a, int n_stripes, size_t smem, cudaStream_t st) {
    switch (CPL) {
        case 1: return launch_c<P, 1>(TB, a, n_stripes, smem, st);
        case 2: return launch_c<P, 2>(TB, a, n_stripes, smem, st);
        case 4: return launch_c<P, 4>(TB, a, n_stripes, smem, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_grid_dft_n256(int P, int TB, int CPL, const GridArgs &a, int n_stripes, size_t smem,
                                   cudaStream_t st) {
    return P == 1 ? launch_p<1>(TB, CPL, a, n_stripes, smem, st) : launch_p<2>(TB, CPL, a, n_stripes, smem, st);
}

}  // namespace moff
