// moff_internal.h -- argument blocks and launchers shared by the host code
// (moff_api.cu) and the kernel translation units.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/moff.h"

namespace moff {

constexpr int kBlock = 256;   // threads per CTA of every imaging kernel
constexpr int kPfbGroup = 32; // antenna-pols per F-stage CTA

// Gridding + row transform (Eq. m6 steps 1-3, first axis).  One CTA owns
// one stripe of `rows` grid rows of one channel and walks `nt` samples.
struct GridArgs {
    const uint8_t *volt;      // voltages; sample t of channel c at volt + t*volt_tstride + c*A*P
    long long volt_tstride;   // bytes between consecutive samples
    int t0, nt;               // first sample and sample count of this launch
    int c0, nc;               // first channel and channel count of this launch
    int A;                    // antennas
    int rows;                 // grid rows per stripe
    int max_nloc, max_ncon;   // per-stripe maxima (shared-memory carve)
    const float2 *gains;      // [C][A][P]
    const int *st_ant_off;    // [n_stripes + 1]
    const int *st_ant;        // antennas touching each stripe
    const int *st_cell_off;   // [n_stripes][P*rows*N + 1] contribution offsets per cell
    const long long *st_con_off; // [n_stripes + 1]
    const float2 *con_tap;    // kernel value of each contribution
    const uint16_t *con_y;    // local voltage index (local antenna * P + input pol)
    const float2 *twp;        // pass twiddles of the N-point transform
    float2 *out;              // [nt][nc][P][N][N] row-transformed (or raw, grid-only) field
};

// Column transform + square-and-integrate (Eq. m6 steps 3-4, second axis).
struct ColArgs {
    const float2 *H;          // [nt][nc][P][N][N]
    int nt, c0, nc;
    const float2 *twp;
    double *acc;              // [C][n_prod][N][N] FP64 accumulators (added to)
};

// Polyphase F-stage (Eq. FFTofE).
struct PfbArgs {
    const int8_t *adc;        // [AP][S]
    long long S;              // samples per stream
    int AP;                   // antenna-pol streams
    int F;                    // frames
    int ntaps;
    const float *h;           // [ntaps * M]
    float scale;
    const float2 *twp;        // pass twiddles of the C-point complex transform (sign applied in-kernel)
    const float2 *twM;        // exp(-2 pi i k / M), k < C
    int out_kind;             // 0 codes, 1 spectra
    uint8_t *codes;           // [F][C][AP]
    float2 *spec;             // [F][C][AP]
};

// Shared-memory bytes of the gridding kernel (host and device agree on the carve).
inline size_t grid_smem_bytes(int N, int P, int rows, int max_nloc, int max_ncon, bool csmem, int tw_total) {
    const int ldr = N + N / 16;
    const size_t nf = (size_t)P * rows;
    size_t b = 0;
    b += (size_t)tw_total * 8;
    b += 2 * nf * ldr * 8;                    // ping-pong row buffers
    b += (size_t)max_nloc * P * 8 * 2;        // calibrated voltages + gains
    if (csmem) b += (size_t)max_ncon * 8;     // contribution kernel values
    b += (size_t)(nf * N + 1) * 4;            // cell offsets
    b += (size_t)max_nloc * 4;                // antenna indices
    if (csmem) b += (size_t)max_ncon * 2;     // contribution voltage indices
    return (b + 15) & ~(size_t)15;
}

// Kernel binning of one array (host side): per grid-row stripe, the antennas
// touching it and each cell's kernel contributions in a fixed order.
struct Bins {
    int rows = 0, n_stripes = 0, max_nloc = 0, max_ncon = 0;
    bool csmem = false;
    size_t grid_smem = 0;
    std::vector<int> ant_off, ant_list, cell_off;
    std::vector<long long> con_off;
    std::vector<float2> con_tap;
    std::vector<uint16_t> con_y;
};
moff_status build_bins(int A, int K, int N, int P, bool jones, const double *pos, const float *taps, Bins *b);
std::vector<float2> pass_twiddles_for(int n);   // pass-twiddle table of the n-point transform (FP64-built)
moff_status fail_msg(moff_status s, const char *msg);

int fft_tw_total(int n);                      // pass-twiddle table length for length n
int col_width(int N);                         // columns per column-kernel CTA
size_t col_smem_bytes(int N, int P);
size_t pfb_smem_bytes(int CN);

// Launchers (return the launch error, if any).
cudaError_t launch_grid(int N, int P, bool csmem, bool grid_only, const GridArgs &a, int n_stripes,
                        size_t smem, cudaStream_t st);
cudaError_t launch_cols(int N, int P, const ColArgs &a, cudaStream_t st);
cudaError_t launch_pfb(int CN, const PfbArgs &a, cudaStream_t st);
cudaError_t launch_to_f32(const double *acc, float *out, long long n, cudaStream_t st);

// Per-N instantiations (one translation unit each, compiled in parallel).
#define MOFF_DECLARE_N(NN)                                                                          \
    cudaError_t launch_grid_n##NN(int P, bool csmem, bool grid_only, const GridArgs &a, int n_stripes, \
                                  size_t smem, cudaStream_t st);                                   \
    cudaError_t launch_cols_n##NN(int P, const ColArgs &a, cudaStream_t st);
MOFF_DECLARE_N(32)
MOFF_DECLARE_N(64)
MOFF_DECLARE_N(128)
MOFF_DECLARE_N(256)
MOFF_DECLARE_N(512)
#undef MOFF_DECLARE_N

}  // namespace moff
