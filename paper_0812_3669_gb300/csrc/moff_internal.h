// moff_internal.h -- argument blocks and launchers shared by the host code
// (moff_api.cu) and the kernel translation units.  Not part of the C ABI.
#pragma once
#include <cuda.h>   // CUtensorMap (type only; encoded through the runtime's driver entry point)
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/moff.h"

namespace moff {

constexpr int kBlock = 256;   // threads per CTA of every imaging kernel
constexpr int kPfbGroup = 32; // antenna-pols per F-stage CTA
constexpr int kMaxBeams = 16; // tied-array beam pixels per plan

// Gridding + row transform (Eq. m6 steps 1-3, first axis).  One CTA owns
// one stripe of `rows` grid rows of one channel and walks `nt` samples, TB at
// a time.  Kernel contributions are stored per stripe in 32-cell slices
// (sliced ELL): entry i of lane l of a slice sits at slice_off + 32 i + l, so
// a warp reads 32 consecutive entries per step.
struct GridArgs {
    const uint8_t *volt;      // voltages; sample t of channel c at volt + t*volt_tstride + c*A*P
    long long volt_tstride;   // bytes between consecutive samples
    int t0, nt;               // first sample and sample count of this launch
    int c0, nc;               // first channel and channel count of this launch
    int A;                    // antennas
    int rows;                 // grid rows per stripe
    int max_nloc;             // most antennas touching one stripe (shared-memory carve)
    int max_entries;          // most sliced-ELL entries of one stripe (shared-memory carve, if staged)
    int n_slices;             // 32-cell slices per stripe = P*rows*N/32
    const float2 *gains;      // [C][A][P]
    const int *st_ant_off;    // [n_stripes + 1]
    const int *st_ant;        // antennas touching each stripe, ascending
    const long long *slice_off; // [n_stripes * n_slices + 1] first entry of each slice
    const uint16_t *lane_cell;  // [n_stripes * n_slices * 32] stripe cell of each lane
    const float2 *con_tap;    // kernel value of each entry (0 for padding)
    const uint16_t *con_y;    // local voltage index (local antenna * P + input pol)
    const float2 *twp;        // pass twiddles of the N-point transform
    float2 *out;              // row-transformed (or raw, grid-only) field: slab [P][N][N] of
                              // (sample t, channel cl) at index t * slab_t + cl * slab_c
    long long slab_t, slab_c;
    int pairs;                // 1: each lane sums two horizontally adjacent cells (entries carry two taps)
    int quads;                // 1: each lane sums a 2 x 2 block of cells (entries carry four taps; pairs ignored)
    int wide;                 // 1: twice grid_fft_rows(N) rows per pass
    // Grid rows any kernel footprint reaches (bit ry of word ry / 32, every set of positions and
    // kernels).  With it, a stripe none of whose rows is set writes nothing: the column kernel
    // reads only the set rows.  nullptr: every stripe is written.
    const uint32_t *row_nz;
    // Channel-dependent positions and kernels: chan_group[c] (absolute channel) picks one of
    // several sets; set g's stripe arrays start at st_ant_off + g (n_stripes + 1), slice_off +
    // g (n_stripes n_slices + 1) and lane_cell + g n_stripes n_slices 32, and their values
    // already index the shared st_ant / con_tap / con_y.  nullptr: one set.
    const int *chan_group;
    // Dense tensor-core transform (k_grid_rows_dft): the row-transformed field as FP16 rows
    // [re N][im N] (slab [P][N] rows of 2N halves at index t * slab_t + cl * slab_c), scaled by
    // sy[c] * s_t (powers of two) / N; dft_tab the factored-DFT table image; err set when an
    // MMA does not complete within its wait limit.
    __half *h16;
    const float *sy;
    float s_t;
    const unsigned char *dft_tab;
    int *err;
};

// Dense tensor-core column transform + square-and-integrate (k_cols_dft).
struct ColDftArgs {
    const __half *H;          // FP16 rows [re N][im N]; slab [P][N] at t * slab_t + cl * slab_c
    long long slab_t, slab_c;
    int nt, c0, nc;
    double *acc;              // [C][n_prod][N][N] FP64 accumulators (added to)
    const uint32_t *row_nz;   // rows to read (bit ry); other rows are zero
    const float *sy;          // per-channel voltage scale; the field carries sy[c] * s_t / N
    float s_t;
    const unsigned char *dft_tab;
    int *err;
};

// Dense tensor-core row transform of a gridded field in global memory (k_rows_dft).
struct RowDftArgs {
    const __half *G;          // FP16 gridded field, tile-major [Cb][P][N/8][N/8][Tb][8 cy][re/im][8 cx]
    int Tb;
    __half *H;                // FP16 row-transformed rows [re N][im N]; slab [P][N] at t * slab_t + cl * slab_c;
                              // the value carries 1/N more than the field
    long long slab_t, slab_c;
    int nt, c0, nc;
    const uint32_t *row_nz;   // stripes with no reached row are skipped
    const unsigned char *active;   // [N/8][N/8] 8x8 cell tiles the gridding writes (others zero)
    const unsigned char *dft_tab;
    int *err;
};

// Tensor-core gridding of dense arrays (k_grid_tc, moff_gridtc.cu): per tile of 8 x 8 cells a
// product of the tile's antenna voltages (FP16 planes, raster order of anchors) with the
// tile's kernel values.
struct GridTcArgs {
    int P, N, nt, nc, c0, AP, kp_max;   // AP: plane rows per channel (voltages + kRowSpecPad)
    int stages;                // depth of the A ring (gridtc_stages)
    int boxes;                 // epilogue boxes per warp (1, or 2: a box is filled while the other is stored)
    const int *tile_cell;      // [tiles] (ty << 16) | tx: cells 8 ty .. 8 ty + 7, 8 tx .. 8 tx + 7
    const int *kp;             // [tiles] contraction length (32 per chunk of 16 plane rows)
    const int *chunk_off;      // [tiles + 1]
    const int *chunk_row;      // first plane row (within a channel) of each chunk
    const long long *bimg_off; // [tiles] byte offset of each tile's B image [2 P 64][kp] K-major
    const __half *bimg;
    __half *G;                 // FP16 gridded field, tile-major: [Cb][P][N/8][N/8][Tb][8 cy][re/im][8 cx]
    int Tb;                    // samples per (pol, tile) block of G
    int *err;
};
struct GridTc {
    int kp_max = 0;
    int n_rows = 0;                             // voltage-plane rows per channel (antenna-pols, with copies)
    std::vector<int> perm;                      // [n_rows] plane row -> voltage index (anchor rows ascending, each
                                                // by column, then copies of its first columns; pols interleaved)
    std::vector<int> tile_cell, kp, chunk_off, chunk_row;
    std::vector<long long> bimg_off;
    std::vector<__half> bimg;
    std::vector<unsigned char> active;          // [N/8][N/8]
};
moff_status build_gridtc(int A, int K, int N, int P, bool jones, const double *pos, const float *taps, float scale,
                         GridTc *gt);
size_t gridtc_smem_bytes(int P, int kp_max, int stages, int boxes);
int gridtc_stages(int P, int kp_max, int boxes);
cudaError_t launch_grid_tc(const GridTcArgs &a, const CUtensorMap &are, const CUtensorMap &aim, const CUtensorMap &gmap,
                           int n_tiles, int cgroups, size_t smem, cudaStream_t st);
// Store map of the tile-major gridded field (rows of 128 halves; box 64 x 32, 128-byte swizzle).
cudaError_t encode_gridtc_store_map(CUtensorMap *map, void *G, long long rows);
cudaError_t launch_rows_dft(int N, int P, const RowDftArgs &a, cudaStream_t st);
// The N = 512 row transform as 8 x 64 with the second stage transposed (its own table image).
cudaError_t launch_rows_dft8(int P, const RowDftArgs &a, cudaStream_t st);
std::vector<unsigned char> build_rows8_table();

// Column transform + square-and-integrate (Eq. m6 steps 3-4, second axis).
struct ColArgs {
    const float2 *H;          // FP32 field, or (fp16 path) half2: slab [P][N][N] of (sample t,
                              // channel cl) at index t * slab_t + cl * slab_c
    long long slab_t, slab_c;
    int nt, c0, nc;
    const float2 *twp;
    double *acc;              // [C][n_prod][N][N] FP64 accumulators (added to)
    const uint32_t *row_nz;   // rows to read (bit ry); other rows are zero (nullptr: read all)
    // FP16 field only: value = half2 * row_inv[p*N + ry] * inv_sw / sy[c]
    const float *row_inv;
    const float *sy;
    float inv_sw;
    // feedback calibration: E_t,p(tap_kx, tap_ky) -> etap[t][cl][p] (null: off)
    float2 *etap;
    int tap_kx, tap_ky;
    // tied-array beams: E_t,p at n_beam pixels -> beam_out[beam_t0 + t][c0 + cl][j][p]
    float2 *beam_out;
    int beam_t0, beam_C, n_beam;
    int beam_kx[kMaxBeams], beam_ky[kMaxBeams];
};

// Batching pattern: one persistent launch over every (Tb, Cb) chunk of a block (k_image_persist;
// the work-item queue, the dependencies and the bounded waits are described there).
constexpr int kPersistMaxChunks = 128;
struct PersistArgs {
    GridArgs g;              // chunk-independent gridding arguments (t0 / nt / c0 / nc set per chunk)
    ColArgs ca;              // chunk-independent column arguments
    int n_chunks, n_items;
    int n_stripes, n_strips; // row items and column items per channel of a chunk
    int cb;                  // channel slots per chunk (the counters' row length)
    int rows_extra;          // row items a column item waits for beyond n_stripes (0; tests only)
    int *next;               // queue head
    int *rows_done;          // [chunk][cb] finished row items
    int *cols_done;          // [chunk][cb] finished column items
    int *status;             // 0, or nonzero once a wait ran out of time
    long long budget;        // clock64 cycles per wait
    int4 chunks[kPersistMaxChunks];       // {t0, nt, c0, nc}, in the direct launches' order
    int item0[kPersistMaxChunks + 1];     // first item of each chunk
};

// FP16 tensor-core gridding + row transform: per (pol, grid row, kx tile) a
// product of the row's segment voltages with the segments' row spectra.
struct RowSpecArgs {
    int P, nt, nc, c0, AP, Tpad, kp_max;   // AP: plane rows per channel (voltages + kRowSpecPad)
    const int *kp;             // [P*N] contraction length (64 per chunk) per (pol, row); 0 = empty row
    const int *chunk_off;      // [P*N + 1] first chunk of each (pol, row)
    const int *chunk_row;      // plane row (within a channel) of each chunk's first voltage; a chunk
                               // is 32 consecutive plane rows, read as a TMA tile of re and of im
    const long long *bimg_off; // [P*N*ntiles] byte offset of each B image
    const __half *bimg;        // row spectra, K-major core-matrix images [2*KX][kp]
    const float *sy;           // [C] voltage scales (powers of two)
    float inv_sw;              // 1 / spectrum scale (power of two)
    const float *row_sh;       // [P*N] FP16 output scale (one power of two for every row)
    __half2 *H;                // row-transformed field, FP16, scaled by row_sh: slab [P][N][N] of
                               // (sample t, channel cl) at index t * slab_t + cl * slab_c
    long long slab_t, slab_c;
    int *err;                  // set when a bounded wait gives up
};

// Feedback calibration sums (Sec. 6) over one chunk.
struct FbArgs {
    const uint8_t *volt;      // codes [T][C][A][P]
    long long tstride;        // bytes between samples
    int t0, nt, c0, nc, AP, P;
    const float2 *gains;      // [C][A][P]
    const float2 *etap;       // [nt][nc][P] image pixel towards the calibrator
    double2 *corr;            // [C][A*P] sums of E conj(y), added to
    double *power;            // [C][P] sums of |E|^2, added to
};
cudaError_t launch_fb_corr(const FbArgs &a, cudaStream_t st);
// Autocorrelation sums per (channel, antenna): |y_x|^2, |y_y|^2, y_x conj(y_y) over a chunk
// (FbArgs: corr = [C][A][3] double2 sums; etap and power unused).
cudaError_t launch_auto_acc(const FbArgs &a, cudaStream_t st);
// The autocorrelation image of every channel and product from the sums and the
// kernels' cross-correlation patches X [A][NQ][(2K-1)^2] (FP64; one such block per set of
// kernels, chosen by chan_group[c] when it is not nullptr), into img [C][n_prod][N][N].
cudaError_t launch_auto_image(const double2 *pw, const double2 *X, const int *chan_group, int C, int A, int P, int K,
                              int N, const double2 *wN, double2 *Q, double *img, cudaStream_t st);
cudaError_t launch_sub_to_f32(const double *acc, const double *sub, float *out, long long n, cudaStream_t st);
// beam: [A*P] antenna beams towards the calibrator, or [sets][A*P] picked by chan_group[c].
cudaError_t launch_fb_finish(const double2 *corr, const double *power, const double2 *beam, const int *chan_group,
                             float2 *gains, int C, int AP, int P, int n_ant, float2 *r_out, float2 *delta, int apply,
                             cudaStream_t st);

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
    // four-step variant (C = 1024, 8 taps): twiddles exp(-2 pi i l k2 / C) as [k2][l],
    // and its stream-major output [AP][F][C] before the reorder
    const float2 *tw4;
    uint8_t *codes_sm;
    float2 *spec_sm;
    int frames_per_cta;       // four-step variant: frames one CTA streams (a multiple of 16)
};

// Row stride (in float2) of the TB calibrated voltages of one antenna-pol in
// shared memory: padded so that rows of a warp's random gathers spread over
// all banks; even, so rows are 16-byte aligned for float4 reads.
template <int TB> struct VoltStride { static constexpr int value = TB == 1 ? 1 : (TB == 8 ? 10 : 6); };
inline int volt_stride(int TB) { return TB == 1 ? 1 : (TB == 8 ? 10 : 6); }

// Rows transformed together by one gridding CTA: TB samples x P pols x rows.
inline int grid_fft_rows(int N) { return N >= 256 ? 8 : (N == 128 ? 16 : 32); }

// Radices of the N-point transform's passes (pass 0, 1, 2; 1 = no such pass);
// the device FFT plan (FftPlan<N>) asserts it agrees.
constexpr int fft_radix(int N, int pass) {
    return pass == 0 ? (N == 128 || N == 256 || N >= 1024 ? 16 : 8)
                     : pass == 1 ? (N == 32 ? 4 : (N == 256 || N == 2048 ? 16 : 8)) : (N >= 512 ? 8 : 1);
}

// The gridding kernel's row transform runs in place (one shared buffer of F rows)
// when the CTA's warps share the F rows evenly and, in every pass but the last,
// the slots of a warp's rows are exactly 32 (one per lane, held in registers
// while the warp reads its rows, written back after a warp barrier).  With idle
// lanes the compiler asked for more registers than the CTAs per SM allow.
constexpr bool grid_rows_in_place(int N, int F) {
    const int nw = 8;   // warps per gridding CTA (kBlock / 32)
    if (F % nw) return false;
    const int rpw = F / nw, np = N >= 512 ? 3 : 2;
    for (int p = 0; p + 1 < np; ++p)
        if (rpw * (N / fft_radix(N, p)) != 32) return false;
    return true;
}

// Shared-memory bytes of the gridding kernel (host and device agree on the carve).
inline size_t grid_smem_bytes(int N, int P, int TB, int rows, int max_nloc, int tw_total, int staged_entries = 0,
                              bool pairs = false) {
    const int ldr = N + N / 16;
    const int F = TB * P * rows;
    size_t b = 0;
    b += (size_t)staged_entries * (pairs ? 18 : 10);   // staged kernel entries (one or two float2 taps + u16)
    b += (size_t)tw_total * 8;
    // row buffer of TB samples, and a second one unless the passes run in place (+ alignment)
    b += (grid_rows_in_place(N, F) ? 1 : 2) * (size_t)F * ldr * 8 + 8;
    b += (size_t)volt_stride(TB) * max_nloc * P * 8;   // calibrated voltages of TB samples
    b += (size_t)max_nloc * P * 8 + 8;        // gains (+ padding that 16-byte aligns the staged entries)
    b += (size_t)max_nloc * 4;                // antenna indices
    return (b + 15) & ~(size_t)15;
}

// Shared-memory bytes of the gridding kernel with the tensor-core row transform.
size_t grid_smem_bytes_dft(int N, int P, int TB, int rows, int max_nloc);

// Kernel binning of one array (host side): per grid-row stripe, the antennas
// touching it and each cell's kernel contributions in a fixed order, packed
// as sliced ELL with cells sorted by contribution count.
struct Bins {
    int rows = 0, n_stripes = 0, tb = 1, max_nloc = 0, n_slices = 0, max_entries = 0;
    bool staged = false;   // kernel entries staged in shared memory
    bool pairs = false;    // lanes own pairs of adjacent cells; con_tap holds two taps per entry
    bool wide = false;     // twice grid_fft_rows(N) rows transformed per pass
    bool quads = false;    // lanes own 2 x 2 blocks of cells; con_tap holds four taps per entry
    std::vector<uint32_t> row_nz;   // [N / 32] grid rows any kernel footprint reaches
    size_t grid_smem = 0;
    std::vector<int> ant_off, ant_list;
    std::vector<long long> slice_off;
    std::vector<uint16_t> lane_cell;
    std::vector<float2> con_tap;
    std::vector<uint16_t> con_y;
};
// Gridding-kernel shape: time batch TB (stripe height follows) and whether
// the kernel entries are staged in shared memory.
struct GridChoice {
    int tb = 0;
    bool staged = false;
    bool pairs = false;   // each lane sums two horizontally adjacent cells
    bool wide = false;    // twice grid_fft_rows(N) rows per pass (more gather work per barrier)
    bool quads = false;   // each lane sums a 2 x 2 block of cells (pairs ignored; entries through L2)
};
// force = nullptr: the built-in rule; else exactly that shape (MOFF_EINVAL if infeasible).
// dft: shapes of the gridding kernel with the tensor-core row transform (k_grid_rows_dft).
moff_status build_bins(int A, int K, int N, int P, bool jones, const double *pos, const float *taps, Bins *b,
                       const GridChoice *force = nullptr, bool dft = false);
std::vector<float2> pass_twiddles_for(int n);   // pass-twiddle table of the n-point transform (FP64-built)

// Row spectra of the kernel rows for the tensor-core path (host side).
struct RowSpec {
    int kp_max = 0, ntiles = 1;
    float inv_sw = 1.f;
    std::vector<int> kp;                        // [P*N] 64 per chunk
    std::vector<int> chunk_off, chunk_row;      // chunks per (pol, row); first plane row of each
    std::vector<int> perm;                      // [A*P] plane row -> voltage index (antennas by anchor row)
    std::vector<float> row_sh, row_inv;         // FP16 field scale and its inverse (equal for every (pol, row))
    std::vector<long long> bimg_off;            // in elements
    std::vector<__half> bimg;
};
moff_status build_rowspec(int A, int K, int N, int P, bool jones, const double *pos, const float *taps, RowSpec *rs);
moff_status fail_msg(moff_status s, const char *msg);

int fft_tw_total(int n);                      // pass-twiddle table length for length n
int col_width(int N);                         // columns per column-kernel CTA
size_t col_smem_bytes(int N, int P);
size_t pfb_smem_bytes(int CN);

// Dense tensor-core path (moff_dft_kernels.cu): the factored-DFT table image of an
// N-point transform (B1 | B2 | twiddles; built in FP64), the column kernel, and the
// gridding kernel with the row transform on the tensor cores (TB, CPL as the plain one;
// entries through L2, stripes of grid_fft_rows(N) rows).
// cols = true: the column kernel's image (outputs grouped by eight for packed FP32 epilogues).
std::vector<unsigned char> build_dft_table(int N, bool cols = false);
float dft_kernel_scale(int A, int K, int N, int P, bool jones, const double *pos, const float *taps);
// W = columns per CTA of the column kernel (8 or 16).
size_t cols_dft_smem_bytes(int N, int P, int W);
cudaError_t launch_cols_dft(int N, int P, int W, const ColDftArgs &a, cudaStream_t st);
int cols_dft_width();            // the default W (MOFF_COLS_W=16 selects 16)
bool cols_dft_width_forced();    // MOFF_COLS_W set: the autotuner keeps it
cudaError_t launch_grid_dft(int N, int P, int TB, int CPL, const GridArgs &a, int n_stripes, size_t smem,
                            cudaStream_t st);
cudaError_t launch_grid_dft_n256(int P, int TB, int CPL, const GridArgs &a, int n_stripes, size_t smem, cudaStream_t st);
cudaError_t launch_grid_dft_n512(int P, int TB, int CPL, const GridArgs &a, int n_stripes, size_t smem, cudaStream_t st);

// Launchers (return the launch error, if any).
cudaError_t launch_grid(int N, int P, int TB, bool staged, bool grid_only, const GridArgs &a, int n_stripes,
                        size_t smem, cudaStream_t st);
cudaError_t launch_cols(int N, int P, const ColArgs &a, cudaStream_t st, bool h16 = false);
cudaError_t launch_pfb(int CN, const PfbArgs &a, cudaStream_t st);
// C = 1024, 8 taps, 16-byte aligned ADC: the four-step kernel into codes_sm /
// spec_sm ([AP][F][C]), then the reorder to codes / spec ([F][C][AP]).
cudaError_t launch_pfb1024(const PfbArgs &a, cudaStream_t st);
cudaError_t launch_pfb_reorder(const PfbArgs &a, cudaStream_t st);
cudaError_t launch_to_f32(const double *acc, float *out, long long n, cudaStream_t st);

// Tensor-core path (moff_tc_kernels.cu).
constexpr int kRowSpecMaxK = 256;   // largest contraction length (64 per 32-voltage chunk) held on chip
size_t rowspec_smem_bytes(int N, int kp_max);
int rowspec_ntiles(int N);
cudaError_t launch_gain_scale(const float2 *gains, int C, int AP, float *sy, cudaStream_t st);
// Voltage planes: plane row v < AP of a channel holds voltage perm[v] (antenna * P + input
// pol); rows AP .. APpad - 1 are zero.  APpad = AP + kRowSpecPad.
constexpr int kRowSpecPad = 32;
// Plane rows v < n_rows hold voltage perm[v]; rows n_rows .. APpad - 1 are zero (n_rows < 0: AP).
cudaError_t launch_volt_prep(const uint8_t *volt, long long tstride, int t0, int nt, int c0, int nc, int AP,
                             int APpad, const float2 *gains, const float *sy, const int *perm, int Tpad, __half *yre,
                             __half *yim, cudaStream_t st, int n_rows = -1, const CUtensorMap *smap_re = nullptr,
                             const CUtensorMap *smap_im = nullptr);
// Store maps of the voltage planes for the row plane kernel (box 32 samples x 32 rows, 64-byte swizzle).
cudaError_t encode_plane_store_map(CUtensorMap *map, void *plane, int Tpad, long long rows);
cudaError_t launch_rowspec(int N, const RowSpecArgs &a, const CUtensorMap &hmap, const CUtensorMap &amap_re,
                           const CUtensorMap &amap_im, int cgroups, size_t smem, cudaStream_t st);
// Tensor map of one FP16 voltage plane [rows][Tpad] (rows = Cb * A * P), box 64 samples x
// 32 rows, 128-byte swizzle, rows past the end read as zero: the A loads of k_rowspec_tc.
cudaError_t encode_plane_map(CUtensorMap *map, void *plane, int Tpad, long long rows, int box_rows = 32);
// Tensor map of the FP16 row-transformed field [nt][Cb][P*N][N] (half2 as 32-bit
// elements), box 32 kx x 32 samples, 128-byte swizzle: the store target of
// k_rowspec_tc.  Stores of samples >= nt fall outside the map and are dropped.
cudaError_t encode_field_map(CUtensorMap *map, void *H, int N, int P, int Cb, int nt);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---- served plans (MOFF_SERVED): the hooks the request loop in moff_server.cu uses
size_t plan_scratch_bytes(const moff_plan *pl);             // per-block scratch lent by the server
size_t plan_block_bytes(const moff_plan *pl, int n_time);   // voltage bytes of an n_time block
long long plan_units(const moff_plan *pl, int n_time);      // channel-snapshots of an n_time block
bool plan_is_served(const moff_plan *pl);
int plan_device(const moff_plan *pl);
cudaStream_t plan_stream(const moff_plan *pl);
// Bind the lent scratch, copy a host block behind it when on_device = 0 (the
// lent region then holds plan_block_bytes more), and enqueue the block.
moff_status plan_run_served(moff_plan *pl, void *scratch, const uint8_t *volt, int n_time, int on_device);

// Per-N instantiations (one translation unit each, compiled in parallel).
#define MOFF_DECLARE_N(NN)                                                                          \
    cudaError_t launch_grid_n##NN(int P, int TB, bool staged, bool grid_only, const GridArgs &a, int n_stripes, \
                                  size_t smem, cudaStream_t st);                                   \
    cudaError_t launch_cols_n##NN(int P, const ColArgs &a, cudaStream_t st, bool h16);            \
    cudaError_t launch_persist_n##NN(int P, int cpl, bool wide, const PersistArgs &pa, size_t smem, int sms, \
                                     cudaStream_t st);
MOFF_DECLARE_N(32)
MOFF_DECLARE_N(64)
MOFF_DECLARE_N(128)
MOFF_DECLARE_N(256)
MOFF_DECLARE_N(512)
#undef MOFF_DECLARE_N

}  // namespace moff
