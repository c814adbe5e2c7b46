/*
 * moff.h -- C ABI of the GB300 MOFF imaging library (libmoff.so).
 *
 * The library computes, per frequency channel and time sample, the MOFF
 * correlator image of Morales (arXiv 0812.3669), Sec. 4, Eq. m6:
 *
 *     I'(theta) = < | F^T(theta, r) W^T(r, a) N~(a, a) E'(a) |^2 >_t
 *
 * step 1 (N~):  every 4-bit complex antenna voltage E'(a) is multiplied by a
 *               per (channel, antenna, pol) complex weight -- the noise
 *               weighting of Eq. m4 with the gain calibration folded in;
 * step 2 (W^T): each weighted voltage is scattered onto a regular N x N
 *               aperture grid through that antenna's kernel (its holographic
 *               aperture map, Sec. 3);
 * step 3 (F^T): the gridded field is transformed to the sky with the
 *               unnormalised 2D transform E(k) = sum_r G(r) exp(+2 pi i k.r/N);
 * step 4:       |E|^2 (and, for two pols, the cross products) is summed over
 *               time.
 * An optional F-stage (Sec. 2, Eq. FFTofE; "often implemented as polyphase
 * filters") turns real 8-bit ADC streams into the 4-bit channelised voltages.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Antenna positions are (x, y) in grid-cell units.  A kernel is centred on
 *    the antenna's anchor cell (floor(x + 0.5), floor(y + 0.5)) and the grid
 *    wraps circularly modulo N.
 *  - Complex numbers are interleaved (re, im) float32 pairs.
 *  - Voltage bytes hold a 4-bit two's-complement real part in the high nibble
 *    and the imaginary part in the low nibble.  Layout [T][C][A][P].
 *  - Images are SUMS over time (the paper's average = sum / n_samples) in
 *    natural DFT order, row-major (ky, kx), not shifted.  Single pol: one
 *    product |E|^2.  Two pols: four products XX = |Ex|^2, YY = |Ey|^2,
 *    Re(Ex Ey*), Im(Ex Ey*).  Autocorrelation terms are included.
 *  - All pointer arguments flagged "on_device" are device pointers of the
 *    current CUDA device when the flag is 1, host pointers otherwise.
 *  - Every call returns a moff_status.  On error nothing aborts, the plan is
 *    left as it was, and moff_last_error() returns a message (thread-local).
 *  - A plan is not thread-safe: one host thread at a time may use it.
 *  - All work is enqueued on the plan's CUDA stream; host-pointer inputs are
 *    fully copied before the call returns, so the caller may reuse them.
 */
#ifndef MOFF_H
#define MOFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct moff_plan moff_plan; /* opaque, owned by the library */

typedef enum {
    MOFF_OK = 0,
    MOFF_EINVAL = -1,    /* bad argument (null pointer, size out of range, wrong state of flags) */
    MOFF_ENOMEM = -2,    /* a device or pinned-host allocation failed */
    MOFF_ECUDA = -3,     /* a CUDA call or kernel launch failed */
    MOFF_ESTATE = -4,    /* call not valid in the plan's current state */
    MOFF_ETIMEDOUT = -5, /* a bounded wait ran out before the GPU finished */
    MOFF_EBUSY = -6      /* resource temporarily unavailable */
} moff_status;

/* Plan flags. */
enum {
    MOFF_PREC_FP32 = 0u,      /* all arithmetic in FP32, cross-block sums in FP64 */
    MOFF_PREC_FP16TC = 1u,    /* FP16 tensor-core path (FP16 operands under exact power-of-two
                                 scales, FP32 accumulation, cross-block sums FP64), by one of two
                                 routes (moff_plan_route):
                                 row spectra -- gridding and the row transform (Eq. m6 steps 1-3,
                                   first axis) as one contraction per grid row (weighted voltages x
                                   each kernel row's FP64-built row spectrum); the column transform
                                   and the squaring stay FP32.  Taken where at most 128 antennas
                                   (4 chunks of 32) land their kernel rows on any one grid row per pol;
                                 factored DFT -- N = 256 or 512 (denser arrays, or environment
                                   variable MOFF_TC_DFT=1): both transform axes as factored DFT
                                   contractions (N = 16 x N/16, twiddles between the two factors;
                                   DFT and twiddle tables built in FP64), the column half fused with
                                   the squaring; the gridding as tensor-core contractions over tiles
                                   of 8 x 8 cells (weighted FP16 voltages x each tile's FP16 kernel
                                   values), or, with MOFF_TC_GRID=0 or tiles too large for shared
                                   memory, the FP32 gather fused with the row transform; the fields
                                   between the steps are FP16.  Feedback calibration and tied-array
                                   beams are not available on this route (MOFF_EINVAL). */
    MOFF_FSTAGE = 1u << 1,    /* enable the polyphase F-stage (moff_submit_adc, moff_channelise) */
    MOFF_JONES = 1u << 2,     /* kernels are full 2x2 Jones matrices (n_pol must be 2) */
    MOFF_SERVED = 1u << 3,    /* the plan does not own its per-block scratch (the row-transformed
                                 field; with MOFF_PREC_FP16TC also the FP16 voltage planes): a
                                 moff_server lends it from its pool for each block.  Such a plan
                                 takes blocks only through moff_server_submit. */
    MOFF_AUTOTUNE = 1u << 4,  /* pick the gridding kernel's shape (samples per pass, shared-memory
                                 staging of the kernel entries) by timing every feasible shape on
                                 this array at plan creation; results are cached per array and
                                 device in the process and, if the environment variable
                                 MOFF_TUNE_CACHE names a file, in that file.  FP32 path only. */
    MOFF_GRAPH = 1u << 5,     /* launch each block's kernel sequence as one CUDA graph: captured
                                 the first time a (input buffer, scratch, block length) is seen,
                                 replayed afterwards (8 kept per plan).  Not used while timing is on. */
    MOFF_PERSIST = 1u << 6    /* batching pattern (no counterpart in the paper): every channel and
                                 pol of a block in ONE persistent launch (k_image_persist) whose CTAs
                                 pull work items -- the gridding + row-transform stripes and the
                                 column strips of each (samples x channels) chunk -- from a device
                                 queue; an item waits, on one polling lane bounded by a clock64
                                 budget (about 1 s), for the items it depends on, so chunks overlap
                                 while the FP64 sums still fold in chunk order: the image equals the
                                 direct launches' bit for bit.  A wait that runs out records a status
                                 that the next moff_sync / moff_read_image returns as
                                 MOFF_ETIMEDOUT.  FP32 path of an unserved plan only (MOFF_EINVAL
                                 with MOFF_PREC_FP16TC or MOFF_SERVED); the gridding shape is 4
                                 samples per pass with entries through L2 (MOFF_AUTOTUNE picks among
                                 those).  Blocks with feedback calibration, beams or autocorrelation
                                 subtraction on run the direct launches.  With MOFF_GRAPH the
                                 persistent launch is what the graph replays. */
};

/*
 * moff_plan_create -- build a plan for one array (Sec. 4: the antenna layout,
 * the kernels W and the grid of Eq. m6 step 2 are fixed for an observation).
 *
 *   out       receives the new plan (set to NULL on error).
 *   n_ant     number of antennas A, 1 <= A <= 65536.
 *   pos       host float64 [A][2], (x, y) in grid-cell units.
 *   ksize     kernel side K, odd, 1 <= K <= min(N, 15).
 *   taps      host float32 complex kernels, copied:
 *               without MOFF_JONES: [A][P][K][K][2]       (one kernel per pol)
 *               with    MOFF_JONES: [A][2][2][K][K][2]    ([a][p_out][p_in][dy][dx])
 *   grid_n    grid side N: 32, 64, 128, 256 or 512.
 *   n_chan    number of channels C >= 1 (with MOFF_FSTAGE: a power of two,
 *             32 <= C <= 2048; the F-stage frame is M = 2C real samples).
 *   n_pol     P = 1 or 2 (input pols = output pols).
 *   flags     MOFF_* bits above.
 *   cuda_stream  cudaStream_t to run on (cudaStreamLegacy, 0x1, selects the
 *             legacy default stream), or NULL for a stream the plan creates.
 * The plan owns device memory for kernels, gains (initialised to 1), FP64
 * accumulators [C][n_prod][N][N] and scratch.  Errors: MOFF_EINVAL for any
 * argument out of range, MOFF_ENOMEM, MOFF_ECUDA.
 */
moff_status moff_plan_create(moff_plan **out, int n_ant, const double *pos, int ksize,
                             const float *taps, int grid_n, int n_chan, int n_pol,
                             unsigned flags, void *cuda_stream);

/*
 * moff_set_gains -- the complex weights N~ of Eq. m6 step 1 (Sec. 4: one over
 * the antenna noise, with any calibration folded in; Sec. 6 feeds
 * calibration back through here).  gains: float32 complex [C][A][P][2],
 * copied (host, or device when on_device = 1).  Takes effect for blocks
 * submitted afterwards.
 */
moff_status moff_set_gains(moff_plan *plan, const float *gains, int on_device);

/*
 * moff_set_channel_groups -- channel-dependent antenna positions and kernels.
 * Antenna positions in grid cells (wavelengths) scale with frequency, and so
 * do the kernels that describe each antenna's illumination; Sec. 4 also folds
 * w-projection into the kernels.  The plan takes n_groups sets, each laid out
 * as in moff_plan_create:
 *   pos         host float64 [n_groups][A][2]
 *   taps        host float32 complex [n_groups][A][P][K][K][2] (MOFF_JONES:
 *               [n_groups][A][2][2][K][K][2])
 *   chan_group  host int [C]: the set of each channel (may be NULL when
 *               n_groups = 1, which replaces the creation-time set)
 * All copied.  Channels of one set are imaged exactly as a plan created with
 * that set.  The gridding shape stays the plan's where every set fits it, else
 * the first of the built-in rule's shapes that all sets fit.  Waits for the
 * plan's work in flight; applies to blocks submitted afterwards (the running
 * integration is kept: reset first to start a new one).  Calibrator beams and
 * autocorrelation patches follow the new sets.  FP32 path only.
 * Errors: MOFF_EINVAL (MOFF_PREC_FP16TC plan, n_groups outside [1, C], a
 * chan_group entry outside [0, n_groups), a position not finite, or a set too
 * dense for the gridding kernel; the plan is unchanged), MOFF_ENOMEM, MOFF_ECUDA.
 */
moff_status moff_set_channel_groups(moff_plan *plan, int n_groups, const double *pos, const float *taps,
                                   const int *chan_group);

/*
 * moff_set_fstage -- configure the polyphase F-stage (Sec. 2, Eq. FFTofE).
 *   n_taps  filter length in frames, 1 <= n_taps <= 16.
 *   coeffs  host float32 [n_taps * M] prototype filter h[n], or NULL for the
 *           default sinc(x / M) * Hann window over n_taps * M samples.
 *   scale   requantisation scale: code = clamp(rint(X * scale), -7, 7) per
 *           component, round half to even.
 * Requires MOFF_FSTAGE.  Default after plan creation: 8 taps, default
 * window, scale 1.
 */
moff_status moff_set_fstage(moff_plan *plan, int n_taps, const float *coeffs, float scale);

/*
 * moff_submit -- add a block of 4-bit voltages to the integration (Eq. m6,
 * steps 1-4, summed over the block's samples).
 *   volt    uint8 [n_time][C][A][P].
 *   n_time  samples in the block, >= 1.
 * With on_device = 0 the block is copied to the device before the call
 * returns; a block of 8 MB or more that spans several channel chunks is
 * copied by channel segments (one 2D copy each, on the plan's copy stream),
 * and each chunk's imaging waits only for its own segment, so the copies
 * overlap the imaging (MOFF_STAGE_PIPELINE=0 copies it whole; graph replay
 * always does).  The image is the same either way.  With on_device = 1 the
 * caller keeps the buffer alive and unmodified until moff_sync or
 * moff_read_image returns.
 */
moff_status moff_submit(moff_plan *plan, const uint8_t *volt, int n_time, int on_device);

/*
 * moff_submit_adc -- F-stage then imaging for a block of real ADC samples.
 *   adc     int8 [A][P][n_samp], n_samp a multiple of M = 2C with
 *           n_samp / M >= n_taps.  The block yields F = n_samp/M - n_taps + 1
 *           frames (time samples); blocks are independent (no history is
 *           carried between calls).
 * Requires MOFF_FSTAGE.  Buffer ownership as for moff_submit.
 */
moff_status moff_submit_adc(moff_plan *plan, const int8_t *adc, long long n_samp, int on_device);

/*
 * moff_channelise -- run only the F-stage (Sec. 2, Eq. FFTofE) on one block.
 *   out_kind 0: out = uint8 [F][C][A][P] requantised 4-bit codes.
 *   out_kind 1: out = float32 complex [F][C][A][P][2] unquantised spectra
 *               X_m[k] = sum_j s_m[j] exp(-2 pi i j k / M).
 * Output goes to host memory (out_on_device = 0) or device memory (1).
 * Synchronous: returns when out is written.  Requires MOFF_FSTAGE.
 */
moff_status moff_channelise(moff_plan *plan, const int8_t *adc, long long n_samp, int in_on_device,
                            void *out, int out_kind, int out_on_device);

/*
 * moff_grid_snapshot -- gridded field of one time sample (Eq. m6 steps 1-2),
 * for inspection and testing.
 *   volt  uint8 [C][A][P] of a single sample (host or device per on_device).
 *   chan  channel index whose gains apply.
 *   out   host float32 complex [P][N][N][2].
 * Synchronous.  Does not touch the accumulators.
 */
moff_status moff_grid_snapshot(moff_plan *plan, const uint8_t *volt, int on_device, int chan,
                               float *out);

/*
 * moff_read_image -- the integrated image (Eq. m6, step 4).
 *   out        float32 [C][n_prod][N][N]; host (out_on_device = 0) or device.
 *   n_samples  if not NULL, receives the number of time samples summed.
 *   reset      1: zero the accumulators after reading.
 *   timeout_ms bounded wait for outstanding work (< 0: wait without limit);
 *              on expiry MOFF_ETIMEDOUT and nothing is read or reset.
 */
moff_status moff_read_image(moff_plan *plan, float *out, long long *n_samples, int reset,
                            int timeout_ms, int out_on_device);

/* moff_sync -- bounded wait for all work enqueued on the plan (MOFF_ETIMEDOUT on expiry). */
moff_status moff_sync(moff_plan *plan, int timeout_ms);

/*
 * moff_export_accumulators / moff_import_accumulators -- checkpoint and resume
 * an integration (no counterpart in the paper, whose time average Eq. m6 is a
 * running sum): the FP64 image sums float64 [C][n_prod][N][N] and their sample
 * count.  Export waits for the plan's work (bounded, as moff_read_image, and
 * reports a failed in-kernel wait as MOFF_ETIMEDOUT) and copies them to out
 * (host, or device with out_on_device = 1).  Import replaces the plan's sums and
 * count with in (host: copied before the call returns; device: the caller keeps
 * it until moff_sync), enqueued behind the plan's earlier work.  A plan of the
 * same C, n_prod and N, on any route, continues the integration: its later
 * blocks add to the imported sums exactly as they would have to its own.
 * Feedback-calibration and autocorrelation sums are not included.
 */
moff_status moff_export_accumulators(moff_plan *plan, double *out, long long *n_samples, int out_on_device,
                                     int timeout_ms);
moff_status moff_import_accumulators(moff_plan *plan, const double *in, long long n_samples, int in_on_device);

/* moff_reset -- zero the accumulators and the sample count (enqueued on the plan's stream). */
moff_status moff_reset(moff_plan *plan);

/* moff_plan_info -- sizes chosen at plan creation (any pointer may be NULL). */
moff_status moff_plan_info(const moff_plan *plan, int *n_prod, int *rows_per_stripe,
                           int *time_chunk, int *chan_chunk, long long *device_bytes);

/*
 * moff_plan_route -- which arithmetic the plan's imaging takes: 0 the FP32 path
 * (gather gridding, both transform axes as FP32 FFTs), 1 the FP16 row-spectrum
 * contraction + FP32 column FFT, 2 FP32 gridding + both axes as factored
 * tensor-core DFT contractions, 3 the same transforms with the gridding on the
 * tensor cores too (see MOFF_PREC_FP16TC).  MOFF_EINVAL for a NULL argument.
 */
moff_status moff_plan_route(const moff_plan *plan, int *route);

/*
 * ---- Feedback calibration (Sec. 6, Eqs. FBeq1-FBeq3): correlate the
 * electric-field image pixel towards a calibrator with every antenna's
 * calibrated signal -- feeding the correlator output back to its input.
 *
 * moff_set_calibrator -- from the next block on, also accumulate per channel,
 * pol p and antenna a over the submitted samples
 *     S_p   = sum_t |E_t,p(k)|^2                                  (FBeq1)
 *     R_a,p = sum_t E_t,p(k) conj(y_t,a,p B_a,p)                    (FBeq2)
 * where E_t,p(k) is the image's field at pixel k = (kx, ky) (before squaring),
 * y the calibrated voltage and B_a,p antenna a's kernel placed at its anchor
 * and transformed at k (its share of the pixel per unit voltage), so that
 * sum_a R_a,p = S_p.  Resets both sums.  kx = ky = -1 switches the sums off.
 * MOFF_EINVAL for a pixel outside the image or a MOFF_JONES plan.  moff_reset
 * zeros these sums too.
 */
moff_status moff_set_calibrator(moff_plan *plan, int kx, int ky);

/*
 * moff_read_feedback -- the sums since the calibrator was set (or last reset):
 *   corr    host float32 complex [C][A][P][2]: R (may be NULL);
 *   power   host float64 [C][P]: S (may be NULL);
 *   n_samples  samples summed (may be NULL); reset = 1 zeros the sums after reading;
 *   timeout_ms  bounded wait for outstanding work (< 0: none).
 * MOFF_ESTATE if no calibrator is set.
 */
moff_status moff_read_feedback(moff_plan *plan, float *corr, double *power, long long *n_samples, int reset,
                               int timeout_ms);

/*
 * moff_feedback_gains -- the Sec. 6 gain-error estimate from the current sums,
 *     delta_g_a,p = g_a,p (1 - A conj(R_a,p) / S_p)
 * read with the antenna count A where the paper prints 2N (at convergence the
 * printed factor gives -g, not 0) and with the conjugated ratio (so that
 * g + delta_g moves each antenna's residual gain to the array mean, to first
 * order, for a dominant calibrator).  delta: host float32 complex [C][A][P][2]
 * (may be NULL).  apply = 1 adds delta_g to the plan's gains for the next block.
 * The relative solution leaves the array's overall gain and phase free (Sec. 6).
 */
moff_status moff_feedback_gains(moff_plan *plan, float *delta, int apply);

/*
 * ---- Autocorrelation subtraction.  Software holography (Sec. 3, Eq. RBeamEq)
 * images the visibilities of antenna pairs; the MOFF image <|sum_a c_a|^2>_t
 * (Sec. 4) also holds every antenna's own term.
 *
 * moff_set_autocorr -- on = 1: from the next block on, also sum per channel
 * and antenna |y_x|^2, |y_y|^2 and y_x conj(y_y) (one pol: |y|^2); on = 0: stop.
 * Switching on resets those sums.  MOFF_EINVAL for a MOFF_JONES plan.
 */
moff_status moff_set_autocorr(moff_plan *plan, int on);

/*
 * moff_read_image_cross -- as moff_read_image, minus the autocorrelation part
 *   sum_a P_a,pq K^_a,p(k) conj(K^_a,q(k))
 * (P the antenna's summed products, K^ its kernel's transform; positions drop
 * out): the image of the baselines only.  Done in FP64 before the conversion.
 * MOFF_ESTATE unless the autocorrelation sums cover exactly the image's samples
 * (switch them on before the integration starts).  reset = 1 zeros both, as do
 * moff_reset and moff_read_image with reset = 1.
 */
moff_status moff_read_image_cross(moff_plan *plan, float *out, long long *n_samples, int reset, int timeout_ms,
                                  int out_on_device);

/*
 * ---- Tied-array beams (Sec. 7: the electric-field image can be tapped, each
 * pixel being a calibrated tied-array beam).
 *
 * moff_set_beams -- from the next block on, write the field E_t,p(k_j) (before
 * squaring) at up to 16 pixels k_j = (kx[j], ky[j]) for every sample of each
 * block; n_beams = 0 stops.  MOFF_EINVAL for a pixel outside the image.
 */
moff_status moff_set_beams(moff_plan *plan, int n_beams, const int *kx, const int *ky);

/*
 * moff_read_beams -- the beams of the most recent block: out float32 complex
 * [T][C][n_beams][P][2] (host, or device when out_on_device = 1; may be NULL to
 * query), n_time receives T.  Bounded wait as moff_read_image.  MOFF_ESTATE if
 * no beams are set.
 */
moff_status moff_read_beams(moff_plan *plan, float *out, int *n_time, int timeout_ms, int out_on_device);

/*
 * moff_plan_tuning -- how the gridding kernel's shape was chosen (any pointer
 * may be NULL): time_batch = samples gridded and row-transformed per pass (1, 2,
 * 4 or 8), staged = 1 if kernel entries are staged in shared memory,
 * cells_per_lane = grid cells each lane sums (1; 2 adjacent cells of a row; 4 = a
 * 2 x 2 block), so that one voltage read feeds all of them, source = 0 built-in rule, 1 measured by MOFF_AUTOTUNE at creation, 2 taken
 * from the tuning cache; best_ms = the measured time of the chosen shape (source
 * 1); wide_rows = 1 if twice the usual number of grid rows is transformed per
 * pass (more gather work between barriers).
 */
/*
 * moff_plan_dft_tuning -- the dense FP16 routes' column kernel (any pointer may
 * be NULL): cols_width = columns per CTA (8: two CTAs per SM; 16: one; 0 on
 * other routes), source = 0 default (environment variable MOFF_COLS_W=16 picks
 * 16), 1 measured by MOFF_AUTOTUNE at creation on one chunk of the plan's shape;
 * ms_w8 / ms_w16 = the measured times per chunk (source 1).
 */
moff_status moff_plan_dft_tuning(const moff_plan *plan, int *cols_width, int *source, double *ms_w8, double *ms_w16);

moff_status moff_plan_tuning(const moff_plan *plan, int *time_batch, int *staged, int *cells_per_lane,
                             int *source, double *best_ms, int *wide_rows);

/*
 * moff_set_timing -- when on (1), every kernel the plan launches is bracketed
 * by a pair of CUDA events on the plan's stream, so its device time can be
 * read with moff_timing.  Off (0) by default; switching on clears old records.
 */
moff_status moff_set_timing(moff_plan *plan, int on);

/*
 * moff_timing -- device time of the plan's kernels since timing was switched
 * on (or last reset), for one kernel kind:
 *   0  F-stage polyphase filter bank,
 *   1  calibrate + grid + row transform (Eq. m6 steps 1-2, step 3 first axis;
 *      with MOFF_PREC_FP16TC the tensor-core row contraction),
 *   2  column transform + square-and-integrate (step 3 second axis, step 4),
 *   3  (MOFF_PREC_FP16TC only) voltage decode, weighting and FP16 transpose,
 *   4  F-stage output reorder (the four-step F-stage used for C = 1024 with
 *      8 taps writes stream-major and reorders to [F][C][A][P]),
 *   5  feedback-calibration correlation (when a calibrator is set),
 *   6  autocorrelation sums (when switched on),
 *   7  (tensor-core gridding route only) the row transform of the gridded field,
 *   8  (MOFF_PERSIST) the persistent launch (kinds 1 and 2 of every chunk).
 * On the tensor-core gridding route kind 1 is the cell-tile gridding alone and
 * kind 3 writes the voltage planes it reads.
 * Waits for the recorded work.  total_ms / launches may be NULL.  reset = 1
 * drops the records of every kind after reading.
 */
moff_status moff_timing(moff_plan *plan, int kind, double *total_ms, long long *launches, int reset);

/*
 * moff_image_noalloc -- image one block of voltages without allocating any
 * GPU memory.  (The paper has no counterpart; this is a library service.)
 *
 * For callers that cannot call cudaMalloc -- code that must live inside a
 * memory budget someone else fixed, or that may not block on the allocator --
 * this call takes every input and the output from the caller and keeps all
 * intermediates (kernel lists, twiddles, the row-transformed field, the FP64
 * sums) in one fixed 64 MiB device array inside the library, which every GPU
 * that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 *   n_ant, pos, ksize, taps, grid_n, n_chan, n_pol, flags
 *            as for moff_plan_create (flags: 0 or MOFF_JONES); pos and taps
 *            are host arrays.
 *   volt     device uint8 [n_time][C][A][P], n_time >= 1.
 *   gains    device float32 complex [C][A][P][2].
 *   image    device float32 [C][n_prod][N][N]; overwritten with this
 *            block's sums (Eq. m6 summed over its n_time samples).
 *   cuda_stream  stream for the work (NULL = legacy default stream).
 * The work is enqueued on cuda_stream; the image is ready when the stream
 * reaches it.  Arrays whose kernel lists plus one channel's sums and field
 * exceed 64 MiB are rejected with MOFF_EINVAL.
 * The first call on each device looks up the array's device address (with
 * that device current).  With lazy module loading (the CUDA default) that
 * lookup is also when the library's kernels and the 64 MiB array are loaded
 * onto that device, so a caller inside a fixed memory budget should make its
 * first call during set-up, before the budget is in force.  Every call copies
 * the kernel lists from pageable host memory, so no call may be made while its
 * stream is being captured into a graph: such a call returns MOFF_ESTATE.
 * All calls share the one array: calls whose GPU work overlaps in time (on
 * different streams, or from different threads) race and corrupt each
 * other's results; serialise them.
 */
moff_status moff_image_noalloc(int n_ant, const double *pos, int ksize, const float *taps, int grid_n,
                               int n_chan, int n_pol, unsigned flags, const uint8_t *volt, int n_time,
                               const float *gains, float *image, void *cuda_stream);

/*
 * moff_voltage_planes -- diagnostic (the paper has no counterpart): the FP16
 * voltage planes the row-spectrum or the tensor-core gridding route builds for
 * one channel (on the latter, rows copied for wrapping kernel windows must equal
 * their originals: MOFF_ECUDA otherwise)
 * (Eq. m6 step 1: each 4-bit voltage decoded, times its gain, times the
 * channel's power-of-two scale, rounded to FP16), read back so the decoding can
 * be checked bit for bit.
 *   volt     uint8 [n_time][C][A][P] (host, or device with on_device = 1),
 *            1 <= n_time <= the plan's time chunk (moff_plan_info).
 *   out      host float32 complex [n_time][A][P][2]: the FP16 plane values,
 *            converted exactly, in voltage order.
 *   scale    the channel's power-of-two scale (may be NULL).
 * Synchronous.  MOFF_EINVAL unless the plan takes the row-spectrum or the
 * tensor-core gridding route (moff_plan_route = 1 or 3) and is not served.
 */
moff_status moff_voltage_planes(moff_plan *plan, const uint8_t *volt, int n_time, int on_device, int chan,
                                float *out, float *scale);

/*
 * moff_tc_selftest -- diagnostic: one tensor-core product D = A * B^T with the
 * building blocks the FP16 DFT kernels use (canonical K-major operands in
 * shared memory, TMEM accumulator, tcgen05.mma kind::f16, completion through
 * an mbarrier with a bounded wait, tcgen05.ld).  The paper has no
 * counterpart; it checks the tensor-core path against a host reference.
 *   a  device half [128][k];  b  device half [n][k];  d  device float [128][n].
 *   n  multiple of 32 in [32, 256];  k  multiple of 16 in [16, 256].
 *   mode  bit 0: stage A MN-major (then k <= 64); bit 1: stage B MN-major
 *         (then k <= 64, n <= 128); bit 2: an MN-major operand's descriptor
 *         carries its K-direction core-matrix stride as the leading byte offset;
 *         bit 3: stage A MN-major with the 128-byte swizzle of a TMA load
 *         (then k <= 64).
 * Synchronous on cuda_stream.  MOFF_ETIMEDOUT if the product did not finish
 * within the wait limit (a few seconds).
 */
moff_status moff_tc_selftest(const void *a, const void *b, float *d, int n, int k, int mode, void *cuda_stream);

/*
 * ---- Serving.  The paper has no counterpart: it treats the correlator as a
 * stream of channelised blocks (Sec. 2); this is the library's streaming front
 * end for many arrays at once.
 *
 * moff_server_create -- a request loop on the current device over plans created
 * with MOFF_SERVED (sub-arrays of uneven antenna count and grid size).  Plans keep
 * their kernels, gains and partial integrations resident; each admitted block
 * borrows its plan's scratch (plus room for its voltages when they come from host
 * memory) from one device pool until its GPU work has finished.
 *   hbm_budget_bytes  size of that pool, allocated once here (>= 1024).
 *   n_slots           most blocks on the GPU at once, 1..64; each runs on its plan's
 *                     stream, so blocks of different plans overlap on the device.
 * Errors: MOFF_EINVAL, MOFF_ENOMEM (pool), MOFF_ECUDA.
 */
typedef struct moff_server moff_server; /* opaque, owned by the library */
moff_status moff_server_create(moff_server **out, long long hbm_budget_bytes, int n_slots);

/*
 * moff_server_submit -- queue one voltage block (Eq. m6 steps 1-4 over its
 * samples, added to the plan's integration) and return at once.
 *   plan      created with MOFF_SERVED on the server's device.
 *   volt, n_time, on_device  as for moff_submit, except that the caller keeps the
 *             buffer alive and unmodified until the ticket is done either way (a host
 *             block is copied when the block starts).
 *   ticket    receives the block's id (>= 1).
 * Blocks start in arrival order as slots and pool memory free up: a block whose
 * plan has one on the GPU waits for it (a plan's blocks run in submission order),
 * and a later block may start ahead of one that does not fit yet only if it leaves
 * at least that block's bytes free.  MOFF_ENOMEM: the block can never fit the pool.
 * MOFF_ESTATE: the plan is not MOFF_SERVED, is on another device, or the server is
 * shutting down.  From submit until the plan's last ticket is done, call no other
 * entry point on that plan (thread-safe calls are those on the server).
 */
moff_status moff_server_submit(moff_server *srv, moff_plan *plan, const uint8_t *volt, int n_time,
                               int on_device, long long *ticket);

/*
 * moff_server_poll -- state of a ticket without waiting: 0 queued, 1 on the GPU,
 * 2 done, or the (negative) moff_status its block failed with.  latency_ms (may be
 * NULL) receives the time from submit to the end of the block's GPU work once it is
 * done, else 0.  The last 65536 finished tickets stay known; older ones give
 * MOFF_EINVAL.
 */
moff_status moff_server_poll(moff_server *srv, long long ticket, int *state, double *latency_ms);

/*
 * moff_server_wait -- wait until a ticket (ticket = 0: every block submitted so far)
 * is done; timeout_ms < 0 waits without limit, else MOFF_ETIMEDOUT on expiry.
 * Returns the block's failure status if it failed.
 */
moff_status moff_server_wait(moff_server *srv, long long ticket, int timeout_ms);

/*
 * moff_server_stats -- over the blocks finished since the last reset: the 50th and
 * 99th percentile block latency (ms, submit to end of GPU work, nearest rank), the
 * throughput in channel-snapshots per second (their C x n_time summed, over the span
 * from the window's first submit to its last completion) and their count.  Any output
 * may be NULL.  reset = 1 starts a new window after reading.
 */
moff_status moff_server_stats(moff_server *srv, double *p50_ms, double *p99_ms, double *throughput,
                              long long *completed, int reset);

/*
 * moff_server_destroy -- cancel the blocks that have not started (their tickets end
 * with MOFF_ESTATE), wait for those on the GPU, free the pool.  NULL is a no-op.
 */
moff_status moff_server_destroy(moff_server *srv);

/* moff_plan_destroy -- wait for the plan's work, free everything.  NULL is a no-op. */
moff_status moff_plan_destroy(moff_plan *plan);

/* moff_last_error -- message of the last failed call on this host thread ("" if none). */
const char *moff_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MOFF_H */
