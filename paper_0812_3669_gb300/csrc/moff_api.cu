// moff_api.cu -- C ABI of libmoff: plans, binning, executor.
//
// A plan fixes one array (Morales, arXiv 0812.3669, Sec. 4, Eq. m6): antenna
// anchors, per-antenna kernels W, grid size, channels and pols.  At creation
// the kernels are binned by grid-row stripe into per-cell contribution lists
// (the gather form of the W^T scatter, so every cell sums its contributions
// in one fixed order and results do not depend on scheduling), twiddle
// tables are built in FP64 on the host, and device memory for gains, FP64
// accumulators and the row-transform scratch is reserved.  Submitting a
// block runs, per (channel chunk, time chunk), the gridding/row-transform
// kernel and the column-transform/integrate kernel on the plan's stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/moff.h"
#include "moff_fft.cuh"
#include "moff_image_kernels.cuh"
#include "moff_internal.h"

using namespace moff;

namespace {

thread_local std::string g_err;

moff_status fail(moff_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define MOFF_CK(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            if (e_ == cudaErrorMemoryAllocation) {                                        \
                cudaGetLastError();                                                       \
                return fail(MOFF_ENOMEM, "%s: %s", #call, cudaGetErrorString(e_));        \
            }                                                                             \
            return fail(MOFF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));             \
        }                                                                                 \
    } while (0)

// Host-side fault injection for tests: MOFF_FAULT=alloc:K makes the K-th
// device allocation of the process (counting from 1) report out-of-memory.
std::atomic<long long> g_alloc_count{0};

cudaError_t dev_alloc(void **p, size_t bytes) {
    const long long k = ++g_alloc_count;
    const char *f = getenv("MOFF_FAULT");
    if (f && strncmp(f, "alloc:", 6) == 0 && atoll(f + 6) == k) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes ? bytes : 16);
}

// exp(2 pi i m / L) in FP64 with exact quadrant points.
void root_unity(long long m, long long L, double *c, double *s) {
    m %= L;
    if (m < 0) m += L;
    const long long q = (4 * m) / L, r = (4 * m) % L;
    double cr = 1.0, sr = 0.0;
    if (r != 0) {
        const double ang = (M_PI / 2.0) * (double)r / (double)L;
        cr = std::cos(ang);
        sr = std::sin(ang);
    }
    switch (q) {
        case 0: *c = cr; *s = sr; break;
        case 1: *c = -sr; *s = cr; break;
        case 2: *c = -cr; *s = -sr; break;
        default: *c = sr; *s = -cr; break;
    }
}

template <int N>
std::vector<float2> pass_twiddles() {
    using P = FftPlan<N>;
    using T = FftTw<N>;
    std::vector<float2> t(std::max(T::TOTAL, 1));
    auto fill = [&](int off, int NS, int R) {
        for (int r = 1; r < R; ++r)
            for (int m = 0; m < NS; ++m) {
                double c, s;
                root_unity((long long)m * r, (long long)NS * R, &c, &s);
                t[off + (r - 1) * NS + m] = make_float2((float)c, (float)s);
            }
    };
    fill(T::OFF1, P::R0, P::R1);
    if (P::NP == 3) fill(T::OFF2, P::R0 * P::R1, P::R2);
    return t;
}

std::vector<float2> pass_twiddles_n(int n) {
    switch (n) {
        case 32: return pass_twiddles<32>();
        case 64: return pass_twiddles<64>();
        case 128: return pass_twiddles<128>();
        case 256: return pass_twiddles<256>();
        case 512: return pass_twiddles<512>();
        case 1024: return pass_twiddles<1024>();
        case 2048: return pass_twiddles<2048>();
    }
    return {};
}

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ o, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        o[i] = (float)a[i];
}

}  // namespace

namespace moff {

int fft_tw_total(int n) {
    switch (n) {
        case 32: return FftTw<32>::TOTAL;
        case 64: return FftTw<64>::TOTAL;
        case 128: return FftTw<128>::TOTAL;
        case 256: return FftTw<256>::TOTAL;
        case 512: return FftTw<512>::TOTAL;
        case 1024: return FftTw<1024>::TOTAL;
        case 2048: return FftTw<2048>::TOTAL;
    }
    return 0;
}

int col_width(int N) {
    switch (N) {
        case 32: return ColShape<32>::W;
        case 64: return ColShape<64>::W;
        case 128: return ColShape<128>::W;
        case 256: return ColShape<256>::W;
        case 512: return ColShape<512>::W;
    }
    return 0;
}

size_t col_smem_bytes(int N, int P) {
    switch (N) {
        case 32: return col_smem_bytes_t<32>(P);
        case 64: return col_smem_bytes_t<64>(P);
        case 128: return col_smem_bytes_t<128>(P);
        case 256: return col_smem_bytes_t<256>(P);
        case 512: return col_smem_bytes_t<512>(P);
    }
    return 0;
}

cudaError_t launch_grid(int N, int P, int TB, bool staged, bool go, const GridArgs &a, int n_stripes, size_t smem,
                        cudaStream_t st) {
    switch (N) {
        case 32: return launch_grid_n32(P, TB, staged, go, a, n_stripes, smem, st);
        case 64: return launch_grid_n64(P, TB, staged, go, a, n_stripes, smem, st);
        case 128: return launch_grid_n128(P, TB, staged, go, a, n_stripes, smem, st);
        case 256: return launch_grid_n256(P, TB, staged, go, a, n_stripes, smem, st);
        case 512: return launch_grid_n512(P, TB, staged, go, a, n_stripes, smem, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cols(int N, int P, const ColArgs &a, cudaStream_t st, bool h16) {
    switch (N) {
        case 32: return launch_cols_n32(P, a, st, h16);
        case 64: return launch_cols_n64(P, a, st, h16);
        case 128: return launch_cols_n128(P, a, st, h16);
        case 256: return launch_cols_n256(P, a, st, h16);
        case 512: return launch_cols_n512(P, a, st, h16);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_persist(int N, int P, int cpl, bool wide, const PersistArgs &pa, size_t smem, int sms,
                           cudaStream_t st) {
    switch (N) {
        case 32: return launch_persist_n32(P, cpl, wide, pa, smem, sms, st);
        case 64: return launch_persist_n64(P, cpl, wide, pa, smem, sms, st);
        case 128: return launch_persist_n128(P, cpl, wide, pa, smem, sms, st);
        case 256: return launch_persist_n256(P, cpl, wide, pa, smem, sms, st);
        case 512: return launch_persist_n512(P, cpl, wide, pa, smem, sms, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_to_f32(const double *acc, float *out, long long n, cudaStream_t st) {
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
    k_to_f32<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, st>>>(acc, out, n);
    return cudaGetLastError();
}

}  // namespace moff

struct moff_plan {
    int A = 0, K = 0, N = 0, C = 0, P = 0, nprod = 0;
    unsigned flags = 0;
    bool jones = false, fstage = false;
    int device = 0;
    cudaStream_t st = nullptr, cst = nullptr;
    bool own_stream = false;

    // binning
    int rows = 0, n_stripes = 0, max_nloc = 0, n_slices = 0, tb = 1, max_entries = 0;
    bool staged = false, pairs = false, wide = false, quads = false;
    size_t grid_smem = 0;
    int *d_st_ant_off = nullptr, *d_st_ant = nullptr;
    long long *d_slice_off = nullptr;
    uint16_t *d_lane_cell = nullptr;
    float2 *d_con_tap = nullptr;
    uint16_t *d_con_y = nullptr;
    uint32_t *d_row_nz = nullptr;   // [N / 32] grid rows any kernel footprint reaches
    float2 *d_twp = nullptr;

    float2 *d_gains = nullptr;
    double *d_acc = nullptr;
    float *d_img = nullptr;
    float2 *d_H = nullptr;
    int Tb = 0, Cb = 0;

    void *d_stage[2] = {nullptr, nullptr};
    size_t stage_bytes[2] = {0, 0};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_consumed[2] = {nullptr, nullptr};
    cudaEvent_t ev_done = nullptr;
    long long nsub = 0;

    // F-stage
    int ntaps = 8;
    float scale = 1.f;
    float *d_h = nullptr;
    float2 *d_twpC = nullptr, *d_twM = nullptr;
    uint8_t *d_codes = nullptr;
    size_t codes_bytes = 0;
    float2 *d_spec = nullptr;
    size_t spec_bytes = 0;
    float2 *d_tw4 = nullptr;           // four-step F-stage (C = 1024) twiddles [k2][l]
    void *d_sm = nullptr;              // its stream-major output before the reorder
    size_t sm_bytes = 0;

    // FP16 tensor-core path
    bool tc = false;
    int rs_kp_max = 0, rs_cgroups = 1;
    size_t rs_smem = 0;
    float rs_inv_sw = 1.f;
    int *d_rs_kp = nullptr, *d_rs_chunk_row = nullptr, *d_rs_chunk_off = nullptr, *d_rs_perm = nullptr,
        *d_err = nullptr;
    long long *d_rs_bimg_off = nullptr;
    CUtensorMap a_map_re{}, a_map_im{};   // TMA maps of the voltage planes (d_yre, d_yim)
    CUtensorMap vp_smap_re{}, vp_smap_im{};   // their store maps (row plane kernel)
    bool vp_tma = true;                       // the row plane kernel stores by TMA boxes (MOFF_VP_TMA=0: directly)
    float *d_rs_row_sh = nullptr, *d_rs_row_inv = nullptr;
    CUtensorMap h_map;                 // tensor-core path: store map of the FP16 field
    int h_map_nt = 0;                  // its sample extent
    // served plans: per-block scratch (field, FP16 voltage planes) lent by a moff_server
    bool served = false;
    size_t h_bytes = 0, y_bytes = 0, scratch_bytes = 0;
    __half *d_rs_bimg = nullptr, *d_yre = nullptr, *d_yim = nullptr;
    float *d_sy = nullptr;
    // dense tensor-core transform (MOFF_PREC_FP16TC at N = 256 or 512 where the row-spectrum
    // contraction does not apply, or MOFF_TC_DFT=1): factored-DFT table image, the kernel scale
    // (power of two: the gridded field times sy[c] * dft_s_t stays within FP16), and the
    // gridding kernel's shared memory for a grid-only (FP32 transform) launch
    bool dft = false;
    unsigned char *d_dft_tab = nullptr;     // rows (gridding kernel, row transform)
    unsigned char *d_dft_tab_r8 = nullptr;  // the 8 x 64 row transform's tables (N = 512)
    bool rows8 = false;                     // row transform of the tensor-core gridding route as 8 x 64
    unsigned char *d_dft_tab_c = nullptr;   // the column kernel's image
    int cols_w = 8;                         // columns per CTA of k_cols_dft
    int cols_w_source = 0;                  // 0 default, 1 measured (MOFF_AUTOTUNE)
    double cols_w_ms[2] = {0.0, 0.0};       // measured ms per chunk at W = 8, 16
    float dft_s_t = 1.f;
    size_t grid_smem_fft = 0;
    // ... with the gridding on the tensor cores too (cell tiles; MOFF_TC_GRID=0 keeps the FP32 gather):
    // tile tables, voltage planes in raster order of anchors (TMA maps of 16-row boxes), and the
    // FP16 gridded field (d_G, the row transform's input; the row-transformed field is d_H)
    bool gtc = false;
    int gt_tiles = 0, gt_kp_max = 0, gt_cgroups = 1, gt_rows = 0, gt_stages = 4, gt_boxes = 1;   // gt_rows: plane rows per channel incl. padding
    size_t gt_smem = 0;
    int *d_gt_tile_cell = nullptr, *d_gt_kp = nullptr, *d_gt_chunk_off = nullptr, *d_gt_chunk_row = nullptr,
        *d_gt_perm = nullptr;
    long long *d_gt_bimg_off = nullptr;
    __half *d_gt_bimg = nullptr;
    unsigned char *d_gt_active = nullptr;
    CUtensorMap gt_map_re{}, gt_map_im{}, gt_map_g{};
    __half *d_G = nullptr;

    long long n_samples = 0;
    size_t dev_bytes = 0;
    std::vector<void *> allocs;

    // MOFF_GRAPH: each block's launch sequence captured once per (kind, input,
    // scratch, length) on a private stream and replayed as one graph launch
    bool graphs = false;
    cudaStream_t gst = nullptr;
    struct GraphEnt { int kind; const void *in, *scratch; long long n, stride; cudaGraphExec_t exec; unsigned long long used; };
    std::vector<GraphEnt> gcache;
    unsigned long long gclock = 0;
    // MOFF_PERSIST: each block's chunks in one persistent launch (k_image_persist)
    bool persist = false;
    size_t persist_smem = 0;
    int *d_pq = nullptr;              // queue head, then rows_done and cols_done [kPersistMaxChunks][Cb]
    long long persist_budget = 0;     // clock64 cycles per wait
    int persist_extra = 0;            // tests only: row items a column item waits for beyond the real ones
    int sms = 152;
    // MOFF_AUTOTUNE: how the gridding shape was chosen (0 rule, 1 measured, 2 cache)
    int tune_source = 0;
    double tune_best_ms = 0.0;

    // feedback calibration (Sec. 6): pixel tap, sums, antenna beams towards the pixel
    bool fb_on = false;
    int fb_kx = -1, fb_ky = -1;
    float2 *d_etap = nullptr;          // [Tb][Cb][P]
    double2 *d_fb_corr = nullptr;      // [C][A*P]
    double *d_fb_power = nullptr;      // [C][P]
    double2 *d_fb_beam = nullptr;      // [A*P]
    float2 *d_fb_out = nullptr;        // [C][A*P] staging of R / delta_g
    long long fb_samples = 0;
    std::vector<float> h_taps;         // host copy of the kernels (per-pol plans), one block per set
    std::vector<double> h_pos;         // host copy of the positions, one block per set
    // channel-dependent positions and kernels (moff_set_channel_groups): n_groups sets,
    // d_chan_group [C] the set of each channel (nullptr while there is one set)
    int n_groups = 1;
    int *d_chan_group = nullptr;
    // autocorrelation subtraction: per-antenna power sums and kernel cross-correlation patches
    bool auto_on = false;
    double2 *d_auto_pw = nullptr;      // [C][A][3]
    double2 *d_auto_X = nullptr;       // [A][NQ][(2K-1)^2]
    double2 *d_auto_Q = nullptr;       // [C][NQ][(2K-1)^2]
    double *d_auto_img = nullptr;      // [C][n_prod][N][N]
    double2 *d_wN = nullptr;           // exp(+2 pi i m / N)
    long long auto_samples = 0;
    // tied-array beams: the field at up to kMaxBeams pixels for every sample of the last block
    int n_beam = 0, beam_kx[kMaxBeams] = {}, beam_ky[kMaxBeams] = {};
    float2 *d_beam = nullptr;
    size_t beam_bytes = 0;
    int beam_T = 0, beam_base = 0;     // beam_base: first sample of the block segment being imaged
    // pipelined host-ADC staging: one event per frame segment
    cudaEvent_t seg_ev[16] = {};
    // pipelined host-voltage staging: while set, the chunk loops make the plan stream wait for
    // seg_ev[(c0 / Cb) / chunk_seg] (the copy of that channel segment) before the chunk's launches
    int chunk_seg = 0;

    // optional per-launch timing: (kind, start, stop)
    bool timing = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> ev_pool;
};

namespace {

template <class T>
moff_status palloc(moff_plan *pl, T **p, size_t bytes) {
    void *q = nullptr;
    cudaError_t e = dev_alloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? MOFF_ENOMEM : MOFF_ECUDA, "device allocation of %zu bytes: %s",
                    bytes, cudaGetErrorString(e));
    }
    pl->allocs.push_back(q);
    pl->dev_bytes += bytes;
    *p = reinterpret_cast<T *>(q);
    return MOFF_OK;
}

void pfree(moff_plan *pl, void *p) {
    if (!p) return;
    auto it = std::find(pl->allocs.begin(), pl->allocs.end(), p);
    if (it != pl->allocs.end()) pl->allocs.erase(it);
    cudaFree(p);
}

void destroy_plan(moff_plan *pl) {
    if (!pl) return;
    if (pl->st) cudaStreamSynchronize(pl->st);
    if (pl->cst) cudaStreamSynchronize(pl->cst);
    for (void *p : pl->allocs) cudaFree(p);
    for (int i = 0; i < 2; ++i) {
        if (pl->ev_copied[i]) cudaEventDestroy(pl->ev_copied[i]);
        if (pl->ev_consumed[i]) cudaEventDestroy(pl->ev_consumed[i]);
    }
    if (pl->ev_done) cudaEventDestroy(pl->ev_done);
    for (auto &r : pl->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (cudaEvent_t e : pl->ev_pool) cudaEventDestroy(e);
    for (auto &g : pl->gcache) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : pl->seg_ev)
        if (e) cudaEventDestroy(e);
    if (pl->gst) cudaStreamDestroy(pl->gst);
    if (pl->cst) cudaStreamDestroy(pl->cst);
    if (pl->own_stream && pl->st) cudaStreamDestroy(pl->st);
    delete pl;
}

moff_status wait_event(cudaEvent_t ev, int timeout_ms) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return MOFF_OK;
        if (e != cudaErrorNotReady) return fail(MOFF_ECUDA, "waiting for the GPU: %s", cudaGetErrorString(e));
        if (timeout_ms >= 0) {
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms >= timeout_ms) return fail(MOFF_ETIMEDOUT, "GPU work not finished after %d ms", timeout_ms);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

moff_status sync_plan(moff_plan *pl, int timeout_ms) {
    MOFF_CK(cudaEventRecord(pl->ev_done, pl->st));
    return wait_event(pl->ev_done, timeout_ms);
}

cudaEvent_t pool_event(moff_plan *pl) {
    if (!pl->ev_pool.empty()) {
        cudaEvent_t e = pl->ev_pool.back();
        pl->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one launch with events when timing is on.
struct TimedLaunch {
    moff_plan *pl;
    int kind;
    cudaEvent_t a = nullptr;
    TimedLaunch(moff_plan *p, int k) : pl(p), kind(k) {
        if (pl->timing) {
            a = pool_event(pl);
            cudaEventRecord(a, pl->st);
        }
    }
    void done() {
        if (a) {
            cudaEvent_t b = pool_event(pl);
            cudaEventRecord(b, pl->st);
            pl->recs.push_back(moff_plan::Rec{kind, a, b});
            a = nullptr;
        }
    }
};

void clear_recs(moff_plan *pl) {
    for (auto &r : pl->recs) {
        pl->ev_pool.push_back(r.a);
        pl->ev_pool.push_back(r.b);
    }
    pl->recs.clear();
}

// Report (and clear) a bounded wait that gave up inside a kernel.
moff_status check_device_err(moff_plan *pl) {
    if (!pl->d_err) return MOFF_OK;
    int h = 0;
    MOFF_CK(cudaMemcpy(&h, pl->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        MOFF_CK(cudaMemset(pl->d_err, 0, sizeof(int)));
        return fail(MOFF_ETIMEDOUT, "a bounded wait inside a kernel ran out of time (tensor-core completion or "
                                    "persistent work-queue dependency)");
    }
    return MOFF_OK;
}

// Copy a host block into the next staging buffer on the copy stream; the
// compute stream waits for the copy, and the host waits until the copy has
// finished (so the caller may reuse its buffer).  Returns the device copy.
moff_status stage_in(moff_plan *pl, const void *host, size_t bytes, const void **dev, int *slot) {
    const int i = (int)(pl->nsub & 1);
    if (pl->stage_bytes[i] < bytes) {
        MOFF_CK(cudaEventSynchronize(pl->ev_consumed[i]));
        pfree(pl, pl->d_stage[i]);
        pl->dev_bytes -= pl->stage_bytes[i];
        pl->d_stage[i] = nullptr;
        pl->stage_bytes[i] = 0;
        moff_status s = palloc(pl, &pl->d_stage[i], bytes);
        if (s != MOFF_OK) return s;
        pl->stage_bytes[i] = bytes;
    }
    MOFF_CK(cudaStreamWaitEvent(pl->cst, pl->ev_consumed[i], 0));
    MOFF_CK(cudaMemcpyAsync(pl->d_stage[i], host, bytes, cudaMemcpyHostToDevice, pl->cst));
    MOFF_CK(cudaEventRecord(pl->ev_copied[i], pl->cst));
    MOFF_CK(cudaStreamWaitEvent(pl->st, pl->ev_copied[i], 0));
    *dev = pl->d_stage[i];
    *slot = i;
    return MOFF_OK;
}

// After the compute that reads staging slot i is enqueued: mark it and wait for the copy.
moff_status stage_done(moff_plan *pl, int i) {
    MOFF_CK(cudaEventRecord(pl->ev_consumed[i], pl->st));
    pl->nsub++;
    return wait_event(pl->ev_copied[i], -1);
}

// Channel chunk c0 of a block staged by channel segments: wait for its segment's copy.
inline moff_status chunk_ready(moff_plan *pl, int c0) {
    if (pl->chunk_seg > 0) {
        const int c = c0 / pl->Cb;
        if (c % pl->chunk_seg == 0) MOFF_CK(cudaStreamWaitEvent(pl->st, pl->seg_ev[c / pl->chunk_seg], 0));
    }
    return MOFF_OK;
}

// Host voltages [T][C][A][P] copied to staging slot i by channel segments (one cudaMemcpy2DAsync
// per segment: its channels of every sample) on the copy stream, so imaging of the first
// channel chunks starts while later ones are still in flight.  The launches and so the
// image equal a device-input submit's.
moff_status stage_in_by_channels(moff_plan *pl, const uint8_t *host, int n_time, const void **dev, int *slot) {
    const int i = (int)(pl->nsub & 1);
    const size_t cap = (size_t)pl->C * pl->A * pl->P, bytes = (size_t)n_time * cap;
    if (pl->stage_bytes[i] < bytes) {
        MOFF_CK(cudaEventSynchronize(pl->ev_consumed[i]));
        pfree(pl, pl->d_stage[i]);
        pl->dev_bytes -= pl->stage_bytes[i];
        pl->d_stage[i] = nullptr;
        pl->stage_bytes[i] = 0;
        moff_status s = palloc(pl, &pl->d_stage[i], bytes);
        if (s != MOFF_OK) return s;
        pl->stage_bytes[i] = bytes;
    }
    for (cudaEvent_t &e : pl->seg_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(MOFF_ECUDA, "event creation failed");
    const int nseg_max = (int)(sizeof(pl->seg_ev) / sizeof(pl->seg_ev[0]));
    const int nchunk = (pl->C + pl->Cb - 1) / pl->Cb;
    const int per = (nchunk + nseg_max - 1) / nseg_max;       // channel chunks per segment
    const size_t ap = (size_t)pl->A * pl->P;
    uint8_t *dst = static_cast<uint8_t *>(pl->d_stage[i]);
    MOFF_CK(cudaStreamWaitEvent(pl->cst, pl->ev_consumed[i], 0));
    for (int k = 0, e = 0; k < nchunk; k += per, ++e) {
        const size_t c0 = (size_t)k * pl->Cb, c1 = std::min<size_t>(pl->C, (size_t)(k + per) * pl->Cb);
        MOFF_CK(cudaMemcpy2DAsync(dst + c0 * ap, cap, host + c0 * ap, cap, (c1 - c0) * ap, (size_t)n_time,
                                  cudaMemcpyHostToDevice, pl->cst));
        MOFF_CK(cudaEventRecord(pl->seg_ev[e], pl->cst));
    }
    MOFF_CK(cudaEventRecord(pl->ev_copied[i], pl->cst));
    pl->chunk_seg = per;
    *dev = dst;
    *slot = i;
    return MOFF_OK;
}

// Gridding-kernel arguments of a plan for channels [c0, c0+nc), samples [t0, t0+nt).
GridArgs grid_args(const moff_plan *pl, const uint8_t *volt, long long tstride, int t0, int nt, int c0, int nc) {
    GridArgs g{};
    g.volt = volt;
    g.volt_tstride = tstride;
    g.t0 = t0;
    g.nt = nt;
    g.c0 = c0;
    g.nc = nc;
    g.A = pl->A;
    g.rows = pl->rows;
    g.max_nloc = pl->max_nloc;
    g.max_entries = pl->max_entries;
    g.n_slices = pl->n_slices;
    g.gains = pl->d_gains;
    g.st_ant_off = pl->d_st_ant_off;
    g.st_ant = pl->d_st_ant;
    g.slice_off = pl->d_slice_off;
    g.lane_cell = pl->d_lane_cell;
    g.con_tap = pl->d_con_tap;
    g.con_y = pl->d_con_y;
    g.twp = pl->d_twp;
    g.out = pl->d_H;
    // channel-major slabs: a channel's samples of one chunk are contiguous, so the
    // time batch a CTA writes, and the samples a column CTA reads, share pages
    g.slab_t = 1;
    g.slab_c = pl->Tb;
    g.pairs = pl->pairs ? 1 : 0;
    g.quads = pl->quads ? 1 : 0;
    g.wide = pl->wide ? 1 : 0;
    g.chan_group = pl->d_chan_group;
    g.row_nz = pl->d_row_nz;
    return g;
}

#define MOFF_CK_S(call)                     \
    do {                                    \
        moff_status s_ = (call);            \
        if (s_ != MOFF_OK) return s_;       \
    } while (0)

void set_tap(const moff_plan *pl, ColArgs *ca, int t0) {
    ca->etap = pl->fb_on ? pl->d_etap : nullptr;
    ca->tap_kx = pl->fb_kx;
    ca->tap_ky = pl->fb_ky;
    ca->n_beam = pl->n_beam;
    ca->beam_out = pl->n_beam ? pl->d_beam : nullptr;
    ca->beam_t0 = pl->beam_base + t0;
    ca->beam_C = pl->C;
    for (int j = 0; j < pl->n_beam; ++j) {
        ca->beam_kx[j] = pl->beam_kx[j];
        ca->beam_ky[j] = pl->beam_ky[j];
    }
}

// Feedback calibration and autocorrelation sums of one chunk (after its column
// launch wrote the pixel tap).
moff_status run_feedback(moff_plan *pl, const uint8_t *volt, long long tstride, int t0, int nt, int c0, int nc) {
    if (pl->auto_on) {
        FbArgs f{};
        f.volt = volt;
        f.tstride = tstride;
        f.t0 = t0;
        f.nt = nt;
        f.c0 = c0;
        f.nc = nc;
        f.AP = pl->A * pl->P;
        f.P = pl->P;
        f.gains = pl->d_gains;
        f.corr = pl->d_auto_pw;
        TimedLaunch ta(pl, 6);
        MOFF_CK(launch_auto_acc(f, pl->st));
        ta.done();
    }
    if (!pl->fb_on) return MOFF_OK;
    FbArgs f{};
    f.volt = volt;
    f.tstride = tstride;
    f.t0 = t0;
    f.nt = nt;
    f.c0 = c0;
    f.nc = nc;
    f.AP = pl->A * pl->P;
    f.P = pl->P;
    f.gains = pl->d_gains;
    f.etap = pl->d_etap;
    f.corr = pl->d_fb_corr;
    f.power = pl->d_fb_power;
    TimedLaunch tf(pl, 5);
    MOFF_CK(launch_fb_corr(f, pl->st));
    tf.done();
    return MOFF_OK;
}

moff_status run_image_tc(moff_plan *pl, const uint8_t *volt, int n_time, long long tstride) {
    const int AP = pl->A * pl->P;
    for (int c0 = 0; c0 < pl->C; c0 += pl->Cb) {
        if (moff_status w = chunk_ready(pl, c0); w != MOFF_OK) return w;
        const int nc = std::min(pl->Cb, pl->C - c0);
        for (int t0 = 0; t0 < n_time; t0 += pl->Tb) {
            const int nt = std::min(pl->Tb, n_time - t0);
            TimedLaunch tv(pl, 3);
            MOFF_CK(launch_volt_prep(volt, tstride, t0, nt, c0, nc, AP, AP + kRowSpecPad, pl->d_gains, pl->d_sy,
                                     pl->d_rs_perm, pl->Tb, pl->d_yre, pl->d_yim, pl->st, -1,
                                     pl->vp_tma ? &pl->vp_smap_re : nullptr, pl->vp_tma ? &pl->vp_smap_im : nullptr));
            tv.done();
            RowSpecArgs ra{};
            ra.P = pl->P;
            ra.nt = nt;
            ra.nc = nc;
            ra.c0 = c0;
            ra.AP = AP + kRowSpecPad;
            ra.Tpad = pl->Tb;
            ra.kp_max = pl->rs_kp_max;
            ra.kp = pl->d_rs_kp;
            ra.chunk_off = pl->d_rs_chunk_off;
            ra.chunk_row = pl->d_rs_chunk_row;
            ra.bimg_off = pl->d_rs_bimg_off;
            ra.bimg = pl->d_rs_bimg;
            ra.sy = pl->d_sy;
            ra.inv_sw = pl->rs_inv_sw;
            ra.row_sh = pl->d_rs_row_sh;
            ra.H = reinterpret_cast<__half2 *>(pl->d_H);
            ra.slab_t = pl->Cb;   // [Tb][Cb] slabs: the layout the field's tensor map describes
            ra.slab_c = 1;
            ra.err = pl->d_err;
            if (pl->h_map_nt != nt) {   // a short block: drop the stores of the padding samples
                if (encode_field_map(&pl->h_map, pl->d_H, pl->N, pl->P, pl->Cb, nt) != cudaSuccess)
                    return fail(MOFF_ECUDA, "tensor map of the row-transformed field could not be encoded");
                pl->h_map_nt = nt;
            }
            TimedLaunch tg(pl, 1);
            MOFF_CK(launch_rowspec(pl->N, ra, pl->h_map, pl->a_map_re, pl->a_map_im, std::min(pl->rs_cgroups, nc),
                                   pl->rs_smem, pl->st));
            tg.done();
            ColArgs ca{};
            ca.H = pl->d_H;
            ca.nt = nt;
            ca.c0 = c0;
            ca.nc = nc;
            ca.twp = pl->d_twp;
            ca.acc = pl->d_acc;
            ca.row_nz = pl->d_row_nz;
            ca.slab_t = ra.slab_t;
            ca.slab_c = ra.slab_c;
            ca.row_inv = pl->d_rs_row_inv;
            ca.sy = pl->d_sy;
            ca.inv_sw = pl->rs_inv_sw;
            set_tap(pl, &ca, t0);
            TimedLaunch tc(pl, 2);
            MOFF_CK(launch_cols(pl->N, pl->P, ca, pl->st, true));
            tc.done();
            MOFF_CK_S(run_feedback(pl, volt, tstride, t0, nt, c0, nc));
        }
    }
    return MOFF_OK;
}

constexpr size_t kGraphCache = 8;

void drop_graphs(moff_plan *pl) {
    for (auto &g : pl->gcache) cudaGraphExecDestroy(g.exec);
    pl->gcache.clear();
}

// Run one block's launch sequence `enqueue` (which launches on pl->st).  With
// MOFF_GRAPH (and timing off) the sequence is captured on the plan's private
// capture stream the first time a (kind, input, scratch, length) key is seen
// and replayed as one graph launch on pl->st afterwards.
template <class F>
moff_status launch_block(moff_plan *pl, int kind, const void *in, long long n, long long stride, F &&enqueue) {
    if (!pl->graphs || pl->timing) return enqueue();
    const void *scratch = pl->d_H;
    for (auto &g : pl->gcache)
        if (g.kind == kind && g.in == in && g.scratch == scratch && g.n == n && g.stride == stride) {
            g.used = ++pl->gclock;
            MOFF_CK(cudaGraphLaunch(g.exec, pl->st));
            return MOFF_OK;
        }
    cudaStream_t user = pl->st;
    pl->st = pl->gst;
    if (cudaStreamBeginCapture(pl->gst, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        pl->st = user;
        cudaGetLastError();
        return fail(MOFF_ECUDA, "stream capture could not start");
    }
    moff_status s = enqueue();
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(pl->gst, &graph);
    pl->st = user;
    if (s != MOFF_OK || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return s != MOFF_OK ? s : fail(MOFF_ECUDA, "stream capture failed: %s", cudaGetErrorString(ec));
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return fail(MOFF_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
    }
    if (pl->gcache.size() >= kGraphCache) {
        auto lru = std::min_element(pl->gcache.begin(), pl->gcache.end(),
                                    [](const moff_plan::GraphEnt &a, const moff_plan::GraphEnt &b) { return a.used < b.used; });
        cudaGraphExecDestroy(lru->exec);
        pl->gcache.erase(lru);
    }
    pl->gcache.push_back(moff_plan::GraphEnt{kind, in, scratch, n, stride, exec, ++pl->gclock});
    MOFF_CK(cudaGraphLaunch(exec, pl->st));
    return MOFF_OK;
}

// Dense FP16 path: gridding + row transform on the tensor cores, then the column transform
// + square-and-integrate on the tensor cores, per (Tb, Cb) chunk.
moff_status run_image_dft(moff_plan *pl, const uint8_t *volt, int n_time, long long tstride) {
    const int cpl = pl->quads ? 4 : (pl->pairs ? 2 : 1);
    for (int c0 = 0; c0 < pl->C; c0 += pl->Cb) {
        if (moff_status w = chunk_ready(pl, c0); w != MOFF_OK) return w;
        const int nc = std::min(pl->Cb, pl->C - c0);
        for (int t0 = 0; t0 < n_time; t0 += pl->Tb) {
            const int nt = std::min(pl->Tb, n_time - t0);
            GridArgs g = grid_args(pl, volt, tstride, t0, nt, c0, nc);
            g.out = nullptr;
            g.h16 = reinterpret_cast<__half *>(pl->d_H);
            g.sy = pl->d_sy;
            g.s_t = pl->dft_s_t;
            g.dft_tab = pl->d_dft_tab;
            g.err = pl->d_err;
            TimedLaunch tg(pl, 1);
            MOFF_CK(launch_grid_dft(pl->N, pl->P, pl->tb, cpl, g, pl->n_stripes, pl->grid_smem, pl->st));
            tg.done();
            ColDftArgs ca{};
            ca.H = reinterpret_cast<const __half *>(pl->d_H);
            ca.slab_t = g.slab_t;
            ca.slab_c = g.slab_c;
            ca.nt = nt;
            ca.c0 = c0;
            ca.nc = nc;
            ca.acc = pl->d_acc;
            ca.row_nz = pl->d_row_nz;
            ca.sy = pl->d_sy;
            ca.s_t = pl->dft_s_t;
            ca.dft_tab = pl->d_dft_tab_c;
            ca.err = pl->d_err;
            TimedLaunch tc(pl, 2);
            MOFF_CK(launch_cols_dft(pl->N, pl->P, pl->cols_w, ca, pl->st));
            tc.done();
            MOFF_CK_S(run_feedback(pl, volt, tstride, t0, nt, c0, nc));
        }
    }
    return MOFF_OK;
}

// Dense FP16 path with the gridding on the tensor cores: voltage planes, cell-tile gridding,
// row transform, column transform + square-and-integrate, per (Tb, Cb) chunk.
moff_status run_image_gtc(moff_plan *pl, const uint8_t *volt, int n_time, long long tstride) {
    const int AP = pl->A * pl->P;
    for (int c0 = 0; c0 < pl->C; c0 += pl->Cb) {
        if (moff_status w = chunk_ready(pl, c0); w != MOFF_OK) return w;
        const int nc = std::min(pl->Cb, pl->C - c0);
        for (int t0 = 0; t0 < n_time; t0 += pl->Tb) {
            const int nt = std::min(pl->Tb, n_time - t0);
            TimedLaunch tv(pl, 3);
            MOFF_CK(launch_volt_prep(volt, tstride, t0, nt, c0, nc, AP, pl->gt_rows, pl->d_gains, pl->d_sy,
                                     pl->d_gt_perm, pl->Tb, pl->d_yre, pl->d_yim, pl->st, pl->gt_rows - kRowSpecPad,
                                     pl->vp_tma ? &pl->vp_smap_re : nullptr, pl->vp_tma ? &pl->vp_smap_im : nullptr));
            tv.done();
            GridTcArgs ga{};
            ga.P = pl->P;
            ga.N = pl->N;
            ga.nt = nt;
            ga.nc = nc;
            ga.c0 = c0;
            ga.AP = pl->gt_rows;
            ga.kp_max = pl->gt_kp_max;
            ga.stages = pl->gt_stages;
            ga.boxes = pl->gt_boxes;
            ga.tile_cell = pl->d_gt_tile_cell;
            ga.kp = pl->d_gt_kp;
            ga.chunk_off = pl->d_gt_chunk_off;
            ga.chunk_row = pl->d_gt_chunk_row;
            ga.bimg_off = pl->d_gt_bimg_off;
            ga.bimg = pl->d_gt_bimg;
            ga.G = pl->d_G;
            ga.Tb = pl->Tb;
            ga.err = pl->d_err;
            TimedLaunch tg(pl, 1);
            MOFF_CK(launch_grid_tc(ga, pl->gt_map_re, pl->gt_map_im, pl->gt_map_g, pl->gt_tiles,
                                   std::min(pl->gt_cgroups, nc), pl->gt_smem, pl->st));
            tg.done();
            RowDftArgs ra{};
            ra.G = pl->d_G;
            ra.Tb = pl->Tb;
            ra.H = reinterpret_cast<__half *>(pl->d_H);
            ra.slab_t = 1;
            ra.slab_c = pl->Tb;
            ra.nt = nt;
            ra.c0 = c0;
            ra.nc = nc;
            ra.row_nz = pl->d_row_nz;
            ra.active = pl->d_gt_active;
            ra.dft_tab = pl->rows8 ? pl->d_dft_tab_r8 : pl->d_dft_tab;
            ra.err = pl->d_err;
            TimedLaunch tr(pl, 7);
            MOFF_CK(pl->rows8 ? launch_rows_dft8(pl->P, ra, pl->st) : launch_rows_dft(pl->N, pl->P, ra, pl->st));
            tr.done();
            ColDftArgs ca{};
            ca.H = reinterpret_cast<const __half *>(pl->d_H);
            ca.slab_t = 1;
            ca.slab_c = pl->Tb;
            ca.nt = nt;
            ca.c0 = c0;
            ca.nc = nc;
            ca.acc = pl->d_acc;
            ca.row_nz = pl->d_row_nz;
            ca.sy = pl->d_sy;
            ca.s_t = pl->dft_s_t;
            ca.dft_tab = pl->d_dft_tab_c;
            ca.err = pl->d_err;
            TimedLaunch tc(pl, 2);
            MOFF_CK(launch_cols_dft(pl->N, pl->P, pl->cols_w, ca, pl->st));
            tc.done();
            MOFF_CK_S(run_feedback(pl, volt, tstride, t0, nt, c0, nc));
        }
    }
    return MOFF_OK;
}

// Batching pattern: the block's (Tb, Cb) chunks, in the direct launches' order, as the work items
// of one persistent launch (k_image_persist; up to kPersistMaxChunks chunks per launch).
moff_status run_image_persist(moff_plan *pl, const uint8_t *volt, int n_time, long long tstride) {
    std::vector<int4> chunks;
    for (int c0 = 0; c0 < pl->C; c0 += pl->Cb)
        for (int t0 = 0; t0 < n_time; t0 += pl->Tb)
            chunks.push_back(make_int4(t0, std::min(pl->Tb, n_time - t0), c0, std::min(pl->Cb, pl->C - c0)));
    const int cpl = pl->quads ? 4 : (pl->pairs ? 2 : 1);
    const int n_strips = pl->N / col_width(pl->N);
    for (size_t k0 = 0; k0 < chunks.size(); k0 += kPersistMaxChunks) {
        const int nch = (int)std::min<size_t>(kPersistMaxChunks, chunks.size() - k0);
        PersistArgs pa{};
        pa.g = grid_args(pl, volt, tstride, 0, 0, 0, 0);
        pa.ca.H = pl->d_H;
        pa.ca.slab_t = pa.g.slab_t;
        pa.ca.slab_c = pa.g.slab_c;
        pa.ca.twp = pl->d_twp;
        pa.ca.acc = pl->d_acc;
        pa.ca.row_nz = pl->d_row_nz;
        pa.n_chunks = nch;
        pa.n_stripes = pl->n_stripes;
        pa.n_strips = n_strips;
        pa.cb = pl->Cb;
        pa.rows_extra = pl->persist_extra;
        pa.next = pl->d_pq;
        pa.rows_done = pl->d_pq + 1;
        pa.cols_done = pl->d_pq + 1 + (size_t)kPersistMaxChunks * pl->Cb;
        pa.status = pl->d_err;
        pa.budget = pl->persist_budget;
        int items = 0;
        for (int k = 0; k < nch; ++k) {
            pa.chunks[k] = chunks[k0 + k];
            pa.item0[k] = items;
            items += (pl->n_stripes + n_strips) * pa.chunks[k].w;
        }
        pa.item0[nch] = items;
        pa.n_items = items;
        MOFF_CK(cudaMemsetAsync(pl->d_pq, 0, sizeof(int), pl->st));
        MOFF_CK(cudaMemsetAsync(pa.rows_done, 0, (size_t)nch * pl->Cb * sizeof(int), pl->st));
        MOFF_CK(cudaMemsetAsync(pa.cols_done, 0, (size_t)nch * pl->Cb * sizeof(int), pl->st));
        TimedLaunch tp(pl, 8);
        MOFF_CK(launch_persist(pl->N, pl->P, cpl, pl->wide, pa, pl->persist_smem, pl->sms, pl->st));
        tp.done();
    }
    return MOFF_OK;
}

moff_status run_image(moff_plan *pl, const uint8_t *volt, int n_time, long long tstride) {
    if (pl->gtc) return run_image_gtc(pl, volt, n_time, tstride);
    if (pl->dft) return run_image_dft(pl, volt, n_time, tstride);
    if (pl->tc) return run_image_tc(pl, volt, n_time, tstride);
    if (pl->persist && !pl->fb_on && !pl->auto_on && pl->n_beam == 0) return run_image_persist(pl, volt, n_time, tstride);
    for (int c0 = 0; c0 < pl->C; c0 += pl->Cb) {
        if (moff_status w = chunk_ready(pl, c0); w != MOFF_OK) return w;
        const int nc = std::min(pl->Cb, pl->C - c0);
        for (int t0 = 0; t0 < n_time; t0 += pl->Tb) {
            const int nt = std::min(pl->Tb, n_time - t0);
            GridArgs g = grid_args(pl, volt, tstride, t0, nt, c0, nc);
            TimedLaunch tg(pl, 1);
            MOFF_CK(launch_grid(pl->N, pl->P, pl->tb, pl->staged, false, g, pl->n_stripes, pl->grid_smem, pl->st));
            tg.done();
            ColArgs ca{};
            ca.H = pl->d_H;
            ca.nt = nt;
            ca.c0 = c0;
            ca.nc = nc;
            ca.slab_t = g.slab_t;
            ca.slab_c = g.slab_c;
            ca.twp = pl->d_twp;
            ca.acc = pl->d_acc;
            ca.row_nz = pl->d_row_nz;
            set_tap(pl, &ca, t0);
            TimedLaunch tc(pl, 2);
            MOFF_CK(launch_cols(pl->N, pl->P, ca, pl->st));
            tc.done();
            MOFF_CK_S(run_feedback(pl, volt, tstride, t0, nt, c0, nc));
        }
    }
    return MOFF_OK;
}

// Per-antenna kernel value (re, im) for output pol po, input pol pi at (iy, ix).
inline void tap_at(bool jones, int P, int K, const float *taps, int a, int po, int pi, int iy, int ix, float *re,
                   float *im) {
    long long idx;
    if (jones) {
        idx = ((((long long)a * 2 + po) * 2 + pi) * K + iy) * K + ix;
    } else {
        if (po != pi) { *re = 0.f; *im = 0.f; return; }
        idx = (((long long)a * P + po) * K + iy) * K + ix;
    }
    *re = taps[2 * idx];
    *im = taps[2 * idx + 1];
}

struct Contrib {
    int cell;
    int y;
    float2 tap;
};

}  // namespace

namespace moff {

moff_status fail_msg(moff_status s, const char *msg) { return fail(s, "%s", msg); }

// Bin every antenna's kernel by grid-row stripe into per-cell contribution
// lists (host only).  The stripe height is the largest power of two <= 16
// whose lists fit the gridding kernel's shared-memory budget.
moff_status build_bins(int A, int K, int N, int P, bool jones, const double *pos, const float *taps, Bins *b,
                       const GridChoice *force, bool dft) {
    const int h = K / 2;
    std::vector<int> ax(A), ay(A);
    for (int a = 0; a < A; ++a) {
        const double x = pos[2 * a], y = pos[2 * a + 1];
        if (!std::isfinite(x) || !std::isfinite(y) || std::fabs(x) > 1e9 || std::fabs(y) > 1e9)
            return fail(MOFF_EINVAL, "antenna %d position is not finite or out of range", a);
        long long fx = (long long)std::floor(x + 0.5), fy = (long long)std::floor(y + 0.5);
        ax[a] = (int)(((fx % N) + N) % N);
        ay[a] = (int)(((fy % N) + N) % N);
    }
    const int pin_n = jones ? 2 : 1;   // input pols per output pol
    const int tw_total = fft_tw_total(N);
    const char *wide_env = getenv("MOFF_GRID_WIDE");
    // the tensor-core row transform runs on stripes of grid_fft_rows(N) rows with entries through L2
    const bool wide = !dft && (force ? force->wide : (wide_env && atoi(wide_env) != 0));
    const int F = grid_fft_rows(N) * (wide ? 2 : 1);
    const size_t budget = 110 * 1024;   // two CTAs per SM
    const size_t big = 225 * 1024;      // one CTA per SM: dense arrays, where more samples per pass reuse each tap
    // Contributions per grid cell (p_out, row, col), independent of the stripe shape.
    std::vector<int> cnt_all((size_t)P * N * N, 0);
    for (int a = 0; a < A; ++a)
        for (int po = 0; po < P; ++po)
            for (int k = 0; k < pin_n; ++k) {
                const int pi = jones ? k : po;
                for (int iy = 0; iy < K; ++iy) {
                    const int row = (ay[a] + iy - h + N) % N;
                    for (int ix = 0; ix < K; ++ix) {
                        float re, im;
                        tap_at(jones, P, K, taps, a, po, pi, iy, ix, &re, &im);
                        if (re != 0.f || im != 0.f) cnt_all[((size_t)po * N + row) * N + (ax[a] + ix - h + N) % N]++;
                    }
                }
            }
    // Stripe shape: F = TB * P * rows rows are transformed together.  Prefer
    // kernel entries staged in shared memory, then more samples per pass.
    // The built-in rule takes cell pairs unless MOFF_GRID_PAIRS=0.
    const char *pairs_env = getenv("MOFF_GRID_PAIRS");
    const char *quads_env = getenv("MOFF_GRID_QUADS");
    // 2 x 2 cell blocks per lane (entries through L2, even stripe height); else pairs or single cells
    const bool quads = force ? force->quads : (quads_env && atoi(quads_env) != 0);
    const bool pairs = !quads && (force ? force->pairs : !(pairs_env && atoi(pairs_env) == 0));
    struct Cand { int tb, rows, nloc; long long entries; size_t sm_staged, sm_plain; };
    std::vector<Cand> cands;
    for (int tb = 8; tb >= 1; tb /= 2) {
        int rows = F / (tb * P);
        if (rows < 1) continue;
        rows = std::min(rows, N);
        const int ns = N / rows;
        std::vector<int> nloc(ns, 0), seen(ns, -1);
        for (int a = 0; a < A; ++a)
            for (int iy = 0; iy < K; ++iy) {
                const int s = ((ay[a] + iy - h + N) % N) / rows;
                if (seen[s] != a) { seen[s] = a; nloc[s]++; }
            }
        const int mnl = std::max(1, *std::max_element(nloc.begin(), nloc.end()));
        if ((long long)mnl * P >= 65536) continue;
        long long ment = 0;
        std::vector<int> c((size_t)P * rows * N);
        for (int s = 0; s < ns; ++s) {
            size_t n = 0;
            for (int po = 0; po < P; ++po)
                for (int rl = 0; rl < rows; ++rl)
                    for (int x = 0; x < N; ++x) c[n++] = cnt_all[((size_t)po * N + s * rows + rl) * N + x];
            if (pairs)   // a pair's joint list is at most the sum of its two cells' lists
                for (size_t k = 0; k < c.size() / 2; ++k) c[k] = c[2 * k] + c[2 * k + 1];
            const size_t nu = pairs ? c.size() / 2 : c.size();
            std::sort(c.begin(), c.begin() + nu, [](int x, int y) { return x > y; });
            long long e = 0;
            for (size_t k = 0; k < nu; k += 32) e += 32LL * c[k];
            ment = std::max(ment, e);
        }
        Cand cd{tb, rows, mnl, ment,
                dft ? (size_t)1 << 40
                    : grid_smem_bytes(N, P, tb, rows, mnl, tw_total, (int)std::min<long long>(ment, 1 << 28), pairs),
                dft ? grid_smem_bytes_dft(N, P, tb, rows, mnl) : grid_smem_bytes(N, P, tb, rows, mnl, tw_total, 0, pairs)};
        cands.push_back(cd);
    }
    // Entries are read through L2 by default (more CTAs per SM measured faster
    // than shared-memory staging); MOFF_GRID_STAGE=1 prefers staging.
    const char *stage_env = getenv("MOFF_GRID_STAGE");
    const bool prefer_staged = !dft && stage_env && atoi(stage_env) != 0;
    const Cand *pick = nullptr;
    bool staged = false;
    if (force) {
        for (const Cand &cd : cands)
            if (cd.tb == force->tb) {
                const bool fits = !(dft && force->staged) && (force->staged ? cd.sm_staged : cd.sm_plain) <= big &&
                                  !(quads && (force->staged || cd.rows % 2));
                if (fits) { pick = &cd; staged = force->staged; }
                break;
            }
        if (!pick)
            return fail(MOFF_EINVAL, "gridding shape tb=%d staged=%d quads=%d does not fit", force->tb,
                        (int)force->staged, (int)quads);
    }
    // Pair lanes relieve the voltage reads, so the rule then prefers 4 samples per
    // pass (fewer registers per lane) before 8; single-cell lanes prefer 8.
    std::vector<const Cand *> pref;
    for (int want : pairs || quads ? std::vector<int>{4, 8, 2, 1} : std::vector<int>{8, 4, 2, 1})
        for (const Cand &cd : cands)
            if (cd.tb == want && !(quads && cd.rows % 2)) pref.push_back(&cd);
    if (!pick && prefer_staged && !quads)
        for (const Cand *cd : pref)
            if (cd->sm_staged <= budget) { pick = cd; staged = true; break; }
    if (!pick)
        for (const Cand *cd : pref)
            if (cd->sm_plain <= budget) { pick = cd; break; }
    if (!pick)   // dense arrays: one CTA per SM, still preferring more samples per pass
        for (const Cand *cd : pref)
            if (cd->sm_plain <= big) { pick = cd; break; }
    if (!pick)
        return fail(MOFF_EINVAL, "array too dense for the gridding kernel (antennas per grid row exceed its limits)");
    if (pick->rows * pick->tb * P != F)
        return fail(MOFF_EINVAL, "internal: stripe shape %d x %d x %d does not fill %d rows", pick->tb, P, pick->rows, F);
    b->rows = pick->rows;
    b->tb = pick->tb;
    b->n_stripes = N / pick->rows;
    b->max_nloc = pick->nloc;
    b->staged = staged;
    b->pairs = pairs;
    b->quads = quads;
    b->wide = wide;
    b->max_entries = staged ? (int)pick->entries : 0;
    b->grid_smem = staged ? pick->sm_staged : pick->sm_plain;

    // Per stripe: local antennas (ascending) and every cell's contributions,
    // antenna-major within a cell.
    const int rows = b->rows, ns = b->n_stripes;
    const int ncell = P * rows * N;                 // a multiple of 32 (N >= 32)
    const int cpl = quads ? 4 : (pairs ? 2 : 1);    // cells per lane
    const int nunit = ncell / cpl;                  // lanes: cells, pairs (x even, x + 1) or 2 x 2 blocks
    if (nunit % 32) return fail(MOFF_EINVAL, "internal: %d gridding lanes per stripe is not a multiple of 32", nunit);
    const int nsl = nunit / 32;
    b->n_slices = nsl;
    std::vector<std::vector<int>> sant(ns);
    std::vector<std::vector<Contrib>> scon(ns);
    for (int a = 0; a < A; ++a) {
        for (int iy = 0; iy < K; ++iy) {
            const int s = ((ay[a] + iy - h + N) % N) / rows;
            if (sant[s].empty() || sant[s].back() != a) sant[s].push_back(a);
        }
        for (int po = 0; po < P; ++po)
            for (int k = 0; k < pin_n; ++k) {
                const int pi = jones ? k : po;
                for (int iy = 0; iy < K; ++iy) {
                    const int row = (ay[a] + iy - h + N) % N;
                    const int s = row / rows, rl = row % rows;
                    const int la = (int)sant[s].size() - 1;   // antenna a was appended last
                    for (int ix = 0; ix < K; ++ix) {
                        float re, im;
                        tap_at(jones, P, K, taps, a, po, pi, iy, ix, &re, &im);
                        if (re == 0.f && im == 0.f) continue;
                        const int col = (ax[a] + ix - h + N) % N;
                        scon[s].push_back(Contrib{(po * rows + rl) * N + col, la * P + pi, make_float2(re, im)});
                    }
                }
            }
    }
    b->row_nz.assign((size_t)(N + 31) / 32, 0u);
    for (int a = 0; a < A; ++a)
        for (int iy = 0; iy < K; ++iy) {
            const int row = (ay[a] + iy - h + N) % N;
            b->row_nz[row >> 5] |= 1u << (row & 31);
        }
    b->ant_off.assign(ns + 1, 0);
    b->ant_list.clear();
    b->slice_off.assign((size_t)ns * nsl + 1, 0);
    b->lane_cell.assign((size_t)ns * nsl * 32, 0);
    b->con_tap.clear();
    b->con_y.clear();
    long long base = 0;
    // Per unit (cell, pair of cells or 2 x 2 block) its entry list: (voltage index,
    // tap of each of the unit's cells).  A cell's contributions keep their order
    // (ascending voltage index = antenna-major), so a pair or block lane sums each
    // of its cells in exactly the order a single-cell lane would (plus exact zero terms).
    // Unit of cell (row f, column x): a pair is (f, x / 2), a block (f / 2, x / 2); the
    // cell's slot in the unit is x & 1 (+ 2 (f & 1) in a block).
    struct Ent { int y; float2 t[4]; };
    auto unit_of = [&](int cell, int *slot) {
        if (cpl == 1) { *slot = 0; return cell; }
        if (cpl == 2) { *slot = cell & 1; return cell / 2; }
        const int f = cell / N, x = cell % N;
        *slot = (x & 1) + 2 * (f & 1);
        return (f / 2) * (N / 2) + x / 2;
    };
    auto first_cell = [&](int u) {
        if (cpl == 1) return u;
        if (cpl == 2) return 2 * u;
        return 2 * (u / (N / 2)) * N + 2 * (u % (N / 2));
    };
    std::vector<std::vector<Ent>> lists(nunit);
    std::vector<int> order(nunit);
    const float2 zero = make_float2(0.f, 0.f);
    for (int s = 0; s < ns; ++s) {
        b->ant_off[s + 1] = b->ant_off[s] + (int)sant[s].size();
        b->ant_list.insert(b->ant_list.end(), sant[s].begin(), sant[s].end());
        auto &v = scon[s];
        std::stable_sort(v.begin(), v.end(), [](const Contrib &x, const Contrib &y) { return x.cell < y.cell; });
        for (auto &l : lists) l.clear();
        size_t i = 0;
        while (i < v.size()) {
            const int cell = v[i].cell;
            size_t j = i;
            while (j < v.size() && v[j].cell == cell) ++j;
            int slot = 0;
            auto &L = lists[unit_of(cell, &slot)];
            if (cpl == 1) {
                for (size_t q = i; q < j; ++q) lists[cell].push_back(Ent{v[q].y, {v[q].tap, zero, zero, zero}});
            } else {
                // merge into the unit's list, sorted by voltage index
                std::vector<Ent> merged;
                merged.reserve(L.size() + (j - i));
                size_t a = 0, q = i;
                while (a < L.size() || q < j) {
                    if (q >= j || (a < L.size() && L[a].y < v[q].y)) {
                        merged.push_back(L[a++]);
                    } else if (a < L.size() && L[a].y == v[q].y) {
                        Ent e = L[a++];
                        e.t[slot] = v[q++].tap;
                        merged.push_back(e);
                    } else {
                        Ent e{v[q].y, {zero, zero, zero, zero}};
                        e.t[slot] = v[q++].tap;
                        merged.push_back(e);
                    }
                }
                L.swap(merged);
            }
            i = j;
        }
        // units by decreasing list length (ties by unit index) -> even slices
        for (int u = 0; u < nunit; ++u) order[u] = u;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return lists[x].size() > lists[y].size(); });
        for (int k = 0; k < nsl; ++k) {
            const size_t si = (size_t)s * nsl + k;
            b->slice_off[si] = base;
            size_t len = 0;
            for (int l = 0; l < 32; ++l) len = std::max(len, lists[order[k * 32 + l]].size());
            for (size_t e = 0; e < len; ++e)
                for (int l = 0; l < 32; ++l) {
                    const auto &L = lists[order[k * 32 + l]];
                    const Ent en = e < L.size() ? L[e] : Ent{0, {zero, zero, zero, zero}};
                    for (int c2 = 0; c2 < cpl; ++c2) b->con_tap.push_back(en.t[c2]);
                    b->con_y.push_back((uint16_t)en.y);
                }
            for (int l = 0; l < 32; ++l)
                b->lane_cell[si * 32 + l] = (uint16_t)first_cell(order[k * 32 + l]);
            base += (long long)len * 32;
        }
    }
    b->slice_off[(size_t)ns * nsl] = base;
    return MOFF_OK;
}

std::vector<float2> pass_twiddles_for(int n) { return pass_twiddles_n(n); }

// Power of two s with s * max over grid cells (each output pol) of the sum of |tap| of the
// kernel contributions landing there <= 1: with |y sy[c]| < 2^14 (k_gain_scale) the gridded
// field times sy[c] * s stays below 2^14 in magnitude, and so does every stage of the
// factored transform (each stage's growth is undone by its power-of-two factor).
float dft_kernel_scale(int A, int K, int N, int P, bool jones, const double *pos, const float *taps) {
    const int h = K / 2, pin_n = jones ? 2 : 1;
    std::vector<double> sum((size_t)P * N * N, 0.0);
    for (int a = 0; a < A; ++a) {
        const long long fx = (long long)std::floor(pos[2 * a] + 0.5), fy = (long long)std::floor(pos[2 * a + 1] + 0.5);
        const int ax = (int)(((fx % N) + N) % N), ay = (int)(((fy % N) + N) % N);
        for (int po = 0; po < P; ++po)
            for (int k = 0; k < pin_n; ++k) {
                const int pi = jones ? k : po;
                for (int iy = 0; iy < K; ++iy)
                    for (int ix = 0; ix < K; ++ix) {
                        float re, im;
                        tap_at(jones, P, K, taps, a, po, pi, iy, ix, &re, &im);
                        sum[((size_t)po * N + (ay + iy - h + N) % N) * N + (ax + ix - h + N) % N] +=
                            std::sqrt((double)re * re + (double)im * im);
                    }
            }
    }
    const double mx = *std::max_element(sum.begin(), sum.end());
    if (!(mx > 0.0)) return 1.f;
    int e = 0;
    std::frexp(mx, &e);   // mx in [2^(e-1), 2^e)
    return (float)std::ldexp(1.0, -e);
}

// Row spectra of every kernel row (segment) for the tensor-core path, as
// K-major core-matrix images per (pol, grid row, kx tile) -- see
// moff_tc_kernels.cu.  FP64 sums, one power-of-two scale, FP16 rounding.
moff_status build_rowspec(int A, int K, int N, int P, bool jones, const double *pos, const float *taps, RowSpec *rs) {
    const int h = K / 2;
    std::vector<int> ax(A), ay(A);
    for (int a = 0; a < A; ++a) {
        const double x = pos[2 * a], y = pos[2 * a + 1];
        if (!std::isfinite(x) || !std::isfinite(y) || std::fabs(x) > 1e9 || std::fabs(y) > 1e9)
            return fail(MOFF_EINVAL, "antenna %d position is not finite or out of range", a);
        long long fx = (long long)std::floor(x + 0.5), fy = (long long)std::floor(y + 0.5);
        ax[a] = (int)(((fx % N) + N) % N);
        ay[a] = (int)(((fy % N) + N) % N);
    }
    const int KX = N < 128 ? N : 128, NT = 2 * KX, ntiles = N / KX;
    std::vector<double> cw(N), sw(N);
    for (int m = 0; m < N; ++m) root_unity(m, N, &cw[m], &sw[m]);
    // Voltage planes list antennas by anchor row (then index): plane row v = q * A + rank(a).
    // The kernel rows landing on grid row ry come from the antennas whose anchor row lies in
    // the cyclic window [ry - h, ry + h], consecutive ranks (two runs where the window
    // wraps), so per (output pol, grid row) the A operand is a few runs of consecutive plane
    // rows, cut into chunks of 32 (one TMA tile each of real and imaginary parts).  A chunk
    // slot past its run's end reads another antenna's voltage (or zero past the plane) and
    // gets zero spectra.
    std::vector<int> order(A), rank(A), ays(A);
    for (int a = 0; a < A; ++a) order[a] = a;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ay[x] < ay[y]; });
    for (int i = 0; i < A; ++i) {
        rank[order[i]] = i;
        ays[i] = ay[order[i]];
    }
    rs->perm.assign((size_t)A * P, 0);
    for (int q = 0; q < P; ++q)
        for (int i = 0; i < A; ++i) rs->perm[(size_t)q * A + i] = order[i] * P + q;
    auto first_ge = [&](int y) { return (int)(std::lower_bound(ays.begin(), ays.end(), y) - ays.begin()); };
    // slots (antenna, input pol, kernel row) per (output pol, grid row) in chunk order; a = -1: padding
    struct Seg { int a, q, dy; };
    std::vector<std::vector<Seg>> segs((size_t)P * N);
    rs->ntiles = ntiles;
    rs->kp.assign((size_t)P * N, 0);
    rs->chunk_off.assign((size_t)P * N + 1, 0);
    rs->chunk_row.clear();
    rs->kp_max = 0;
    const int pin_n = jones ? 2 : 1;
    for (int po = 0; po < P; ++po)
        for (int ry = 0; ry < N; ++ry) {
            const size_t r = (size_t)po * N + ry;
            int iv[2][2], niv = 0;      // anchor-row intervals of the window
            if (ry - h < 0) {
                iv[niv][0] = 0; iv[niv][1] = ry + h; ++niv;
                iv[niv][0] = N + ry - h; iv[niv][1] = N - 1; ++niv;
            } else if (ry + h >= N) {
                iv[niv][0] = ry - h; iv[niv][1] = N - 1; ++niv;
                iv[niv][0] = 0; iv[niv][1] = ry + h - N; ++niv;
            } else {
                iv[niv][0] = ry - h; iv[niv][1] = ry + h; ++niv;
            }
            for (int k = 0; k < pin_n; ++k) {
                const int q = jones ? k : po;
                for (int w = 0; w < niv; ++w) {
                    const int lo = first_ge(iv[w][0]), n = first_ge(iv[w][1] + 1) - lo;
                    for (int c0 = 0; c0 < n; c0 += 32) {
                        rs->chunk_row.push_back(q * A + lo + c0);
                        for (int i = 0; i < 32; ++i) {
                            if (c0 + i < n) {
                                const int a = order[lo + c0 + i];
                                segs[r].push_back(Seg{a, q, (ry - ay[a] + h + N) % N});
                            } else {
                                segs[r].push_back(Seg{-1, q, 0});
                            }
                        }
                    }
                }
            }
            rs->chunk_off[r + 1] = (int)rs->chunk_row.size();
            rs->kp[r] = 2 * (int)segs[r].size();
            rs->kp_max = std::max(rs->kp_max, rs->kp[r]);
        }
    if (rs->kp_max > kRowSpecMaxK)
        return fail(MOFF_EINVAL,
                    "tensor-core path: the kernel rows landing on one grid row need %d voltage chunks of 32 (at most "
                    "%d); use the FP32 path", rs->kp_max / 64, kRowSpecMaxK / 64);
    // spectra in FP64, then one power-of-two scale for the whole plan
    std::vector<std::vector<double>> spec_re((size_t)P * N), spec_im((size_t)P * N);
    double mx = 0.0;
    for (size_t r = 0; r < (size_t)P * N; ++r) {
        const int po = (int)(r / N);
        const auto &sg = segs[r];
        spec_re[r].assign(sg.size() * N, 0.0);
        spec_im[r].assign(sg.size() * N, 0.0);
        for (size_t j = 0; j < sg.size(); ++j) {
            if (sg[j].a < 0) continue;   // padding slot: zero spectrum
            for (int dx = 0; dx < K; ++dx) {
                float tr, ti;
                tap_at(jones, P, K, taps, sg[j].a, po, sg[j].q, sg[j].dy, dx, &tr, &ti);
                if (tr == 0.f && ti == 0.f) continue;
                const long long col = (ax[sg[j].a] + dx - h + N) % N;
                for (int kx = 0; kx < N; ++kx) {
                    const int m = (int)((kx * col) % N);
                    spec_re[r][j * N + kx] += (double)tr * cw[m] - (double)ti * sw[m];
                    spec_im[r][j * N + kx] += (double)tr * sw[m] + (double)ti * cw[m];
                }
            }
            for (int kx = 0; kx < N; ++kx)
                mx = std::max(mx, std::max(std::fabs(spec_re[r][j * N + kx]), std::fabs(spec_im[r][j * N + kx])));
        }
    }
    int e = 0;
    if (mx > 0.0) std::frexp(mx, &e);        // mx in [2^(e-1), 2^e)
    const double scale = std::ldexp(1.0, 14 - e);
    rs->inv_sw = (float)std::ldexp(1.0, e - 14);
    // FP16 field scale per (pol, row): the accumulator is sum_j (y s_y)(S_j s_w) with
    // |y s_y| < 2^14, so |re|, |im| <= 2^14 * sum_j max_kx (|S_j re| + |S_j im|) s_w; keep that below 2^15.
    rs->row_sh.assign((size_t)P * N, 1.f);
    rs->row_inv.assign((size_t)P * N, 1.f);
    float sh = 1.f;
    bool any = false;
    for (size_t r = 0; r < (size_t)P * N; ++r) {
        double bound = 0.0;
        for (size_t j = 0; j < segs[r].size(); ++j) {
            double m = 0.0;
            for (int kx = 0; kx < N; ++kx)
                m = std::max(m, std::fabs(spec_re[r][j * N + kx]) + std::fabs(spec_im[r][j * N + kx]));
            bound += m * scale;
        }
        bound *= 16384.0;
        int eb = 0;
        if (bound > 0.0) std::frexp(bound, &eb);          // bound in [2^(eb-1), 2^eb)
        rs->row_sh[r] = bound > 0.0 ? (float)std::ldexp(1.0, 15 - eb) : 1.f;
        rs->row_inv[r] = bound > 0.0 ? (float)std::ldexp(1.0, eb - 15) : 1.f;
        if (bound > 0.0 && (!any || rs->row_sh[r] < sh)) {
            sh = rs->row_sh[r];
            any = true;
        }
    }
    // One scale for all rows: the smallest row scale keeps every row in FP16 range, and
    // a power-of-two scale changes no rounding (FP16 rounding is relative), so the column
    // kernel transforms the scaled rows and undoes one scale per channel.
    rs->row_sh.assign((size_t)P * N, sh);
    rs->row_inv.assign((size_t)P * N, 1.f / sh);
    // B images: row n < KX -> real part of H at kx = tile*KX + n; n >= KX -> imaginary part.
    //   Hr = sum_j yr Sr - yi Si ; Hi = sum_j yr Si + yi Sr
    // Slot j = 32 c + i: chunk c's K rows 64 c + i (yr, the real plane's tile) and 64 c + 32 + i (yi).
    rs->bimg_off.assign((size_t)P * N * ntiles, 0);
    rs->bimg.clear();
    for (size_t r = 0; r < (size_t)P * N; ++r) {
        const int kp = rs->kp[r];
        const int ns = (int)segs[r].size();
        for (int t = 0; t < ntiles; ++t) {
            rs->bimg_off[r * ntiles + t] = (long long)rs->bimg.size();
            if (!kp) continue;
            std::vector<__half> img((size_t)NT * kp, __float2half_rn(0.f));
            for (int n = 0; n < NT; ++n) {
                const int kx = t * KX + (n % KX);
                const bool imag_row = n >= KX;
                for (int j = 0; j < ns; ++j) {
                    const double sr = spec_re[r][(size_t)j * N + kx] * scale, si = spec_im[r][(size_t)j * N + kx] * scale;
                    const double b0 = imag_row ? si : sr;       // coefficient of yr
                    const double b1 = imag_row ? sr : -si;      // coefficient of yi
                    const int kre = 64 * (j / 32) + (j % 32);
                    for (int k = kre; k <= kre + 32; k += 32) {
                        const size_t off = ((size_t)(n >> 3) * (kp >> 3) * 128 + (size_t)(k >> 3) * 128 +
                                            (size_t)(n & 7) * 16 + (size_t)(k & 7) * 2) / 2;
                        img[off] = __double2half(k == kre ? b0 : b1);
                    }
                }
            }
            rs->bimg.insert(rs->bimg.end(), img.begin(), img.end());
        }
    }
    return MOFF_OK;
}


}  // namespace moff

namespace {

// Kernel bins of n_sets sets of positions and kernels ([sets][A] blocks laid out as for
// moff_plan_create) with one common gridding shape, concatenated into one Bins: set g's
// stripe offsets, slice offsets and lane cells follow set g - 1's, with their values
// rebased so that one antenna list and one entry list serve all sets (GridArgs::chan_group).
// One set: the built-in rule or force.  Several: the shape in force (else the rule's
// preferences) that every set fits, with shared memory sized for the densest set.
moff_status build_bin_sets(const moff_plan *pl, int n_sets, const double *pos, const float *taps,
                           const GridChoice *force, Bins *out) {
    const int A = pl->A, K = pl->K, N = pl->N, P = pl->P;
    if (n_sets == 1) return build_bins(A, K, N, P, pl->jones, pos, taps, out, force, pl->dft);
    const size_t pos_set = (size_t)A * 2;
    const size_t tap_set = (size_t)A * P * (pl->jones ? 2 : 1) * K * K * 2;
    std::vector<GridChoice> cands;
    if (force) cands.push_back(*force);
    for (bool pr : {pl->pairs, !pl->pairs})
        for (int tb : {4, 8, 2, 1}) cands.push_back(GridChoice{tb, false, pr, false, false});
    const int nthr = (int)std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 32u));
    std::vector<Bins> bins(n_sets);
    std::vector<moff_status> st(n_sets);
    for (const GridChoice &ch : cands) {
        std::vector<std::thread> workers;
        for (int w = 0; w < std::min(nthr, n_sets); ++w)
            workers.emplace_back([&, w] {
                for (int g = w; g < n_sets; g += nthr) {
                    bins[g] = Bins{};
                    st[g] = build_bins(A, K, N, P, pl->jones, pos + g * pos_set, taps + g * tap_set, &bins[g], &ch,
                                       pl->dft);
                }
            });
        for (std::thread &t : workers) t.join();
        int bad = -1;
        for (int g = 0; g < n_sets && bad < 0; ++g)
            if (st[g] != MOFF_OK) bad = g;
        if (bad >= 0) {
            if (&ch == &cands.back()) {   // the message of the first set that fits no shape
                Bins tmp;
                return build_bins(A, K, N, P, pl->jones, pos + bad * pos_set, taps + bad * tap_set, &tmp, &ch, pl->dft);
            }
            continue;
        }
        Bins &o = *out;
        o = Bins{};
        const Bins &b0 = bins[0];
        o.rows = b0.rows; o.tb = b0.tb; o.n_stripes = b0.n_stripes; o.n_slices = b0.n_slices;
        o.staged = b0.staged; o.pairs = b0.pairs; o.wide = b0.wide; o.quads = b0.quads;
        o.row_nz.assign(b0.row_nz.size(), 0u);
        for (const Bins &b : bins)
            for (size_t w = 0; w < o.row_nz.size(); ++w) o.row_nz[w] |= b.row_nz[w];
        for (const Bins &b : bins) {
            if (b.n_slices != b0.n_slices || b.n_stripes != b0.n_stripes)
                return fail(MOFF_EINVAL, "internal: sets binned to different stripe shapes");
            o.max_nloc = std::max(o.max_nloc, b.max_nloc);
            o.max_entries = std::max(o.max_entries, b.max_entries);
        }
        o.grid_smem = pl->dft ? grid_smem_bytes_dft(N, P, o.tb, o.rows, o.max_nloc)
                              : grid_smem_bytes(N, P, o.tb, o.rows, o.max_nloc, fft_tw_total(N),
                                                o.staged ? o.max_entries : 0, o.pairs);
        if (o.grid_smem > 225 * 1024) continue;
        const size_t tpe = o.quads ? 4 : (o.pairs ? 2 : 1);
        long long ebase = 0;
        int abase = 0;
        for (const Bins &b : bins) {
            if (b.slice_off.back() != (long long)b.con_y.size() || b.con_tap.size() != tpe * b.con_y.size())
                return fail(MOFF_EINVAL, "internal: inconsistent kernel bins");
            for (int v : b.ant_off) o.ant_off.push_back(v + abase);
            for (long long v : b.slice_off) o.slice_off.push_back(v + ebase);
            o.ant_list.insert(o.ant_list.end(), b.ant_list.begin(), b.ant_list.end());
            o.lane_cell.insert(o.lane_cell.end(), b.lane_cell.begin(), b.lane_cell.end());
            o.con_tap.insert(o.con_tap.end(), b.con_tap.begin(), b.con_tap.end());
            o.con_y.insert(o.con_y.end(), b.con_y.begin(), b.con_y.end());
            abase += (int)b.ant_list.size();
            ebase += (long long)b.con_y.size();
        }
        return MOFF_OK;
    }
    return fail(MOFF_EINVAL, "no gridding shape fits every set of positions and kernels in shared memory");
}

// Upload bins and adopt their shape; the plan keeps its old bins if an allocation fails.
moff_status upload_bins(moff_plan *pl, const Bins &b) {
    int *ant_off = nullptr, *ant = nullptr;
    long long *soff = nullptr;
    uint16_t *lcell = nullptr, *cy = nullptr;
    float2 *ctap = nullptr;
    uint32_t *rnz = nullptr;
    auto undo = [&](moff_status s) {
        pfree(pl, ant_off); pfree(pl, ant); pfree(pl, soff); pfree(pl, lcell); pfree(pl, ctap); pfree(pl, cy);
        pfree(pl, rnz);
        return s;
    };
    moff_status s;
    if ((s = palloc(pl, &ant_off, b.ant_off.size() * 4)) != MOFF_OK) return undo(s);
    if ((s = palloc(pl, &ant, std::max<size_t>(b.ant_list.size(), 1) * 4)) != MOFF_OK) return undo(s);
    if ((s = palloc(pl, &soff, b.slice_off.size() * 8)) != MOFF_OK) return undo(s);
    if ((s = palloc(pl, &lcell, b.lane_cell.size() * 2)) != MOFF_OK) return undo(s);
    if ((s = palloc(pl, &ctap, std::max<size_t>(b.con_tap.size(), 1) * 8)) != MOFF_OK) return undo(s);
    if ((s = palloc(pl, &cy, std::max<size_t>(b.con_y.size(), 1) * 2)) != MOFF_OK) return undo(s);
    if ((s = palloc(pl, &rnz, b.row_nz.size() * 4)) != MOFF_OK) return undo(s);
    bool ok = cudaMemcpy(rnz, b.row_nz.data(), b.row_nz.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(ant_off, b.ant_off.data(), b.ant_off.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(soff, b.slice_off.data(), b.slice_off.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(lcell, b.lane_cell.data(), b.lane_cell.size() * 2, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && !b.ant_list.empty())
        ok = cudaMemcpy(ant, b.ant_list.data(), b.ant_list.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && !b.con_tap.empty())
        ok = cudaMemcpy(ctap, b.con_tap.data(), b.con_tap.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(cy, b.con_y.data(), b.con_y.size() * 2, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) return undo(fail(MOFF_ECUDA, "upload of the kernel bins failed"));
    pfree(pl, pl->d_st_ant_off); pfree(pl, pl->d_st_ant); pfree(pl, pl->d_slice_off);
    pfree(pl, pl->d_lane_cell); pfree(pl, pl->d_con_tap); pfree(pl, pl->d_con_y); pfree(pl, pl->d_row_nz);
    pl->d_row_nz = rnz;
    pl->d_st_ant_off = ant_off; pl->d_st_ant = ant; pl->d_slice_off = soff;
    pl->d_lane_cell = lcell; pl->d_con_tap = ctap; pl->d_con_y = cy;
    pl->rows = b.rows;
    pl->tb = b.tb;
    pl->staged = b.staged;
    pl->pairs = b.pairs;
    pl->quads = b.quads;
    pl->wide = b.wide;
    pl->max_entries = b.max_entries;
    pl->n_stripes = b.n_stripes;
    pl->max_nloc = b.max_nloc;
    pl->n_slices = b.n_slices;
    pl->grid_smem = b.grid_smem;
    pl->grid_smem_fft = pl->dft ? grid_smem_bytes(pl->N, pl->P, b.tb, b.rows, b.max_nloc, fft_tw_total(pl->N), 0, b.pairs)
                                : b.grid_smem;
    return MOFF_OK;
}

moff_status bin_plan(moff_plan *pl, const double *pos, const float *taps, const GridChoice *force = nullptr) {
    Bins b;
    moff_status s = build_bin_sets(pl, 1, pos, taps, force, &b);
    return s != MOFF_OK ? s : upload_bins(pl, b);
}

moff_status upload_fstage(moff_plan *pl, int ntaps, const float *coeffs, float scale) {
    const int M = 2 * pl->C;
    const long long L = (long long)ntaps * M;
    std::vector<float> h(L);
    if (coeffs) {
        for (long long n = 0; n < L; ++n) {
            if (!std::isfinite(coeffs[n])) return fail(MOFF_EINVAL, "filter coefficient %lld is not finite", n);
            h[n] = coeffs[n];
        }
    } else {
        // sinc one channel wide, Hann window over the whole filter
        for (long long n = 0; n < L; ++n) {
            const double x = ((double)n - (double)(L - 1) / 2.0) / (double)M;
            const double sinc = x == 0.0 ? 1.0 : std::sin(M_PI * x) / (M_PI * x);
            const double win = L > 1 ? 0.5 - 0.5 * std::cos(2.0 * M_PI * (double)n / (double)(L - 1)) : 1.0;
            h[n] = (float)(sinc * win);
        }
    }
    MOFF_CK(cudaMemcpyAsync(pl->d_h, h.data(), L * 4, cudaMemcpyHostToDevice, pl->st));
    MOFF_CK(cudaStreamSynchronize(pl->st));
    drop_graphs(pl);   // captured F-stage launches hold the old scale and taps
    pl->ntaps = ntaps;
    pl->scale = scale;
    return MOFF_OK;
}

moff_status check_plan(const moff_plan *pl) {
    if (!pl) return fail(MOFF_EINVAL, "plan is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != pl->device) return fail(MOFF_ESTATE, "plan belongs to device %d but device %d is current", pl->device, dev);
    return MOFF_OK;
}

// Entry points that need the plan's own scratch.
moff_status check_unserved(const moff_plan *pl) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (pl->served) return fail(MOFF_ESTATE, "plan was created with MOFF_SERVED: submit its blocks with moff_server_submit");
    return MOFF_OK;
}

// The four-step F-stage applies to C = 1024, 8 taps and a 16-byte aligned ADC block.
bool pfb_four_step(const moff_plan *pl, const int8_t *adc, int F, int kind) {
    return pl->C == 1024 && pl->ntaps == 8 && pl->d_tw4 && ((uintptr_t)adc & 15u) == 0 && F <= 65535 &&
           pl->A * pl->P <= 65535 &&
           pl->sm_bytes >= (size_t)F * pl->C * pl->A * pl->P * (kind == 0 ? 1 : 8);
}

moff_status run_pfb(moff_plan *pl, const int8_t *adc, long long n_samp, int F, int kind, void *out) {
    PfbArgs p{};
    p.adc = adc;
    p.S = n_samp;
    p.AP = pl->A * pl->P;
    p.F = F;
    p.ntaps = pl->ntaps;
    p.h = pl->d_h;
    p.scale = pl->scale;
    p.twp = pl->d_twpC;
    p.twM = pl->d_twM;
    p.out_kind = kind;
    p.codes = kind == 0 ? reinterpret_cast<uint8_t *>(out) : nullptr;
    p.spec = kind == 1 ? reinterpret_cast<float2 *>(out) : nullptr;
    TimedLaunch tp(pl, 0);
    if (pfb_four_step(pl, adc, F, kind)) {
        p.tw4 = pl->d_tw4;
        p.codes_sm = kind == 0 ? static_cast<uint8_t *>(pl->d_sm) : nullptr;
        p.spec_sm = kind == 1 ? static_cast<float2 *>(pl->d_sm) : nullptr;
        MOFF_CK(launch_pfb1024(p, pl->st));
        tp.done();
        TimedLaunch tr(pl, 4);
        MOFF_CK(launch_pfb_reorder(p, pl->st));
        tr.done();
        return MOFF_OK;
    }
    MOFF_CK(launch_pfb(pl->C, p, pl->st));
    tp.done();
    return MOFF_OK;
}

// Beam output for a block of n_time samples (allocated before any capture).
moff_status ensure_beams(moff_plan *pl, int n_time) {
    if (!pl->n_beam) return MOFF_OK;
    const size_t need = (size_t)n_time * pl->C * pl->n_beam * pl->P * 8;
    if (pl->beam_bytes >= need) return MOFF_OK;
    moff_status s = sync_plan(pl, -1);
    if (s != MOFF_OK) return s;
    pfree(pl, pl->d_beam);
    pl->dev_bytes -= pl->beam_bytes;
    pl->d_beam = nullptr;
    pl->beam_bytes = 0;
    drop_graphs(pl);   // captured launches hold the old buffer
    if ((s = palloc(pl, &pl->d_beam, need)) != MOFF_OK) return s;
    pl->beam_bytes = need;
    return MOFF_OK;
}

// Stream-major scratch of the four-step F-stage for F frames (allocated before
// any capture; a no-op when that path does not apply).
moff_status ensure_sm(moff_plan *pl, int F, int kind) {
    if (pl->C != 1024 || pl->ntaps != 8) return MOFF_OK;
    const size_t need = (size_t)F * pl->C * pl->A * pl->P * (kind == 0 ? 1 : 8);
    if (pl->sm_bytes >= need) return MOFF_OK;
    moff_status s = sync_plan(pl, -1);
    if (s != MOFF_OK) return s;
    pfree(pl, pl->d_sm);
    pl->dev_bytes -= pl->sm_bytes;
    pl->d_sm = nullptr;
    pl->sm_bytes = 0;
    if ((s = palloc(pl, &pl->d_sm, need)) != MOFF_OK) return s;
    pl->sm_bytes = need;
    return MOFF_OK;
}

moff_status check_adc(moff_plan *pl, const int8_t *adc, long long n_samp, int *F) {
    if (!pl->fstage) return fail(MOFF_ESTATE, "plan was created without MOFF_FSTAGE");
    if (!adc) return fail(MOFF_EINVAL, "adc is NULL");
    const long long M = 2LL * pl->C;
    if (n_samp <= 0 || n_samp % M != 0) return fail(MOFF_EINVAL, "n_samp (%lld) must be a positive multiple of 2*n_chan = %lld", n_samp, M);
    const long long f = n_samp / M - pl->ntaps + 1;
    if (f < 1) return fail(MOFF_EINVAL, "n_samp (%lld) shorter than one filter (%d frames of %lld)", n_samp, pl->ntaps, M);
    if (f > (1LL << 30)) return fail(MOFF_EINVAL, "too many frames");
    *F = (int)f;
    return MOFF_OK;
}

// ---- MOFF_AUTOTUNE: the gridding kernel's shape (time batch, and whether the
// kernel entries are staged in shared memory) measured on the plan's own array.
// Results are cached per (array, device) in the process and, when
// MOFF_TUNE_CACHE names a file, in that file (one "key tb staged" per line).
std::mutex g_tune_mu;
std::map<std::string, GridChoice> g_tune_cache;
bool g_tune_loaded = false;

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ULL) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ULL;
    return h;
}

std::string tune_key(const moff_plan *pl, const double *pos, const float *taps) {
    const size_t ntap = (size_t)pl->A * (pl->jones ? 4 : pl->P) * pl->K * pl->K * 2;
    uint64_t h = fnv1a(pos, (size_t)pl->A * 2 * sizeof(double));
    h = fnv1a(taps, ntap * sizeof(float), h);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, pl->device);
    h = fnv1a(prop.name, strlen(prop.name), h);
    char buf[128];
    // the prefix changes with the gridding kernels, so picks timed on an older build are not reused
    snprintf(buf, sizeof buf, "%s-A%d-K%d-N%d-P%d-J%d-T%d-C%d-sm%d-%016llx",
             pl->dft ? "gdft1" : (pl->persist ? "gpst1" : "grid6"), pl->A, pl->K,
             pl->N, pl->P, (int)pl->jones, pl->Tb, std::min(pl->Cb, pl->C), prop.multiProcessorCount,
             (unsigned long long)h);
    return buf;
}

// MOFF_AUTOTUNE on the dense FP16 routes: the column kernel's width (8 or 16 columns per CTA)
// timed on one chunk of the plan's own shape over a zeroed field (it adds zeros to the
// accumulators, which are cleared afterwards anyway).
moff_status tune_cols_width(moff_plan *pl) {
    if (!pl->d_H || cols_dft_width_forced()) return MOFF_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(MOFF_ECUDA, "event creation failed");
    }
    ColDftArgs ca{};
    ca.H = reinterpret_cast<const __half *>(pl->d_H);
    ca.slab_t = 1;
    ca.slab_c = pl->Tb;
    ca.nt = pl->Tb;
    ca.c0 = 0;
    ca.nc = std::min(pl->Cb, pl->C);
    ca.acc = pl->d_acc;
    ca.row_nz = pl->d_row_nz;
    ca.sy = pl->d_sy;
    ca.s_t = pl->dft_s_t;
    ca.dft_tab = pl->d_dft_tab_c;
    ca.err = pl->d_err;
    cudaError_t e = cudaMemsetAsync(pl->d_H, 0, pl->h_bytes, pl->st);
    const int ws[2] = {8, 16};
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = launch_cols_dft(pl->N, pl->P, ws[i], ca, pl->st);                  // warm
        if (e == cudaSuccess) e = cudaEventRecord(e0, pl->st);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = launch_cols_dft(pl->N, pl->P, ws[i], ca, pl->st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, pl->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        pl->cols_w_ms[i] = ms / 2.0;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_acc, 0, (size_t)pl->C * pl->nprod * pl->N * pl->N * 8, pl->st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(MOFF_ECUDA, "column-kernel tuning failed: %s", cudaGetErrorString(e));
    pl->cols_w = pl->cols_w_ms[1] < pl->cols_w_ms[0] ? 16 : 8;
    pl->cols_w_source = 1;
    return check_device_err(pl);
}

moff_status tune_grid(moff_plan *pl, const double *pos, const float *taps, GridChoice *out) {
    const std::string key = tune_key(pl, pos, taps);
    const char *path = getenv("MOFF_TUNE_CACHE");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (!g_tune_loaded && path) {
            if (FILE *f = fopen(path, "r")) {
                char k[256];
                int tb = 0, st = 0, pr = 0, wd = 0, qd = 0;
                while (fscanf(f, "%255s %d %d %d %d %d", k, &tb, &st, &pr, &wd, &qd) == 6)
                    g_tune_cache[k] = GridChoice{tb, st != 0, pr != 0, wd != 0, qd != 0};
                fclose(f);
            }
        }
        g_tune_loaded = true;
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second;
            pl->tune_source = 2;
            return MOFF_OK;
        }
    }
    // one chunk of the plan's own shape (Tb samples x Cb channels) into its field scratch
    // (a temporary one for a served plan), so the timing sees the launch the plan will make
    const int N = pl->N, P = pl->P, A = pl->A, nt = pl->Tb;
    const int nc = std::min(pl->Cb, pl->C);
    const long long tstride = (long long)nc * A * P;
    void *volt = nullptr, *gains = nullptr, *Htmp = nullptr, *twp = nullptr, *sy = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<float2> tw = pass_twiddles_n(N);
    auto cleanup = [&] {
        cudaFree(volt); cudaFree(gains); cudaFree(Htmp); cudaFree(twp); cudaFree(sy);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (!pl->d_H && cudaMalloc(&Htmp, pl->h_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(MOFF_ENOMEM, "autotuner scratch allocation failed");
    }
    void *H = pl->d_H ? static_cast<void *>(pl->d_H) : Htmp;
    if (cudaMalloc(&volt, (size_t)nt * tstride) != cudaSuccess || cudaMalloc(&gains, (size_t)nc * A * P * 8) != cudaSuccess ||
        cudaMalloc(&twp, tw.size() * 8) != cudaSuccess || cudaMalloc(&sy, (size_t)nc * 4) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(MOFF_ENOMEM, "autotuner scratch allocation failed");
    }
    // every voltage (3, 5), unit gains: the gridding work does not depend on the values
    std::vector<float2> one((size_t)nc * A * P, make_float2(1.f, 0.f));
    std::vector<float> ones((size_t)nc, 1.f);
    if (cudaMemsetAsync(volt, 0x35, (size_t)nt * tstride, pl->st) != cudaSuccess ||
        cudaMemcpy(sy, ones.data(), ones.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(gains, one.data(), one.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(twp, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        cleanup();
        return fail(MOFF_ECUDA, "autotuner set-up failed");
    }
    GridChoice best{};
    float best_ms = 0.f;
    for (int tb = 8; tb >= 1; tb /= 2)
        for (int cand = 0; cand < 10; ++cand) {
            // cand 0-7: staged x pairs x wide; 8, 9: 2 x 2 blocks (entries through L2), without and with wide.
            // The tensor-core row transform: entries through L2, no wide stripes (cand 0, 2, 8).
            if (pl->dft && cand != 0 && cand != 2 && cand != 8) continue;
            // the persistent launch is built for 4 samples per pass with entries through L2
            if (pl->persist && (tb != 4 || (cand < 8 && (cand & 1)))) continue;
            const GridChoice ch = cand < 8 ? GridChoice{tb, (cand & 1) != 0, (cand & 2) != 0, (cand & 4) != 0, false}
                                           : GridChoice{tb, false, false, cand == 9, true};
            moff_plan tmp;
            tmp.A = A; tmp.K = pl->K; tmp.N = N; tmp.C = nc; tmp.P = P; tmp.jones = pl->jones;
            tmp.device = pl->device;
            tmp.dft = pl->dft;
            if (bin_plan(&tmp, pos, taps, &ch) != MOFF_OK) {
                for (void *q : tmp.allocs) cudaFree(q);
                continue;
            }
            tmp.d_twp = static_cast<float2 *>(twp);
            tmp.d_gains = static_cast<float2 *>(gains);
            tmp.d_H = static_cast<float2 *>(H);
            tmp.Tb = nt;
            tmp.Cb = nc;
            GridArgs g = grid_args(&tmp, static_cast<const uint8_t *>(volt), tstride, 0, nt, 0, nc);
            if (pl->dft) {
                g.out = nullptr;
                g.h16 = static_cast<__half *>(H);
                g.sy = static_cast<const float *>(sy);
                g.s_t = pl->dft_s_t;
                g.dft_tab = pl->d_dft_tab;
                g.err = pl->d_err;
            }
            const int cpl = tmp.quads ? 4 : (tmp.pairs ? 2 : 1);
            auto launch = [&] {
                return pl->dft ? launch_grid_dft(N, P, tmp.tb, cpl, g, tmp.n_stripes, tmp.grid_smem, pl->st)
                               : launch_grid(N, P, tmp.tb, tmp.staged, false, g, tmp.n_stripes, tmp.grid_smem, pl->st);
            };
            float ms = 0.f;
            bool ok = launch() == cudaSuccess;
            for (int r = 0; ok && r < 3; ++r) {
                float t = 0.f;
                ok = cudaEventRecord(e0, pl->st) == cudaSuccess && launch() == cudaSuccess &&
                     cudaEventRecord(e1, pl->st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                     cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
                if (ok && (r == 0 || t < ms)) ms = t;
            }
            cudaStreamSynchronize(pl->st);
            for (void *q : tmp.allocs) cudaFree(q);
            if (!ok) {
                cleanup();
                cudaGetLastError();
                return fail(MOFF_ECUDA, "autotuner launch failed");
            }
            if (getenv("MOFF_TUNE_VERBOSE"))
                fprintf(stderr, "moff autotune: tb=%d staged=%d pairs=%d wide=%d quads=%d  %.4f ms\n", ch.tb,
                        (int)ch.staged, (int)ch.pairs, (int)ch.wide, (int)ch.quads, ms);
            if (best.tb == 0 || ms < best_ms) {
                best = ch;
                best_ms = ms;
            }
        }
    cleanup();
    if (best.tb == 0) return fail(MOFF_EINVAL, "array too dense for the gridding kernel (no feasible shape)");
    *out = best;
    pl->tune_source = 1;
    pl->tune_best_ms = best_ms;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    if (path)
        if (FILE *f = fopen(path, "a")) {
            fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), best.tb, (int)best.staged, (int)best.pairs, (int)best.wide,
                    (int)best.quads);
            fclose(f);
        }
    return MOFF_OK;
}

// Every antenna's beam towards the calibrator pixel (kx, ky), per set of positions and
// kernels: B_a,p = sum_{dy,dx} taps[a][p][dy][dx] exp(+2 pi i (ky (ay + dy - h) + kx (ax + dx - h)) / N),
// FP64 [sets][A][P].
moff_status upload_fb_beams(moff_plan *pl, int kx, int ky) {
    const int A = pl->A, P = pl->P, K = pl->K, N = pl->N, h = K / 2, G = pl->n_groups;
    std::vector<double2> beam((size_t)G * A * P);
    for (int ga = 0; ga < G * A; ++ga) {      // antenna ga % A of set ga / A ([sets][A] host blocks)
        const long long fx = (long long)std::floor(pl->h_pos[2 * (size_t)ga] + 0.5);
        const long long fy = (long long)std::floor(pl->h_pos[2 * (size_t)ga + 1] + 0.5);
        const long long ax = ((fx % N) + N) % N, ay = ((fy % N) + N) % N;
        for (int p = 0; p < P; ++p) {
            double br = 0.0, bi = 0.0;
            for (int dy = 0; dy < K; ++dy)
                for (int dx = 0; dx < K; ++dx) {
                    const float *t = &pl->h_taps[((((size_t)ga * P + p) * K + dy) * K + dx) * 2];
                    const long long m = ((long long)ky * (ay + dy - h) + (long long)kx * (ax + dx - h)) % N;
                    double c, sn;
                    root_unity(m < 0 ? m + N : m, N, &c, &sn);
                    br += (double)t[0] * c - (double)t[1] * sn;
                    bi += (double)t[0] * sn + (double)t[1] * c;
                }
            beam[(size_t)ga * P + p] = make_double2(br, bi);
        }
    }
    double2 *d = nullptr;
    moff_status s = palloc(pl, &d, beam.size() * 16);
    if (s != MOFF_OK) return s;
    if (cudaMemcpy(d, beam.data(), beam.size() * 16, cudaMemcpyHostToDevice) != cudaSuccess) {
        pfree(pl, d);
        return fail(MOFF_ECUDA, "upload of the calibrator beams failed");
    }
    pfree(pl, pl->d_fb_beam);
    pl->d_fb_beam = d;
    return MOFF_OK;
}

// The kernels' cross-correlation patches of every set, X_a,q(u) = sum_{d - d' = u}
// T_a,p[d] conj(T_a,p'[d']) with q = (p, p') in {(x,x), (y,y), (x,y)}, FP64 [sets][A][NQ][U].
moff_status upload_auto_patches(moff_plan *pl) {
    const int A = pl->A, P = pl->P, K = pl->K, L = 2 * K - 1, U = L * L, NQ = P == 1 ? 1 : 3, G = pl->n_groups;
    std::vector<double2> X((size_t)G * A * NQ * U, make_double2(0.0, 0.0));
    const int qp[3][2] = {{0, 0}, {1, 1}, {0, 1}};
    for (int ga = 0; ga < G * A; ++ga)           // antenna ga % A of set ga / A ([sets][A] host blocks)
        for (int q = 0; q < NQ; ++q) {
            const float *T0 = &pl->h_taps[(((size_t)ga * P + qp[q][0]) * K * K) * 2];
            const float *T1 = &pl->h_taps[(((size_t)ga * P + qp[q][1]) * K * K) * 2];
            double2 *Xa = &X[((size_t)ga * NQ + q) * U];
            for (int dy = 0; dy < K; ++dy)
                for (int dx = 0; dx < K; ++dx) {
                    const double ar = T0[(dy * K + dx) * 2], ai = T0[(dy * K + dx) * 2 + 1];
                    if (ar == 0.0 && ai == 0.0) continue;
                    for (int ey = 0; ey < K; ++ey)
                        for (int ex = 0; ex < K; ++ex) {
                            const double br = T1[(ey * K + ex) * 2], bi = -T1[(ey * K + ex) * 2 + 1];
                            double2 &x = Xa[(dy - ey + K - 1) * L + (dx - ex + K - 1)];
                            x.x += ar * br - ai * bi;
                            x.y += ar * bi + ai * br;
                        }
                }
        }
    double2 *d = nullptr;
    moff_status s = palloc(pl, &d, X.size() * 16);
    if (s != MOFF_OK) return s;
    if (cudaMemcpy(d, X.data(), X.size() * 16, cudaMemcpyHostToDevice) != cudaSuccess) {
        pfree(pl, d);
        return fail(MOFF_ECUDA, "upload of the autocorrelation patches failed");
    }
    pfree(pl, pl->d_auto_X);
    pl->d_auto_X = d;
    return MOFF_OK;
}

}  // namespace

namespace moff {

size_t plan_scratch_bytes(const moff_plan *pl) { return pl->scratch_bytes; }
size_t plan_block_bytes(const moff_plan *pl, int n_time) { return (size_t)n_time * pl->C * pl->A * pl->P; }
long long plan_units(const moff_plan *pl, int n_time) { return (long long)n_time * pl->C; }
bool plan_is_served(const moff_plan *pl) { return pl->served; }
int plan_device(const moff_plan *pl) { return pl->device; }
cudaStream_t plan_stream(const moff_plan *pl) { return pl->st; }

moff_status plan_run_served(moff_plan *pl, void *scratch, const uint8_t *volt, int n_time, int on_device) {
    moff_status sb = ensure_beams(pl, n_time);
    if (sb != MOFF_OK) return sb;
    unsigned char *base = static_cast<unsigned char *>(scratch);
    pl->d_H = reinterpret_cast<float2 *>(base);
    size_t off = align_up(pl->h_bytes, 1024);
    if (pl->gtc) {
        pl->d_G = reinterpret_cast<__half *>(base + off);
        off += align_up(pl->h_bytes, 1024);
        pl->d_yre = reinterpret_cast<__half *>(base + off);
        off += align_up(pl->y_bytes, 1024);
        pl->d_yim = reinterpret_cast<__half *>(base + off);
        off += align_up(pl->y_bytes, 1024);
        const long long rows = (long long)pl->Cb * pl->gt_rows;
        if (encode_plane_map(&pl->gt_map_re, pl->d_yre, pl->Tb, rows, 16) != cudaSuccess ||
            encode_plane_map(&pl->gt_map_im, pl->d_yim, pl->Tb, rows, 16) != cudaSuccess ||
            encode_plane_store_map(&pl->vp_smap_re, pl->d_yre, pl->Tb, rows) != cudaSuccess ||
            encode_plane_store_map(&pl->vp_smap_im, pl->d_yim, pl->Tb, rows) != cudaSuccess)
            return fail(MOFF_ECUDA, "tensor maps of the voltage planes could not be encoded");
        if (encode_gridtc_store_map(&pl->gt_map_g, pl->d_G, (long long)(pl->h_bytes / 256)) != cudaSuccess)
            return fail(MOFF_ECUDA, "tensor map of the gridded field could not be encoded");
    }
    if (pl->tc && !pl->dft) {
        pl->d_yre = reinterpret_cast<__half *>(base + off);
        off += align_up(pl->y_bytes, 1024);
        pl->d_yim = reinterpret_cast<__half *>(base + off);
        off += align_up(pl->y_bytes, 1024);
        if (encode_field_map(&pl->h_map, pl->d_H, pl->N, pl->P, pl->Cb, pl->Tb) != cudaSuccess)
            return fail(MOFF_ECUDA, "tensor map of the row-transformed field could not be encoded");
        const long long rows = (long long)pl->Cb * (pl->A * pl->P + kRowSpecPad);
        if (encode_plane_map(&pl->a_map_re, pl->d_yre, pl->Tb, rows) != cudaSuccess ||
            encode_plane_map(&pl->a_map_im, pl->d_yim, pl->Tb, rows) != cudaSuccess ||
            encode_plane_store_map(&pl->vp_smap_re, pl->d_yre, pl->Tb, rows) != cudaSuccess ||
            encode_plane_store_map(&pl->vp_smap_im, pl->d_yim, pl->Tb, rows) != cudaSuccess)
            return fail(MOFF_ECUDA, "tensor maps of the voltage planes could not be encoded");
        pl->h_map_nt = pl->Tb;
    }
    const long long tstride = (long long)pl->C * pl->A * pl->P;
    const uint8_t *src = volt;
    if (!on_device) {
        uint8_t *dst = base + off;
        MOFF_CK(cudaMemcpyAsync(dst, volt, plan_block_bytes(pl, n_time), cudaMemcpyHostToDevice, pl->st));
        src = dst;
    }
    moff_status s = launch_block(pl, 0, src, n_time, tstride, [&] { return run_image(pl, src, n_time, tstride); });
    if (s != MOFF_OK) return s;
    pl->n_samples += n_time;
    if (pl->fb_on) pl->fb_samples += n_time;
    if (pl->auto_on) pl->auto_samples += n_time;
    pl->beam_T = n_time;
    return MOFF_OK;
}

}  // namespace moff

extern "C" {

const char *moff_last_error(void) { return g_err.c_str(); }

moff_status moff_plan_create(moff_plan **out, int n_ant, const double *pos, int ksize, const float *taps, int grid_n,
                             int n_chan, int n_pol, unsigned flags, void *cuda_stream) {
    if (!out) return fail(MOFF_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_ant < 1 || n_ant > 65536) return fail(MOFF_EINVAL, "n_ant (%d) must be in [1, 65536]", n_ant);
    if (!pos || !taps) return fail(MOFF_EINVAL, "pos and taps must not be NULL");
    if (grid_n != 32 && grid_n != 64 && grid_n != 128 && grid_n != 256 && grid_n != 512)
        return fail(MOFF_EINVAL, "grid_n (%d) must be 32, 64, 128, 256 or 512", grid_n);
    if (ksize < 1 || ksize % 2 == 0 || ksize > 15 || ksize > grid_n)
        return fail(MOFF_EINVAL, "ksize (%d) must be odd, in [1, 15] and <= grid_n", ksize);
    if (n_chan < 1) return fail(MOFF_EINVAL, "n_chan (%d) must be >= 1", n_chan);
    if (n_pol != 1 && n_pol != 2) return fail(MOFF_EINVAL, "n_pol (%d) must be 1 or 2", n_pol);
    if (flags & ~(unsigned)(MOFF_FSTAGE | MOFF_JONES | MOFF_PREC_FP16TC | MOFF_SERVED | MOFF_AUTOTUNE | MOFF_GRAPH |
                            MOFF_PERSIST))
        return fail(MOFF_EINVAL, "unknown flag bits 0x%x", flags);
    if ((flags & MOFF_PERSIST) && (flags & (MOFF_PREC_FP16TC | MOFF_SERVED)))
        return fail(MOFF_EINVAL, "MOFF_PERSIST runs the FP32 path of an unserved plan");
    if ((flags & MOFF_JONES) && n_pol != 2) return fail(MOFF_EINVAL, "MOFF_JONES requires n_pol = 2");
    if ((flags & MOFF_FSTAGE) && (!is_pow2(n_chan) || n_chan < 32 || n_chan > 2048))
        return fail(MOFF_EINVAL, "with MOFF_FSTAGE n_chan (%d) must be a power of two in [32, 2048]", n_chan);

    moff_plan *pl = new moff_plan();
    pl->A = n_ant;
    pl->K = ksize;
    pl->N = grid_n;
    pl->C = n_chan;
    pl->P = n_pol;
    pl->nprod = n_pol == 1 ? 1 : 4;
    pl->flags = flags;
    pl->jones = (flags & MOFF_JONES) != 0;
    pl->fstage = (flags & MOFF_FSTAGE) != 0;
    pl->tc = (flags & MOFF_PREC_FP16TC) != 0;
    pl->served = (flags & MOFF_SERVED) != 0;
    pl->persist = (flags & MOFF_PERSIST) != 0;
    // FP16 path at N = 256 / 512: the row-spectrum contraction where the array's rows are sparse
    // enough for it, else (or with MOFF_TC_DFT=1) the factored DFT contractions
    RowSpec rs_probe;
    bool have_probe = false;
    if (pl->tc && (grid_n == 256 || grid_n == 512)) {
        const char *e = getenv("MOFF_TC_DFT");
        if (e && atoi(e) == 1) {
            pl->dft = true;
        } else if (!(e && atoi(e) == 0)) {
            if (build_rowspec(n_ant, ksize, grid_n, n_pol, (flags & MOFF_JONES) != 0, pos, taps, &rs_probe) == MOFF_OK)
                have_probe = true;
            else
                pl->dft = true;   // too dense for the row-spectrum contraction (or invalid: reported below)
        }
    }
    pl->graphs = (flags & MOFF_GRAPH) != 0;
    if (!pl->jones) {
        pl->h_taps.assign(taps, taps + (size_t)n_ant * n_pol * ksize * ksize * 2);
        pl->h_pos.assign(pos, pos + (size_t)n_ant * 2);
    }
    auto bail = [&](moff_status s) {
        std::string msg = g_err;
        destroy_plan(pl);
        g_err = msg;
        return s;
    };
    if (cudaGetDevice(&pl->device) != cudaSuccess) return bail(fail(MOFF_ECUDA, "no CUDA device"));
    if (cuda_stream) {
        pl->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&pl->st, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "stream creation failed"));
        pl->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&pl->cst, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(MOFF_ECUDA, "copy stream creation failed"));
    if (const char *e = getenv("MOFF_VP_TMA")) pl->vp_tma = atoi(e) != 0;
    for (int i = 0; i < 2; ++i) {
        if (cudaEventCreateWithFlags(&pl->ev_copied[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->ev_consumed[i], cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "event creation failed"));
    }
    if (cudaEventCreateWithFlags(&pl->ev_done, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(MOFF_ECUDA, "event creation failed"));
    if (pl->graphs && cudaStreamCreateWithFlags(&pl->gst, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(MOFF_ECUDA, "capture stream creation failed"));

    moff_status s = MOFF_OK;

    // twiddles of the N-point imaging transform
    {
        std::vector<float2> tw = pass_twiddles_n(grid_n);
        if ((s = palloc(pl, &pl->d_twp, tw.size() * 8)) != MOFF_OK) return bail(s);
        if (cudaMemcpy(pl->d_twp, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "twiddle upload failed"));
    }
    // gains = 1
    {
        const size_t n = (size_t)n_chan * n_ant * n_pol;
        if ((s = palloc(pl, &pl->d_gains, n * 8)) != MOFF_OK) return bail(s);
        std::vector<float2> one(n, make_float2(1.f, 0.f));
        if (cudaMemcpy(pl->d_gains, one.data(), n * 8, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "gain upload failed"));
    }
    // Tensor-core gridding tables (FP16 path, factored-DFT route): B images scaled by the same power
    // of two as the gather's FP16 field (the kernel scale), so the row transform sees one field.
    GridTc gtab;
    if (pl->dft) {
        const char *e = getenv("MOFF_TC_GRID");
        if (!(e && atoi(e) == 0)) {
            pl->dft_s_t = dft_kernel_scale(n_ant, ksize, grid_n, n_pol, pl->jones, pos, taps);
            if ((s = build_gridtc(n_ant, ksize, grid_n, n_pol, pl->jones, pos, taps, pl->dft_s_t, &gtab)) != MOFF_OK)
                return bail(s);
            // one CTA per SM: the tile's kernel matrix, the A ring and the barriers must fit shared memory
            pl->gtc = !gtab.tile_cell.empty() && gridtc_stages(n_pol, gtab.kp_max, 1) > 0;
            pl->gt_rows = gtab.n_rows + kRowSpecPad;
        }
    }
    // accumulators and image staging
    {
        const size_t n = (size_t)n_chan * pl->nprod * grid_n * grid_n;
        if ((s = palloc(pl, &pl->d_acc, n * 8)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_img, n * 4)) != MOFF_OK) return bail(s);
        if (cudaMemset(pl->d_acc, 0, n * 8) != cudaSuccess) return bail(fail(MOFF_ECUDA, "memset failed"));
    }
    // row-transform scratch: Tb samples x Cb channels per chunk
    {
        // FP32 field (float2) on the FP32 path, FP16 (half2) on the tensor-core path
        const size_t per = (size_t)n_pol * grid_n * grid_n * (pl->tc ? 4 : 8);
        // served plans borrow their scratch per block from a shared pool: keep it modest (the tensor-core
        // gridding route reads each tile's kernel matrix once per launch, so it wants more channels per chunk)
        long long budget = pl->served ? (pl->gtc ? (8192LL << 20) : (2048LL << 20)) : (32768LL << 20);
        if (const char *e = getenv("MOFF_SCRATCH_MB")) budget = std::max(1LL, (long long)(atof(e) * 1048576.0));
        // channels split into equal chunks (no ragged last chunk)
        auto balance = [&](long long cb_max) {
            const long long n = (n_chan + cb_max - 1) / cb_max;
            return (n_chan + n - 1) / n;
        };
        if (pl->gtc) {
            // 128 samples per chunk (the tensor-core gridding's product height): the FP16 gridded and
            // row-transformed fields and the FP16 voltage planes of every sample of every channel
            const size_t per_c = 128 * (2 * per + (size_t)pl->gt_rows * 4);
            pl->Tb = 128;
            pl->Cb = (int)balance(std::max(1LL, std::min<long long>(n_chan, budget / (long long)per_c)));
        } else if (pl->dft) {
            // FP16 field only; up to 128 samples per chunk (FP32 sums per chunk, then FP64)
            const long long cb = balance(std::max(1LL, std::min<long long>(n_chan, budget / (long long)(32 * per))));
            const long long tb = std::max(1LL, std::min<long long>(128, budget / (long long)(cb * per)));
            pl->Cb = (int)cb;
            pl->Tb = (int)tb;
        } else if (pl->tc) {
            // the tensor-core path works on 128 samples per product
            const size_t per_c = 128 * per + ((size_t)n_ant * n_pol + kRowSpecPad) * 128 * 4;
            pl->Tb = 128;
            pl->Cb = (int)balance(std::max(1LL, std::min<long long>(n_chan, budget / (long long)per_c)));
        } else {
            const long long cb = balance(std::max(1LL, std::min<long long>(n_chan, budget / (long long)(32 * per))));
            const long long tb = std::max(1LL, std::min<long long>(128, budget / (long long)(cb * per)));
            pl->Cb = (int)cb;
            pl->Tb = (int)tb;
        }
        pl->h_bytes = (size_t)pl->Tb * pl->Cb * per;
        if (pl->gtc) pl->y_bytes = (size_t)pl->Cb * pl->gt_rows * pl->Tb * 2;
        if (!pl->served) {
            if ((s = palloc(pl, &pl->d_H, pl->h_bytes)) != MOFF_OK) return bail(s);
            if (pl->gtc) {
                if ((s = palloc(pl, &pl->d_G, pl->h_bytes)) != MOFF_OK) return bail(s);
                if ((s = palloc(pl, &pl->d_yre, pl->y_bytes)) != MOFF_OK) return bail(s);
                if ((s = palloc(pl, &pl->d_yim, pl->y_bytes)) != MOFF_OK) return bail(s);
                const long long rows = (long long)pl->Cb * pl->gt_rows;
                if (encode_plane_map(&pl->gt_map_re, pl->d_yre, pl->Tb, rows, 16) != cudaSuccess ||
                    encode_plane_map(&pl->gt_map_im, pl->d_yim, pl->Tb, rows, 16) != cudaSuccess ||
                    encode_plane_store_map(&pl->vp_smap_re, pl->d_yre, pl->Tb, rows) != cudaSuccess ||
                    encode_plane_store_map(&pl->vp_smap_im, pl->d_yim, pl->Tb, rows) != cudaSuccess)
                    return bail(fail(MOFF_ECUDA, "tensor maps of the voltage planes could not be encoded"));
                if (encode_gridtc_store_map(&pl->gt_map_g, pl->d_G, (long long)(pl->h_bytes / 256)) != cudaSuccess)
                    return bail(fail(MOFF_ECUDA, "tensor map of the gridded field could not be encoded"));
            }
            if (pl->tc && !pl->dft && encode_field_map(&pl->h_map, pl->d_H, grid_n, n_pol, pl->Cb, pl->Tb) != cudaSuccess)
                return bail(fail(MOFF_ECUDA, "tensor map of the row-transformed field could not be encoded"));
            pl->h_map_nt = pl->Tb;
        }
    }
    if (pl->dft) {
        // factored-DFT tables, and the kernel scale: every cell's sum of |tap| over its contributions
        // (all output pols) times dft_s_t is at most 1, so |G| sy[c] dft_s_t <= 2^14
        std::vector<unsigned char> tab = build_dft_table(grid_n), tabc = build_dft_table(grid_n, true);
        if ((s = palloc(pl, &pl->d_dft_tab, tab.size())) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_dft_tab_c, tabc.size())) != MOFF_OK) return bail(s);
        if (cudaMemcpy(pl->d_dft_tab, tab.data(), tab.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(pl->d_dft_tab_c, tabc.data(), tabc.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "tensor-core DFT table upload failed"));
        if (!pl->gtc) pl->dft_s_t = dft_kernel_scale(n_ant, ksize, grid_n, n_pol, pl->jones, pos, taps);
        // the 8 x 64 row transform on the 512 grid: 2.76 against 3.31 ms per wide-field launch for the
        // 16 x 32 one (MOFF_ROWS8=0 keeps that)
        if (const char *e = getenv("MOFF_ROWS8"); pl->gtc && grid_n == 512 && !(e && atoi(e) == 0)) {
            std::vector<unsigned char> t8 = build_rows8_table();
            if ((s = palloc(pl, &pl->d_dft_tab_r8, t8.size())) != MOFF_OK) return bail(s);
            if (cudaMemcpy(pl->d_dft_tab_r8, t8.data(), t8.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(MOFF_ECUDA, "row-transform table upload failed"));
            pl->rows8 = true;
        }
        if ((s = palloc(pl, &pl->d_sy, (size_t)n_chan * 4)) != MOFF_OK) return bail(s);
        if (pl->gtc) {
            pl->gt_tiles = (int)gtab.tile_cell.size();
            pl->gt_kp_max = gtab.kp_max;
            // one epilogue box per warp and the deepest A ring: on the wide-field array a second box
            // per warp (4 stages instead of 8) measured 3.14 against 2.76 ms per launch
            // (MOFF_GT_BOXES=2 selects it where it fits)
            const char *gb = getenv("MOFF_GT_BOXES");
            pl->gt_boxes = (gb && atoi(gb) == 2 && gridtc_stages(n_pol, gtab.kp_max, 2) > 0) ? 2 : 1;
            pl->gt_stages = gridtc_stages(n_pol, gtab.kp_max, pl->gt_boxes);
            pl->gt_smem = gridtc_smem_bytes(n_pol, gtab.kp_max, pl->gt_stages, pl->gt_boxes);
            // channel groups: about two CTAs' worth of tiles per SM over a launch
            int sms = 152;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
            pl->gt_cgroups = std::max(1, std::min(pl->Cb, (2 * sms + pl->gt_tiles - 1) / pl->gt_tiles));
            if (const char *e = getenv("MOFF_TC_CGROUPS")) pl->gt_cgroups = std::max(1, std::min(pl->Cb, atoi(e)));
            auto up = [&](auto **dst, const auto &v) -> moff_status {
                moff_status st = palloc(pl, dst, std::max<size_t>(v.size(), 1) * sizeof(v[0]));
                if (st != MOFF_OK) return st;
                if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice) != cudaSuccess)
                    return fail(MOFF_ECUDA, "tensor-core gridding table upload failed");
                return MOFF_OK;
            };
            if ((s = up(&pl->d_gt_tile_cell, gtab.tile_cell)) != MOFF_OK || (s = up(&pl->d_gt_kp, gtab.kp)) != MOFF_OK ||
                (s = up(&pl->d_gt_chunk_off, gtab.chunk_off)) != MOFF_OK ||
                (s = up(&pl->d_gt_chunk_row, gtab.chunk_row)) != MOFF_OK || (s = up(&pl->d_gt_perm, gtab.perm)) != MOFF_OK ||
                (s = up(&pl->d_gt_bimg_off, gtab.bimg_off)) != MOFF_OK || (s = up(&pl->d_gt_bimg, gtab.bimg)) != MOFF_OK ||
                (s = up(&pl->d_gt_active, gtab.active)) != MOFF_OK)
                return bail(s);
        }
        if ((s = palloc(pl, &pl->d_err, 16)) != MOFF_OK) return bail(s);
        if (cudaMemset(pl->d_err, 0, 16) != cudaSuccess) return bail(fail(MOFF_ECUDA, "memset failed"));
        if (launch_gain_scale(pl->d_gains, n_chan, n_ant * n_pol, pl->d_sy, pl->st) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "gain scale kernel failed"));
    }
    // gridding shape: measured on the plan's own chunk (MOFF_AUTOTUNE), else the built-in rule
    {
        GridChoice tuned;
        if ((flags & MOFF_AUTOTUNE) && (!pl->tc || pl->dft) && !pl->gtc) {
            if ((s = tune_grid(pl, pos, taps, &tuned)) != MOFF_OK) return bail(s);
        }
        if ((s = bin_plan(pl, pos, taps, pl->tune_source ? &tuned : nullptr)) != MOFF_OK) return bail(s);
        if (pl->persist && (pl->tb != 4 || pl->staged)) {
            GridChoice ch{4, false, pl->pairs, pl->wide, pl->quads};
            if ((s = bin_plan(pl, pos, taps, &ch)) != MOFF_OK) return bail(s);
        }
    }
    if (pl->dft) {   // the column kernel's width: the default, or timed (needs the plan's reached-row mask)
        pl->cols_w = cols_dft_width();
        if ((flags & MOFF_AUTOTUNE) && (s = tune_cols_width(pl)) != MOFF_OK) return bail(s);
    }
    if (pl->persist) {
        pl->persist_smem = std::max(pl->grid_smem, col_smem_bytes(grid_n, n_pol));
        if (pl->persist_smem > 227 * 1024)
            return bail(fail(MOFF_EINVAL, "MOFF_PERSIST: the persistent kernel needs %zu bytes of shared memory",
                             pl->persist_smem));
        cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, pl->device);
        const size_t nq = 1 + 2 * (size_t)kPersistMaxChunks * pl->Cb;
        if ((s = palloc(pl, &pl->d_pq, nq * sizeof(int))) != MOFF_OK) return bail(s);
        if (!pl->d_err) {
            if ((s = palloc(pl, &pl->d_err, 16)) != MOFF_OK) return bail(s);
            if (cudaMemset(pl->d_err, 0, 16) != cudaSuccess) return bail(fail(MOFF_ECUDA, "memset failed"));
        }
        // about one second of SM clock per wait (MOFF_PERSIST_BUDGET_US shortens it); MOFF_PERSIST_EXTRA
        // (tests) makes column items wait for row items that do not exist, so their waits run out
        double us = 1e6;
        if (const char *e = getenv("MOFF_PERSIST_BUDGET_US")) us = std::max(1.0, atof(e));
        int clk_khz = 2070000;
        cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, pl->device);
        pl->persist_budget = (long long)(us * 1e-3 * (double)std::max(clk_khz, 100000));
        if (const char *e = getenv("MOFF_PERSIST_EXTRA")) pl->persist_extra = std::max(0, atoi(e));
    }
    if (pl->tc && !pl->dft) {
        RowSpec rs;
        if (have_probe)
            rs = std::move(rs_probe);
        else if ((s = build_rowspec(n_ant, ksize, grid_n, n_pol, pl->jones, pos, taps, &rs)) != MOFF_OK)
            return bail(s);
        pl->rs_kp_max = std::max(rs.kp_max, 16);
        pl->rs_inv_sw = rs.inv_sw;
        pl->rs_smem = rowspec_smem_bytes(grid_n, pl->rs_kp_max);
        const int items = n_pol * grid_n * rs.ntiles;
        // channel groups: about twelve CTAs per SM over the launch (a sweep on the benchmark array: 3, 8, 19,
        // 38 groups gave 33.0, 31.0, 31.6, 34.2 ms per step)
        pl->rs_cgroups = std::max(1, std::min(pl->Cb, (12 * 152 + items - 1) / items));
        if (const char *e = getenv("MOFF_TC_CGROUPS")) pl->rs_cgroups = std::max(1, std::min(pl->Cb, atoi(e)));
        const size_t ny = (size_t)pl->Cb * (n_ant * n_pol + kRowSpecPad) * pl->Tb;
        if ((s = palloc(pl, &pl->d_rs_kp, rs.kp.size() * 4)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_rs_chunk_off, rs.chunk_off.size() * 4)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_rs_chunk_row, std::max<size_t>(rs.chunk_row.size(), 1) * 4)) != MOFF_OK)
            return bail(s);
        if ((s = palloc(pl, &pl->d_rs_perm, rs.perm.size() * 4)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_rs_bimg_off, rs.bimg_off.size() * 8)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_rs_bimg, std::max<size_t>(rs.bimg.size(), 8) * 2)) != MOFF_OK) return bail(s);
        pl->y_bytes = ny * 2;
        if (!pl->served) {
            if ((s = palloc(pl, &pl->d_yre, ny * 2)) != MOFF_OK) return bail(s);
            if ((s = palloc(pl, &pl->d_yim, ny * 2)) != MOFF_OK) return bail(s);
            const long long rows = (long long)pl->Cb * (n_ant * n_pol + kRowSpecPad);
            if (encode_plane_map(&pl->a_map_re, pl->d_yre, pl->Tb, rows) != cudaSuccess ||
                encode_plane_map(&pl->a_map_im, pl->d_yim, pl->Tb, rows) != cudaSuccess ||
                encode_plane_store_map(&pl->vp_smap_re, pl->d_yre, pl->Tb, rows) != cudaSuccess ||
                encode_plane_store_map(&pl->vp_smap_im, pl->d_yim, pl->Tb, rows) != cudaSuccess)
                return bail(fail(MOFF_ECUDA, "tensor maps of the voltage planes could not be encoded"));
        }
        if ((s = palloc(pl, &pl->d_sy, (size_t)n_chan * 4)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_err, 16)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_rs_row_sh, rs.row_sh.size() * 4)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_rs_row_inv, rs.row_inv.size() * 4)) != MOFF_OK) return bail(s);
        if (cudaMemcpy(pl->d_rs_row_sh, rs.row_sh.data(), rs.row_sh.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(pl->d_rs_row_inv, rs.row_inv.data(), rs.row_inv.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "tensor-core row scales upload failed"));
        if (cudaMemcpy(pl->d_rs_kp, rs.kp.data(), rs.kp.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(pl->d_rs_chunk_off, rs.chunk_off.data(), rs.chunk_off.size() * 4, cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            (!rs.chunk_row.empty() && cudaMemcpy(pl->d_rs_chunk_row, rs.chunk_row.data(), rs.chunk_row.size() * 4,
                                                 cudaMemcpyHostToDevice) != cudaSuccess) ||
            cudaMemcpy(pl->d_rs_perm, rs.perm.data(), rs.perm.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(pl->d_rs_bimg_off, rs.bimg_off.data(), rs.bimg_off.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
            (!rs.bimg.empty() &&
             cudaMemcpy(pl->d_rs_bimg, rs.bimg.data(), rs.bimg.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) ||
            cudaMemset(pl->d_err, 0, 16) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "tensor-core table upload failed"));
        if (launch_gain_scale(pl->d_gains, n_chan, n_ant * n_pol, pl->d_sy, pl->st) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "gain scale kernel failed"));
    }
    // F-stage tables
    if (pl->fstage) {
        const int CN = n_chan, M = 2 * CN;
        std::vector<float2> tw = pass_twiddles_n(CN);
        std::vector<float2> twM(CN);
        for (int k = 0; k < CN; ++k) {
            double c, sn;
            root_unity(-(long long)k, M, &c, &sn);
            twM[k] = make_float2((float)c, (float)sn);
        }
        if ((s = palloc(pl, &pl->d_twpC, tw.size() * 8)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_twM, twM.size() * 8)) != MOFF_OK) return bail(s);
        if ((s = palloc(pl, &pl->d_h, (size_t)16 * M * 4)) != MOFF_OK) return bail(s);
        if (cudaMemcpy(pl->d_twpC, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(pl->d_twM, twM.data(), twM.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(MOFF_ECUDA, "F-stage table upload failed"));
        if ((s = upload_fstage(pl, 8, nullptr, 1.f)) != MOFF_OK) return bail(s);
        if (CN == 1024) {
            // exp(-2 pi i l k2 / 1024) stored [k2][l] for the four-step transform
            std::vector<float2> t4(1024);
            for (int k2 = 0; k2 < 32; ++k2)
                for (int l = 0; l < 32; ++l) {
                    double c, sn;
                    root_unity(-(long long)l * k2, 1024, &c, &sn);
                    t4[k2 * 32 + l] = make_float2((float)c, (float)sn);
                }
            if ((s = palloc(pl, &pl->d_tw4, t4.size() * 8)) != MOFF_OK) return bail(s);
            if (cudaMemcpy(pl->d_tw4, t4.data(), t4.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(MOFF_ECUDA, "F-stage table upload failed"));
        }
    }
    pl->scratch_bytes = align_up(pl->h_bytes, 1024) + (pl->tc && !pl->dft ? 2 * align_up(pl->y_bytes, 1024) : 0) +
                        (pl->gtc ? align_up(pl->h_bytes, 1024) + 2 * align_up(pl->y_bytes, 1024) : 0);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(fail(MOFF_ECUDA, "plan set-up failed"));
    if (const char *lg = getenv("MOFF_LOG"); lg && atoi(lg) > 0) {   // the plan's decisions, one line on stderr
        static const char *routes[4] = {"fp32", "fp16_rowspec", "fp16_dft", "fp16_tcgrid"};
        const int route = pl->gtc ? 3 : (pl->dft ? 2 : (pl->tc ? 1 : 0));
        fprintf(stderr,
                "moff: plan A=%d K=%d N=%d C=%d P=%d route=%s chunk=%dx%d grid(tb=%d cells/lane=%d wide=%d staged=%d "
                "source=%d) cols_w=%d rows8=%d persist=%d scratch=%.1f MB device=%.1f MB\n",
                n_ant, ksize, grid_n, n_chan, n_pol, routes[route], pl->Tb, pl->Cb, pl->tb,
                pl->quads ? 4 : (pl->pairs ? 2 : 1), (int)pl->wide, (int)pl->staged, pl->tune_source,
                pl->dft ? pl->cols_w : 0, (int)pl->rows8, (int)pl->persist, pl->scratch_bytes / 1048576.0,
                pl->dev_bytes / 1048576.0);
    }
    *out = pl;
    g_err.clear();
    return MOFF_OK;
}

moff_status moff_plan_destroy(moff_plan *plan) {
    if (!plan) return MOFF_OK;
    destroy_plan(plan);
    return MOFF_OK;
}

moff_status moff_set_gains(moff_plan *pl, const float *gains, int on_device) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (!gains) return fail(MOFF_EINVAL, "gains is NULL");
    const size_t bytes = (size_t)pl->C * pl->A * pl->P * 8;
    MOFF_CK(cudaMemcpyAsync(pl->d_gains, gains, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, pl->st));
    if (pl->tc) MOFF_CK(launch_gain_scale(pl->d_gains, pl->C, pl->A * pl->P, pl->d_sy, pl->st));
    if (!on_device) return sync_plan(pl, -1);
    return MOFF_OK;
}

moff_status moff_set_channel_groups(moff_plan *pl, int n_groups, const double *pos, const float *taps,
                                   const int *chan_group) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (pl->tc) return fail(MOFF_EINVAL, "channel-dependent positions and kernels run on the FP32 path (not MOFF_PREC_FP16TC)");
    if (n_groups < 1 || n_groups > pl->C) return fail(MOFF_EINVAL, "n_groups (%d) must be in [1, C = %d]", n_groups, pl->C);
    if (!pos || !taps) return fail(MOFF_EINVAL, "pos and taps must not be NULL");
    if (n_groups > 1 && !chan_group) return fail(MOFF_EINVAL, "chan_group must not be NULL with more than one set");
    if (chan_group)
        for (int c = 0; c < pl->C; ++c)
            if (chan_group[c] < 0 || chan_group[c] >= n_groups)
                return fail(MOFF_EINVAL, "chan_group[%d] = %d outside [0, %d)", c, chan_group[c], n_groups);
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    const GridChoice cur{pl->tb, pl->staged, pl->pairs, pl->wide, pl->quads};
    Bins b;
    if ((s = build_bin_sets(pl, n_groups, pos, taps, &cur, &b)) != MOFF_OK) return s;
    int *d_grp = nullptr;
    if (n_groups > 1) {
        if ((s = palloc(pl, &d_grp, (size_t)pl->C * 4)) != MOFF_OK) return s;
        if (cudaMemcpy(d_grp, chan_group, (size_t)pl->C * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            pfree(pl, d_grp);
            return fail(MOFF_ECUDA, "upload of the channel sets failed");
        }
    }
    if ((s = upload_bins(pl, b)) != MOFF_OK) {
        pfree(pl, d_grp);
        return s;
    }
    pfree(pl, pl->d_chan_group);
    pl->d_chan_group = d_grp;
    pl->n_groups = n_groups;
    if (!pl->jones) {
        pl->h_pos.assign(pos, pos + (size_t)n_groups * pl->A * 2);
        pl->h_taps.assign(taps, taps + (size_t)n_groups * pl->A * pl->P * pl->K * pl->K * 2);
    }
    drop_graphs(pl);   // captured launches hold the old bins
    if (pl->fb_on && (s = upload_fb_beams(pl, pl->fb_kx, pl->fb_ky)) != MOFF_OK) return s;
    if (pl->auto_on && (s = upload_auto_patches(pl)) != MOFF_OK) return s;
    return MOFF_OK;
}

moff_status moff_set_fstage(moff_plan *pl, int n_taps, const float *coeffs, float scale) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (!pl->fstage) return fail(MOFF_ESTATE, "plan was created without MOFF_FSTAGE");
    if (n_taps < 1 || n_taps > 16) return fail(MOFF_EINVAL, "n_taps (%d) must be in [1, 16]", n_taps);
    if (!std::isfinite(scale) || scale <= 0.f) return fail(MOFF_EINVAL, "scale must be finite and > 0");
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    return upload_fstage(pl, n_taps, coeffs, scale);
}

moff_status moff_submit(moff_plan *pl, const uint8_t *volt, int n_time, int on_device) {
    moff_status s = check_unserved(pl);
    if (s != MOFF_OK) return s;
    if (!volt) return fail(MOFF_EINVAL, "volt is NULL");
    if (n_time < 1) return fail(MOFF_EINVAL, "n_time (%d) must be >= 1", n_time);
    const long long tstride = (long long)pl->C * pl->A * pl->P;
    const size_t bytes = (size_t)n_time * tstride;
    if ((s = ensure_beams(pl, n_time)) != MOFF_OK) return s;
    auto image = [&](const uint8_t *src) {
        return launch_block(pl, 0, src, n_time, tstride, [&] { return run_image(pl, src, n_time, tstride); });
    };
    if (on_device) {
        if ((s = image(volt)) != MOFF_OK) return s;
    } else {
        const void *dev = nullptr;
        int slot = 0;
        // blocks of several channel chunks are copied by channel segments that overlap the imaging
        // (not under graph replay, whose captured launches carry no per-segment waits)
        static const bool pipeline = !(getenv("MOFF_STAGE_PIPELINE") && atoi(getenv("MOFF_STAGE_PIPELINE")) == 0);
        const bool by_chan = pipeline && !pl->graphs && !pl->persist && pl->Cb < pl->C && bytes >= ((size_t)8 << 20);
        if ((s = by_chan ? stage_in_by_channels(pl, volt, n_time, &dev, &slot) : stage_in(pl, volt, bytes, &dev, &slot)) !=
            MOFF_OK)
            return s;
        s = image(reinterpret_cast<const uint8_t *>(dev));
        pl->chunk_seg = 0;
        if (s != MOFF_OK) return s;
        if (by_chan) MOFF_CK(cudaStreamWaitEvent(pl->st, pl->ev_copied[slot], 0));
        if ((s = stage_done(pl, slot)) != MOFF_OK) return s;
    }
    pl->n_samples += n_time;
    if (pl->fb_on) pl->fb_samples += n_time;
    if (pl->auto_on) pl->auto_samples += n_time;
    pl->beam_T = n_time;
    return MOFF_OK;
}

// Host ADC block staged in frame segments: each segment's copy (cudaMemcpy2DAsync
// of its sample range, every stream, on the copy stream) is followed on the
// plan's stream by that segment's F-stage and imaging, so later copies overlap
// earlier compute.  Segments overlap by n_taps - 1 frames of samples.
constexpr int kSegFrames = 128;

moff_status submit_adc_pipelined(moff_plan *pl, const int8_t *adc, long long n_samp, int F) {
    const int i = (int)(pl->nsub & 1);
    const size_t abytes = (size_t)pl->A * pl->P * n_samp;
    moff_status s = MOFF_OK;
    if (pl->stage_bytes[i] < abytes) {
        MOFF_CK(cudaEventSynchronize(pl->ev_consumed[i]));
        pfree(pl, pl->d_stage[i]);
        pl->dev_bytes -= pl->stage_bytes[i];
        pl->d_stage[i] = nullptr;
        pl->stage_bytes[i] = 0;
        if ((s = palloc(pl, &pl->d_stage[i], abytes)) != MOFF_OK) return s;
        pl->stage_bytes[i] = abytes;
    }
    for (cudaEvent_t &e : pl->seg_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(MOFF_ECUDA, "event creation failed");
    const int nseg_max = (int)(sizeof(pl->seg_ev) / sizeof(pl->seg_ev[0]));
    // segments hold whole imaging chunks (so the launches, and the image, equal a device-input submit's)
    const int step = pl->tc ? pl->Tb : ((kSegFrames + pl->Tb - 1) / pl->Tb) * pl->Tb;
    int seg = step;
    while ((F + seg - 1) / seg > nseg_max) seg += step;
    const long long M = 2LL * pl->C, tstride = (long long)pl->C * pl->A * pl->P;
    const int AP = pl->A * pl->P;
    int8_t *dst = static_cast<int8_t *>(pl->d_stage[i]);
    MOFF_CK(cudaStreamWaitEvent(pl->cst, pl->ev_consumed[i], 0));
    int e = 0;
    for (int f0 = 0; f0 < F; f0 += seg, ++e) {
        const int f1 = std::min(F, f0 + seg);
        const long long c0 = (long long)f0 * M, c1 = (long long)(f1 + pl->ntaps - 1) * M;
        MOFF_CK(cudaMemcpy2DAsync(dst + c0, (size_t)n_samp, adc + c0, (size_t)n_samp, (size_t)(c1 - c0), (size_t)AP,
                                  cudaMemcpyHostToDevice, pl->cst));
        MOFF_CK(cudaEventRecord(pl->seg_ev[e], pl->cst));
        MOFF_CK(cudaStreamWaitEvent(pl->st, pl->seg_ev[e], 0));
        uint8_t *codes = pl->d_codes + (size_t)f0 * tstride;
        if ((s = run_pfb(pl, dst + c0, n_samp, f1 - f0, 0, codes)) != MOFF_OK) break;
        pl->beam_base = f0;
        if ((s = run_image(pl, codes, f1 - f0, tstride)) != MOFF_OK) break;
    }
    pl->beam_base = 0;
    MOFF_CK(cudaEventRecord(pl->ev_copied[i], pl->cst));
    MOFF_CK(cudaEventRecord(pl->ev_consumed[i], pl->st));
    pl->nsub++;
    moff_status w = wait_event(pl->ev_copied[i], -1);   // the caller's buffer is free once copied
    return s != MOFF_OK ? s : w;
}

moff_status moff_submit_adc(moff_plan *pl, const int8_t *adc, long long n_samp, int on_device) {
    moff_status s = check_unserved(pl);
    if (s != MOFF_OK) return s;
    int F = 0;
    if ((s = check_adc(pl, adc, n_samp, &F)) != MOFF_OK) return s;
    const size_t cbytes = (size_t)F * pl->C * pl->A * pl->P;
    if (pl->codes_bytes < cbytes) {
        if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
        pfree(pl, pl->d_codes);
        pl->dev_bytes -= pl->codes_bytes;
        pl->d_codes = nullptr;
        pl->codes_bytes = 0;
        if ((s = palloc(pl, &pl->d_codes, cbytes)) != MOFF_OK) return s;
        pl->codes_bytes = cbytes;
    }
    if ((s = ensure_sm(pl, F, 0)) != MOFF_OK) return s;
    if ((s = ensure_beams(pl, F)) != MOFF_OK) return s;
    const size_t abytes = (size_t)pl->A * pl->P * n_samp;
    static const bool pipeline = !(getenv("MOFF_STAGE_PIPELINE") && atoi(getenv("MOFF_STAGE_PIPELINE")) == 0);
    if (pipeline && !on_device && !pl->graphs && F > kSegFrames) {
        if ((s = submit_adc_pipelined(pl, adc, n_samp, F)) != MOFF_OK) return s;
    } else {
        const int8_t *src = adc;
        int slot = -1;
        if (!on_device) {
            const void *dev = nullptr;
            if ((s = stage_in(pl, adc, abytes, &dev, &slot)) != MOFF_OK) return s;
            src = reinterpret_cast<const int8_t *>(dev);
        }
        s = launch_block(pl, 1, src, n_samp, (long long)(void *)pl->d_codes, [&] {
            moff_status r = run_pfb(pl, src, n_samp, F, 0, pl->d_codes);
            return r != MOFF_OK ? r : run_image(pl, pl->d_codes, F, (long long)pl->C * pl->A * pl->P);
        });
        if (s != MOFF_OK) return s;
        if (slot >= 0 && (s = stage_done(pl, slot)) != MOFF_OK) return s;
    }
    pl->n_samples += F;
    if (pl->fb_on) pl->fb_samples += F;
    if (pl->auto_on) pl->auto_samples += F;
    pl->beam_T = F;
    return MOFF_OK;
}

moff_status moff_channelise(moff_plan *pl, const int8_t *adc, long long n_samp, int in_on_device, void *out, int out_kind,
                            int out_on_device) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    int F = 0;
    if ((s = check_adc(pl, adc, n_samp, &F)) != MOFF_OK) return s;
    if (!out) return fail(MOFF_EINVAL, "out is NULL");
    if (out_kind != 0 && out_kind != 1) return fail(MOFF_EINVAL, "out_kind must be 0 (codes) or 1 (spectra)");
    const size_t n = (size_t)F * pl->C * pl->A * pl->P;
    const size_t obytes = out_kind == 0 ? n : n * 8;
    void *dst = out;
    if (!out_on_device) {
        if (out_kind == 0) {
            if (pl->codes_bytes < n) {
                if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
                pfree(pl, pl->d_codes);
                pl->dev_bytes -= pl->codes_bytes;
                pl->d_codes = nullptr;
                pl->codes_bytes = 0;
                if ((s = palloc(pl, &pl->d_codes, n)) != MOFF_OK) return s;
                pl->codes_bytes = n;
            }
            dst = pl->d_codes;
        } else {
            if (pl->spec_bytes < obytes) {
                if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
                pfree(pl, pl->d_spec);
                pl->dev_bytes -= pl->spec_bytes;
                pl->d_spec = nullptr;
                pl->spec_bytes = 0;
                if ((s = palloc(pl, &pl->d_spec, obytes)) != MOFF_OK) return s;
                pl->spec_bytes = obytes;
            }
            dst = pl->d_spec;
        }
    }
    if ((s = ensure_sm(pl, F, out_kind)) != MOFF_OK) return s;
    const size_t abytes = (size_t)pl->A * pl->P * n_samp;
    const int8_t *src = adc;
    int slot = -1;
    if (!in_on_device) {
        const void *dev = nullptr;
        if ((s = stage_in(pl, adc, abytes, &dev, &slot)) != MOFF_OK) return s;
        src = reinterpret_cast<const int8_t *>(dev);
    }
    if ((s = run_pfb(pl, src, n_samp, F, out_kind, dst)) != MOFF_OK) return s;
    if (slot >= 0 && (s = stage_done(pl, slot)) != MOFF_OK) return s;
    if (!out_on_device) MOFF_CK(cudaMemcpyAsync(out, dst, obytes, cudaMemcpyDeviceToHost, pl->st));
    return sync_plan(pl, -1);
}

moff_status moff_grid_snapshot(moff_plan *pl, const uint8_t *volt, int on_device, int chan, float *out) {
    moff_status s = check_unserved(pl);
    if (s != MOFF_OK) return s;
    if (!volt || !out) return fail(MOFF_EINVAL, "volt and out must not be NULL");
    if (chan < 0 || chan >= pl->C) return fail(MOFF_EINVAL, "chan (%d) out of range [0, %d)", chan, pl->C);
    // the snapshot is written as FP32 into the field scratch (FP16-sized on the tensor-core path)
    if (pl->h_bytes < (size_t)pl->P * pl->N * pl->N * 8)
        return fail(MOFF_EINVAL, "the plan's field scratch is too small for an FP32 snapshot");
    const size_t bytes = (size_t)pl->C * pl->A * pl->P;
    const uint8_t *src = volt;
    int slot = -1;
    if (!on_device) {
        const void *dev = nullptr;
        if ((s = stage_in(pl, volt, bytes, &dev, &slot)) != MOFF_OK) return s;
        src = reinterpret_cast<const uint8_t *>(dev);
    }
    GridArgs g = grid_args(pl, src, 0, 0, 1, chan, 1);
    MOFF_CK(launch_grid(pl->N, pl->P, pl->tb, false, true, g, pl->n_stripes, pl->grid_smem_fft, pl->st));
    if (slot >= 0 && (s = stage_done(pl, slot)) != MOFF_OK) return s;
    MOFF_CK(cudaMemcpyAsync(out, pl->d_H, (size_t)pl->P * pl->N * pl->N * 8, cudaMemcpyDeviceToHost, pl->st));
    return sync_plan(pl, -1);
}

moff_status moff_voltage_planes(moff_plan *pl, const uint8_t *volt, int n_time, int on_device, int chan, float *out,
                                float *scale) {
    moff_status s = check_unserved(pl);
    if (s != MOFF_OK) return s;
    if (!pl->tc || (pl->dft && !pl->gtc))
        return fail(MOFF_EINVAL, "voltage planes exist only on the row-spectrum and tensor-core gridding routes");
    if (!volt || !out) return fail(MOFF_EINVAL, "volt and out must not be NULL");
    if (n_time < 1 || n_time > pl->Tb) return fail(MOFF_EINVAL, "n_time (%d) must be in [1, %d]", n_time, pl->Tb);
    if (chan < 0 || chan >= pl->C) return fail(MOFF_EINVAL, "chan (%d) out of range [0, %d)", chan, pl->C);
    // row-spectrum route: one plane row per antenna-pol; tensor-core gridding route: raster order of
    // the anchors plus copies of the rows whose kernel window wraps (every copy written out again)
    const int AP = pl->A * pl->P;
    const bool gt = pl->gtc;
    const int APpad = gt ? pl->gt_rows : AP + kRowSpecPad, nrows = gt ? pl->gt_rows - kRowSpecPad : AP;
    const int *dperm = gt ? pl->d_gt_perm : pl->d_rs_perm;
    const long long tstride = (long long)pl->C * AP;
    const uint8_t *src = volt;
    int slot = -1;
    if (!on_device) {
        const void *dev = nullptr;
        if ((s = stage_in(pl, volt, (size_t)n_time * tstride, &dev, &slot)) != MOFF_OK) return s;
        src = reinterpret_cast<const uint8_t *>(dev);
    }
    MOFF_CK(launch_volt_prep(src, tstride, 0, n_time, chan, 1, AP, APpad, pl->d_gains, pl->d_sy, dperm, pl->Tb,
                             pl->d_yre, pl->d_yim, pl->st, nrows, pl->vp_tma ? &pl->vp_smap_re : nullptr,
                             pl->vp_tma ? &pl->vp_smap_im : nullptr));
    if (slot >= 0 && (s = stage_done(pl, slot)) != MOFF_OK) return s;
    std::vector<__half> re((size_t)nrows * pl->Tb), im((size_t)nrows * pl->Tb);
    std::vector<int> perm(nrows);
    float sy = 0.f;
    MOFF_CK(cudaMemcpyAsync(re.data(), pl->d_yre, re.size() * 2, cudaMemcpyDeviceToHost, pl->st));
    MOFF_CK(cudaMemcpyAsync(im.data(), pl->d_yim, im.size() * 2, cudaMemcpyDeviceToHost, pl->st));
    MOFF_CK(cudaMemcpyAsync(perm.data(), dperm, (size_t)nrows * 4, cudaMemcpyDeviceToHost, pl->st));
    MOFF_CK(cudaMemcpyAsync(&sy, pl->d_sy + chan, 4, cudaMemcpyDeviceToHost, pl->st));
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    std::vector<char> seen(AP, 0);
    for (int v = 0; v < nrows; ++v) {
        if (perm[v] < 0 || perm[v] >= AP) return fail(MOFF_ECUDA, "voltage-plane row %d maps outside the array", v);
        const bool copy = seen[perm[v]] != 0;    // a row copied for a wrapping kernel window: must equal its original
        seen[perm[v]] = 1;
        for (int t = 0; t < n_time; ++t) {
            const size_t o = ((size_t)t * AP + perm[v]) * 2;
            const float r = __half2float(re[(size_t)v * pl->Tb + t]), i = __half2float(im[(size_t)v * pl->Tb + t]);
            if (copy && (out[o] != r || out[o + 1] != i))
                return fail(MOFF_ECUDA, "a copied voltage-plane row differs from its original (row %d)", v);
            out[o] = r;
            out[o + 1] = i;
        }
    }
    if (scale) *scale = sy;
    return MOFF_OK;
}

moff_status moff_read_image(moff_plan *pl, float *out, long long *n_samples, int reset, int timeout_ms, int out_on_device) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (!out) return fail(MOFF_EINVAL, "out is NULL");
    if ((s = sync_plan(pl, timeout_ms)) != MOFF_OK) return s;
    if ((s = check_device_err(pl)) != MOFF_OK) return s;
    const long long n = (long long)pl->C * pl->nprod * pl->N * pl->N;
    MOFF_CK(launch_to_f32(pl->d_acc, out_on_device ? out : pl->d_img, n, pl->st));
    if (!out_on_device) MOFF_CK(cudaMemcpyAsync(out, pl->d_img, (size_t)n * 4, cudaMemcpyDeviceToHost, pl->st));
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    if (n_samples) *n_samples = pl->n_samples;
    if (reset) {
        MOFF_CK(cudaMemsetAsync(pl->d_acc, 0, (size_t)n * 8, pl->st));
        pl->n_samples = 0;
        if (pl->auto_on) {   // the autocorrelation sums follow the integration
            MOFF_CK(cudaMemsetAsync(pl->d_auto_pw, 0, (size_t)pl->C * pl->A * 3 * 16, pl->st));
            pl->auto_samples = 0;
        }
    }
    return MOFF_OK;
}

moff_status moff_sync(moff_plan *pl, int timeout_ms) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if ((s = sync_plan(pl, timeout_ms)) != MOFF_OK) return s;
    return check_device_err(pl);
}

moff_status moff_export_accumulators(moff_plan *pl, double *out, long long *n_samples, int out_on_device,
                                     int timeout_ms) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (!out) return fail(MOFF_EINVAL, "out is NULL");
    if ((s = sync_plan(pl, timeout_ms)) != MOFF_OK) return s;
    if ((s = check_device_err(pl)) != MOFF_OK) return s;
    const size_t bytes = (size_t)pl->C * pl->nprod * pl->N * pl->N * 8;
    MOFF_CK(cudaMemcpyAsync(out, pl->d_acc, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            pl->st));
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    if (n_samples) *n_samples = pl->n_samples;
    return MOFF_OK;
}

moff_status moff_import_accumulators(moff_plan *pl, const double *in, long long n_samples, int in_on_device) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (!in) return fail(MOFF_EINVAL, "in is NULL");
    if (n_samples < 0) return fail(MOFF_EINVAL, "n_samples (%lld) must be >= 0", n_samples);
    const size_t bytes = (size_t)pl->C * pl->nprod * pl->N * pl->N * 8;
    // enqueued behind the plan's work; a host source is read before the call returns
    MOFF_CK(cudaMemcpyAsync(pl->d_acc, in, bytes, in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            pl->st));
    if (!in_on_device && (s = sync_plan(pl, -1)) != MOFF_OK) return s;
    pl->n_samples = n_samples;
    return MOFF_OK;
}

moff_status moff_reset(moff_plan *pl) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    MOFF_CK(cudaMemsetAsync(pl->d_acc, 0, (size_t)pl->C * pl->nprod * pl->N * pl->N * 8, pl->st));
    pl->n_samples = 0;
    if (pl->fb_on) {
        MOFF_CK(cudaMemsetAsync(pl->d_fb_corr, 0, (size_t)pl->C * pl->A * pl->P * 16, pl->st));
        MOFF_CK(cudaMemsetAsync(pl->d_fb_power, 0, (size_t)pl->C * pl->P * 8, pl->st));
        pl->fb_samples = 0;
    }
    if (pl->auto_on) {
        MOFF_CK(cudaMemsetAsync(pl->d_auto_pw, 0, (size_t)pl->C * pl->A * 3 * 16, pl->st));
        pl->auto_samples = 0;
    }
    return MOFF_OK;
}

moff_status moff_set_autocorr(moff_plan *pl, int on) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    drop_graphs(pl);   // the captured launch sequences change
    if (!on) {
        pl->auto_on = false;
        return MOFF_OK;
    }
    if (pl->jones) return fail(MOFF_EINVAL, "autocorrelation subtraction needs one kernel per pol (not MOFF_JONES)");
    const int A = pl->A, P = pl->P, K = pl->K, N = pl->N, L = 2 * K - 1, U = L * L, NQ = P == 1 ? 1 : 3;
    if (!pl->d_auto_pw) {
        if ((s = palloc(pl, &pl->d_auto_pw, (size_t)pl->C * A * 3 * 16)) != MOFF_OK) return s;
        if ((s = palloc(pl, &pl->d_auto_Q, (size_t)pl->C * NQ * U * 16)) != MOFF_OK) return s;
        if ((s = palloc(pl, &pl->d_auto_img, (size_t)pl->C * pl->nprod * N * N * 8)) != MOFF_OK) return s;
        if ((s = palloc(pl, &pl->d_wN, (size_t)N * 16)) != MOFF_OK) return s;
    }
    if ((s = upload_auto_patches(pl)) != MOFF_OK) return s;
    std::vector<double2> w(N);
    for (int m = 0; m < N; ++m) {
        double c, sn;
        root_unity(m, N, &c, &sn);
        w[m] = make_double2(c, sn);
    }
    MOFF_CK(cudaMemcpy(pl->d_wN, w.data(), w.size() * 16, cudaMemcpyHostToDevice));
    MOFF_CK(cudaMemsetAsync(pl->d_auto_pw, 0, (size_t)pl->C * A * 3 * 16, pl->st));
    pl->auto_on = true;
    pl->auto_samples = 0;
    return sync_plan(pl, -1);
}

moff_status moff_read_image_cross(moff_plan *pl, float *out, long long *n_samples, int reset, int timeout_ms,
                                  int out_on_device) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (!out) return fail(MOFF_EINVAL, "out is NULL");
    if (!pl->auto_on) return fail(MOFF_ESTATE, "autocorrelation sums are off (moff_set_autocorr)");
    if (pl->auto_samples != pl->n_samples)
        return fail(MOFF_ESTATE, "autocorrelation sums cover %lld of the image's %lld samples (switch them on before the "
                    "integration starts, or reset)", pl->auto_samples, pl->n_samples);
    if ((s = sync_plan(pl, timeout_ms)) != MOFF_OK) return s;
    if ((s = check_device_err(pl)) != MOFF_OK) return s;
    const long long n = (long long)pl->C * pl->nprod * pl->N * pl->N;
    MOFF_CK(launch_auto_image(pl->d_auto_pw, pl->d_auto_X, pl->d_chan_group, pl->C, pl->A, pl->P, pl->K, pl->N, pl->d_wN, pl->d_auto_Q,
                              pl->d_auto_img, pl->st));
    MOFF_CK(launch_sub_to_f32(pl->d_acc, pl->d_auto_img, out_on_device ? out : pl->d_img, n, pl->st));
    if (!out_on_device) MOFF_CK(cudaMemcpyAsync(out, pl->d_img, (size_t)n * 4, cudaMemcpyDeviceToHost, pl->st));
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    if (n_samples) *n_samples = pl->n_samples;
    if (reset) {
        MOFF_CK(cudaMemsetAsync(pl->d_acc, 0, (size_t)n * 8, pl->st));
        MOFF_CK(cudaMemsetAsync(pl->d_auto_pw, 0, (size_t)pl->C * pl->A * 3 * 16, pl->st));
        pl->n_samples = 0;
        pl->auto_samples = 0;
    }
    return MOFF_OK;
}

moff_status moff_set_beams(moff_plan *pl, int n_beams, const int *kx, const int *ky) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (n_beams < 0 || n_beams > kMaxBeams) return fail(MOFF_EINVAL, "n_beams (%d) must be in [0, %d]", n_beams, kMaxBeams);
    if (n_beams && (!kx || !ky)) return fail(MOFF_EINVAL, "kx and ky must not be NULL");
    if (n_beams && pl->dft)
        return fail(MOFF_EINVAL, "tied-array beams are not available on the factored-DFT tensor-core route");
    for (int j = 0; j < n_beams; ++j)
        if (kx[j] < 0 || kx[j] >= pl->N || ky[j] < 0 || ky[j] >= pl->N)
            return fail(MOFF_EINVAL, "beam %d pixel (%d, %d) outside the %d x %d image", j, kx[j], ky[j], pl->N, pl->N);
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    pl->n_beam = n_beams;
    for (int j = 0; j < n_beams; ++j) {
        pl->beam_kx[j] = kx[j];
        pl->beam_ky[j] = ky[j];
    }
    pl->beam_T = 0;
    if (pl->d_beam) {   // a buffer sized for another beam count: drop it
        pfree(pl, pl->d_beam);
        pl->dev_bytes -= pl->beam_bytes;
        pl->d_beam = nullptr;
        pl->beam_bytes = 0;
    }
    drop_graphs(pl);
    return MOFF_OK;
}

moff_status moff_read_beams(moff_plan *pl, float *out, int *n_time, int timeout_ms, int out_on_device) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (!pl->n_beam) return fail(MOFF_ESTATE, "no beams set (moff_set_beams)");
    if ((s = sync_plan(pl, timeout_ms)) != MOFF_OK) return s;
    if ((s = check_device_err(pl)) != MOFF_OK) return s;
    if (n_time) *n_time = pl->beam_T;
    if (out && pl->beam_T) {
        const size_t bytes = (size_t)pl->beam_T * pl->C * pl->n_beam * pl->P * 8;
        MOFF_CK(cudaMemcpyAsync(out, pl->d_beam, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                pl->st));
        return sync_plan(pl, -1);
    }
    return MOFF_OK;
}

moff_status moff_set_calibrator(moff_plan *pl, int kx, int ky) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (kx < 0 && ky < 0) {
        if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
        pl->fb_on = false;
        drop_graphs(pl);
        return MOFF_OK;
    }
    if (pl->jones) return fail(MOFF_EINVAL, "feedback calibration needs one kernel per pol (not MOFF_JONES)");
    if (pl->dft) return fail(MOFF_EINVAL, "feedback calibration is not available on the factored-DFT tensor-core route");
    if (kx < 0 || kx >= pl->N || ky < 0 || ky >= pl->N)
        return fail(MOFF_EINVAL, "calibrator pixel (%d, %d) outside the %d x %d image", kx, ky, pl->N, pl->N);
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    const int P = pl->P;
    const size_t AP = (size_t)pl->A * P;
    if (!pl->d_etap) {
        if ((s = palloc(pl, &pl->d_etap, (size_t)pl->Tb * pl->Cb * P * 8)) != MOFF_OK) return s;
        if ((s = palloc(pl, &pl->d_fb_corr, (size_t)pl->C * AP * 16)) != MOFF_OK) return s;
        if ((s = palloc(pl, &pl->d_fb_power, (size_t)pl->C * P * 8)) != MOFF_OK) return s;
        if ((s = palloc(pl, &pl->d_fb_out, (size_t)pl->C * AP * 8)) != MOFF_OK) return s;
    }
    if ((s = upload_fb_beams(pl, kx, ky)) != MOFF_OK) return s;
    MOFF_CK(cudaMemsetAsync(pl->d_fb_corr, 0, (size_t)pl->C * AP * 16, pl->st));
    MOFF_CK(cudaMemsetAsync(pl->d_fb_power, 0, (size_t)pl->C * P * 8, pl->st));
    pl->fb_kx = kx;
    pl->fb_ky = ky;
    pl->fb_on = true;
    pl->fb_samples = 0;
    drop_graphs(pl);   // the captured launch sequences change
    return sync_plan(pl, -1);
}

moff_status moff_read_feedback(moff_plan *pl, float *corr, double *power, long long *n_samples, int reset,
                               int timeout_ms) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (!pl->fb_on) return fail(MOFF_ESTATE, "no calibrator set (moff_set_calibrator)");
    if ((s = sync_plan(pl, timeout_ms)) != MOFF_OK) return s;
    if ((s = check_device_err(pl)) != MOFF_OK) return s;
    const size_t n = (size_t)pl->C * pl->A * pl->P;
    if (corr) {
        MOFF_CK(launch_fb_finish(pl->d_fb_corr, pl->d_fb_power, pl->d_fb_beam, pl->d_chan_group, pl->d_gains, pl->C, pl->A * pl->P, pl->P,
                                 pl->A, pl->d_fb_out, nullptr, 0, pl->st));
        MOFF_CK(cudaMemcpyAsync(corr, pl->d_fb_out, n * 8, cudaMemcpyDeviceToHost, pl->st));
    }
    if (power) MOFF_CK(cudaMemcpyAsync(power, pl->d_fb_power, (size_t)pl->C * pl->P * 8, cudaMemcpyDeviceToHost, pl->st));
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    if (n_samples) *n_samples = pl->fb_samples;
    if (reset) {
        MOFF_CK(cudaMemsetAsync(pl->d_fb_corr, 0, n * 16, pl->st));
        MOFF_CK(cudaMemsetAsync(pl->d_fb_power, 0, (size_t)pl->C * pl->P * 8, pl->st));
        pl->fb_samples = 0;
    }
    return MOFF_OK;
}

moff_status moff_feedback_gains(moff_plan *pl, float *delta, int apply) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (!pl->fb_on) return fail(MOFF_ESTATE, "no calibrator set (moff_set_calibrator)");
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    const size_t n = (size_t)pl->C * pl->A * pl->P;
    MOFF_CK(launch_fb_finish(pl->d_fb_corr, pl->d_fb_power, pl->d_fb_beam, pl->d_chan_group, pl->d_gains, pl->C, pl->A * pl->P, pl->P,
                             pl->A, nullptr, pl->d_fb_out, apply ? 1 : 0, pl->st));
    if (apply && pl->tc) MOFF_CK(launch_gain_scale(pl->d_gains, pl->C, pl->A * pl->P, pl->d_sy, pl->st));
    if (delta) MOFF_CK(cudaMemcpyAsync(delta, pl->d_fb_out, n * 8, cudaMemcpyDeviceToHost, pl->st));
    return sync_plan(pl, -1);
}

moff_status moff_plan_tuning(const moff_plan *pl, int *time_batch, int *staged, int *cells_per_lane, int *source,
                             double *best_ms, int *wide_rows) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (time_batch) *time_batch = pl->tb;
    if (staged) *staged = pl->staged ? 1 : 0;
    if (cells_per_lane) *cells_per_lane = pl->quads ? 4 : (pl->pairs ? 2 : 1);
    if (source) *source = pl->tune_source;
    if (best_ms) *best_ms = pl->tune_best_ms;
    if (wide_rows) *wide_rows = pl->wide ? 1 : 0;
    return MOFF_OK;
}

moff_status moff_plan_dft_tuning(const moff_plan *pl, int *cols_width, int *source, double *ms_w8, double *ms_w16) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (cols_width) *cols_width = pl->dft ? pl->cols_w : 0;
    if (source) *source = pl->cols_w_source;
    if (ms_w8) *ms_w8 = pl->cols_w_ms[0];
    if (ms_w16) *ms_w16 = pl->cols_w_ms[1];
    return MOFF_OK;
}

moff_status moff_set_timing(moff_plan *pl, int on) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    clear_recs(pl);
    pl->timing = on != 0;
    return MOFF_OK;
}

moff_status moff_timing(moff_plan *pl, int kind, double *total_ms, long long *launches, int reset) {
    moff_status s = check_plan(pl);
    if (s != MOFF_OK) return s;
    if (kind < 0 || kind > 8) return fail(MOFF_EINVAL, "kind (%d) must be in [0, 8]", kind);
    if ((s = sync_plan(pl, -1)) != MOFF_OK) return s;
    double tot = 0.0;
    long long n = 0;
    for (auto &r : pl->recs) {
        if (r.kind != kind) continue;
        float ms = 0.f;
        MOFF_CK(cudaEventElapsedTime(&ms, r.a, r.b));
        tot += ms;
        ++n;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = n;
    if (reset) clear_recs(pl);
    return MOFF_OK;
}

moff_status moff_plan_route(const moff_plan *pl, int *route) {
    if (!pl || !route) return fail(MOFF_EINVAL, "plan and route must not be NULL");
    *route = pl->gtc ? 3 : (pl->dft ? 2 : (pl->tc ? 1 : 0));
    return MOFF_OK;
}

moff_status moff_plan_info(const moff_plan *pl, int *n_prod, int *rows_per_stripe, int *time_chunk, int *chan_chunk,
                           long long *device_bytes) {
    if (!pl) return fail(MOFF_EINVAL, "plan is NULL");
    if (n_prod) *n_prod = pl->nprod;
    if (rows_per_stripe) *rows_per_stripe = pl->rows;
    if (time_chunk) *time_chunk = pl->Tb;
    if (chan_chunk) *chan_chunk = pl->Cb;
    if (device_bytes) *device_bytes = (long long)pl->dev_bytes;
    return MOFF_OK;
}

}  // extern "C"
