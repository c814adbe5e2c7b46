// moff_noalloc.cu -- moff_image_noalloc: the imaging path for callers that
// must not allocate GPU memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory budget
// fixed by someone else (a pre-sized pool or a real-time pipeline that may not
// block on the allocator), or a host program that was handed only device
// buffers.  For them this entry point images one block of voltages with every
// intermediate -- the kernel lists, the twiddles, the row-transformed field
// and the FP64 sums -- placed in one file-scope __device__ array of fixed size
// (kNoallocScratchBytes, 64 MiB) that every GPU loading the library holds
// until the process exits.  The caller passes all inputs and the output; the
// function calls no cudaMalloc, cudaFree or allocating library routine.
//
// The same two kernels as moff_submit do the work (calibrate + grid + row
// transform, then column transform + square-and-integrate); only the memory
// they are pointed at differs.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/moff.h"
#include "moff_internal.h"

namespace moff {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

moff_status failf(moff_status s, const char *fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return fail_msg(s, buf);
}

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in, never a device address; the real
// address is looked up once per device, with that device current.
moff_status scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return failf(MOFF_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return failf(MOFF_EINVAL, "device index %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return failf(MOFF_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return MOFF_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace moff

using namespace moff;

extern "C" moff_status moff_image_noalloc(int n_ant, const double *pos, int ksize, const float *taps, int grid_n,
                                          int n_chan, int n_pol, unsigned flags, const uint8_t *volt, int n_time,
                                          const float *gains, float *image, void *cuda_stream) {
    if (n_ant < 1 || n_ant > 65536) return failf(MOFF_EINVAL, "n_ant (%d) must be in [1, 65536]", n_ant);
    if (!pos || !taps || !volt || !gains || !image)
        return failf(MOFF_EINVAL, "pos, taps, volt, gains and image must not be NULL");
    if (grid_n != 32 && grid_n != 64 && grid_n != 128 && grid_n != 256 && grid_n != 512)
        return failf(MOFF_EINVAL, "grid_n (%d) must be 32, 64, 128, 256 or 512", grid_n);
    if (ksize < 1 || ksize % 2 == 0 || ksize > 15 || ksize > grid_n)
        return failf(MOFF_EINVAL, "ksize (%d) must be odd, in [1, 15] and <= grid_n", ksize);
    if (n_chan < 1) return failf(MOFF_EINVAL, "n_chan (%d) must be >= 1", n_chan);
    if (n_pol != 1 && n_pol != 2) return failf(MOFF_EINVAL, "n_pol (%d) must be 1 or 2", n_pol);
    if (flags & ~(unsigned)MOFF_JONES) return failf(MOFF_EINVAL, "only MOFF_JONES may be set (flags 0x%x)", flags);
    const bool jones = (flags & MOFF_JONES) != 0;
    if (jones && n_pol != 2) return failf(MOFF_EINVAL, "MOFF_JONES requires n_pol = 2");
    if (n_time < 1) return failf(MOFF_EINVAL, "n_time (%d) must be >= 1", n_time);

    const int N = grid_n, P = n_pol, C = n_chan, nprod = P == 1 ? 1 : 4;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    {   // the host lists are copied from pageable memory: not capturable
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(st, &cs);
        if (e != cudaSuccess) return failf(MOFF_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
        if (cs != cudaStreamCaptureStatusNone)
            return failf(MOFF_ESTATE, "moff_image_noalloc cannot run while its stream is being captured");
    }

    Bins b;
    moff_status s = build_bins(n_ant, ksize, N, P, jones, pos, taps, &b);
    if (s != MOFF_OK) return s;
    const std::vector<float2> tw = pass_twiddles_for(N);

    // Scratch layout: twiddles | lists | FP64 sums of a channel chunk | row-transformed field.
    size_t off = 0;
    const size_t o_tw = off;        off = align256(off + tw.size() * 8);
    const size_t o_ant_off = off;   off = align256(off + b.ant_off.size() * 4);
    const size_t o_ant = off;       off = align256(off + std::max<size_t>(b.ant_list.size(), 1) * 4);
    const size_t o_soff = off;      off = align256(off + b.slice_off.size() * 8);
    const size_t o_lcell = off;     off = align256(off + b.lane_cell.size() * 2);
    const size_t o_tap = off;       off = align256(off + std::max<size_t>(b.con_tap.size(), 1) * 8);
    const size_t o_cy = off;        off = align256(off + std::max<size_t>(b.con_y.size(), 1) * 2);
    const size_t fixed = off;
    const size_t per_acc = (size_t)nprod * N * N * 8;   // FP64 sums of one channel
    const size_t per_h = (size_t)P * N * N * 8;         // row-transformed field of one sample of one channel
    if (fixed + per_acc + per_h > kNoallocScratchBytes)
        return failf(MOFF_EINVAL,
                     "this array needs %zu bytes of scratch for one channel and sample, more than the %zu-byte "
                     "no-allocation limit",
                     fixed + per_acc + per_h, kNoallocScratchBytes);
    const size_t room = kNoallocScratchBytes - fixed;
    int Tb = std::min(n_time, 16);
    while (Tb > 1 && room / (per_acc + (size_t)Tb * per_h) < 1) Tb /= 2;
    const int Cb = (int)std::min<size_t>((size_t)C, room / (per_acc + (size_t)Tb * per_h));
    const size_t o_acc = fixed;
    const size_t o_H = align256(o_acc + (size_t)Cb * per_acc);

    void *base = nullptr;
    if ((s = scratch_address(&base)) != MOFF_OK) return s;
    unsigned char *sc = static_cast<unsigned char *>(base);

#define NA_CK(call)                                                                                 \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return failf(MOFF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

    // Host lists are pageable: each copy has read its source before it returns.
    NA_CK(cudaMemcpyAsync(sc + o_tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(sc + o_ant_off, b.ant_off.data(), b.ant_off.size() * 4, cudaMemcpyHostToDevice, st));
    if (!b.ant_list.empty())
        NA_CK(cudaMemcpyAsync(sc + o_ant, b.ant_list.data(), b.ant_list.size() * 4, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(sc + o_soff, b.slice_off.data(), b.slice_off.size() * 8, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(sc + o_lcell, b.lane_cell.data(), b.lane_cell.size() * 2, cudaMemcpyHostToDevice, st));
    if (!b.con_tap.empty()) {
        NA_CK(cudaMemcpyAsync(sc + o_tap, b.con_tap.data(), b.con_tap.size() * 8, cudaMemcpyHostToDevice, st));
        NA_CK(cudaMemcpyAsync(sc + o_cy, b.con_y.data(), b.con_y.size() * 2, cudaMemcpyHostToDevice, st));
    }

    const long long tstride = (long long)C * n_ant * P;
    double *acc = reinterpret_cast<double *>(sc + o_acc);
    for (int c0 = 0; c0 < C; c0 += Cb) {
        const int nc = std::min(Cb, C - c0);
        // the array keeps the previous call's contents: the sums start at zero
        NA_CK(cudaMemsetAsync(acc, 0, (size_t)nc * per_acc, st));
        for (int t0 = 0; t0 < n_time; t0 += Tb) {
            const int nt = std::min(Tb, n_time - t0);
            GridArgs g{};
            g.volt = volt;
            g.volt_tstride = tstride;
            g.t0 = t0;
            g.nt = nt;
            g.c0 = c0;
            g.nc = nc;
            g.A = n_ant;
            g.rows = b.rows;
            g.max_nloc = b.max_nloc;
            g.max_entries = b.max_entries;
            g.n_slices = b.n_slices;
            g.gains = reinterpret_cast<const float2 *>(gains);
            g.st_ant_off = reinterpret_cast<const int *>(sc + o_ant_off);
            g.st_ant = reinterpret_cast<const int *>(sc + o_ant);
            g.slice_off = reinterpret_cast<const long long *>(sc + o_soff);
            g.lane_cell = reinterpret_cast<const uint16_t *>(sc + o_lcell);
            g.con_tap = reinterpret_cast<const float2 *>(sc + o_tap);
            g.con_y = reinterpret_cast<const uint16_t *>(sc + o_cy);
            g.twp = reinterpret_cast<const float2 *>(sc + o_tw);
            g.out = reinterpret_cast<float2 *>(sc + o_H);
            g.slab_t = 1;
            g.slab_c = Tb;
            g.pairs = b.pairs ? 1 : 0;
            g.quads = b.quads ? 1 : 0;
            g.wide = b.wide ? 1 : 0;
            NA_CK(launch_grid(N, P, b.tb, b.staged, false, g, b.n_stripes, b.grid_smem, st));
            ColArgs ca{};
            ca.H = reinterpret_cast<const float2 *>(sc + o_H);
            ca.nt = nt;
            ca.c0 = 0;              // sums of this chunk are indexed from its first channel
            ca.nc = nc;
            ca.slab_t = g.slab_t;
            ca.slab_c = g.slab_c;
            ca.twp = reinterpret_cast<const float2 *>(sc + o_tw);
            ca.acc = acc;
            NA_CK(launch_cols(N, P, ca, st));
        }
        NA_CK(launch_to_f32(acc, image + (size_t)c0 * nprod * N * N, (long long)nc * nprod * N * N, st));
    }
#undef NA_CK
    return MOFF_OK;
}
