// moff_tc_kernels.cu -- FP16 tensor-core variant of Eq. m6 steps 1-3 (first
// axis) of Morales (arXiv 0812.3669): gridding and the row transform as one
// dense contraction per grid row.
//
// The row transform of the gridded field is linear in the weighted voltages:
//   H(ry, kx) = sum_rx G(ry, rx) e^{+2 pi i kx rx / N}
//             = sum_{segments j on row ry} y_j * S_j(kx),
// where a segment is one row dy of one antenna-pol kernel (Eq. m6 step 2) and
// S_j(kx) = sum_dx taps[dy][dx] e^{+2 pi i kx (anchor_x + dx - K/2) / N} is its
// row spectrum, computed once per plan in FP64.  Per (pol, grid row) this is a
// product (samples x 2 nseg) * (2 nseg x 2 KX) in real arithmetic, run on the
// tensor cores with FP16 operands (exact power-of-two scales) and FP32
// accumulation in TMEM.  The second transform axis and the squaring stay in
// the FP32 column kernel.
//
//   k_gain_scale   per-channel power-of-two scale keeping weighted voltages in FP16 range
//   k_volt_prep    decode, weight, scale and transpose the voltages to FP16 planes [c][voltage][t],
//                  antennas ordered by anchor row so a grid row's segments are consecutive plane rows
//   k_rowspec_tc   per (pol, row, kx tile): B = row spectra resident in shared memory,
//                  A = 128 samples of the row's segment voltages (TMA tiles of 32 plane rows,
//                  128-byte swizzled, MN-major),
//                  D = TMEM (double buffered), epilogue writes the row-transformed field in
//                  FP16 under an exact power-of-two scale (undone by the column kernel).
#include <cuda_fp16.h>

#include "moff_fft.cuh"
#include "moff_internal.h"
#include "moff_tc.cuh"

namespace moff {
namespace {

// One weighted voltage y = (g s) x of a 4+4-bit code b (real part in the high nibble), with gs = g s
// the gain times the channel's power-of-two scale.  A nibble u reads (u xor 8) - 8: (u xor 8) goes
// into the low mantissa bits of 2^23, and one packed subtraction of 2^23 + 8 leaves the integer
// exactly (no integer-to-float conversion); then re = gs.re x.re - gs.im x.im and im = gs.re x.im +
// gs.im x.re, each one rounded product and one fused multiply-add, both parts in two packed
// instructions.  Returns the pair as FP16 (round to nearest) for samples b0 (low half) and b1.
__device__ __forceinline__ float2 weigh_tc(float2 gs, uint32_t b) {
    const uint32_t bre = ((b >> 4) & 15u) ^ 0x4B000008u, bim = (b & 15u) ^ 0x4B000008u;
    float2 x, p, y;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %4};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(x.x), "=f"(x.y)
        : "r"(bre), "r"(bim), "f"(8388616.0f));
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(p.x), "=f"(p.y)
        : "f"(-gs.y), "f"(gs.y), "f"(x.y), "f"(x.x));
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %2};\n\tmov.b64 rb, {%3, %4};\n\tmov.b64 rc, {%5, %6};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(y.x), "=f"(y.y)
        : "f"(gs.x), "f"(x.x), "f"(x.y), "f"(p.x), "f"(p.y));
    return y;
}
__device__ __forceinline__ void weigh2_tc(float2 gs, uint32_t b0, uint32_t b1, uint32_t &re, uint32_t &im) {
    const float2 y0 = weigh_tc(gs, b0), y1 = weigh_tc(gs, b1);
    const __half2 hr = __floats2half2_rn(y0.x, y1.x), hi = __floats2half2_rn(y0.y, y1.y);
    re = *reinterpret_cast<const uint32_t *>(&hr);
    im = *reinterpret_cast<const uint32_t *>(&hi);
}

// s_y[c] = 2^e with 16 * max|g_c| * 2^e in [2^13, 2^14): |y| <= |g| (|x_re| + |x_im|) <= 16 |g|.
__global__ void k_gain_scale(const float2 *__restrict__ gains, int AP, float *__restrict__ sy) {
    const int c = blockIdx.x;
    float m = 0.f;
    for (int i = threadIdx.x; i < AP; i += blockDim.x) {
        const float2 g = gains[(long long)c * AP + i];
        m = fmaxf(m, fmaxf(fabsf(g.x), fabsf(g.y)));
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) {
            float s = 1.f;
            if (m > 0.f) {
                int e;
                frexpf(16.f * m, &e);            // 16 m in [2^(e-1), 2^e)
                s = ldexpf(1.f, 14 - e);         // 16 m s in [2^13, 2^14)
            }
            sy[c] = s;
        }
    }
}

// Voltages of samples [t0, t0+nt) of channels [c0, c0+nc) -> FP16 planes
// Yre/Yim [nc][APpad][Tpad] (t contiguous), zero for t >= nt and for rows v >= AP (the
// pad rows a chunk running past the last voltage reads); plane row v < AP holds voltage
// perm[v].  A CTA stages the voltage bytes of TT samples of one channel (coalesced
// 16-byte loads) and writes every plane row's TT samples (half2 per sample pair).
__global__ void __launch_bounds__(256) k_volt_prep(const uint8_t *__restrict__ volt, long long tstride, int t0, int nt,
                                                   int c0, int AP, int APpad, const float2 *__restrict__ gains,
                                                   const float *__restrict__ sy, const int *__restrict__ perm, int Tpad,
                                                   int TT, __half *__restrict__ yre, __half *__restrict__ yim,
                                                   int n_rows) {
    extern __shared__ __align__(16) unsigned char s_v[];   // [TT][APr] voltage bytes
    const int cl = blockIdx.y, c = c0 + cl;
    const int tb = blockIdx.x * TT;
    const int APr = (AP + 15) & ~15, nq = APr / 16;
    const float s = sy[c];
    const uint8_t *vc = volt + (long long)c * AP;
    const bool vec = (AP & 15) == 0 && (tstride & 15) == 0 && ((reinterpret_cast<uintptr_t>(vc)) & 15) == 0;
    for (int i = threadIdx.x; i < TT * nq; i += blockDim.x) {
        const int tt = i / nq, q = i - tt * nq, t = tb + tt;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (t < nt) {
            const uint8_t *src = vc + (long long)(t0 + t) * tstride + q * 16;
            if (vec) {
                v = *reinterpret_cast<const uint4 *>(src);
            } else {
                uint32_t w[4] = {0u, 0u, 0u, 0u};
                for (int u = 0; u < 16 && q * 16 + u < AP; ++u) w[u >> 2] |= (uint32_t)src[u] << (8 * (u & 3));
                v = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        *reinterpret_cast<uint4 *>(s_v + tt * APr + q * 16) = v;
    }
    __syncthreads();
    if (TT >= 8) {   // 8 samples of one plane row per thread: one 16-byte store per plane
        const int ng = TT / 8;
        for (int i = threadIdx.x; i < APpad * ng; i += blockDim.x) {
            const int v = i / ng, t8 = 8 * (i - v * ng);
            uint4 re = make_uint4(0u, 0u, 0u, 0u), im = re;
            if (v < n_rows) {
                const int sv = perm[v];
                const float2 g = gains[(long long)c * AP + sv], gs = make_float2(g.x * s, g.y * s);
                uint32_t hr[4], hi[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    weigh2_tc(gs, s_v[(t8 + 2 * u) * APr + sv], s_v[(t8 + 2 * u + 1) * APr + sv], hr[u], hi[u]);
                re = make_uint4(hr[0], hr[1], hr[2], hr[3]);
                im = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            }
            const long long o = ((long long)cl * APpad + v) * Tpad + tb + t8;   // 16-byte aligned (Tpad % 8 == 0)
            *reinterpret_cast<uint4 *>(yre + o) = re;
            *reinterpret_cast<uint4 *>(yim + o) = im;
        }
        return;
    }
    const int np = TT / 2;
    for (int i = threadIdx.x; i < APpad * np; i += blockDim.x) {
        const int v = i / np, tp = 2 * (i - v * np), t = tb + tp;
        uint32_t re = 0u, im = 0u;
        if (v < n_rows) {
            const int sv = perm[v];
            const float2 g = gains[(long long)c * AP + sv];
            weigh2_tc(make_float2(g.x * s, g.y * s), s_v[tp * APr + sv], s_v[(tp + 1) * APr + sv], re, im);
        }
        const long long o = ((long long)cl * APpad + v) * Tpad + t;   // t even, Tpad even: 4-byte aligned
        *reinterpret_cast<uint32_t *>(yre + o) = re;
        *reinterpret_cast<uint32_t *>(yim + o) = im;
    }
}

// 16-byte asynchronous global -> shared copies for the plane kernel's staging ring.
__device__ __forceinline__ void vp_cp16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void vp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most n (0..3) of this thread's copy groups are still in flight
__device__ __forceinline__ void vp_wait(int n) {
    if (n <= 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else if (n == 2) asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    else asm volatile("cp.async.wait_group 3;\n" ::: "memory");
}

// Large arrays (a channel's voltage bytes of eight samples exceed the staging budget): one
// thread per plane row, all Tpad samples in passes of 32.  A warp whose 32 plane rows hold 32
// consecutive voltages (the common case: antennas in raster order) copies each sample's 32 bytes
// as two or three aligned 16-byte pieces into a three-pass ring in shared memory (cp.async, up to
// two passes ahead of the one it converts) and picks its byte there; other warps read one byte
// per sample and row.  With store maps (use_tma) a warp whose 32 rows all lie inside the channel's
// APpad rows writes each pass's 32 rows x 32 samples of each plane as one TMA box (64-byte
// swizzle: piece k of row r at k ^ ((r >> 1) & 3)); other rows are stored directly as four
// 16-byte pieces per plane.  vec_ok: 16-byte aligned voltage rows (tstride and A P multiples of 16).
constexpr int kVpRing = 3;
constexpr int kVpRingBytes = kVpRing * 8 * 32 * 48;
constexpr int kVpBoxBytes = 2 * 32 * 64;                 // one warp's re and im boxes
constexpr size_t kVpSmem = 1024 + kVpRingBytes + 8 * kVpBoxBytes;
__global__ void __launch_bounds__(256, 3) k_volt_prep_rows(const uint8_t *__restrict__ volt, long long tstride, int t0,
                                                        int nt, int c0, int AP, int APpad, int n_rows,
                                                        const float2 *__restrict__ gains, const float *__restrict__ sy,
                                                        const int *__restrict__ perm, int Tpad, int vec_ok,
                                                        __half *__restrict__ yre, __half *__restrict__ yim,
                                                        const __grid_constant__ CUtensorMap smap_re,
                                                        const __grid_constant__ CUtensorMap smap_im, int use_tma) {
    extern __shared__ __align__(1024) unsigned char vp_smem[];
    unsigned char *base_s = vp_smem + ((1024u - (tc::smem_u32(vp_smem) & 1023u)) & 1023u);
    auto ring = [&](int slot, int wp, int t) { return base_s + ((slot * 8 + wp) * 32 + t) * 48; };
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int cl = blockIdx.y, c = c0 + cl;
    const int v0 = v - lane;
    const bool boxed = use_tma && v0 + 32 <= APpad;      // warp-uniform
    unsigned char *bre = base_s + kVpRingBytes + wp * kVpBoxBytes, *bim = bre + kVpBoxBytes / 2;
    const bool have = v < n_rows;
    const int sv = have ? perm[v] : 0;
    const int sv0 = __shfl_sync(0xffffffffu, sv, 0);
    const bool contig = vec_ok && __all_sync(0xffffffffu, have && sv == sv0 + lane);
    const int np = Tpad / 32;
    // contiguous warps: bytes [row0, row0 + 32) of each sample are pieces [a0 + 16 k, a0 + 16 k + 16), k < npc,
    // all inside the channel's A P bytes (c A P and A P are multiples of 16, sv0 + 32 <= A P)
    const long long row0 = (long long)c * AP + sv0, a0 = row0 & ~15LL;
    const int off = (int)(row0 - a0), npc = (off + 47) >> 4;
    auto issue = [&](int p) {      // pass p's 32 samples into ring slot p mod 3 (zero past the block)
        const uint8_t *src = volt + (long long)(t0 + 32 * p) * tstride + a0;
        for (int i = lane; i < 32 * npc; i += 32) {
            const int t = i / npc, k = i - t * npc;
            unsigned char *d = ring(p % kVpRing, wp, t) + 16 * k;
            if (32 * p + t < nt) vp_cp16(d, src + (long long)t * tstride + 16 * k);
            else *reinterpret_cast<uint4 *>(d) = make_uint4(0u, 0u, 0u, 0u);
        }
        vp_commit();
    };
    int issued = 0;
    if (contig)
        for (; issued < np && issued < kVpRing - 1; ++issued) issue(issued);
    const float2 g = have ? gains[(long long)c * AP + sv] : make_float2(0.f, 0.f);
    const float2 gs = make_float2(g.x * sy[c], g.y * sy[c]);
    for (int p = 0; p < np; ++p) {
        const int tb = 32 * p;
        uint32_t b[32];
        if (contig) {
            if (issued < np) issue(issued++);
            vp_wait(issued - 1 - p);                 // pass p's group has landed
            __syncwarp();
#pragma unroll
            for (int t = 0; t < 32; ++t) b[t] = ring(p % kVpRing, wp, t)[off + lane];
            __syncwarp();                            // read by every lane before the slot is refilled
        } else {
            const uint8_t *src = volt + (long long)(t0 + tb) * tstride + (long long)c * AP + sv;
#pragma unroll
            for (int t = 0; t < 32; ++t) b[t] = have && tb + t < nt ? (uint32_t)__ldg(src + (long long)t * tstride) : 0u;
        }
        if (!boxed && v >= APpad) continue;
        uint32_t re[16], im[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) re[i] = im[i] = 0u;
        if (have) {
#pragma unroll
            for (int t = 0; t < 32; t += 2) weigh2_tc(gs, b[t], b[t + 1], re[t >> 1], im[t >> 1]);
        }
        if (boxed) {
            if (p > 0) {                             // the previous pass's stores have read the boxes
                if (lane == 0) tc::bulk_wait_read<0>();
                __syncwarp();
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int o = lane * 64 + ((k ^ ((lane >> 1) & 3)) << 4);
                *reinterpret_cast<uint4 *>(bre + o) = make_uint4(re[4 * k], re[4 * k + 1], re[4 * k + 2], re[4 * k + 3]);
                *reinterpret_cast<uint4 *>(bim + o) = make_uint4(im[4 * k], im[4 * k + 1], im[4 * k + 2], im[4 * k + 3]);
            }
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                const int y = cl * APpad + v0;
                tc::tma_store_2d(&smap_re, tc::smem_u32(bre), tb, y);
                tc::tma_store_2d(&smap_im, tc::smem_u32(bim), tb, y);
                tc::bulk_commit();
            }
            continue;
        }
        uint4 *ore = reinterpret_cast<uint4 *>(yre + ((long long)cl * APpad + v) * Tpad + tb);
        uint4 *oim = reinterpret_cast<uint4 *>(yim + ((long long)cl * APpad + v) * Tpad + tb);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ore[k] = make_uint4(re[4 * k], re[4 * k + 1], re[4 * k + 2], re[4 * k + 3]);
            oim[k] = make_uint4(im[4 * k], im[4 * k + 1], im[4 * k + 2], im[4 * k + 3]);
        }
    }
    if (boxed && lane == 0) tc::bulk_wait_all();
}

template <int N>
struct TcShape {
    static constexpr int KX = N < 128 ? N : 128;     // kx per tile
    static constexpr int NT = 2 * KX;                // MMA N: real parts then imaginary parts
    static constexpr int NTILES = N / KX;
    static constexpr int TCOLS = 2 * NT <= 32 ? 32 : 2 * NT;   // two TMEM accumulators
};

// Warp roles: warps 0-7 drain the TMEM accumulators (lane quarter w % 4, kx half
// w / 4), one lane of warp 8 loads A with TMA, one lane of warp 9 issues the MMAs.
// A: ring of kAStages K-chunks of 64 = 32 consecutive plane rows (real parts,
// then imaginary parts) x 128 samples, MN-major with the 128-byte swizzle: two
// 64-sample halves of 8 KB, each 64 rows of 128 bytes; four TMA tiles of
// 64 samples x 32 rows per chunk.  B: resident; accumulators: two in TMEM;
// epilogue: each warp converts its 32 samples x 32 kx to FP16 into a
// 128-byte-swizzled box in shared memory and one lane hands it to the TMA unit
// (bulk tensor store); a warp reuses its box once the store has read it.
constexpr int kEpiWarps = 8;   // two per TMEM lane quarter, each draining half of the kx columns
constexpr int kTcRoleThreads = (kEpiWarps + 2) * 32;
constexpr int kAStages = 4, kKChunk = 64;
constexpr int kAChunkBytes = 128 * kKChunk * 2;
constexpr int kAHalfBytes = kAChunkBytes / 2;          // one 64-sample half: 64 rows x 128 bytes
constexpr int kBoxBytes = 32 * 128;                 // 32 samples x 32 kx x half2
constexpr int kEpiBufs = 1;                         // boxes per warp
constexpr long long kWaitCycles = 4000000000LL;     // ~2 s at the SM clock

template <int N>
__global__ void __launch_bounds__(kTcRoleThreads, 1)
    k_rowspec_tc(const RowSpecArgs a, const __grid_constant__ CUtensorMap hmap,
                 const __grid_constant__ CUtensorMap amap_re, const __grid_constant__ CUtensorMap amap_im) {
    using S = TcShape<N>;
    constexpr int KX = S::KX, NT = S::NT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int item = blockIdx.x;                      // (p * N + ry) * NTILES + tile
    const int tile = item % S::NTILES;
    const int pr = item / S::NTILES;
    const int p = pr / N, ry = pr % N;
    const int kp = a.kp[pr];
    const int ch0 = a.chunk_off[pr];

    const int cper = (a.nc + gridDim.y - 1) / gridDim.y;
    const int cb = blockIdx.y * cper, ce = min(a.nc, cb + cper);
    if (cb >= ce) return;
    const int ntb = (a.nt + 127) / 128;
    const int nitems = (ce - cb) * ntb;

    // No kernel row lands on this grid row: its row-transformed field is zero, and the
    // column kernel never reads it (the plan's reached-row mask clears it there), so
    // nothing is written.
    if (kp == 0) return;
    const int nchunk = kp / kKChunk;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzled TMA boxes need 1024-byte alignment: round the base up (the size includes the slack)
    unsigned char *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *sB = smem;                                  // NT x kp, K-major (resident)
    unsigned char *sA = sB + (size_t)NT * a.kp_max * 2;        // kAStages x [128 x 64], MN-major, 1024-aligned
    unsigned char *sE = sA + (size_t)kAStages * kAChunkBytes;  // [kEpiWarps][kEpiBufs] boxes, 1024-aligned
    uint64_t *bars = reinterpret_cast<uint64_t *>(sE + kEpiWarps * kEpiBufs * kBoxBytes);
    uint64_t *a_full = bars, *a_empty = bars + kAStages, *d_full = bars + 2 * kAStages,
             *d_empty = bars + 2 * kAStages + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * kAStages + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.bimg + a.bimg_off[item]);
        uint4 *dst = reinterpret_cast<uint4 *>(sB);
        const int n16 = NT * kp * 2 / 16;
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    if (tid == 0) {
        for (int b = 0; b < kAStages; ++b) {
            tc::mbar_init(&a_full[b], 1);        // the producer's arrive + the chunk's TMA bytes
            tc::mbar_init(&a_empty[b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&d_full[b], 1);
            tc::mbar_init(&d_empty[b], kEpiWarps * 32);
        }
        *abort_flag = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, S::TCOLS);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();   // resident B written by generic stores, read by the tensor core
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == kEpiWarps) {
        // ---------------- producer (one lane): chunk g (global counter) into stage g % kAStages,
        // four TMA tiles (re / im x two 64-sample halves) completing on a_full.
        if (lane == 0) {
            int g = 0;
            for (int i = 0; i < nitems && !*abort_flag; ++i) {
                const int cl = cb + i / ntb, t0b = (i % ntb) * 128;
                bool ok = true;
                for (int ch = 0; ch < nchunk; ++ch, ++g) {
                    const int st = g % kAStages;
                    if (!tc::mbar_wait_abortable(&a_empty[st], (uint32_t)(((g / kAStages) & 1) ^ 1), kWaitCycles,
                                                 abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = tc::smem_u32(sA + st * kAChunkBytes);
                    const int y = cl * a.AP + a.chunk_row[ch0 + ch];
                    tc::mbar_arrive_expect_tx(&a_full[st], kAChunkBytes);
#pragma unroll
                    for (int hm = 0; hm < 2; ++hm) {
                        tc::tma_load_2d(sa + hm * kAHalfBytes, &amap_re, t0b + 64 * hm, y, &a_full[st]);
                        tc::tma_load_2d(sa + hm * kAHalfBytes + kAHalfBytes / 2, &amap_im, t0b + 64 * hm, y,
                                        &a_full[st]);
                    }
                }
                if (!ok) break;
            }
            // tiles still landing (the MMA lane stopped early): let them finish before the
            // shared memory is released
            for (int gg = g - kAStages > 0 ? g - kAStages : 0; gg < g; ++gg)
                tc::mbar_wait_bounded(&a_full[gg % kAStages], (uint32_t)((gg / kAStages) & 1), kWaitCycles);
        }
        __syncwarp();
    } else if (warp == kEpiWarps + 1) {
        // ---------------- MMA issuer (one lane)
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(128, NT, /*a_mn=*/true, /*b_mn=*/false);
            const uint32_t sb_sbo = (uint32_t)(kp / 8) * 128;
            const uint32_t sbb = tc::smem_u32(sB);
            int g = 0;
            bool ok = true;
            for (int i = 0; i < nitems && ok; ++i) {
                const int b = i & 1;
                ok = tc::mbar_wait_abortable(&d_empty[b], (uint32_t)(((i >> 1) & 1) ^ 1), kWaitCycles, abort_flag);
                if (!ok) break;
                const uint32_t d = tbase + (uint32_t)(b * NT);
                for (int ch = 0; ch < nchunk; ++ch, ++g) {
                    const int st = g % kAStages;
                    ok = tc::mbar_wait_abortable(&a_full[st], (uint32_t)((g / kAStages) & 1), kWaitCycles, abort_flag);
                    if (!ok) break;
                    tc::fence_after_sync();
                    const uint32_t sa = tc::smem_u32(sA + st * kAChunkBytes);
                    for (int ks = 0; ks < kKChunk / 16; ++ks) {
                        // 128-byte swizzled MN-major: LBO = the 64-sample halves' stride, SBO = 8 rows
                        const uint64_t ad = tc::smem_desc_sw128(sa + ks * 16 * 128, kAHalfBytes, 1024);
                        const uint64_t bd = tc::smem_desc(sbb + (ch * (kKChunk / 8) + 2 * ks) * 128, 128, sb_sbo);
                        tc::mma_f16(d, ad, bd, idesc, ch > 0 || ks > 0);
                    }
                    tc::mma_commit(&a_empty[st]);   // stage free once these MMAs finish
                }
                if (ok) tc::mma_commit(&d_full[b]); // accumulator ready
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps 0-7: TMEM lanes 32 (w % 4) .. + 31 = samples
        unsigned char *sw = sE + warp * kEpiBufs * kBoxBytes;
        int nbox = 0;
        for (int i = 0; i < nitems; ++i) {
            const int b = i & 1;
            if (!tc::mbar_wait_abortable(&d_full[b], (uint32_t)((i >> 1) & 1), kWaitCycles, abort_flag)) break;
            tc::fence_after_sync();
            const int q4 = warp & 3;                     // TMEM lane quarter of this warp
            const int cl = cb + i / ntb, t0w = (i % ntb) * 128 + q4 * 32;
            const float inv = a.row_sh[pr];   // exact power of two: FP16 range for every row
            const uint32_t dcol = tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * NT);
            // kx columns of this warp: the 32-column boxes dealt out to the warps of its lane quarter
            constexpr int kPerQuarter = kEpiWarps / 4;
            const int nbx = KX / 32, per = (nbx + kPerQuarter - 1) / kPerQuarter;
            const int kx_lo = min(nbx, (warp >> 2) * per) * 32, kx_hi = min(nbx, (warp >> 2) * per + per) * 32;
            const int nb = (kx_hi - kx_lo) / 32;
#pragma unroll 1
            for (int k0 = kx_lo, bi = 0; k0 < kx_hi; k0 += 32, ++nbox, ++bi) {
                float vr[32], vi[32];
                tc::tmem_ld32(dcol + (uint32_t)k0, vr);
                tc::tmem_ld32(dcol + (uint32_t)(KX + k0), vi);
                if (bi == nb - 1) {                      // this item's last TMEM read: the accumulator is free
                    tc::fence_before_sync();
                    tc::mbar_arrive(&d_empty[b]);
                }
                // lane = sample t0w + lane: its 32 kx as eight 16-byte chunks of one 128-byte row,
                // chunk q stored at q ^ (row % 8) (the tensor map's 128-byte swizzle); packed
                // before waiting for the box so the conversion overlaps the previous store's read
                uint4 pk[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    __half2 h[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) h[u] = __floats2half2_rn(vr[4 * q + u] * inv, vi[4 * q + u] * inv);
                    pk[q] = *reinterpret_cast<const uint4 *>(h);
                }
                unsigned char *box = sw + (nbox % kEpiBufs) * kBoxBytes;
                if (nbox >= kEpiBufs) {                  // the store that last read this box is done with it
                    if (lane == 0) tc::bulk_wait_read<kEpiBufs - 1>();
                    __syncwarp();
                }
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *reinterpret_cast<uint4 *>(box + lane * 128 + ((q ^ (lane & 7)) << 4)) = pk[q];
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    // a box wholly past the block's samples is not issued (the map clips partial ones)
                    if (t0w < a.nt) tc::tma_store_4d(&hmap, tc::smem_u32(box), tile * KX + k0, p * N + ry, cl, t0w);
                    tc::bulk_commit();
                }
            }
            if (nb == 0) {                               // no kx columns for this warp (narrow grids)
                tc::fence_before_sync();
                tc::mbar_arrive(&d_empty[b]);
            }
        }
        if (lane == 0) tc::bulk_wait_all();
    }
    if (*abort_flag && tid == 0) atomicExch(a.err, tc::kErrWaitTimeout);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, S::TCOLS);
}

}  // namespace

size_t rowspec_smem_bytes(int N, int kp_max) {
    const int KX = N < 128 ? N : 128, NT = 2 * KX;
    size_t b = 1024 + (size_t)NT * kp_max * 2 + (size_t)kAStages * kAChunkBytes +
               (size_t)kEpiWarps * kEpiBufs * kBoxBytes + (size_t)(2 * kAStages + 4) * 8 + 8;
    b = (b + 127) & ~(size_t)127;
    // one CTA per SM: two CTAs must never wait on each other's TMEM columns
    return b < 120 * 1024 ? 120 * 1024 : b;
}

int rowspec_ntiles(int N) { return N < 128 ? 1 : N / 128; }

cudaError_t launch_gain_scale(const float2 *gains, int C, int AP, float *sy, cudaStream_t st) {
    k_gain_scale<<<C, 256, 0, st>>>(gains, AP, sy);
    return cudaGetLastError();
}

cudaError_t launch_volt_prep(const uint8_t *volt, long long tstride, int t0, int nt, int c0, int nc, int AP,
                             int APpad, const float2 *gains, const float *sy, const int *perm, int Tpad, __half *yre,
                             __half *yim, cudaStream_t st, int n_rows, const CUtensorMap *smap_re,
                             const CUtensorMap *smap_im) {
    // samples per CTA: 32, or fewer (even, dividing Tpad) so the staged bytes stay within 96 KB
    const size_t APr = (size_t)((AP + 15) & ~15);
    const int rows = n_rows < 0 ? AP : n_rows;
    if (8 * APr > 96 * 1024 && Tpad % 32 == 0) {   // too large to stage 8 samples: one thread per plane row
        dim3 grid((APpad + 255) / 256, nc);
        const int vec_ok = tstride % 16 == 0 && AP % 16 == 0 && ((uintptr_t)volt & 15) == 0;
        const int use_tma = smap_re && smap_im ? 1 : 0;
        CUtensorMap none{};
        cudaError_t e = cudaFuncSetAttribute(k_volt_prep_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVpSmem);
        if (e != cudaSuccess) return e;
        k_volt_prep_rows<<<grid, 256, kVpSmem, st>>>(volt, tstride, t0, nt, c0, AP, APpad, rows, gains, sy, perm, Tpad,
                                                     vec_ok, yre, yim, use_tma ? *smap_re : none,
                                                     use_tma ? *smap_im : none, use_tma);
        return cudaGetLastError();
    }
    int TT = 32;
    while (TT > 2 && (TT * APr > 96 * 1024 || Tpad % TT)) TT /= 2;
    if (Tpad % TT || TT * APr > 200 * 1024) return cudaErrorInvalidValue;
    const size_t smem = TT * APr;
    cudaError_t e = cudaFuncSetAttribute(k_volt_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(Tpad / TT, nc);
    k_volt_prep<<<grid, 256, smem, st>>>(volt, tstride, t0, nt, c0, AP, APpad, gains, sy, perm, Tpad, TT, yre, yim,
                                         rows);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_rowspec_t(const RowSpecArgs &a, const CUtensorMap &hmap, const CUtensorMap &are,
                             const CUtensorMap &aim, int cgroups, size_t smem, cudaStream_t st) {
    auto k = k_rowspec_tc<N>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(a.P * N * TcShape<N>::NTILES, cgroups), kTcRoleThreads, smem, st>>>(a, hmap, are, aim);
    return cudaGetLastError();
}

cudaError_t launch_rowspec(int N, const RowSpecArgs &a, const CUtensorMap &hmap, const CUtensorMap &amap_re,
                           const CUtensorMap &amap_im, int cgroups, size_t smem, cudaStream_t st) {
    switch (N) {
        case 32: return launch_rowspec_t<32>(a, hmap, amap_re, amap_im, cgroups, smem, st);
        case 64: return launch_rowspec_t<64>(a, hmap, amap_re, amap_im, cgroups, smem, st);
        case 128: return launch_rowspec_t<128>(a, hmap, amap_re, amap_im, cgroups, smem, st);
        case 256: return launch_rowspec_t<256>(a, hmap, amap_re, amap_im, cgroups, smem, st);
        case 512: return launch_rowspec_t<512>(a, hmap, amap_re, amap_im, cgroups, smem, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t encode_plane_map(CUtensorMap *map, void *plane, int Tpad, long long rows, int box_rows) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const cuuint64_t dims[2] = {(cuuint64_t)Tpad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Tpad * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, plane, dims, strides, box,
                                                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Store map of the voltage planes for the row plane kernel: rows of Tpad halves, box 32 samples x
// 32 rows, 64-byte swizzle.
cudaError_t encode_plane_store_map(CUtensorMap *map, void *plane, int Tpad, long long rows) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const cuuint64_t dims[2] = {(cuuint64_t)Tpad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Tpad * 2};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, plane, dims, strides, box,
                                                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                                    CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_field_map(CUtensorMap *map, void *H, int N, int P, int Cb, int nt) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const cuuint64_t row = (cuuint64_t)N * 4, slab = (cuuint64_t)P * N * row;
    const cuuint64_t dims[4] = {(cuuint64_t)N, (cuuint64_t)P * N, (cuuint64_t)Cb, (cuuint64_t)nt};
    const cuuint64_t strides[3] = {row, slab, slab * (cuuint64_t)Cb};
    const cuuint32_t box[4] = {32, 1, 1, 32};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, H, dims, strides, box, estr,
                                                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                                    CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace moff
