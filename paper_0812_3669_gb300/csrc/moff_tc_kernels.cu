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
//   k_volt_prep    decode, weight, scale and transpose the voltages to FP16 planes [c][voltage][t]
//   k_rowspec_tc   per (pol, row, kx tile): B = row spectra resident in shared memory,
//                  A = 128 samples of the row's segment voltages (cp.async, MN-major),
//                  D = TMEM (double buffered), epilogue writes the row-transformed field in
//                  FP16 under an exact power-of-two scale (undone by the column kernel).
#include <cuda_fp16.h>

#include "moff_fft.cuh"
#include "moff_internal.h"
#include "moff_tc.cuh"

namespace moff {
namespace {

__device__ __forceinline__ float2 decode4_tc(uint32_t b) {
    const int hi = (int)((b >> 4) & 15u), lo = (int)(b & 15u);
    return make_float2((float)(hi - ((hi & 8) << 1)), (float)(lo - ((lo & 8) << 1)));
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
// Yre/Yim [nc][AP][Tpad] (t contiguous), zero for t >= nt.  Tile 32 t x 64 voltages:
// each thread loads four voltages of one sample (4 bytes) and stores two samples of
// one voltage (half2) per plane.
__global__ void __launch_bounds__(256) k_volt_prep(const uint8_t *__restrict__ volt, long long tstride, int t0, int nt,
                                                   int c0, int AP, const float2 *__restrict__ gains,
                                                   const float *__restrict__ sy, int Tpad, __half *__restrict__ yre,
                                                   __half *__restrict__ yim) {
    __shared__ float2 tile[32][65];
    const int cl = blockIdx.z, c = c0 + cl;
    const int v0 = blockIdx.x * 64, tb = blockIdx.y * 32;
    const float s = sy[c];
    const bool vec = (AP & 3) == 0 && (tstride & 3) == 0 && ((uintptr_t)volt & 3) == 0;
    for (int i = threadIdx.x; i < 32 * 16; i += 256) {
        const int tt = i / 16, v4 = (i % 16) * 4;
        const int t = tb + tt;
        uint32_t b4 = 0;
        if (t < nt) {
            const uint8_t *src = volt + (long long)(t0 + t) * tstride + (long long)c * AP + v0 + v4;
            if (vec && v0 + v4 + 3 < AP) {
                b4 = *reinterpret_cast<const uint32_t *>(src);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (v0 + v4 + u < AP) b4 |= (uint32_t)src[u] << (8 * u);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int vi = v0 + v4 + u;
            float2 y = make_float2(0.f, 0.f);
            if (t < nt && vi < AP) {
                y = cmul(gains[(long long)c * AP + vi], decode4_tc((b4 >> (8 * u)) & 0xffu));
                y.x *= s;
                y.y *= s;
            }
            tile[tt][v4 + u] = y;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * 16; i += 256) {
        const int v = i / 16, tt = (i % 16) * 2;
        const int t = tb + tt, vi = v0 + v;
        if (vi < AP && t < Tpad) {
            const long long o = ((long long)cl * AP + vi) * Tpad + t;   // t even, Tpad even: 4-byte aligned
            *reinterpret_cast<__half2 *>(yre + o) = __floats2half2_rn(tile[tt][v].x, tile[tt + 1][v].x);
            *reinterpret_cast<__half2 *>(yim + o) = __floats2half2_rn(tile[tt][v].y, tile[tt + 1][v].y);
        }
    }
}


template <int N>
struct TcShape {
    static constexpr int KX = N < 128 ? N : 128;     // kx per tile
    static constexpr int NT = 2 * KX;                // MMA N: real parts then imaginary parts
    static constexpr int NTILES = N / KX;
    static constexpr int TCOLS = 2 * NT <= 32 ? 32 : 2 * NT;   // two TMEM accumulators
};

__device__ __forceinline__ void cp_async16_tc(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_u32(smem_dst)), "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_tc() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_tc() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait_tc() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory"); }

// Warp roles: warps 0-3 drain the TMEM accumulators (one lane quarter each),
// warps 4-15 stage A in K-chunks of 64 with cp.async, warp 16 issues the MMAs
// (one lane).  A: 3-stage ring of [128 samples x 64] MN-major chunks; B:
// resident; accumulators: two in TMEM; epilogue: each warp converts its 32
// samples x 32 kx to FP16 into a 128-byte-swizzled box in shared memory and
// one lane hands it to the TMA unit (bulk tensor store), two boxes in flight
// per warp.  Per-thread global stores from four warps could not keep enough
// writes in flight; the bulk stores can.
constexpr int kEpiWarps = 4, kProdWarps = 12;   // 12 producer warps keep more A gathers in flight
constexpr int kTcRoleThreads = (kEpiWarps + kProdWarps + 1) * 32;
constexpr int kAStages = 3, kKChunk = 64;
constexpr int kAChunkBytes = 128 * kKChunk * 2;
constexpr int kBoxBytes = 32 * 128;                 // 32 samples x 32 kx x half2
constexpr int kEpiBufs = 2;                         // boxes per warp
constexpr long long kWaitCycles = 4000000000LL;     // ~2 s at the SM clock

template <int N>
__global__ void __launch_bounds__(kTcRoleThreads, 1)
    k_rowspec_tc(const RowSpecArgs a, const __grid_constant__ CUtensorMap hmap) {
    using S = TcShape<N>;
    constexpr int KX = S::KX, NT = S::NT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int item = blockIdx.x;                      // (p * N + ry) * NTILES + tile
    const int tile = item % S::NTILES;
    const int pr = item / S::NTILES;
    const int p = pr / N, ry = pr % N;
    const int kp = a.kp[pr];
    const int nseg = (int)(a.seg_off[pr + 1] - a.seg_off[pr]);

    const int cper = (a.nc + gridDim.y - 1) / gridDim.y;
    const int cb = blockIdx.y * cper, ce = min(a.nc, cb + cper);
    if (cb >= ce) return;
    const int ntb = (a.nt + 127) / 128;
    const int nitems = (ce - cb) * ntb;
    const long long hrow = (long long)p * N * N + (long long)ry * N + tile * KX;   // within one (t, c) slab
    const long long hslab = (long long)a.P * N * N;

    if (kp == 0) {   // no kernel row lands here: the row-transformed field is zero
        for (int it = 0; it < nitems; ++it) {
            const int cl = cb + it / ntb, t0b = (it % ntb) * 128;
            for (int i = tid; i < 128 * KX; i += blockDim.x) {
                const int tt = i / KX, kx = i % KX, t = t0b + tt;
                if (t < a.nt) a.H[((long long)t * a.slab_t + (long long)cl * a.slab_c) * hslab + hrow + kx] =
                    __floats2half2_rn(0.f, 0.f);
            }
        }
        return;
    }
    const int nchunk = (kp + kKChunk - 1) / kKChunk;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzled TMA boxes need 1024-byte alignment: round the base up (the size includes the slack)
    unsigned char *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *sB = smem;                                  // NT x kp, K-major (resident)
    unsigned char *sA = sB + (size_t)NT * a.kp_max * 2;        // kAStages x [128 x 64], MN-major
    unsigned char *sE = sA + (size_t)kAStages * kAChunkBytes;  // [4 warps][kEpiBufs] boxes, 1024-aligned
    uint64_t *bars = reinterpret_cast<uint64_t *>(sE + kEpiWarps * kEpiBufs * kBoxBytes);
    uint64_t *a_full = bars, *a_empty = bars + kAStages, *d_full = bars + 2 * kAStages,
             *d_empty = bars + 2 * kAStages + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * kAStages + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    int *s_seg = reinterpret_cast<int *>(tslot + 2);

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.bimg + a.bimg_off[item]);
        uint4 *dst = reinterpret_cast<uint4 *>(sB);
        const int n16 = NT * kp * 2 / 16;
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
        for (int j = tid; j < nseg; j += blockDim.x) s_seg[j] = a.seg_y[a.seg_off[pr] + j];
    }
    if (tid == 0) {
        for (int b = 0; b < kAStages; ++b) {
            tc::mbar_init(&a_full[b], kProdWarps * 32);
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

    if (warp >= kEpiWarps && warp < kEpiWarps + kProdWarps) {
        // ---------------- producers: chunk g (global counter) into stage g % kAStages.
        // Up to kAStages chunks are in flight: after issuing chunk g the
        // producers wait only for chunk g - (kAStages - 1) and release it.
        const int ptid = tid - kEpiWarps * 32;
        int g = 0;
        for (int i = 0; i < nitems && !*abort_flag; ++i) {
            const int cl = cb + i / ntb, t0b = (i % ntb) * 128;
            const __half *re = a.yre + (long long)cl * a.AP * a.Tpad + t0b;
            const __half *im = a.yim + (long long)cl * a.AP * a.Tpad + t0b;
            for (int ch = 0; ch < nchunk; ++ch, ++g) {
                const int st = g % kAStages;
                if (!tc::mbar_wait_abortable(&a_empty[st], (uint32_t)(((g / kAStages) & 1) ^ 1), kWaitCycles,
                                             abort_flag))
                    break;
                unsigned char *sa = sA + st * kAChunkBytes;
                for (int q = ptid; q < kKChunk * 16; q += kProdWarps * 32) {
                    // a warp covers 8 consecutive k x 4 sample groups: four 128-byte bank
                    // sweeps in shared memory, 64 contiguous bytes per segment in global
                    const int kk = ((q >> 7) << 3) | (q & 7), m8 = (q >> 3) & 15;
                    const int k = ch * kKChunk + kk, j = k >> 1;
                    unsigned char *d = sa + m8 * 128 + (kk >> 3) * 2048 + (kk & 7) * 16;
                    if (k < kp && j < nseg) {
                        cp_async16_tc(d, ((k & 1) ? im : re) + (long long)s_seg[j] * a.Tpad + m8 * 8);
                    } else {
                        *reinterpret_cast<uint4 *>(d) = make_uint4(0u, 0u, 0u, 0u);
                    }
                }
                cp_async_commit_tc();
                if (g >= kAStages - 1) {
                    cp_async_wait_tc<kAStages - 1>();          // chunk g - (kAStages-1) has landed
                    tc::fence_async_smem();
                    tc::mbar_arrive(&a_full[(g - (kAStages - 1)) % kAStages]);
                }
            }
        }
        // release the chunks still in flight, oldest first
        const int g0 = g - (kAStages - 1) > 0 ? g - (kAStages - 1) : 0;
        cp_async_wait_all_tc();
        tc::fence_async_smem();
        for (int gg = g0; gg < g; ++gg) tc::mbar_arrive(&a_full[gg % kAStages]);
    } else if (warp == kEpiWarps + kProdWarps) {
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
                    const int kend = min(kKChunk, kp - ch * kKChunk);
                    for (int ks = 0; ks < kend / 16; ++ks) {
                        const uint64_t ad = tc::smem_desc(sa + ks * 2 * 2048, 2048, 128);   // MN-major: LBO = K stride
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
        // ---------------- epilogue warps 0-3: TMEM lanes 32w..32w+31 = samples
        unsigned char *sw = sE + warp * kEpiBufs * kBoxBytes;
        int nbox = 0;
        for (int i = 0; i < nitems; ++i) {
            const int b = i & 1;
            if (!tc::mbar_wait_abortable(&d_full[b], (uint32_t)((i >> 1) & 1), kWaitCycles, abort_flag)) break;
            tc::fence_after_sync();
            const int cl = cb + i / ntb, t0w = (i % ntb) * 128 + warp * 32;
            const float inv = a.row_sh[pr];   // exact power of two: FP16 range for every row
            const uint32_t dcol = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * NT);
#pragma unroll 1
            for (int k0 = 0; k0 < KX; k0 += 32, ++nbox) {
                float vr[32], vi[32];
                tc::tmem_ld32(dcol + (uint32_t)k0, vr);
                tc::tmem_ld32(dcol + (uint32_t)(KX + k0), vi);
                unsigned char *box = sw + (nbox % kEpiBufs) * kBoxBytes;
                if (nbox >= kEpiBufs) {                  // the store that last read this box is done with it
                    if (lane == 0) tc::bulk_wait_read<kEpiBufs - 1>();
                    __syncwarp();
                }
                // lane = sample t0w + lane: its 32 kx as eight 16-byte chunks of one 128-byte row,
                // chunk q stored at q ^ (row % 8) (the tensor map's 128-byte swizzle)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    __half2 h[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) h[u] = __floats2half2_rn(vr[4 * q + u] * inv, vi[4 * q + u] * inv);
                    *reinterpret_cast<uint4 *>(box + lane * 128 + ((q ^ (lane & 7)) << 4)) =
                        *reinterpret_cast<const uint4 *>(h);
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    // a box wholly past the block's samples is not issued (the map clips partial ones)
                    if (t0w < a.nt) tc::tma_store_4d(&hmap, tc::smem_u32(box), tile * KX + k0, p * N + ry, cl, t0w);
                    tc::bulk_commit();
                }
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&d_empty[b]);
        }
        if (lane == 0) tc::bulk_wait_all();
    }
    if (*abort_flag && tid == 0) atomicExch(a.err, tc::kErrWaitTimeout);
    cp_async_wait_all_tc();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, S::TCOLS);
}

}  // namespace

size_t rowspec_smem_bytes(int N, int kp_max, int max_seg) {
    const int KX = N < 128 ? N : 128, NT = 2 * KX;
    size_t b = 1024 + (size_t)NT * kp_max * 2 + (size_t)kAStages * kAChunkBytes +
               (size_t)kEpiWarps * kEpiBufs * kBoxBytes + (size_t)(2 * kAStages + 4) * 8 + 8 + (size_t)max_seg * 4;
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
                             const float2 *gains, const float *sy, int Tpad, __half *yre, __half *yim,
                             cudaStream_t st) {
    dim3 grid((AP + 63) / 64, (Tpad + 31) / 32, nc);
    k_volt_prep<<<grid, 256, 0, st>>>(volt, tstride, t0, nt, c0, AP, gains, sy, Tpad, yre, yim);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_rowspec_t(const RowSpecArgs &a, const CUtensorMap &hmap, int cgroups, size_t smem,
                             cudaStream_t st) {
    auto k = k_rowspec_tc<N>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(a.P * N * TcShape<N>::NTILES, cgroups), kTcRoleThreads, smem, st>>>(a, hmap);
    return cudaGetLastError();
}

cudaError_t launch_rowspec(int N, const RowSpecArgs &a, const CUtensorMap &hmap, int cgroups, size_t smem,
                           cudaStream_t st) {
    switch (N) {
        case 32: return launch_rowspec_t<32>(a, hmap, cgroups, smem, st);
        case 64: return launch_rowspec_t<64>(a, hmap, cgroups, smem, st);
        case 128: return launch_rowspec_t<128>(a, hmap, cgroups, smem, st);
        case 256: return launch_rowspec_t<256>(a, hmap, cgroups, smem, st);
        case 512: return launch_rowspec_t<512>(a, hmap, cgroups, smem, st);
    }
    return cudaErrorInvalidValue;
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
