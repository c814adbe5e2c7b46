// moff_image_kernels.cuh -- the per-channel imaging hot path of the MOFF
// correlator (Morales, arXiv 0812.3669, Sec. 4, Eq. m6), FP32.
//
//   k_grid_rows : step 1 (complex weight per antenna), step 2 (scatter through
//                 each antenna's kernel, written as a deterministic gather per
//                 grid cell) and the first axis of step 3 (row transforms).
//                 One CTA = one stripe of grid rows of one channel walking a
//                 chunk of samples TB at a time: each kernel entry is read
//                 once (coalesced, sliced-ELL order, from L2) per TB samples,
//                 and the TB x P x rows rows are transformed in place.
//   k_cols_acc  : second axis of step 3 (column transforms) fused with step 4
//                 (|E|^2 and the cross-pol products summed over the chunk in
//                 registers, then added to FP64 accumulators).
// The row-transformed field goes through global memory between the two.
#pragma once
#include <cuda_fp16.h>

#include "moff_dft.cuh"
#include "moff_fft.cuh"
#include "moff_internal.h"

namespace moff {

// 4-bit two's-complement nibbles: real part high, imaginary part low.
__device__ __forceinline__ float2 decode4(uint32_t b) {
    const int hi = (int)((b >> 4) & 15u), lo = (int)(b & 15u);
    return make_float2((float)(hi - ((hi & 8) << 1)), (float)(lo - ((lo & 8) << 1)));
}

// One Stockham pass over the F rows held in shared memory (row f at
// src + f*LDR, padded index) into dst, or -- LAST -- into the global row
// returned by `rowptr(f)` (nullptr: row not stored).  When the warps can
// share the rows evenly, warp w owns rows [w F/NW, (w+1) F/NW) in every pass,
// so a pass reads only what its own warp wrote and a warp barrier orders the
// passes; otherwise the slots are dealt out over the block and a block barrier
// ends each pass.  IP (in place, dst == src): each lane holds one slot, reads
// it, and writes it back after the warp has read all its rows.  No barrier
// after a LAST pass.
template <int N, int F, int R, int NS, bool LAST, bool IP, class RowPtr>
__device__ __forceinline__ void rows_pass(const float2 *src, float2 *dst, const float2 *tw, RowPtr rowptr) {
    constexpr int LDR = PaddedLen<N>::value;
    constexpr int NSL = N / R;
    constexpr int NW = kBlock / 32;
    constexpr bool WL = F % NW == 0;                 // warp-local rows
    constexpr int SLOTS = WL ? (F / NW) * NSL : F * NSL;
    constexpr int STEP = WL ? 32 : kBlock;
    const int base = WL ? (int)(threadIdx.x >> 5) * (F / NW) : 0;
    if constexpr (IP && !LAST) {
        static_assert(WL && SLOTS == 32, "in-place pass: one slot per lane");
        const int sl = (int)(threadIdx.x & 31);
        const int fl = sl / NSL, j = sl - fl * NSL, f = base + fl;
        float2 v[R];
        const float2 *in = src + f * LDR;
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[pad_load<NSL>(j, r)];
        twiddle<R, NS, 1>(v, j, tw);
        dft<R, 1>(v);
        __syncwarp();                                // the warp's rows are read
        float2 *out = dst + f * LDR;
#pragma unroll
        for (int r = 0; r < R; ++r) out[pad_store<R, NS>(j, r)] = v[r];
        __syncwarp();
    } else {
        for (int sl = WL ? (int)(threadIdx.x & 31) : (int)threadIdx.x; sl < SLOTS; sl += STEP) {
            const int fl = sl / NSL, j = sl - fl * NSL, f = base + fl;
            const float2 *in = src + f * LDR;
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = in[pad_load<NSL>(j, r)];
            twiddle<R, NS, 1>(v, j, tw);
            dft<R, 1>(v);
            if constexpr (LAST) {
                float2 *o = rowptr(f);
                if (o) {
#pragma unroll
                    for (int r = 0; r < R; ++r) o[j + r * NSL] = v[r];
                }
            } else {
                float2 *out = dst + f * LDR;
#pragma unroll
                for (int r = 0; r < R; ++r) out[pad_store<R, NS>(j, r)] = v[r];
            }
        }
        if constexpr (!LAST) {
            if constexpr (WL) __syncwarp();
            else __syncthreads();
        }
    }
}

// Stripe height of the gridding kernel: TB samples x P pols x ROWS rows = F rows per pass.
template <int N, int P, int TB, bool WIDE = false>
struct GridShape {
    // rows per pass: grid_fft_rows(N), or twice that for the wide variant
    static constexpr int FR = (N >= 256 ? 8 : (N == 128 ? 16 : 32)) * (WIDE ? 2 : 1);
    static constexpr int ROWS_ = FR / (TB * P);
    static constexpr int ROWS = ROWS_ < 1 ? 1 : (ROWS_ > N ? N : ROWS_);
    static constexpr int PR = P * ROWS;
    static constexpr int F = TB * PR;
    // one row buffer (passes in place)
    static constexpr bool IN_PLACE = grid_rows_in_place(N, F);
};

// CTAs per SM the register allocation is sized for when the row passes run in
// place (one row buffer, so more CTAs fit an SM's shared memory): four (64
// registers) up to 4 samples per pass, three (80) for 2 x 2 block lanes at 4
// samples on wide stripes, two (128) for 2 x 2 blocks at 4 samples otherwise and at
// 8 samples.
template <int N, int P, int TB, int CPL, bool WIDE>
constexpr int grid_min_blocks() {
    if (TB >= 8) return 2;
    if (CPL == 4 && TB == 4) return WIDE ? 3 : 2;
    return 4;
}

static_assert(fft_radix(32, 0) == FftPlan<32>::R0 && fft_radix(32, 1) == FftPlan<32>::R1 &&
              fft_radix(64, 0) == FftPlan<64>::R0 && fft_radix(64, 1) == FftPlan<64>::R1 &&
              fft_radix(128, 0) == FftPlan<128>::R0 && fft_radix(128, 1) == FftPlan<128>::R1 &&
              fft_radix(256, 0) == FftPlan<256>::R0 && fft_radix(256, 1) == FftPlan<256>::R1 &&
              fft_radix(512, 0) == FftPlan<512>::R0 && fft_radix(512, 1) == FftPlan<512>::R1 &&
              fft_radix(512, 2) == FftPlan<512>::R2 && fft_radix(1024, 0) == FftPlan<1024>::R0 &&
              fft_radix(1024, 1) == FftPlan<1024>::R1 && fft_radix(2048, 1) == FftPlan<2048>::R1,
              "host radix table matches the FFT plan");

// CPL = grid cells per lane: 1, 2 (cells (f, e), (f, e + 1) of one row) or 4 (the 2 x 2
// block (f, e), (f, e + 1), (f + 1, e), (f + 1, e + 1), f even); each entry carries CPL taps.
// DFT: the row transform runs as factored DFT contractions on the tensor cores
// (moff_dft.cuh) and the field leaves as FP16 rows [re N][im N] (a.h16).
// (s, cl): this CTA's stripe and channel of the launch; n_str: stripes per set (the grid's x extent).
template <int N, int P, int TB, bool STAGED, bool GRID_ONLY, int CPL, bool WIDE, bool DFT = false>
__device__ __forceinline__ void grid_rows(const GridArgs &a, const int s, const int cl, const int n_str) {
    constexpr bool PAIRS = CPL >= 2;
    using FP = FftPlan<N>;
    using TW = FftTw<N>;
    using GS = GridShape<N, P, TB, WIDE>;
    constexpr int LDR = PaddedLen<N>::value;
    constexpr int YS = VoltStride<TB>::value;
    constexpr int ROWS = GS::ROWS, PR = GS::PR, F = GS::F;
    constexpr int YPT = 2;                // voltages per thread whose bytes are prefetched

    const int c = a.c0 + cl;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nsl = a.n_slices;
    const int grp = a.chan_group ? a.chan_group[c] : 0;      // this channel's set of positions and kernels
    const long long gs = (long long)grp * n_str + s;         // stripe s of that set
    const int *sao = a.st_ant_off + grp + gs;                // set g's offsets start at g (n_stripes + 1)
    const int ant0 = sao[0];
    const int nloc = sao[1] - ant0;
    const int nyi = nloc * P;
    const long long *soff = a.slice_off + grp + gs * nsl;
    const uint16_t *lcell = a.lane_cell + gs * nsl * 32;
    const long long e0 = soff[0];

    if (nloc == 0) {   // no kernel reaches these rows: their field (and its transform) is zero
        if (!GRID_ONLY && a.row_nz) {   // rows the column kernel will not read are not written
            bool any = false;
            for (int rl = 0; rl < ROWS; ++rl) {
                const int ry = s * ROWS + rl;
                any |= ((a.row_nz[ry >> 5] >> (ry & 31)) & 1u) != 0;
            }
            if (!any) return;
        }
        if constexpr (DFT) {   // FP16 rows [re N][im N]: 8 halves per 16-byte store
            constexpr int PER_T16 = P * ROWS * 2 * N / 8;
            for (int i = tid; i < a.nt * PER_T16; i += kBlock) {
                const int t = i / PER_T16, e = 8 * (i - t * PER_T16);
                const int p = e / (ROWS * 2 * N), rem = e - p * (ROWS * 2 * N), rl = rem / (2 * N), x = rem - rl * 2 * N;
                __half *o = a.h16 + (((long long)t * a.slab_t + (long long)cl * a.slab_c) * P * N + (long long)p * N +
                                     (long long)s * ROWS + rl) * 2 * N + x;
                *reinterpret_cast<uint4 *>(o) = make_uint4(0u, 0u, 0u, 0u);
            }
            return;
        }
        constexpr int PER_T = P * ROWS * N / 2;     // 16-byte stores per sample
        for (int i = tid; i < a.nt * PER_T; i += kBlock) {
            const int t = i / PER_T, e = 2 * (i - t * PER_T);
            const int p = e / (ROWS * N), rem = e - p * (ROWS * N), rl = rem / N, x = rem - rl * N;
            float2 *o = a.out + (((long long)t * a.slab_t + (long long)cl * a.slab_c) * P * N + (long long)p * N +
                                 (long long)s * ROWS + rl) * N + x;
            *reinterpret_cast<float4 *>(o) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }

    // Carve (matches grid_smem_bytes; DFT: the transform region replaces the pass
    // twiddles and the second row buffer).
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool IP = GS::IN_PLACE;                 // row passes in place (FFT variant)
    constexpr bool ONEBUF = GS::IN_PLACE || DFT;      // one row buffer
    constexpr size_t DREG = DFT ? (dft_row_region_bytes(N, F) + 15) / 16 * 16 : 0;
    unsigned char *s_dft = smem;
    float2 *s_tw = reinterpret_cast<float2 *>(smem + DREG);
    float2 *s_buf = s_tw + (DFT ? 0 : TW::TOTAL);      // gridded rows
    float2 *s_alt = ONEBUF ? s_buf : s_buf + F * LDR;  // second buffer of the row passes (none in place)
    float2 *s_y = s_alt + ((F * LDR + 1) & ~1);        // [nloc*P][YS]: TB samples, padded row (16-byte aligned)
    float2 *s_g = s_y + YS * a.max_nloc * P;
    // staged kernel values (CPL per entry, read as 16-byte vectors when CPL >= 2: 16-byte aligned)
    float2 *s_tap = reinterpret_cast<float2 *>((reinterpret_cast<uintptr_t>(s_g + a.max_nloc * P) + 15) & ~uintptr_t(15));
    constexpr int TPE = CPL;                           // taps per entry
    int *s_ant = reinterpret_cast<int *>(s_tap + (STAGED ? TPE * a.max_entries : 0));
    uint16_t *s_cy = reinterpret_cast<uint16_t *>(s_ant + a.max_nloc);   // staged voltage indices

    if constexpr (!DFT) {
        for (int i = tid; i < TW::TOTAL; i += kBlock) s_tw[i] = a.twp[i];
    }
    // DFT: table image, the MMA mbarrier and this CTA's TMEM columns
    uint64_t *s_mbar = reinterpret_cast<uint64_t *>(s_dft + (DFT ? dft_row_region_bytes(N, F) - 16 : 0));
    uint32_t *s_tslot = reinterpret_cast<uint32_t *>(s_mbar + 1);
    constexpr int TCOLS = DFT ? dft_row_tmem_cols(N, F) : 32;
    if constexpr (DFT) {
        dftc::load_table(s_dft + (size_t)F * (N / 16) * 64, a.dft_tab, DftShape<N>::TAB_BYTES);
        if (tid == 0) tc::mbar_init(s_mbar, 1);
        if (warp == 0) {
            tc::tmem_alloc(s_tslot, TCOLS);
            tc::tmem_relinquish();
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
    }
    for (int i = tid; i < nloc; i += kBlock) s_ant[i] = a.st_ant[ant0 + i];
    for (int i = tid; i < nyi; i += kBlock) {
        const int la = i / P, q = i - la * P;
        s_g[i] = a.gains[((long long)c * a.A + a.st_ant[ant0 + la]) * P + q];
    }
    if constexpr (STAGED) {
        const int ne = (int)(soff[nsl] - e0);
        for (int i = tid; i < TPE * ne; i += kBlock) s_tap[i] = __ldg(a.con_tap + TPE * e0 + i);
        for (int i = tid; i < ne; i += kBlock) s_cy[i] = __ldg(a.con_y + e0 + i);
    }
    __syncthreads();
    uint32_t tbase = 0, mphase = 0;
    float sG = 1.f;
    bool dft_ok = true;
    if constexpr (DFT) {
        tc::fence_after_sync();
        tbase = *s_tslot;
        sG = a.sy[c] * a.s_t;
    }

    // Voltage bytes: thread owns local voltages yi = tid + m*kBlock and their TB samples.
    const bool pre = nyi <= YPT * kBlock;
    const uint8_t *vchan = a.volt + (long long)c * a.A * P;
    uint32_t vb[YPT][TB];
    auto fetch = [&](int tbn) {
        const int nbn = min(TB, a.nt - tbn);
#pragma unroll
        for (int m = 0; m < YPT; ++m) {
            const int yi = tid + m * kBlock;
            const int la = yi / P, q = yi - la * P;
            const uint8_t *src = vchan + (long long)(a.t0 + tbn) * a.volt_tstride +
                                 (yi < nyi ? (long long)s_ant[la] * P + q : 0);
#pragma unroll
            for (int t = 0; t < TB; ++t) vb[m][t] = (yi < nyi && t < nbn) ? src[t * a.volt_tstride] : 0u;
        }
    };
    if (pre) fetch(0);

    const int ry0 = s * ROWS;
    for (int tb0 = 0; tb0 < a.nt; tb0 += TB) {
        const int nb = min(TB, a.nt - tb0);
        // Step 1: decode and weight the voltages of the antennas touching this stripe.
        if (pre) {
#pragma unroll
            for (int m = 0; m < YPT; ++m) {
                const int yi = tid + m * kBlock;
                if (yi < nyi) {
                    const float2 g = s_g[yi];
                    float2 *yrow = s_y + yi * YS;
#pragma unroll
                    for (int t = 0; t < TB; ++t) yrow[t] = t < nb ? cmul(g, decode4(vb[m][t])) : make_float2(0.f, 0.f);
                }
            }
            if (tb0 + TB < a.nt) fetch(tb0 + TB);     // in flight during this pass
        } else {
            for (int yi = tid; yi < nyi; yi += kBlock) {
                const int la = yi / P, q = yi - la * P;
                const float2 g = s_g[yi];
                const uint8_t *src = vchan + (long long)(a.t0 + tb0) * a.volt_tstride + (long long)s_ant[la] * P + q;
                float2 *yrow = s_y + yi * YS;
                for (int t = 0; t < TB; ++t)
                    yrow[t] = t < nb ? cmul(g, decode4(src[t * a.volt_tstride])) : make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
        // Step 2: every cell sums its kernel contributions (fixed order), for TB
        // samples.  Entries are fetched U at a time so their latencies overlap.
        // With CPL = 2 a lane owns cells (e, e + 1) of one row, with CPL = 4 a 2 x 2 block;
        // each entry carries every cell's tap, so one read of a voltage row feeds CPL cells.
        // Slices come longest first; warps take them in snake order (w, 2W-1-w, 2W+w, ...)
        // so that each warp's total stays close to the mean.
        constexpr int NW = kBlock / 32;
        for (int r = 0; r * NW < nsl; ++r) {
            const int k = r * NW + ((r & 1) ? NW - 1 - warp : warp);
            if (k >= nsl) continue;
            const long long b0 = soff[k];
            const int len = (int)((soff[k + 1] - b0) >> 5);
            const int cell = lcell[k * 32 + lane];
            const float2 *tp = (STAGED ? s_tap + TPE * (b0 - e0) : a.con_tap + TPE * b0) + TPE * lane;
            const uint16_t *yp = (STAGED ? s_cy + (b0 - e0) : a.con_y + b0) + lane;
            float2 acc[TPE][TB];
#pragma unroll
            for (int c2 = 0; c2 < TPE; ++c2)
#pragma unroll
                for (int t = 0; t < TB; ++t) acc[c2][t] = make_float2(0.f, 0.f);
            constexpr int U = PAIRS ? 2 : 4;
            // Entries i0 .. i0 + U - 1 (zero past the slice): taps and voltage indices.
            auto load_ent = [&](int i0, float2 (&tv)[U][TPE], int (&yv)[U]) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool ok = i0 + u < len;
                    const float2 *tq = tp + TPE * 32 * (i0 + u);
                    if constexpr (CPL == 4) {
                        float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f), r4 = q4;
                        if (ok) {
                            q4 = __ldg(reinterpret_cast<const float4 *>(tq));
                            r4 = __ldg(reinterpret_cast<const float4 *>(tq) + 1);
                        }
                        tv[u][0] = make_float2(q4.x, q4.y);
                        tv[u][1] = make_float2(q4.z, q4.w);
                        tv[u][2] = make_float2(r4.x, r4.y);
                        tv[u][3] = make_float2(r4.z, r4.w);
                    } else if constexpr (PAIRS) {
                        float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (ok) q4 = STAGED ? *reinterpret_cast<const float4 *>(tq) : __ldg(reinterpret_cast<const float4 *>(tq));
                        tv[u][0] = make_float2(q4.x, q4.y);
                        tv[u][TPE - 1] = make_float2(q4.z, q4.w);
                    } else {
                        tv[u][0] = ok ? (STAGED ? tq[0] : __ldg(tq)) : make_float2(0.f, 0.f);
                    }
                    yv[u] = ok ? (int)(STAGED ? yp[32 * (i0 + u)] : __ldg(yp + 32 * (i0 + u))) : 0;
                }
            };
            // The next group's entries are loaded while this group is summed, so the
            // L2 latency of the entries overlaps the arithmetic.
            float2 tv[U][TPE];
            int yv[U];
            load_ent(0, tv, yv);
            for (int i0 = 0; i0 < len; i0 += U) {
                float2 tn[U][TPE];
                int yn[U];
                load_ent(i0 + U, tn, yn);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float2 *yy = s_y + yv[u] * YS;
                    if constexpr (TB >= 2) {
#pragma unroll
                        for (int t = 0; t < TB; t += 2) {
                            const float4 q = *reinterpret_cast<const float4 *>(yy + t);
#pragma unroll
                            for (int c2 = 0; c2 < TPE; ++c2) {
                                const float2 w = tv[u][c2];
                                acc[c2][t].x = fmaf(w.x, q.x, fmaf(-w.y, q.y, acc[c2][t].x));
                                acc[c2][t].y = fmaf(w.x, q.y, fmaf(w.y, q.x, acc[c2][t].y));
                                acc[c2][t + 1].x = fmaf(w.x, q.z, fmaf(-w.y, q.w, acc[c2][t + 1].x));
                                acc[c2][t + 1].y = fmaf(w.x, q.w, fmaf(w.y, q.z, acc[c2][t + 1].y));
                            }
                        }
                    } else {
                        const float2 y = yy[0];
#pragma unroll
                        for (int c2 = 0; c2 < TPE; ++c2) {
                            const float2 w = tv[u][c2];
                            acc[c2][0].x = fmaf(w.x, y.x, fmaf(-w.y, y.y, acc[c2][0].x));
                            acc[c2][0].y = fmaf(w.x, y.y, fmaf(w.y, y.x, acc[c2][0].y));
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    yv[u] = yn[u];
#pragma unroll
                    for (int c2 = 0; c2 < TPE; ++c2) tv[u][c2] = tn[u][c2];
                }
            }
            const int f = cell / N, e = cell - f * N;
#pragma unroll
            for (int c2 = 0; c2 < TPE; ++c2) {
                float2 *dst = s_buf + (f + (c2 >> 1)) * LDR + pad16(e + (c2 & 1));
#pragma unroll
                for (int t = 0; t < TB; ++t) dst[t * PR * LDR] = acc[c2][t];
            }
        }
        __syncthreads();

        // Global row of transform row fa = t*PR + p*ROWS + rl (nullptr past the chunk).
        float2 *outb = a.out;
        auto rowptr = [&](int fa) -> float2 * {
            const int t = fa / PR, f = fa - t * PR;
            if (t >= nb) return nullptr;
            const int p = f / ROWS, rl = f - p * ROWS;
            return outb + (((long long)(tb0 + t) * a.slab_t + (long long)cl * a.slab_c) * P * N + (long long)p * N +
                           ry0 + rl) * N;
        };
        if constexpr (DFT) {
            // Global FP16 row [re N][im N] of transform row fa (nullptr past the chunk).
            auto rowout = [&](int fa) -> __half * {
                const int t = fa / PR, f = fa - t * PR;
                if (t >= nb) return nullptr;
                const int p = f / ROWS, rl = f - p * ROWS;
                return a.h16 + (((long long)(tb0 + t) * a.slab_t + (long long)cl * a.slab_c) * P * N +
                                (long long)p * N + ry0 + rl) * 2 * N;
            };
            dft_ok = dftc::rows_dft<N, F, LDR, kBlock>(s_buf, sG, s_dft, s_mbar, tbase, mphase,
                                                      reinterpret_cast<__half *>(s_buf), rowout);
            if (!dft_ok) break;   // uniform: the wait's result is agreed by a block barrier
            continue;
        }
        if constexpr (GRID_ONLY) {
            for (int i = tid; i < F * N; i += kBlock) {
                const int fa = i / N, e = i - fa * N;
                float2 *o = rowptr(fa);
                if (o) o[e] = s_buf[fa * LDR + pad16(e)];
            }
            __syncthreads();
            continue;
        }
        // Step 3, first axis: N-point transform of every row (ping-pong buffers, or one in place).
        rows_pass<N, F, FP::R0, 1, false, IP>(s_buf, s_alt, s_tw, rowptr);
        if constexpr (FP::NP == 3) {
            rows_pass<N, F, FP::R1, FP::R0, false, IP>(s_alt, s_buf, s_tw + TW::OFF1, rowptr);
            rows_pass<N, F, FP::R2, FP::R0 * FP::R1, true, IP>(s_buf, nullptr, s_tw + TW::OFF2, rowptr);
        } else {
            rows_pass<N, F, FP::R1, FP::R0, true, IP>(s_alt, nullptr, s_tw + TW::OFF1, rowptr);
        }
        // (the next iteration's first barrier orders these reads before any rewrite)
    }
    if constexpr (DFT) {
        if (!dft_ok && tid == 0) atomicExch(a.err, tc::kErrWaitTimeout);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (warp == 0) tc::tmem_dealloc(tbase, TCOLS);
    }
}

// Row transform out of place: the register count is the compiler's choice (an
// explicit minimum of one CTA per SM lets it take about twice as many).
template <int N, int P, int TB, bool STAGED, bool GRID_ONLY, int CPL, bool WIDE>
__global__ void __launch_bounds__(kBlock) k_grid_rows(const GridArgs a) {
    grid_rows<N, P, TB, STAGED, GRID_ONLY, CPL, WIDE>(a, blockIdx.x, blockIdx.y, gridDim.x);
}

// Gridding with the row transform on the tensor cores (FP16 field out).
template <int N, int P, int TB, int CPL>
__global__ void __launch_bounds__(kBlock) k_grid_rows_dft(const GridArgs a) {
    grid_rows<N, P, TB, false, false, CPL, false, true>(a, blockIdx.x, blockIdx.y, gridDim.x);
}

// Row transform in place: registers capped so that grid_min_blocks CTAs fit an SM.
template <int N, int P, int TB, bool STAGED, bool GRID_ONLY, int CPL, bool WIDE>
__global__ void __launch_bounds__(kBlock, grid_min_blocks<N, P, TB, CPL, WIDE>()) k_grid_rows_ip(const GridArgs a) {
    grid_rows<N, P, TB, STAGED, GRID_ONLY, CPL, WIDE>(a, blockIdx.x, blockIdx.y, gridDim.x);
}

template <int N>
struct ColShape {
    using FP = FftPlan<N>;
    static constexpr int RL = FP::NP == 3 ? FP::R2 : FP::R1;   // radix of the last pass
    static constexpr int W = kBlock * RL / N;                  // columns per CTA
    static constexpr int NS = N / RL;                          // slots per column in the last pass
};

// (sx, cl): this CTA's column strip and channel of the launch.
template <int N, int P, bool H16, bool TAPS>
__device__ __forceinline__ void cols_acc(const ColArgs &a, const int sx, const int cl) {
    using FP = FftPlan<N>;
    using TW = FftTw<N>;
    using CS = ColShape<N>;
    constexpr int W = CS::W;
    constexpr int RL = CS::RL;
    constexpr int NPROD = P == 1 ? 1 : 4;
    constexpr int TILE = P * N * W;                 // elements per sample: [P][N][W]
    constexpr int EB = H16 ? 4 : 8;                 // bytes per input element (half2 or float2)
    constexpr int CHUNKS = TILE * EB / 16;          // 16-byte pieces per tile
    constexpr int ROWCH = W * EB / 16;              // pieces per tile row

    const int kx0 = sx * W;
    const int c = a.c0 + cl;
    const int tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *s_tw = reinterpret_cast<float2 *>(smem);
    unsigned char *s_in = reinterpret_cast<unsigned char *>(s_tw + ((TW::TOTAL + 1) & ~1));  // 2 staging tiles
    float2 *s_a = reinterpret_cast<float2 *>(s_in + 2 * TILE * EB);   // pass outputs
    float2 *s_b = s_a + TILE;                      // second pass buffer (3-pass lengths only)

    for (int i = tid; i < TW::TOTAL; i += kBlock) s_tw[i] = a.twp[i];
    // FP16 field: one power-of-two scale for every row of the channel, so the transform
    // runs on the scaled values (exactly proportional) and the scale is undone on the
    // field taps and, squared, on the chunk's sums
    const float sc = H16 ? a.row_inv[0] * a.inv_sw / a.sy[c] : 1.f;

    // Rows no kernel reaches are zero: cleared once in both staging tiles and never read.
    // Piece q = tid + k kBlock of a tile is read only if bit k of `act` is set.
    static_assert(CHUNKS % kBlock == 0 && CHUNKS / kBlock <= 32, "staging pieces per thread");
    constexpr int ITER = CHUNKS / kBlock;
    uint32_t act = 0;
#pragma unroll
    for (int k = 0; k < ITER; ++k) {
        const int q = tid + k * kBlock, row = q / ROWCH, part = q - row * ROWCH, ry = row % N;
        if (!a.row_nz || ((a.row_nz[ry >> 5] >> (ry & 31)) & 1u)) {
            act |= 1u << k;
        } else {
            *reinterpret_cast<uint4 *>(s_in + (row * W) * EB + part * 16) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(s_in + TILE * EB + (row * W) * EB + part * 16) = make_uint4(0u, 0u, 0u, 0u);
        }
    }

    // Stage sample tt's [P][N][W] tile of the row-transformed field.
    auto stage = [&](int tt, unsigned char *dst) {
        const unsigned char *src = reinterpret_cast<const unsigned char *>(a.H) +
                                   (((long long)tt * a.slab_t + (long long)cl * a.slab_c) * P * N * N + kx0) * EB;
#pragma unroll
        for (int k = 0; k < ITER; ++k) {
            const int q = tid + k * kBlock, row = q / ROWCH, part = q - row * ROWCH;   // row = p*N + ry
            if ((act >> k) & 1u) cp_async16(dst + (row * W) * EB + part * 16, src + (long long)row * N * EB + part * 16);
        }
        cp_async_commit();
    };

    float acc[NPROD][RL];
#pragma unroll
    for (int q = 0; q < NPROD; ++q)
#pragma unroll
        for (int r = 0; r < RL; ++r) acc[q][r] = 0.f;

    const int colL = tid % W, jL = tid / W;
    // tied-array beam pixels this thread holds (bit j: beam j), fixed for the CTA; the
    // thread's pixels are ky = jL + r NS (r < RL) of column kx0 + colL
    uint32_t bmask = 0;
    if constexpr (TAPS) {
        for (int j = 0; j < a.n_beam; ++j) {
            const int ky = a.beam_ky[j];
            if (kx0 + colL == a.beam_kx[j] && ky >= jL && (ky - jL) % CS::NS == 0) bmask |= 1u << j;
        }
    }
    if (a.nt > 0) stage(0, s_in);

    for (int tt = 0; tt < a.nt; ++tt) {
        if (tt + 1 < a.nt) {
            stage(tt + 1, s_in + ((tt + 1) & 1) * TILE * EB);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const unsigned char *tin = s_in + (tt & 1) * TILE * EB;
        auto in_at = [&](int p, int row, int col) -> float2 {
            const int e = (p * N + row) * W + col;
            if constexpr (H16) {
                return __half22float2(reinterpret_cast<const __half2 *>(tin)[e]);
            } else {
                return reinterpret_cast<const float2 *>(tin)[e];
            }
        };
        {   // pass 0: staged tile -> registers -> s_a.  FP32 field: one (pol, slot) per thread and
            // turn (every thread busy); FP16 field: both pols of a slot per thread (measured faster there)
            constexpr int R = FP::R0, NSL = N / R;
            constexpr int PS = H16 ? 1 : P;     // pols spread over threads
            for (int it = tid; it < PS * W * NSL; it += kBlock) {
                const int p0 = it / (W * NSL), sl = it - p0 * (W * NSL);
                const int col = sl % W, j = sl / W;
#pragma unroll
                for (int pp = 0; pp < P / PS; ++pp) {
                    const int p = p0 + pp;
                    float2 v[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) v[r] = in_at(p, j + r * NSL, col);
                    dft<R, 1>(v);
#pragma unroll
                    for (int r = 0; r < R; ++r) s_a[(p * N + stockham_out<R, 1>(j, r)) * W + col] = v[r];
                }
            }
        }
        __syncthreads();
        if constexpr (FP::NP == 3) {
            constexpr int R = FP::R1, NS = FP::R0, NSL = N / R;
            for (int it = tid; it < P * W * NSL; it += kBlock) {
                const int p = it / (W * NSL), sl = it - p * (W * NSL);
                const int col = sl % W, j = sl / W;
                float2 v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = s_a[(p * N + j + r * NSL) * W + col];
                twiddle<R, NS, 1>(v, j, s_tw + TW::OFF1);
                dft<R, 1>(v);
#pragma unroll
                for (int r = 0; r < R; ++r) s_b[(p * N + stockham_out<R, NS>(j, r)) * W + col] = v[r];
            }
            __syncthreads();
        }
        {   // last pass: shared -> registers, then step 4 in registers
            constexpr int NS = CS::NS;
            const float2 *src = FP::NP == 3 ? s_b : s_a;
            const float2 *tw = s_tw + (FP::NP == 3 ? TW::OFF2 : TW::OFF1);
            float2 vx[RL];
#pragma unroll
            for (int r = 0; r < RL; ++r) vx[r] = src[(jL + r * NS) * W + colL];
            twiddle<RL, NS, 1>(vx, jL, tw);
            dft<RL, 1>(vx);
            // feedback calibration: this thread holds ky = jL + r NS of column kx0 + colL
            const bool tap = TAPS && a.etap && kx0 + colL == a.tap_kx && (a.tap_ky - jL) % NS == 0 && a.tap_ky >= jL;
            // tied-array beams: the field at each beam pixel this thread holds, every sample
            auto beams = [&](const float2 (&v)[RL], int p) {
                for (uint32_t m = bmask; m; m &= m - 1) {
                    const int j = __ffs(m) - 1;
                    const int rj = (a.beam_ky[j] - jL) / NS;
                    float2 val = v[0];
#pragma unroll
                    for (int r = 1; r < RL; ++r)
                        if (r == rj) val = v[r];
                    a.beam_out[(((long long)(a.beam_t0 + tt) * a.beam_C + c) * a.n_beam + j) * P + p] =
                        make_float2(val.x * sc, val.y * sc);
                }
            };
            if constexpr (P == 1) {
                if (tap) {
#pragma unroll
                    for (int r = 0; r < RL; ++r)
                        if (jL + r * NS == a.tap_ky)
                            a.etap[(long long)tt * a.nc + cl] = make_float2(vx[r].x * sc, vx[r].y * sc);
                }
                if (TAPS && bmask) beams(vx, 0);
#pragma unroll
                for (int r = 0; r < RL; ++r) acc[0][r] = fmaf(vx[r].x, vx[r].x, fmaf(vx[r].y, vx[r].y, acc[0][r]));
            } else {
                float2 vy[RL];
#pragma unroll
                for (int r = 0; r < RL; ++r) vy[r] = src[(N + jL + r * NS) * W + colL];
                twiddle<RL, NS, 1>(vy, jL, tw);
                dft<RL, 1>(vy);
                if (tap) {
#pragma unroll
                    for (int r = 0; r < RL; ++r)
                        if (jL + r * NS == a.tap_ky) {
                            a.etap[((long long)tt * a.nc + cl) * 2] = make_float2(vx[r].x * sc, vx[r].y * sc);
                            a.etap[((long long)tt * a.nc + cl) * 2 + 1] = make_float2(vy[r].x * sc, vy[r].y * sc);
                        }
                }
                if (TAPS && bmask) {
                    beams(vx, 0);
                    beams(vy, 1);
                }
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    acc[0][r] = fmaf(vx[r].x, vx[r].x, fmaf(vx[r].y, vx[r].y, acc[0][r]));
                    acc[1][r] = fmaf(vy[r].x, vy[r].x, fmaf(vy[r].y, vy[r].y, acc[1][r]));
                    acc[2][r] = fmaf(vx[r].x, vy[r].x, fmaf(vx[r].y, vy[r].y, acc[2][r]));
                    acc[3][r] = fmaf(vx[r].y, vy[r].x, fmaf(-vx[r].x, vy[r].y, acc[3][r]));
                }
            }
        }
        // s_a is rewritten by the next pass 0 only after the next barrier.
    }

    // Fold this chunk's FP32 sums into the FP64 accumulators (one owner per pixel).
    const double sc2 = (double)sc * (double)sc;
    const int kx = kx0 + colL;
#pragma unroll
    for (int q = 0; q < NPROD; ++q) {
        double *d = a.acc + ((long long)c * NPROD + q) * N * N + kx;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            const int ky = jL + r * CS::NS;
            // read through L2: in a persistent launch another SM folded the previous chunk
            d[(long long)ky * N] = __ldcg(d + (long long)ky * N) + (H16 ? (double)acc[q][r] * sc2 : (double)acc[q][r]);
        }
    }
}

template <int N, int P, bool H16, bool TAPS>
__global__ void __launch_bounds__(kBlock) k_cols_acc(const ColArgs a) {
    cols_acc<N, P, H16, TAPS>(a, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------------------------
// Batching pattern: every (Tb, Cb) chunk of a block in ONE persistent launch.  Each CTA pulls
// work items from a device queue (an atomic counter over the item list, in chunk order: the
// chunk's gridding + row-transform items, then its column items) until the queue is empty.
// An item waits (one polling lane, bounded by a clock64 budget) for the items it depends on:
//   row item (k, stripe, cl)   the column items of chunk k - 1 for channel slot cl (they read
//                              the field scratch it overwrites);
//   column item (k, strip, cl) the row items of chunk k for cl, and, when chunk k - 1 holds the
//                              same channels, its column items for cl (both add to the same FP64
//                              accumulators: chunks fold in order, so the sums equal the direct
//                              launches' bit for bit).
// Every dependency is on an earlier item of the queue, which a running CTA has claimed, so the
// launch always progresses.  A wait that runs out of budget (or sees another CTA's failure)
// records MOFF_ETIMEDOUT in the status word and the CTA leaves; no asynchronous copy is in
// flight at any wait.
__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One lane: wait until *cnt >= need, within budget; false if it ran out or a CTA failed.
__device__ __forceinline__ bool persist_wait(const int *cnt, int need, const PersistArgs &pa) {
    const long long t0 = clock64();
    while (ld_acquire_gpu(cnt) < need) {
        if (ld_acquire_gpu(pa.status) != 0 || clock64() - t0 > pa.budget) return false;
        __nanosleep(256);
    }
    return true;
}

// Item it of the queue: chunk k (item0[k] <= it < item0[k + 1]); within it, nc * n_stripes row
// items (stripe fastest, as the direct launch's grid), then nc * n_strips column items.
__device__ __forceinline__ int4 persist_item(const PersistArgs &pa, int it) {
    int lo = 0, hi = pa.n_chunks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pa.item0[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    const int r = it - pa.item0[lo], nr = pa.n_stripes * pa.chunks[lo].w;
    if (r < nr) return make_int4(lo, 0, r % pa.n_stripes, r / pa.n_stripes);
    const int rc = r - nr;
    return make_int4(lo, 1, rc % pa.n_strips, rc / pa.n_strips);
}

template <int N, int P, int TB, int CPL, bool WIDE>
__global__ void __launch_bounds__(kBlock) k_image_persist(const __grid_constant__ PersistArgs pa) {
    __shared__ int4 s_w;
    __shared__ int s_go;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const int it = ld_acquire_gpu(pa.status) != 0 ? pa.n_items : atomicAdd(pa.next, 1);
            int go = it < pa.n_items;
            int4 w = make_int4(0, 0, 0, 0);
            if (go) {
                w = persist_item(pa, it);
                const int k = w.x, cl = w.w;
                if (w.y == 0) {
                    if (k > 0) go = persist_wait(pa.cols_done + (k - 1) * pa.cb + cl, pa.n_strips, pa);
                } else {
                    go = persist_wait(pa.rows_done + k * pa.cb + cl, pa.n_stripes + pa.rows_extra, pa);
                    if (go && k > 0 && pa.chunks[k - 1].z == pa.chunks[k].z)
                        go = persist_wait(pa.cols_done + (k - 1) * pa.cb + cl, pa.n_strips, pa);
                }
                if (!go) atomicCAS(pa.status, 0, 1);
            }
            s_w = w;
            s_go = go;
        }
        __syncthreads();
        if (!s_go) break;
        const int4 w = s_w;
        const int4 ch = pa.chunks[w.x];
        if (w.y == 0) {
            GridArgs g = pa.g;
            g.t0 = ch.x;
            g.nt = ch.y;
            g.c0 = ch.z;
            g.nc = ch.w;
            grid_rows<N, P, TB, false, false, CPL, WIDE>(g, w.z, w.w, pa.n_stripes);
        } else {
            ColArgs ca = pa.ca;
            ca.nt = ch.y;
            ca.c0 = ch.z;
            ca.nc = ch.w;
            cols_acc<N, P, false, false>(ca, w.z, w.w);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd((w.y == 0 ? pa.rows_done : pa.cols_done) + w.x * pa.cb + w.w, 1);
    }
}

template <int N, int P, int CPL, bool WIDE>
cudaError_t launch_persist_t(const PersistArgs &pa, size_t smem, int sms, cudaStream_t st) {
    auto k = k_image_persist<N, P, 4, CPL, WIDE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBlock, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::max(1, std::min(pa.n_items, per_sm * sms));
    k<<<grid, kBlock, smem, st>>>(pa);
    return cudaGetLastError();
}

// The persistent launch runs the gridding shape with 4 samples per pass and kernel entries read
// through L2; CPL and wide stripes as the plan chose them.
template <int N, int P>
cudaError_t launch_persist_p(int cpl, bool wide, const PersistArgs &pa, size_t smem, int sms, cudaStream_t st) {
    if (cpl == 4) {
        if constexpr (GridShape<N, P, 4, true>::ROWS % 2 == 0 && GridShape<N, P, 4, false>::ROWS % 2 == 0)
            return wide ? launch_persist_t<N, P, 4, true>(pa, smem, sms, st) : launch_persist_t<N, P, 4, false>(pa, smem, sms, st);
        return cudaErrorInvalidValue;
    }
    if (cpl == 2)
        return wide ? launch_persist_t<N, P, 2, true>(pa, smem, sms, st) : launch_persist_t<N, P, 2, false>(pa, smem, sms, st);
    return wide ? launch_persist_t<N, P, 1, true>(pa, smem, sms, st) : launch_persist_t<N, P, 1, false>(pa, smem, sms, st);
}

#define MOFF_DEFINE_PERSIST_N(NN)                                                                    \
    cudaError_t launch_persist_n##NN(int P, int cpl, bool wide, const PersistArgs &pa, size_t smem, int sms, \
                                     cudaStream_t st) {                                             \
        return P == 1 ? launch_persist_p<NN, 1>(cpl, wide, pa, smem, sms, st)                       \
                      : launch_persist_p<NN, 2>(cpl, wide, pa, smem, sms, st);                      \
    }

template <int N>
size_t col_smem_bytes_t(int P, bool h16 = false) {
    using FP = FftPlan<N>;
    const size_t tile = (size_t)P * N * ColShape<N>::W;
    return (size_t)((FftTw<N>::TOTAL + 1) & ~1) * 8 + tile * (h16 ? 4 : 8) * 2 + tile * 8 * (FP::NP == 3 ? 2 : 1);
}

template <int N, int P, int TB, bool ST, bool GO, int CPL, bool WD>
cudaError_t launch_grid_t(const GridArgs &a, int n_stripes, size_t smem, cudaStream_t st) {
    // 2 x 2 blocks need an even stripe height and entries read through L2
    if constexpr (CPL == 4 && (ST || GridShape<N, P, TB, WD>::ROWS % 2 != 0)) {
        return cudaErrorInvalidValue;
    } else {
    void (*k)(GridArgs);
    if constexpr (GridShape<N, P, TB, WD>::IN_PLACE) k = k_grid_rows_ip<N, P, TB, ST, GO, CPL, WD>;
    else k = k_grid_rows<N, P, TB, ST, GO, CPL, WD>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(n_stripes, a.nc), kBlock, smem, st>>>(a);
    return cudaGetLastError();
    }
}

template <int N, int P, bool ST, bool GO, int CPL, bool WD>
cudaError_t launch_grid_s(int TB, const GridArgs &a, int n_stripes, size_t smem, cudaStream_t st) {
    switch (TB) {
        case 1: return launch_grid_t<N, P, 1, ST, GO, CPL, WD>(a, n_stripes, smem, st);
        case 2: return launch_grid_t<N, P, 2, ST, GO, CPL, WD>(a, n_stripes, smem, st);
        case 4: return launch_grid_t<N, P, 4, ST, GO, CPL, WD>(a, n_stripes, smem, st);
        case 8: return launch_grid_t<N, P, 8, ST, GO, CPL, WD>(a, n_stripes, smem, st);
    }
    return cudaErrorInvalidValue;
}

// The stripe height is a compile-time function of TB, so the grid-only
// variant runs with the plan's TB too (and stores only the first sample).
template <int N, int P, int CPL, bool WD>
cudaError_t launch_grid_q(int TB, bool staged, bool go, const GridArgs &a, int n_stripes, size_t smem,
                          cudaStream_t st) {
    if (go) return launch_grid_s<N, P, false, true, CPL, WD>(TB, a, n_stripes, smem, st);
    if (CPL == 4) return staged ? cudaErrorInvalidValue : launch_grid_s<N, P, false, false, CPL, WD>(TB, a, n_stripes, smem, st);
    return staged ? launch_grid_s<N, P, true, false, CPL, WD>(TB, a, n_stripes, smem, st)
                  : launch_grid_s<N, P, false, false, CPL, WD>(TB, a, n_stripes, smem, st);
}

template <int N, int P, bool WD>
cudaError_t launch_grid_w(int TB, bool staged, bool go, const GridArgs &a, int n_stripes, size_t smem,
                          cudaStream_t st) {
    if (a.quads) return launch_grid_q<N, P, 4, WD>(TB, staged, go, a, n_stripes, smem, st);
    return a.pairs ? launch_grid_q<N, P, 2, WD>(TB, staged, go, a, n_stripes, smem, st)
                   : launch_grid_q<N, P, 1, WD>(TB, staged, go, a, n_stripes, smem, st);
}

template <int N, int P>
cudaError_t launch_grid_p(int TB, bool staged, bool go, const GridArgs &a, int n_stripes, size_t smem,
                          cudaStream_t st) {
    return a.wide ? launch_grid_w<N, P, true>(TB, staged, go, a, n_stripes, smem, st)
                  : launch_grid_w<N, P, false>(TB, staged, go, a, n_stripes, smem, st);
}

template <int N, int P, bool H16>
cudaError_t launch_cols_t(const ColArgs &a, cudaStream_t st) {
    // pixel taps (feedback calibration, beams) compiled in only where asked for
    auto k = (a.etap || a.n_beam) ? k_cols_acc<N, P, H16, true> : k_cols_acc<N, P, H16, false>;
    const size_t smem = col_smem_bytes_t<N>(P, H16);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(N / ColShape<N>::W, a.nc), kBlock, smem, st>>>(a);
    return cudaGetLastError();
}

#define MOFF_DEFINE_N(NN)                                                                            \
    cudaError_t launch_grid_n##NN(int P, int TB, bool staged, bool go, const GridArgs &a, int n_stripes, \
                                  size_t smem, cudaStream_t st) {                                    \
        return P == 1 ? launch_grid_p<NN, 1>(TB, staged, go, a, n_stripes, smem, st)                 \
                      : launch_grid_p<NN, 2>(TB, staged, go, a, n_stripes, smem, st);                \
    }                                                                                                \
    cudaError_t launch_cols_n##NN(int P, const ColArgs &a, cudaStream_t st, bool h16) {              \
        if (h16) return P == 1 ? launch_cols_t<NN, 1, true>(a, st) : launch_cols_t<NN, 2, true>(a, st); \
        return P == 1 ? launch_cols_t<NN, 1, false>(a, st) : launch_cols_t<NN, 2, false>(a, st);      \
    }

}  // namespace moff
