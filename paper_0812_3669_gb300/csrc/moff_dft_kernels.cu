// moff_dft_kernels.cu -- the column half of Eq. m6 step 3 (Morales, arXiv
// 0812.3669) as factored DFT contractions on the tensor cores, fused with step 4
// (|E|^2 and the cross-pol products summed over a chunk, then added to the FP64
// accumulators), for the dense FP16 path.  The row half runs inside the
// gridding kernel (k_grid_rows_dft, moff_dft.cuh).
//
//   k_cols_dft  one CTA = 16 columns of one channel walking a chunk of samples.
//               Per sample: the FP16 field's 16-column strip (cp.async, 32-byte
//               pieces of the reached rows) lands as the stage-1 A operand
//               (rows (b, x), k = (a, re/im)); stage 1 on the tensor cores; the
//               twiddled FP32 result is written back as the stage-2 A operand
//               (128-byte swizzled, rows (c, x)); stage 2 leaves E in TMEM,
//               where the epilogue squares and sums it.  Loads of sample t + 1 and
//               stage 1 of sample t run while the epilogue of sample t - 1 works.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdlib>
#include <cstring>

#include "moff_dft.cuh"
#include "moff_fft.cuh"
#include "moff_internal.h"
#include "moff_tc.cuh"

namespace moff {
namespace {

// exp(2 pi i m / L) with the angle reduced exactly (m mod L), in FP64.
void unit_root(long long m, long long L, double *c, double *s) {
    long long r = m % L;
    if (r < 0) r += L;
    const double ang = 2.0 * 3.14159265358979323846264338327950288 * (double)r / (double)L;
    *c = std::cos(ang);
    *s = std::sin(ang);
}

// Byte offset of element (n, k) of a K-major operand image with K columns
// (8 x 8 core matrices of 128 bytes; along K 128 bytes apart, along rows (K/8) * 128).
size_t kmajor_at(int n, int k, int K) {
    return (size_t)(n >> 3) * (K >> 3) * 128 + (size_t)(k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

template <int N, int P, int W>
struct ColDftShape {
    using S = DftShape<N>;
    static_assert(W == 8 || W == 16, "columns per CTA");
    static constexpr int N2 = S::N2;
    static constexpr int H = W / 8;                    // 16-byte pieces per (pol, row, re/im) of the strip
    static constexpr int M1 = W * N2;                  // stage-1 rows per pol: m = W b + x
    static constexpr int T1 = M1 / 128;
    static constexpr int LBO1 = (M1 / 8) * 128;        // stage-1 A: K-direction core-matrix stride
    static constexpr int A1P = M1 * S::K1 * 2;         // bytes of one pol's stage-1 A
    static constexpr int M2 = 16 * W;                  // stage-2 rows per pol: m2 = 8 W c_hi + 8 x + c_lo
    static constexpr int T2 = M2 / 128;
    static constexpr int A2P = M2 * S::K2 * 2;         // bytes of one pol's stage-2 A (128-byte swizzled)
    static constexpr int D1 = P * T1 * S::C1;          // TMEM columns: stage-1 accumulators
    static constexpr int D2 = P * T2 * S::C2;          // then stage-2 accumulators
    static constexpr int TC_ = D1 + D2;
    static constexpr int TCOLS = TC_ <= 32 ? 32 : (TC_ <= 64 ? 64 : (TC_ <= 128 ? 128 : (TC_ <= 256 ? 256 : 512)));
    static constexpr int NPIECE = P * N * 2 * H;       // 16-byte pieces per sample: (p, ry, re/im, h)
    static constexpr int ITER = NPIECE / kBlock;
    static constexpr int ROWS_K = kBlock / (2 * H);    // grid rows covered by one piece round of the block
    // warp groups per stage-2 tile: with one tile (W = 8) the two groups split the d range
    static constexpr int DSPLIT = 2 / T2;
    static constexpr int ND = N2 / DSPLIT;             // d values per thread
    static constexpr int MINB = W == 8 ? 2 : 1;        // CTAs per SM
    static constexpr size_t SMEM = 1024 + (size_t)P * A2P + 2 * (size_t)P * A1P + S::TAB_BYTES + 32;
    static_assert(T2 >= 1 && T2 <= 2 && T1 >= 1 && TC_ * MINB <= 512 && NPIECE % kBlock == 0 && ITER <= 32 &&
                      ND % 8 == 0 && (2 * H * N) % kBlock == 0 && ROWS_K % N2 == 0 && SMEM * MINB <= 225 * 1024,
                  "column-kernel shape");
};

template <int N, int P, int W>
__global__ void __launch_bounds__(kBlock, ColDftShape<N, P, W>::MINB) k_cols_dft(const ColDftArgs a) {
    using S = DftShape<N>;
    using CS = ColDftShape<N, P, W>;
    constexpr int N2 = S::N2, K2 = S::K2, C2 = S::C2, H = CS::H, ND = CS::ND;
    constexpr int NPROD = P == 1 ? 1 : 4;
    const int x0 = blockIdx.x * W, cl = blockIdx.y, c = a.c0 + cl;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp & 3;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the swizzled stage-2 operand needs a 1024-byte aligned base (the size includes the slack)
    unsigned char *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *sA2 = smem;                                   // [P][A2P]
    unsigned char *sA1 = sA2 + P * CS::A2P;                      // [2 buffers][P][A1P]
    unsigned char *sTab = sA1 + 2 * P * CS::A1P;
    const unsigned char *sB1 = sTab, *sB2 = sTab + S::B1_BYTES;
    const float4 *sTw = reinterpret_cast<const float4 *>(sB2 + S::B2_BYTES);   // [c pair][b]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sTab + S::TAB_BYTES);   // [0] stage 1, [1] stage 2
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);

    dftc::load_table(sTab, a.dft_tab, S::TAB_BYTES);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, CS::TCOLS);
        tc::tmem_relinquish();
    }
    // Piece i = k kBlock + tid of a sample: pol p, row ry, re/im ri, column piece h (i = ((p N + ry) 2
    // + ri) H + h).  With kBlock a divisor of 2 H N, k fixes p and ry's multiple of ROWS_K (PK, RYK
    // below, compile-time) and the thread fixes ry mod ROWS_K = r0, ri and h: every offset is a thread
    // constant plus a compile-time one.  In the stage-1 operand the piece is the 8 rows m = W b + 8 h
    // + (0..7) at k = 2 a + ri (ry = N2 a + b).  Rows no kernel reaches are zero: cleared once in both
    // buffers and never loaded.
    const int h0 = tid % H, ri0 = (tid / H) & 1, r0 = tid / (2 * H);
    const int a0 = r0 / N2, b0 = r0 - a0 * N2, kt = 2 * a0 + ri0;
    // 2 a = 2 (RYK / N2) + 2 a0: the compile-time part is a multiple of 8 when ROWS_K is one of 4 N2,
    // else (16 columns at N = 512) kt and the compile-time part share one core-matrix row group
    constexpr bool KSPLIT8 = CS::ROWS_K % (4 * N2) == 0;
    const uint32_t dst_t = (uint32_t)((H * b0 + h0) * 128) +
                           (KSPLIT8 ? (uint32_t)((kt >> 3) * CS::LBO1 + (kt & 7) * 16) : (uint32_t)(kt * 16));
    const long long src_t = (long long)(2 * r0 + ri0) * N + x0 + 8 * h0;
    auto piece_dst = [&](int k) -> uint32_t {      // k compile-time after unrolling
        const int PK = (k * kBlock) / (2 * H * N), RYK = ((k * kBlock) % (2 * H * N)) / (2 * H), AK = RYK / N2;
        return (uint32_t)(PK * CS::A1P + ((2 * AK) >> 3) * CS::LBO1 + ((2 * AK) & 7) * 16) + dst_t;
    };
    auto piece_src = [&](int k) -> long long {
        const int PK = (k * kBlock) / (2 * H * N), RYK = ((k * kBlock) % (2 * H * N)) / (2 * H);
        return (long long)(PK * N + RYK) * 2 * N + src_t;
    };
    uint32_t act = 0;
#pragma unroll
    for (int k = 0; k < CS::ITER; ++k) {
        const int ry = (((k * kBlock) % (2 * H * N)) / (2 * H)) + r0;
        if ((a.row_nz[ry >> 5] >> (ry & 31)) & 1u) {
            act |= 1u << k;
        } else {
            const uint32_t d = piece_dst(k);
            *reinterpret_cast<uint4 *>(sA1 + d) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(sA1 + P * CS::A1P + d) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    auto stage = [&](int tt, int buf) {
        const __half *src = a.H + ((long long)tt * a.slab_t + (long long)cl * a.slab_c) * P * N * 2 * N;
        unsigned char *dst = sA1 + buf * P * CS::A1P;
#pragma unroll
        for (int k = 0; k < CS::ITER; ++k)
            if ((act >> k) & 1u) cp_async16(dst + piece_dst(k), src + piece_src(k));
        cp_async_commit();
    };
    auto issue_s1 = [&](int buf) {
        tc::fence_after_sync();
        const uint32_t id1 = tc::idesc_f16(128, S::C1, true, false);
        const uint32_t a0 = tc::smem_u32(sA1 + buf * P * CS::A1P), b0 = tc::smem_u32(sB1);
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int j = 0; j < CS::T1; ++j)
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                    tc::mma_f16(tbase + (uint32_t)((p * CS::T1 + j) * S::C1),
                                tc::smem_desc(a0 + p * CS::A1P + j * 2048 + ks * 2 * CS::LBO1, CS::LBO1, 128),
                                tc::smem_desc(b0 + ks * 256, 128, 512), id1, ks > 0);
        tc::mma_commit(&mbar[0]);
    };
    auto issue_s2 = [&]() {
        tc::fence_after_sync();
        const uint32_t id2 = tc::idesc_f16(128, C2, true, false);
        const uint32_t a0 = tc::smem_u32(sA2), b0 = tc::smem_u32(sB2);
        constexpr uint32_t SBOB = (K2 / 8) * 128;
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int j = 0; j < CS::T2; ++j)
#pragma unroll
                for (int ks = 0; ks < K2 / 16; ++ks)
                    tc::mma_f16(tbase + (uint32_t)(CS::D1 + (p * CS::T2 + j) * C2),
                                tc::smem_desc_sw128(a0 + p * CS::A2P + j * 2 * K2 * 128 + ks * 2048, K2 * 128, 1024),
                                tc::smem_desc(b0 + ks * 256, 128, SBOB), id2, ks > 0);
        tc::mma_commit(&mbar[1]);
    };
    // Twiddle stage 1's result and write it as stage 2's A: thread (b, x) of tile (p, j) writes, for
    // c = 8 ch .. 8 ch + 7 (one TMEM load of 16 columns each: real parts, then imaginary parts), the
    // re piece at k = b and the im piece at k = N2 + b of row group m2 = 8 W ch + 8 x.  Outputs c and
    // c + 1 go through packed FP32 arithmetic as a pair (t = (re w, -im w) / 16 of both):
    //   re = Xr re w - Xi im w,   im = Xi re w + Xr im w.
    auto epi1 = [&]() {
        for (int idx = warp >> 2; idx < P * CS::T1; idx += kBlock / 128) {
            const int p = idx / CS::T1, j = idx - p * CS::T1;
            const int m = 128 * j + 32 * q + lane, b = m / W, x = m % W;
            unsigned char *a2 = sA2 + p * CS::A2P;
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
                float v[16];
                tc::tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(idx * S::C1 + 16 * ch), v);
                uint32_t re[4], im[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 t = sTw[(4 * ch + i) * N2 + b];
                    const float2 xr = make_float2(v[2 * i], v[2 * i + 1]), xi = make_float2(v[8 + 2 * i], v[9 + 2 * i]);
                    const float2 wr = make_float2(t.x, t.y), nwi = make_float2(t.z, t.w);
                    const float2 yr = dftc::fma2(xi, nwi, dftc::mul2(xr, wr));
                    const float2 yi = dftc::sub2(dftc::mul2(xi, wr), dftc::mul2(xr, nwi));
                    re[i] = dftc::pack_hh(yr.x, yr.y);
                    im[i] = dftc::pack_hh(yi.x, yi.y);
                }
                const int m2 = ch * 8 * W + x * 8;
                const int hb = (m2 >> 6) * K2 * 128, cg = (m2 & 63) >> 3;
                const int kr = b, ki = N2 + b;
                *reinterpret_cast<uint4 *>(a2 + hb + kr * 128 + ((cg ^ (kr & 7)) << 4)) =
                    make_uint4(re[0], re[1], re[2], re[3]);
                *reinterpret_cast<uint4 *>(a2 + hb + ki * 128 + ((cg ^ (ki & 7)) << 4)) =
                    make_uint4(im[0], im[1], im[2], im[3]);
            }
        }
    };
    // Square and sum: warp group g = warp / 4 takes stage-2 tile j2 (two tiles) or half the d range
    // (one tile); lane quarter q's row l = 32 q + lane of the tile is m2 = 128 j2 + l = 8 W c_hi + 8 x
    // + c_lo: pixels (ky = 8 c_hi + c_lo + 16 d, kx = x0 + x) for the group's d.
    const int g = warp >> 2;
    const int j2 = CS::T2 == 2 ? g : 0, dbase = CS::T2 == 2 ? 0 : g * ND;
    // sums of d and d + 1 side by side (packed FP32)
    float2 acc[NPROD][ND / 2];
#pragma unroll
    for (int pq = 0; pq < NPROD; ++pq)
#pragma unroll
        for (int d = 0; d < ND / 2; ++d) acc[pq][d] = make_float2(0.f, 0.f);
    auto epi2 = [&]() {
#pragma unroll
        for (int db = 0; db < ND / 8; ++db) {         // 8 d per TMEM load of each pol: real parts, then imaginary
            const uint32_t col = (uint32_t)(CS::D1 + j2 * C2 + 2 * dbase + 16 * db);
            float ex[16];
            tc::tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + col, ex);
            if constexpr (P == 1) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 xr = make_float2(ex[2 * i], ex[2 * i + 1]), xi = make_float2(ex[8 + 2 * i], ex[9 + 2 * i]);
                    float2 &s0 = acc[0][4 * db + i];
                    s0 = dftc::fma2(xr, xr, dftc::fma2(xi, xi, s0));
                }
            } else {
                float ey[16];
                tc::tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + col + (uint32_t)(CS::T2 * C2), ey);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 xr = make_float2(ex[2 * i], ex[2 * i + 1]), xi = make_float2(ex[8 + 2 * i], ex[9 + 2 * i]);
                    const float2 yr = make_float2(ey[2 * i], ey[2 * i + 1]), yi = make_float2(ey[8 + 2 * i], ey[9 + 2 * i]);
                    const int dp = 4 * db + i;
                    acc[0][dp] = dftc::fma2(xr, xr, dftc::fma2(xi, xi, acc[0][dp]));
                    acc[1][dp] = dftc::fma2(yr, yr, dftc::fma2(yi, yi, acc[1][dp]));
                    acc[2][dp] = dftc::fma2(xr, yr, dftc::fma2(xi, yi, acc[2][dp]));
                    acc[3][dp] = dftc::sub2(dftc::fma2(xi, yr, acc[3][dp]), dftc::mul2(xr, yi));
                }
            }
        }
    };

    bool ok = true;
    if (a.nt > 0) stage(0, 0);
    for (int t = 0; t < a.nt; ++t) {
        const int buf = t & 1;
        cp_async_wait<0>();                    // sample t's strip has landed
        tc::fence_async_smem();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) issue_s1(buf);
        if (t + 1 < a.nt) stage(t + 1, buf ^ 1);   // its buffer was read by stage 1 of t - 1 (done)
        if (t > 0) {
            ok &= tc::mbar_wait_bounded(&mbar[1], (uint32_t)((t - 1) & 1), dftc::kWaitCycles);
            tc::fence_after_sync();
            epi2();
        }
        ok &= tc::mbar_wait_bounded(&mbar[0], (uint32_t)(t & 1), dftc::kWaitCycles);
        tc::fence_after_sync();
        epi1();
        tc::fence_async_smem();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) issue_s2();
    }
    if (ok && a.nt > 0) {
        ok &= tc::mbar_wait_bounded(&mbar[1], (uint32_t)((a.nt - 1) & 1), dftc::kWaitCycles);
        tc::fence_after_sync();
        epi2();
    }
    cp_async_wait<0>();
    tc::fence_before_sync();
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();
    if (ok) {
        // undo the field's scale s_G / (16 N) (exact powers of two), squared, and fold into FP64
        const double un = 16.0 * (double)N / ((double)a.sy[c] * (double)a.s_t);
        const double sc2 = un * un;
        const int m2 = 128 * j2 + 32 * q + lane;
        const int x = (m2 % (8 * W)) >> 3, cy = 8 * (m2 / (8 * W)) + (m2 & 7);
#pragma unroll
        for (int pq = 0; pq < NPROD; ++pq) {
            double *dst = a.acc + ((long long)c * NPROD + pq) * N * N + x0 + x;
#pragma unroll
            for (int d = 0; d < ND; ++d)
                dst[(long long)(cy + 16 * (dbase + d)) * N] += (double)((d & 1) ? acc[pq][d >> 1].y : acc[pq][d >> 1].x) * sc2;
        }
    } else if (tid == 0) {
        atomicExch(a.err, tc::kErrWaitTimeout);
    }
    if (warp == 0) tc::tmem_dealloc(tbase, CS::TCOLS);
}

// ---------------------------------------------------------------------------------------------
// Row transform of a gridded field that is already in global memory (FP16 rows [re N][im N],
// written by the tensor-core gridding): one CTA = a stripe of RS grid rows (both pols) of one
// channel walking a chunk of samples.  Per sample the F = P RS rows land by 16-byte cp.async
// pieces as the stage-1 A operand, MN-major (row m = f N2 + b, k = 2 a + re/im: each piece is 8
// consecutive b of one (f, a, re/im)); pieces of cells no tile reaches are zero, cleared once.
// Stage 1, twiddle, stage 2 and the FP16 store of the row-transformed rows as in the gridding
// kernel's row transform; loads of sample t + 1 and stage 1 of sample t overlap the epilogue of
// sample t - 1.
template <int N, int P>
struct RowDftShape {
    using S = DftShape<N>;
    static constexpr int RS = 8 / P;                    // grid rows per stripe (8 transform rows, inside one tile band)
    static constexpr int F = P * RS;                    // transform rows per sample, f = p RS + rl
    static constexpr int N2 = S::N2;
    static constexpr int M1 = F * N2, T1 = M1 / 128;    // stage-1 rows (f, b)
    static constexpr int LBO1 = (M1 / 8) * 128;
    static constexpr int A1B = M1 * S::K1 * 2;
    static constexpr int M2 = 16 * F, T2 = M2 / 128;    // stage-2 rows (f, c)
    static constexpr int LBO2 = (M2 / 8) * 128;
    static constexpr int A2B = M2 * S::K2 * 2;
    static constexpr int D1 = T1 * S::C1, D2 = T2 * S::C2;
    static constexpr int TC_ = D1 + D2;
    static constexpr int TCOLS = TC_ <= 32 ? 32 : (TC_ <= 64 ? 64 : (TC_ <= 128 ? 128 : (TC_ <= 256 ? 256 : 512)));
    static constexpr int NPIECE = F * 16 * 2 * (N2 / 8);   // (f, a, re/im, b8)
    static constexpr int ITER = NPIECE / kBlock;
    static constexpr size_t SMEM = 16 + 2 * (size_t)A1B + A2B + S::TAB_BYTES + 32;
    static_assert(M1 % 128 == 0 && M2 % 128 == 0 && NPIECE % kBlock == 0 && ITER <= 32, "row-transform shape");
};

template <int N, int P>
__global__ void __launch_bounds__(kBlock) k_rows_dft(const RowDftArgs a) {
    using S = DftShape<N>;
    using RD = RowDftShape<N, P>;
    constexpr int N2 = S::N2, K2 = S::K2, C2 = S::C2, F = RD::F, RS = RD::RS;
    const int s = blockIdx.x, cl = blockIdx.y, c = a.c0 + cl;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp & 3;
    const int ry0 = s * RS;
    {   // stripes no kernel reaches carry no field: nothing to transform or store
        bool any = false;
        for (int rl = 0; rl < RS; ++rl) any |= ((a.row_nz[(ry0 + rl) >> 5] >> ((ry0 + rl) & 31)) & 1u) != 0;
        if (!any) return;
    }
    (void)c;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *sA1 = smem;                                   // [2][A1B]
    unsigned char *sA2 = sA1 + 2 * RD::A1B;
    unsigned char *sTab = sA2 + RD::A2B;
    const unsigned char *sB1 = sTab, *sB2 = sTab + S::B1_BYTES;
    const float2 *sTw = reinterpret_cast<const float2 *>(sB2 + S::B2_BYTES);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sTab + S::TAB_BYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);

    dftc::load_table(sTab, a.dft_tab, S::TAB_BYTES);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, RD::TCOLS);
        tc::tmem_relinquish();
    }
    // Piece i = k kBlock + tid = ((f 16 + aa) 2 + ri) (N2/8) + b8: with 32 (N2/8) a divisor of
    // kBlock, k fixes f's high part (FK, compile-time) and the thread fixes (f mod FPK, aa, ri, b8).
    constexpr int B8N = N2 / 8, FPK = kBlock / (32 * B8N);   // rows f per k step
    static_assert(kBlock % (32 * B8N) == 0, "piece enumeration");
    const int b8_0 = tid % B8N, ri_0 = (tid / B8N) & 1, aa_0 = (tid / (2 * B8N)) & 15, f_0 = tid / (32 * B8N);
    auto piece = [&](int k, int &f, int &aa, int &ri, int &b8) {
        f = k * FPK + f_0;
        aa = aa_0;
        ri = ri_0;
        b8 = b8_0;
    };
    auto piece_dst = [&](int f, int aa, int ri, int b8) -> uint32_t {
        const int k = 2 * aa + ri;
        return (uint32_t)((f * (N2 / 8) + b8) * 128 + (k >> 3) * RD::LBO1 + (k & 7) * 16);
    };
    const int ty = ry0 >> 3, nty = N / 8;   // the stripe lies in one tile row (RS <= 8, aligned)
    uint32_t act = 0;
#pragma unroll
    for (int k = 0; k < RD::ITER; ++k) {
        int f, aa, ri, b8;
        piece(k, f, aa, ri, b8);
        const int tx = (N2 * aa + 8 * b8) >> 3;
        if (a.active[ty * nty + tx]) {
            act |= 1u << k;
        } else {
            const uint32_t d = piece_dst(f, aa, ri, b8);
            *reinterpret_cast<uint4 *>(sA1 + d) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(sA1 + RD::A1B + d) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const float sc = 1.0f / (float)N2;

    // output row f of sample tt: [re N][im N] halves
    auto row_base = [&](int tt, int f) -> long long {
        const int p = f / RS, rl = f - p * RS;
        return (((long long)tt * a.slab_t + (long long)cl * a.slab_c) * P + p) * N * 2 * N +
               (long long)(ry0 + rl) * 2 * N;
    };
    // input piece: the tile-major field, [channel][pol][tile row][tile col][sample][cy][re/im][cx]
    const long long tstride = (long long)a.Tb * 128;
    auto load = [&](int tt, int buf) {
        unsigned char *dst = sA1 + buf * RD::A1B;
#pragma unroll
        for (int k = 0; k < RD::ITER; ++k) {
            if ((act >> k) & 1u) {
                int f, aa, ri, b8;
                piece(k, f, aa, ri, b8);
                const int p = f / RS, ry = ry0 + (f - p * RS), tx = (N2 * aa + 8 * b8) >> 3;
                const __half *src = a.G + ((((long long)cl * P + p) * nty + ty) * nty + tx) * tstride +
                                    (long long)tt * 128 + ((ry & 7) * 2 + ri) * 8;
                cp_async16(dst + piece_dst(f, aa, ri, b8), src);
            }
        }
        cp_async_commit();
    };
    auto issue_s1 = [&](int buf) {
        tc::fence_after_sync();
        const uint32_t id1 = tc::idesc_f16(128, S::C1, true, false);
        const uint32_t a0 = tc::smem_u32(sA1 + buf * RD::A1B), b0 = tc::smem_u32(sB1);
#pragma unroll
        for (int j = 0; j < RD::T1; ++j)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                tc::mma_f16(tbase + (uint32_t)(j * S::C1),
                            tc::smem_desc(a0 + j * 2048 + ks * 2 * RD::LBO1, RD::LBO1, 128),
                            tc::smem_desc(b0 + ks * 256, 128, 512), id1, ks > 0);
        tc::mma_commit(&mbar[0]);
    };
    auto issue_s2 = [&]() {
        tc::fence_after_sync();
        const uint32_t id2 = tc::idesc_f16(128, C2, true, false);
        const uint32_t a0 = tc::smem_u32(sA2), b0 = tc::smem_u32(sB2);
        constexpr uint32_t SBOB = (K2 / 8) * 128;
#pragma unroll
        for (int j = 0; j < RD::T2; ++j)
#pragma unroll
            for (int ks = 0; ks < K2 / 16; ++ks)
                tc::mma_f16(tbase + (uint32_t)(RD::D1 + j * C2),
                            tc::smem_desc(a0 + j * 2048 + ks * 2 * RD::LBO2, RD::LBO2, 128),
                            tc::smem_desc(b0 + ks * 256, 128, SBOB), id2, ks > 0);
        tc::mma_commit(&mbar[1]);
    };
    // twiddle, then stage-2 A: thread (f, b) writes 8 consecutive c at k = b (re) and N2 + b (im)
    auto epi1 = [&]() {
        for (int u = warp >> 2; u < RD::T1; u += kBlock / 128) {
            const int m = 128 * u + 32 * q + lane;
            const int f = m / N2, b = m - f * N2;
            float v[32];
            tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * u), v);
            uint32_t re[8], im[8];
#pragma unroll
            for (int cc = 0; cc < 16; cc += 2) {
                const float2 t0 = sTw[cc * N2 + b], t1 = sTw[(cc + 1) * N2 + b];
                re[cc >> 1] = dftc::pack_hh(v[2 * cc] * t0.x - v[2 * cc + 1] * t0.y,
                                            v[2 * cc + 2] * t1.x - v[2 * cc + 3] * t1.y);
                im[cc >> 1] = dftc::pack_hh(v[2 * cc] * t0.y + v[2 * cc + 1] * t0.x,
                                            v[2 * cc + 2] * t1.y + v[2 * cc + 3] * t1.x);
            }
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
                const int mg = 2 * f + ch, kr = b, ki = N2 + b;
                *reinterpret_cast<uint4 *>(sA2 + mg * 128 + (kr >> 3) * RD::LBO2 + (kr & 7) * 16) =
                    make_uint4(re[4 * ch], re[4 * ch + 1], re[4 * ch + 2], re[4 * ch + 3]);
                *reinterpret_cast<uint4 *>(sA2 + mg * 128 + (ki >> 3) * RD::LBO2 + (ki & 7) * 16) =
                    make_uint4(im[4 * ch], im[4 * ch + 1], im[4 * ch + 2], im[4 * ch + 3]);
            }
        }
    };
    // stage-2 accumulators -> FP16 (x 1/N2) rows: lane (f, c) holds k = c + 16 d; even lanes store
    // the real parts of (c, c + 1), odd lanes the imaginary parts (pairs swapped by one shuffle)
    auto epi2 = [&](int tt) {
        constexpr int NCB = C2 / 32;
        for (int u = warp >> 2; u < RD::T2 * NCB; u += kBlock / 128) {
            const int j = u / NCB, cb2 = u - j * NCB;
            const int m2 = 128 * j + 32 * q + lane;
            const int f = m2 >> 4, cc = m2 & 15, odd = cc & 1;
            float v[32];
            tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(RD::D1 + j * C2 + 32 * cb2), v);
            __half *row = a.H + row_base(tt, f) + (odd ? N : 0) + (cc & ~1) + 16 * 16 * cb2;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float re = v[2 * i] * sc, im = v[2 * i + 1] * sc;
                const float re_o = __shfl_xor_sync(0xffffffffu, re, 1), im_o = __shfl_xor_sync(0xffffffffu, im, 1);
                *reinterpret_cast<__half2 *>(row + 16 * i) = odd ? __floats2half2_rn(im_o, im) : __floats2half2_rn(re, re_o);
            }
        }
    };

    bool ok = true;
    if (a.nt > 0) load(0, 0);
    for (int t = 0; t < a.nt; ++t) {
        const int buf = t & 1;
        cp_async_wait<0>();
        tc::fence_async_smem();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) issue_s1(buf);
        if (t + 1 < a.nt) load(t + 1, buf ^ 1);
        if (t > 0) {
            ok &= tc::mbar_wait_bounded(&mbar[1], (uint32_t)((t - 1) & 1), dftc::kWaitCycles);
            tc::fence_after_sync();
            epi2(t - 1);
        }
        ok &= tc::mbar_wait_bounded(&mbar[0], (uint32_t)(t & 1), dftc::kWaitCycles);
        tc::fence_after_sync();
        epi1();
        tc::fence_async_smem();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) issue_s2();
    }
    if (ok && a.nt > 0) {
        ok &= tc::mbar_wait_bounded(&mbar[1], (uint32_t)((a.nt - 1) & 1), dftc::kWaitCycles);
        tc::fence_after_sync();
        epi2(a.nt - 1);
    }
    cp_async_wait<0>();
    tc::fence_before_sync();
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();
    if (!ok && tid == 0) atomicExch(a.err, tc::kErrWaitTimeout);
    if (warp == 0) tc::tmem_dealloc(tbase, RD::TCOLS);
}

template <int N, int P>
cudaError_t launch_rows_dft_t(const RowDftArgs &a, cudaStream_t st) {
    auto k = k_rows_dft<N, P>;
    const size_t smem = RowDftShape<N, P>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(N / RowDftShape<N, P>::RS, a.nc), kBlock, smem, st>>>(a);
    return cudaGetLastError();
}

template <int N, int P, int W>
cudaError_t launch_cols_dft_t(const ColDftArgs &a, cudaStream_t st) {
    auto k = k_cols_dft<N, P, W>;
    const size_t smem = ColDftShape<N, P, W>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(N / W, a.nc), kBlock, smem, st>>>(a);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------------
// Row transform for N = 512 as 8 x 64 with the second stage transposed.  With n = b + 64 a
// (a < 8, b < 64): stage 1 is the 8-point DFT over a, [F 64 rows (f, b)] x [16 (a, re/im)] ->
// 16 (re/im, c) columns per row; the twiddle exp(+2 pi i b c / 512) / 8 is formed from w_b =
// exp(+2 pi i b / 512) by complex products in FP32 and applied there, the result rounded to FP16 into
// the stage-2 operand Y'[(f, c)][(re/im, b)] (MN-major); stage 2 is the 64-point DFT over b as the
// product D[(re/im, d)][(f, c)] = T[(re/im, d)][(re/im, b)] . Y', the DFT matrix T in real form the
// K-major A operand.  T's four 64 x 64 blocks are C, -S / S, C (C, S the cosine and sine matrices),
// kept once as [-S; C; S]: the real-input k-steps read rows C, S from the middle block on, the
// imaginary-input ones -S, C from the top.  TMEM lane (re/im, d) then holds outputs k = c + 8 d,
// c < 8, of every row f: eight consecutive outputs of one part, one 16-byte store per row, a warp's
// 32 lanes (32 consecutive d) writing 512 contiguous bytes.  Output scale 1/8 x 1/64 = 1/512, as the
// 16 x 32 kernel's.  73 KB of shared memory, 128 TMEM columns: three CTAs per SM.
template <int P>
struct RowDft8Shape {
    static constexpr int N = 512, N1 = 8, N2 = 64;
    static constexpr int RS = 8 / P, F = P * RS;          // 8 transform rows per stripe, f = p RS + rl
    static constexpr int M1 = F * N2, T1 = M1 / 128;      // stage-1 rows (f, b): four tiles
    static constexpr int K1 = 16, C1 = 16;                // (a, re/im) -> (re/im, c)
    static constexpr int LBO1 = (M1 / 8) * 128;
    static constexpr int A1B = M1 * K1 * 2;
    static constexpr int NB = F * N1;                     // stage-2 N: (f, c)
    static constexpr int K2 = 2 * N2;                     // stage-2 K: (re/im, b)
    static constexpr int LBOB = (NB / 8) * 128;           // K-direction stride of the stage-2 B operand
    static constexpr int BB = NB * K2 * 2;
    static constexpr int B1_BYTES = C1 * K1 * 2;
    static constexpr int TSBO = (N2 / 8) * 128;           // row-group stride of the [-S; C; S] image (K = 64)
    static constexpr int T_BYTES = 3 * N2 * N2 * 2;
    static constexpr int W_BYTES = N2 * 8;                // float2 w_b
    static constexpr int TAB_BYTES = B1_BYTES + T_BYTES + W_BYTES;
    static constexpr int D1 = T1 * C1;                    // TMEM: stage-1 accumulators, then NB stage-2 columns
    static constexpr int TCOLS = 128;
    static constexpr int NPIECE = F * N1 * 2 * (N2 / 8);  // 16-byte pieces per sample: (f, a, re/im, b8)
    static constexpr int ITER = NPIECE / kBlock;
    static constexpr size_t SMEM = 16 + 2 * (size_t)A1B + BB + TAB_BYTES + 32;
    static_assert(D1 + NB <= TCOLS && NPIECE % kBlock == 0 && kBlock == 256 && T1 == 4 && TAB_BYTES % 16 == 0,
                  "8 x 64 row-transform shape");
};

__device__ __forceinline__ float2 cmul8(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

template <int P>
__global__ void __launch_bounds__(kBlock) k_rows_dft8(const RowDftArgs a) {
    using RD = RowDft8Shape<P>;
    constexpr int N = RD::N, N2 = RD::N2, RS = RD::RS;
    const int s = blockIdx.x, cl = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp & 3;
    const int ry0 = s * RS;
    {   // stripes no kernel reaches carry no field: nothing to transform or store
        bool any = false;
        for (int rl = 0; rl < RS; ++rl) any |= ((a.row_nz[(ry0 + rl) >> 5] >> ((ry0 + rl) & 31)) & 1u) != 0;
        if (!any) return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *sA1 = smem;                                   // [2][A1B]
    unsigned char *sB = sA1 + 2 * RD::A1B;                       // stage-2 B operand Y'
    unsigned char *sTab = sB + RD::BB;
    const unsigned char *sB1 = sTab, *sT = sTab + RD::B1_BYTES;
    const float2 *sW = reinterpret_cast<const float2 *>(sT + RD::T_BYTES);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sTab + RD::TAB_BYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);

    dftc::load_table(sTab, a.dft_tab, RD::TAB_BYTES);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, RD::TCOLS);
        tc::tmem_relinquish();
    }
    // Piece i = k kBlock + tid = ((f 8 + aa) 2 + ri) 8 + b8: the thread fixes (aa, ri, b8) and f mod 2,
    // k fixes f's high part.  In the stage-1 operand the piece is the 8 rows m = 64 f + 8 b8 + (0..7)
    // at k = 2 aa + ri; pieces of tiles no kernel reaches are zero, cleared once.
    const int b8 = tid & 7, ri = (tid >> 3) & 1, aa = (tid >> 4) & 7, f0 = tid >> 7;
    const int kk = 2 * aa + ri;
    const uint32_t dst_t = (uint32_t)(b8 * 128 + (kk >> 3) * RD::LBO1 + (kk & 7) * 16);
    const int ty = ry0 >> 3, nty = N / 8, tx = 8 * aa + b8;   // the stripe lies in one tile row
    const bool active = a.active[ty * nty + tx] != 0;
    if (!active) {
#pragma unroll
        for (int k = 0; k < RD::ITER; ++k) {
            const uint32_t d = (uint32_t)((2 * k + f0) * 8 * 128) + dst_t;
            *reinterpret_cast<uint4 *>(sA1 + d) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(sA1 + RD::A1B + d) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const float sc = 1.0f / (float)N2;

    // output row f of sample tt: [re N][im N] halves
    auto row_base = [&](int tt, int f) -> long long {
        const int p = f / RS, rl = f - p * RS;
        return (((long long)tt * a.slab_t + (long long)cl * a.slab_c) * P + p) * N * 2 * N +
               (long long)(ry0 + rl) * 2 * N;
    };
    // input piece: the tile-major field, [channel][pol][tile row][tile col][sample][cy][re/im][cx]
    const long long tstride = (long long)a.Tb * 128;
    auto load = [&](int tt, int buf) {
        if (active) {
            unsigned char *dst = sA1 + buf * RD::A1B;
#pragma unroll
            for (int k = 0; k < RD::ITER; ++k) {
                const int f = 2 * k + f0, p = f / RS, ry = ry0 + (f - p * RS);
                const __half *src = a.G + ((((long long)cl * P + p) * nty + ty) * nty + tx) * tstride +
                                    (long long)tt * 128 + ((ry & 7) * 2 + ri) * 8;
                cp_async16(dst + (uint32_t)(f * 8 * 128) + dst_t, src);
            }
        }
        cp_async_commit();
    };
    auto issue_s1 = [&](int buf) {
        tc::fence_after_sync();
        const uint32_t id1 = tc::idesc_f16(128, RD::C1, true, false);
        const uint32_t a0 = tc::smem_u32(sA1 + buf * RD::A1B), b0 = tc::smem_u32(sB1);
#pragma unroll
        for (int j = 0; j < RD::T1; ++j)
            tc::mma_f16(tbase + (uint32_t)(j * RD::C1), tc::smem_desc(a0 + j * 2048, RD::LBO1, 128),
                        tc::smem_desc(b0, 128, (RD::K1 / 8) * 128), id1, false);
        tc::mma_commit(&mbar[0]);
    };
    auto issue_s2 = [&]() {
        tc::fence_after_sync();
        const uint32_t id2 = tc::idesc_f16(128, RD::NB, false, true);
        const uint32_t t0 = tc::smem_u32(sT), b0 = tc::smem_u32(sB);
#pragma unroll
        for (int ks = 0; ks < RD::K2 / 16; ++ks) {
            // k-steps 0-3 (real parts of Y'): rows C, S from block 1; 4-7 (imaginary parts): -S, C from block 0
            const uint32_t ta = t0 + (ks < 4 ? (uint32_t)(8 * RD::TSBO) : 0u) + (uint32_t)((ks & 3) * 256);
            tc::mma_f16(tbase + (uint32_t)RD::D1, tc::smem_desc(ta, 128, RD::TSBO),
                        tc::smem_desc(b0 + ks * 2 * RD::LBOB, RD::LBOB, 128), id2, ks > 0);
        }
        tc::mma_commit(&mbar[1]);
    };
    // twiddle, then the stage-2 operand: thread (f, b) writes the eight c of its row at k = b (re)
    // and k = N2 + b (im) of n-group f
    auto epi1 = [&]() {
        for (int u = warp >> 2; u < RD::T1; u += kBlock / 128) {
            const int m = 128 * u + 32 * q + lane, f = m / N2, b = m - f * N2;
            float v[16];
            tc::tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(u * RD::C1), v);
            float2 w[8];
            w[0] = make_float2(1.f, 0.f);
            w[1] = sW[b];
            w[2] = cmul8(w[1], w[1]);
            w[3] = cmul8(w[2], w[1]);
            w[4] = cmul8(w[2], w[2]);
            w[5] = cmul8(w[4], w[1]);
            w[6] = cmul8(w[3], w[3]);
            w[7] = cmul8(w[4], w[3]);
            uint32_t re[4], im[4];
#pragma unroll
            for (int cc = 0; cc < 8; cc += 2) {
                const float2 t0 = w[cc], t1 = w[cc + 1];
                re[cc >> 1] = dftc::pack_hh((v[cc] * t0.x - v[8 + cc] * t0.y) * 0.125f,
                                            (v[cc + 1] * t1.x - v[9 + cc] * t1.y) * 0.125f);
                im[cc >> 1] = dftc::pack_hh((v[cc] * t0.y + v[8 + cc] * t0.x) * 0.125f,
                                            (v[cc + 1] * t1.y + v[9 + cc] * t1.x) * 0.125f);
            }
            const int kr = b, ki = N2 + b;
            *reinterpret_cast<uint4 *>(sB + f * 128 + (kr >> 3) * RD::LBOB + (kr & 7) * 16) =
                make_uint4(re[0], re[1], re[2], re[3]);
            *reinterpret_cast<uint4 *>(sB + f * 128 + (ki >> 3) * RD::LBOB + (ki & 7) * 16) =
                make_uint4(im[0], im[1], im[2], im[3]);
        }
    };
    // stage-2 accumulators -> FP16 (x 1/N2) rows: lane (re/im, d) of warp group g holds the eight c
    // of rows f = 4 g .. 4 g + 3
    auto epi2 = [&](int tt) {
        const int g = warp >> 2, m2 = 32 * q + lane, part = m2 / N2, d = m2 - part * N2;
        float v[32];
        tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(RD::D1 + 32 * g), v);
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) {
            uint32_t h[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) h[u] = dftc::pack_hh(v[8 * fl + 2 * u] * sc, v[8 * fl + 2 * u + 1] * sc);
            *reinterpret_cast<uint4 *>(a.H + row_base(tt, 4 * g + fl) + part * N + 8 * d) = make_uint4(h[0], h[1], h[2], h[3]);
        }
    };

    bool ok = true;
    if (a.nt > 0) load(0, 0);
    for (int t = 0; t < a.nt; ++t) {
        const int buf = t & 1;
        cp_async_wait<0>();
        tc::fence_async_smem();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) issue_s1(buf);
        if (t + 1 < a.nt) load(t + 1, buf ^ 1);
        if (t > 0) {
            ok &= tc::mbar_wait_bounded(&mbar[1], (uint32_t)((t - 1) & 1), dftc::kWaitCycles);
            tc::fence_after_sync();
            epi2(t - 1);
        }
        ok &= tc::mbar_wait_bounded(&mbar[0], (uint32_t)(t & 1), dftc::kWaitCycles);
        tc::fence_after_sync();
        epi1();
        tc::fence_async_smem();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) issue_s2();
    }
    if (ok && a.nt > 0) {
        ok &= tc::mbar_wait_bounded(&mbar[1], (uint32_t)((a.nt - 1) & 1), dftc::kWaitCycles);
        tc::fence_after_sync();
        epi2(a.nt - 1);
    }
    cp_async_wait<0>();
    tc::fence_before_sync();
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();
    if (!ok && tid == 0) atomicExch(a.err, tc::kErrWaitTimeout);
    if (warp == 0) tc::tmem_dealloc(tbase, RD::TCOLS);
}

template <int P>
cudaError_t launch_rows_dft8_t(const RowDftArgs &a, cudaStream_t st) {
    auto k = k_rows_dft8<P>;
    const size_t smem = RowDft8Shape<P>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(512 / RowDft8Shape<P>::RS, a.nc), kBlock, smem, st>>>(a);
    return cudaGetLastError();
}


}  // namespace

// B1 [n = 2c + re/im][k = 2a + re/im] = the real form of exp(+2 pi i a c / 16);
// B2 [n = 2d + re/im][k = re/im N2 + b] = that of exp(+2 pi i b d / N2) (both K-major
// images); twiddles [c][b] = exp(+2 pi i b c / N) / 16.  All in FP64, then rounded once.
// cols: the column kernel's image.  Output columns grouped by eight: n = 16 (c / 8) + 8 re/im
// + c mod 8 (and the same for d), so one 16-column TMEM load returns the real parts of eight
// outputs, then their imaginary parts, and neighbouring outputs pair up for packed FP32 arithmetic;
// twiddles as float4 (re w_c, re w_{c+1}, -im w_c, -im w_{c+1}) / 16 per (c pair, b).
std::vector<unsigned char> build_dft_table(int N, bool cols) {
    const int N2 = N / 16, K2 = 2 * N2;
    std::vector<unsigned char> img((size_t)dft_table_bytes(N), 0);
    auto put = [&](size_t off, double v) {
        const __half h = __float2half_rn((float)v);
        std::memcpy(img.data() + off, &h, 2);
    };
    auto col = [&](int o, int ri) { return cols ? 16 * (o >> 3) + 8 * ri + (o & 7) : 2 * o + ri; };
    for (int cc = 0; cc < 16; ++cc)
        for (int aa = 0; aa < 16; ++aa) {
            double wc, ws;
            unit_root((long long)aa * cc, 16, &wc, &ws);
            put(kmajor_at(col(cc, 0), 2 * aa, 32), wc);
            put(kmajor_at(col(cc, 0), 2 * aa + 1, 32), -ws);
            put(kmajor_at(col(cc, 1), 2 * aa, 32), ws);
            put(kmajor_at(col(cc, 1), 2 * aa + 1, 32), wc);
        }
    const size_t b2 = 2048;
    for (int d = 0; d < N2; ++d)
        for (int b = 0; b < N2; ++b) {
            double vc, vs;
            unit_root((long long)b * d, N2, &vc, &vs);
            put(b2 + kmajor_at(col(d, 0), b, K2), vc);
            put(b2 + kmajor_at(col(d, 0), N2 + b, K2), -vs);
            put(b2 + kmajor_at(col(d, 1), b, K2), vs);
            put(b2 + kmajor_at(col(d, 1), N2 + b, K2), vc);
        }
    const size_t tw = b2 + (size_t)K2 * K2 * 2;
    for (int cc = 0; cc < 16; ++cc)
        for (int b = 0; b < N2; ++b) {
            double wc, ws;
            unit_root((long long)b * cc, N, &wc, &ws);
            if (cols) {
                float *q = reinterpret_cast<float *>(img.data() + tw + ((size_t)(cc >> 1) * N2 + b) * 16);
                q[cc & 1] = (float)(wc / 16.0);
                q[2 + (cc & 1)] = (float)(-ws / 16.0);
            } else {
                const float2 v = make_float2((float)(wc / 16.0), (float)(ws / 16.0));
                std::memcpy(img.data() + tw + ((size_t)cc * N2 + b) * 8, &v, 8);
            }
        }
    return img;
}

// Tables of the 8 x 64 row transform (N = 512), all in FP64 then rounded once: B1 [n = 8 re/im + c]
// [k = 2 a + re/im] = the real form of exp(+2 pi i a c / 8) (K-major, 16 x 16); the stage-2 DFT
// matrix's blocks [-S; C; S] (S, C [d][b] = sin, cos of 2 pi b d / 64; K-major, 192 rows x 64);
// w_b = exp(+2 pi i b / 512) as float2.
std::vector<unsigned char> build_rows8_table() {
    constexpr int B1B = 16 * 16 * 2, TB = 3 * 64 * 64 * 2;
    std::vector<unsigned char> img((size_t)B1B + TB + 64 * 8, 0);
    auto put = [&](size_t off, double v) {
        const __half h = __float2half_rn((float)v);
        std::memcpy(img.data() + off, &h, 2);
    };
    for (int c = 0; c < 8; ++c)
        for (int aa = 0; aa < 8; ++aa) {
            double wc, ws;
            unit_root((long long)aa * c, 8, &wc, &ws);
            put(kmajor_at(c, 2 * aa, 16), wc);
            put(kmajor_at(c, 2 * aa + 1, 16), -ws);
            put(kmajor_at(8 + c, 2 * aa, 16), ws);
            put(kmajor_at(8 + c, 2 * aa + 1, 16), wc);
        }
    for (int d = 0; d < 64; ++d)
        for (int b = 0; b < 64; ++b) {
            double vc, vs;
            unit_root((long long)b * d, 64, &vc, &vs);
            put(B1B + kmajor_at(d, b, 64), -vs);
            put(B1B + kmajor_at(64 + d, b, 64), vc);
            put(B1B + kmajor_at(128 + d, b, 64), vs);
        }
    for (int b = 0; b < 64; ++b) {
        double wc, ws;
        unit_root(b, 512, &wc, &ws);
        const float2 v = make_float2((float)wc, (float)ws);
        std::memcpy(img.data() + B1B + TB + (size_t)b * 8, &v, 8);
    }
    return img;
}

cudaError_t launch_rows_dft8(int P, const RowDftArgs &a, cudaStream_t st) {
    return P == 1 ? launch_rows_dft8_t<1>(a, st) : launch_rows_dft8_t<2>(a, st);
}

// Columns per CTA by default: 8 (two CTAs per SM, so one CTA's epilogue runs while the other
// waits on its MMAs) unless MOFF_COLS_W=16 (one CTA per SM); MOFF_AUTOTUNE times both.
int cols_dft_width() { return (getenv("MOFF_COLS_W") && atoi(getenv("MOFF_COLS_W")) == 16) ? 16 : 8; }
bool cols_dft_width_forced() { return getenv("MOFF_COLS_W") != nullptr; }

size_t cols_dft_smem_bytes(int N, int P, int W) {
    if (W == 16) {
        if (N == 512) return P == 1 ? ColDftShape<512, 1, 16>::SMEM : ColDftShape<512, 2, 16>::SMEM;
        if (N == 256) return P == 1 ? ColDftShape<256, 1, 16>::SMEM : ColDftShape<256, 2, 16>::SMEM;
    } else {
        if (N == 512) return P == 1 ? ColDftShape<512, 1, 8>::SMEM : ColDftShape<512, 2, 8>::SMEM;
        if (N == 256) return P == 1 ? ColDftShape<256, 1, 8>::SMEM : ColDftShape<256, 2, 8>::SMEM;
    }
    return 0;
}

cudaError_t launch_cols_dft(int N, int P, int W, const ColDftArgs &a, cudaStream_t st) {
    if (W == 16) {
        if (N == 512) return P == 1 ? launch_cols_dft_t<512, 1, 16>(a, st) : launch_cols_dft_t<512, 2, 16>(a, st);
        if (N == 256) return P == 1 ? launch_cols_dft_t<256, 1, 16>(a, st) : launch_cols_dft_t<256, 2, 16>(a, st);
    } else {
        if (N == 512) return P == 1 ? launch_cols_dft_t<512, 1, 8>(a, st) : launch_cols_dft_t<512, 2, 8>(a, st);
        if (N == 256) return P == 1 ? launch_cols_dft_t<256, 1, 8>(a, st) : launch_cols_dft_t<256, 2, 8>(a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rows_dft(int N, int P, const RowDftArgs &a, cudaStream_t st) {
    if (N == 512) return P == 1 ? launch_rows_dft_t<512, 1>(a, st) : launch_rows_dft_t<512, 2>(a, st);
    if (N == 256) return P == 1 ? launch_rows_dft_t<256, 1>(a, st) : launch_rows_dft_t<256, 2>(a, st);
    return cudaErrorInvalidValue;
}

size_t grid_smem_bytes_dft(int N, int P, int TB, int rows, int max_nloc) {
    const int ldr = N + N / 16;
    const int F = TB * P * rows;
    size_t b = (dft_row_region_bytes(N, F) + 15) / 16 * 16;
    b += (size_t)F * ldr * 8 + 8;                       // one row buffer (+ alignment)
    b += (size_t)volt_stride(TB) * max_nloc * P * 8;    // calibrated voltages of TB samples
    b += (size_t)max_nloc * P * 8 + 8;                  // gains (+ padding)
    b += (size_t)max_nloc * 4;                          // antenna indices
    return (b + 15) & ~(size_t)15;
}

cudaError_t launch_grid_dft(int N, int P, int TB, int CPL, const GridArgs &a, int n_stripes, size_t smem,
                            cudaStream_t st) {
    if (N == 512) return launch_grid_dft_n512(P, TB, CPL, a, n_stripes, smem, st);
    if (N == 256) return launch_grid_dft_n256(P, TB, CPL, a, n_stripes, smem, st);
    return cudaErrorInvalidValue;
}

}  // namespace moff
