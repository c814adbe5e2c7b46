// moff_dft.cuh -- Eq. m6 step 3 of Morales (arXiv 0812.3669) as factored DFT
// contractions on the 5th-generation tensor cores (tcgen05, FP16 operands,
// FP32 accumulation in TMEM): the precision pattern's "2D FFT as tensor-core
// DFT-matrix contractions" for grids of N = 256 and 512.
//
// One N-point transform E(k) = sum_r G(r) w^{kr}, w = exp(+2 pi i / N), is
// split with N = 16 * N2 (Fig. 1 rows d-e draw the Cooley-Tukey stages of the
// same transform): r = N2 a + b, k = c + 16 d with a, c < 16 and b, d < N2,
//     stage 1   X(b, c)  = sum_a G(N2 a + b) exp(+2 pi i a c / 16)
//     twiddle   X'(b, c) = X(b, c) w^{b c}
//     stage 2   E(c + 16 d) = sum_b X'(b, c) exp(+2 pi i b d / N2)
// (w^{kr} = exp(2 pi i ac/16) w^{bc} exp(2 pi i bd/N2) because w^{16 N2 a d} = 1).
// Both stages are real products D = A B^T with complex values split into
// (re, im): stage 1 has K = 32 (k = 2a + re/im) and 32 output columns
// (n = 2c + re/im), stage 2 has K = 2 N2 (k = (re/im) N2 + b) and 2 N2 output
// columns (n = 2d + re/im).  The DFT matrices B1, B2 and the twiddles are built
// once per plan in FP64 (moff_dft_kernels.cu) and copied into shared memory by
// every CTA as one image: [B1 | B2 | twiddle table].
//
// Scaling (every FP16 operand is a value times an exact power of two, so no
// rounding changes and nothing can overflow): the gridded field enters FP16 at
// magnitude <= 2^14 (per-channel voltage scale x per-plan kernel scale), the
// twiddle table carries 1/16 (stage 1 grows magnitudes by at most 16) and stage
// 2's output is multiplied by 1/N2, so every intermediate stays <= 2^14.  The
// column kernel undoes the accumulated factor s_G / (16 N) once per chunk.
#pragma once
#include <cuda_fp16.h>

#include "moff_fft.cuh"
#include "moff_tc.cuh"

namespace moff {

// 16-byte asynchronous global -> shared copies (completion tracked per group).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory"); }

template <int N>
struct DftShape {
    static_assert(N == 256 || N == 512, "factored tensor-core DFT: N = 256 or 512");
    static constexpr int N1 = 16;               // stage-1 length
    static constexpr int N2 = N / 16;           // stage-2 length
    static constexpr int K1 = 32;               // stage-1 contraction (16 complex)
    static constexpr int C1 = 32;               // stage-1 output columns (16 complex)
    static constexpr int K2 = 2 * N2;           // stage-2 contraction
    static constexpr int C2 = 2 * N2;           // stage-2 output columns
    static constexpr int B1_BYTES = C1 * K1 * 2;
    static constexpr int B2_BYTES = C2 * K2 * 2;
    static constexpr int TW_BYTES = 16 * N2 * 8;   // float2 [c][b]
    static constexpr int TAB_BYTES = B1_BYTES + B2_BYTES + TW_BYTES;
};
__host__ __device__ constexpr int dft_table_bytes(int N) {
    return 2048 + (2 * (N / 16)) * (2 * (N / 16)) * 2 + 16 * (N / 16) * 8;
}

// Shared-memory bytes of the gridding kernel's transform region (row variant):
// one operand buffer (stage-1 A, then stage-2 A, F * N2 * 64 bytes), the table
// image, one mbarrier and the TMEM address slot.
__host__ __device__ constexpr size_t dft_row_region_bytes(int N, int F) {
    return (size_t)F * (N / 16) * 64 + (size_t)dft_table_bytes(N) + 16;
}
// TMEM columns of the row variant (stage-2 accumulators reuse stage 1's).
__host__ __device__ constexpr int dft_row_tmem_cols(int N, int F) {
    const int n2 = N / 16;
    const int c1 = (F * n2 / 128) * 32, c2 = (16 * F / 128) * 2 * n2;
    const int c = c1 > c2 ? c1 : c2;
    return c <= 32 ? 32 : (c <= 64 ? 64 : (c <= 128 ? 128 : (c <= 256 ? 256 : 512)));
}

namespace dftc {

// Packed FP32 pairs (one instruction for both lanes; each lane rounds as its scalar form).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

constexpr long long kWaitCycles = 200000000LL;   // ~0.1 s at the SM clock (an MMA group takes microseconds)

__device__ __forceinline__ uint32_t pack_h2(float re, float im) {
    const __half2 h = __floats2half2_rn(re, im);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack_hh(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Copy the table image (B1 | B2 | twiddles) into shared memory (16-byte pieces).
__device__ __forceinline__ void load_table(unsigned char *dst, const unsigned char *src, int bytes) {
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

// Row transform of the F gridded rows of one gridding pass (FP32 in shared
// memory, row f at src + f * LDR, element e at pad16(e)) on the tensor cores;
// the FP16 result goes, row f as [re N][im N], to rowout(f) (nullptr: not
// stored), through a staging copy in `stage` (may alias src: src is read
// first).  All kBlock threads call it; thread 0 issues the MMAs.  sG: the
// FP16 scale of the field.  `region`: dft_row_region_bytes(N, F) bytes
// (16-byte aligned) whose table image is already loaded; `mbar` initialised
// with count 1; `phase` counts its completed phases.  Returns false (the same
// value in every thread) when an MMA does not complete within the wait limit.
template <int N, int F, int LDR, int NTHREADS, class RowOut>
__device__ __forceinline__ bool rows_dft(const float2 *src, float sG, unsigned char *region, uint64_t *mbar,
                                         uint32_t tbase, uint32_t &phase, __half *stage, RowOut rowout) {
    using S = DftShape<N>;
    constexpr int N2 = S::N2;
    constexpr int M1 = F * N2;                 // stage-1 rows (f, b)
    constexpr int M2 = 16 * F;                 // stage-2 rows (f, c)
    constexpr int T1 = M1 / 128, T2 = M2 / 128;
    static_assert(M1 % 128 == 0 && M2 % 128 == 0, "row transform: F must be a multiple of 8");
    constexpr int NW = NTHREADS / 32;
    static_assert(NW % 4 == 0, "whole warpgroups");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp & 3;
    unsigned char *sA = region;                              // stage-1 A, then stage-2 A
    const unsigned char *sB1 = region + F * N2 * 64;
    const unsigned char *sB2 = sB1 + S::B1_BYTES;
    const float2 *sTw = reinterpret_cast<const float2 *>(sB2 + S::B2_BYTES);

    // (1) stage-1 A, K-major: row m = f N2 + b holds (re, im) of G(f, N2 a + b), a < 16,
    //     as k = 2a + re/im; 16-byte piece kc carries a = 4 kc .. 4 kc + 3.
    for (int m = tid; m < M1; m += NTHREADS) {
        const int f = m / N2, b = m - f * N2;
        const float2 *row = src + f * LDR;
        uint32_t w[16];
#pragma unroll
        for (int a = 0; a < 16; ++a) {
            const float2 g = row[pad16(N2 * a + b)];
            w[a] = pack_h2(g.x * sG, g.y * sG);
        }
        unsigned char *dst = sA + (m >> 3) * 512 + (m & 7) * 16;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
            *reinterpret_cast<uint4 *>(dst + kc * 128) = make_uint4(w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t id1 = tc::idesc_f16(128, S::C1, false, false);
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB1);
#pragma unroll
        for (int j = 0; j < T1; ++j)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                tc::mma_f16(tbase + 32 * j, tc::smem_desc(a0 + j * 8192 + ks * 256, 128, 512),
                            tc::smem_desc(b0 + ks * 256, 128, 512), id1, ks > 0);
        tc::mma_commit(mbar);
    }
    bool ok = tc::mbar_wait_bounded(mbar, phase & 1, kWaitCycles);
    ++phase;
    ok = __syncthreads_and(ok);
    if (!ok) return false;
    tc::fence_after_sync();

    // (2) twiddle, then stage-2 A (MN-major, no swizzle; rows m2 = 16 f + c, k = re/im N2 + b):
    //     thread (f, b) writes 16-byte pieces of 8 consecutive c at k = b and k = N2 + b.
    constexpr uint32_t LBO2 = (M2 / 8) * 128;   // K-direction core-matrix stride
    for (int u = warp >> 2; u < T1; u += NW / 4) {
        const int m = 128 * u + 32 * q + lane;
        const int f = m / N2, b = m - f * N2;
        float v[32];
        tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * u), v);
        uint32_t re[8], im[8];
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
            const float2 t0 = sTw[c * N2 + b], t1 = sTw[(c + 1) * N2 + b];
            const float x0r = v[2 * c] * t0.x - v[2 * c + 1] * t0.y, x0i = v[2 * c] * t0.y + v[2 * c + 1] * t0.x;
            const float x1r = v[2 * c + 2] * t1.x - v[2 * c + 3] * t1.y,
                        x1i = v[2 * c + 2] * t1.y + v[2 * c + 3] * t1.x;
            re[c >> 1] = pack_hh(x0r, x1r);
            im[c >> 1] = pack_hh(x0i, x1i);
        }
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            const int mg = 2 * f + ch;                       // core-matrix row (m2 >> 3)
            const uint4 pr = make_uint4(re[4 * ch], re[4 * ch + 1], re[4 * ch + 2], re[4 * ch + 3]);
            const uint4 pi = make_uint4(im[4 * ch], im[4 * ch + 1], im[4 * ch + 2], im[4 * ch + 3]);
            const int kr = b, ki = N2 + b;
            *reinterpret_cast<uint4 *>(sA + mg * 128 + (kr >> 3) * LBO2 + (kr & 7) * 16) = pr;
            *reinterpret_cast<uint4 *>(sA + mg * 128 + (ki >> 3) * LBO2 + (ki & 7) * 16) = pi;
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t id2 = tc::idesc_f16(128, S::C2, true, false);
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB2);
        constexpr uint32_t SBOB = (S::K2 / 8) * 128;
#pragma unroll
        for (int j = 0; j < T2; ++j)
#pragma unroll
            for (int ks = 0; ks < S::K2 / 16; ++ks)
                tc::mma_f16(tbase + j * S::C2, tc::smem_desc(a0 + j * 2048 + ks * 2 * LBO2, LBO2, 128),
                            tc::smem_desc(b0 + ks * 256, 128, SBOB), id2, ks > 0);
        tc::mma_commit(mbar);
    }
    ok = tc::mbar_wait_bounded(mbar, phase & 1, kWaitCycles);
    ++phase;
    ok = __syncthreads_and(ok);
    if (!ok) return false;
    tc::fence_after_sync();

    // (3) stage-2 accumulators -> FP16 (x 1/N2) staging rows [f][re/im][N + 8]
    constexpr int SLD = N + 8;
    constexpr int NCB = S::C2 / 32;                           // 32-column blocks per tile
    constexpr float inv = 1.0f / (float)N2;
    for (int u = warp >> 2; u < T2 * NCB; u += NW / 4) {
        const int j = u / NCB, cb = u - j * NCB;
        const int m2 = 128 * j + 32 * q + lane;
        const int f = m2 >> 4, c = m2 & 15;
        float v[32];
        tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(j * S::C2 + 32 * cb), v);
        __half *sr = stage + (2 * f) * SLD + c + 16 * 16 * cb;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            sr[16 * i] = __float2half_rn(v[2 * i] * inv);
            sr[SLD + 16 * i] = __float2half_rn(v[2 * i + 1] * inv);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    // (4) staging -> global rows, 16-byte pieces
    constexpr int PR = N / 8;
    for (int i = tid; i < F * 2 * PR; i += NTHREADS) {
        const int rr = i / PR, pc = i - rr * PR;
        __half *o = rowout(rr >> 1);
        if (o) *reinterpret_cast<uint4 *>(o + (rr & 1) * N + 8 * pc) =
                   *reinterpret_cast<const uint4 *>(stage + rr * SLD + 8 * pc);
    }
    return true;
}

}  // namespace dftc
}  // namespace moff
