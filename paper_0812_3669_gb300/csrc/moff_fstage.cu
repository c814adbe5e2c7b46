// moff_fstage.cu -- polyphase filter-bank F-stage (Morales, arXiv 0812.3669,
// Sec. 2, Eq. FFTofE: each antenna stream is transformed into narrow
// channels, "often implemented as polyphase filters"; Fig. 1 row b).
//
// For frame m of stream ap (M = 2C real samples per frame, n_taps frames per
// filter):
//   s_m[j] = sum_{p < n_taps} h[p M + j] adc[(m + p) M + j]          (FIR)
//   X_m[k] = sum_j s_m[j] exp(-2 pi i j k / M),  k < C                (real DFT)
// The real M-point DFT is done as a C-point complex transform of
// z[n] = s[2n] + i s[2n+1] followed by the even/odd split
//   X[k] = (Z[k] + conj Z[C-k]) / 2 - (i/2) exp(-2 pi i k / M) (Z[k] - conj Z[C-k]).
// The FIR is fused into the first transform pass (no shared-memory round trip),
// and the requantised 4-bit codes are staged in shared memory so each CTA
// writes whole [k][32 streams] rows of the [F][C][A][P] output.
#include "moff_fft.cuh"
#include "moff_internal.h"

namespace moff {

template <int CN>
struct PfbShape {
    static constexpr int NB = (2048 / CN) < 1 ? 1 : ((2048 / CN) > kPfbGroup ? kPfbGroup : (2048 / CN));
    static constexpr int LD = PaddedLen<CN>::value;
};

template <int CN>
__global__ void __launch_bounds__(kBlock) k_pfb(const PfbArgs a) {
    using FP = FftPlan<CN>;
    using TW = FftTw<CN>;
    constexpr int NB = PfbShape<CN>::NB;
    constexpr int LD = PfbShape<CN>::LD;
    constexpr int M = 2 * CN;
    constexpr int GA = kPfbGroup;

    const int m = blockIdx.y;
    const int ap0 = blockIdx.x * GA;
    const int tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *s_tw = reinterpret_cast<float2 *>(smem);
    float2 *s_twM = s_tw + TW::TOTAL;
    float2 *s_b0 = s_twM + CN;
    float2 *s_b1 = s_b0 + NB * LD;
    uint8_t *s_codes = reinterpret_cast<uint8_t *>(s_b1 + NB * LD);   // [CN][GA]

    for (int i = tid; i < TW::TOTAL; i += kBlock) s_tw[i] = a.twp[i];
    for (int i = tid; i < CN; i += kBlock) s_twM[i] = a.twM[i];
    __syncthreads();

    for (int b0 = 0; b0 < GA; b0 += NB) {
        {   // FIR fused with the first transform pass
            constexpr int R = FP::R0, NSL = CN / R;
            for (int sl = tid; sl < NB * NSL; sl += kBlock) {
                const int f = sl / NSL, j = sl - f * NSL;
                const int ap = ap0 + b0 + f;
                float2 v[R];
                if (ap < a.AP) {
                    const int8_t *x = a.adc + (long long)ap * a.S + (long long)m * M;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int n2 = 2 * (j + r * NSL);
                        float sr = 0.f, si = 0.f;
                        for (int p = 0; p < a.ntaps; ++p) {
                            const char2 d = *reinterpret_cast<const char2 *>(x + (long long)p * M + n2);
                            const float2 hh = *reinterpret_cast<const float2 *>(a.h + p * M + n2);
                            sr = fmaf(hh.x, (float)d.x, sr);
                            si = fmaf(hh.y, (float)d.y, si);
                        }
                        v[r] = make_float2(sr, si);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) v[r] = make_float2(0.f, 0.f);
                }
                dft<R, -1>(v);
                float2 *dst = s_b1 + f * LD;
#pragma unroll
                for (int r = 0; r < R; ++r) dst[pad16(stockham_out<R, 1>(j, r))] = v[r];
            }
        }
        __syncthreads();
        {
            constexpr int R = FP::R1, NS = FP::R0, NSL = CN / R;
            for (int sl = tid; sl < NB * NSL; sl += kBlock) {
                const int f = sl / NSL, j = sl - f * NSL;
                const float2 *src = s_b1 + f * LD;
                float2 v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = src[pad16(j + r * NSL)];
                twiddle<R, NS, -1>(v, j, s_tw + TW::OFF1);
                dft<R, -1>(v);
                float2 *dst = s_b0 + f * LD;
#pragma unroll
                for (int r = 0; r < R; ++r) dst[pad16(stockham_out<R, NS>(j, r))] = v[r];
            }
        }
        __syncthreads();
        if constexpr (FP::NP == 3) {
            constexpr int R = FP::R2, NS = FP::R0 * FP::R1, NSL = CN / R;
            for (int sl = tid; sl < NB * NSL; sl += kBlock) {
                const int f = sl / NSL, j = sl - f * NSL;
                const float2 *src = s_b0 + f * LD;
                float2 v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = src[pad16(j + r * NSL)];
                twiddle<R, NS, -1>(v, j, s_tw + TW::OFF2);
                dft<R, -1>(v);
                float2 *dst = s_b1 + f * LD;
#pragma unroll
                for (int r = 0; r < R; ++r) dst[pad16(stockham_out<R, NS>(j, r))] = v[r];
            }
            __syncthreads();
        }
        const float2 *Z = FP::NP == 3 ? s_b1 : s_b0;
        for (int sl = tid; sl < NB * CN; sl += kBlock) {
            const int f = sl / CN, k = sl - f * CN;
            const int ap = ap0 + b0 + f;
            const float2 zk = Z[f * LD + pad16(k)];
            const float2 zm = Z[f * LD + pad16((CN - k) & (CN - 1))];
            const float2 zc = make_float2(zm.x, -zm.y);
            const float2 ev = cscale(cadd(zk, zc), 0.5f);
            const float2 d = csub(zk, zc);
            const float2 od = make_float2(0.5f * d.y, -0.5f * d.x);   // -(i/2) d
            const float2 X = cadd(ev, cmul(s_twM[k], od));
            if (a.out_kind == 0) {
                int qr = (int)rintf(X.x * a.scale);
                int qi = (int)rintf(X.y * a.scale);
                qr = qr < -7 ? -7 : (qr > 7 ? 7 : qr);
                qi = qi < -7 ? -7 : (qi > 7 ? 7 : qi);
                s_codes[k * GA + b0 + f] = (uint8_t)(((qr & 15) << 4) | (qi & 15));
            } else if (ap < a.AP) {
                a.spec[((long long)m * CN + k) * a.AP + ap] = X;
            }
        }
        __syncthreads();
    }
    if (a.out_kind == 0) {
        for (int i = tid; i < CN * GA; i += kBlock) {
            const int k = i / GA, b = i - k * GA;
            const int ap = ap0 + b;
            if (ap < a.AP) a.codes[((long long)m * CN + k) * a.AP + ap] = s_codes[i];
        }
    }
}

// ---------------------------------------------------------------------------
// Four-step variant for C = 1024 channels (M = 2048) and 8 taps, the
// benchmark F-stage.  One CTA streams one antenna-pol through kPfbFrames
// consecutive frames:
//   FIR   thread t owns samples 4t..4t+3 of every frame; the last 8 frames of
//         those samples (the FIR window) stay in registers and the filter in
//         shared memory, so each ADC byte is read once and each frame costs
//         one 4-byte load, eight 16-byte shared loads and 32 FMAs per thread.
//         16 frames go to shared memory as z[n] = s[2n] + i s[2n+1].
//   FFT   each warp transforms one frame: z[l + 32 n2] -> 32-point DFT over
//         n2 in registers, twiddle w^{l k2} (w = exp(-2 pi i / 1024)), a
//         32 x 32 transpose through the frame's own shared-memory rows, a
//         second 32-point DFT -> Z[j + 32 k1] in lane j.  No CTA barrier
//         inside the transform.
//   split X[k] = (Z[k] + conj Z[C-k]) / 2 - (i/2) exp(-2 pi i k / M)
//         (Z[k] - conj Z[C-k]) with Z[C-k] taken from lane (32 - j) % 32 by
//         shuffle; requantised (or raw) outputs go out stream-major
//         [AP][F][C] in 32-byte runs, and k_to_time_major reorders them.
constexpr int kPfbFrames = 256;    // frames per CTA unless PfbArgs::frames_per_cta says otherwise (64 -> 256:
                                   // 10.3 -> 9.9 ms per benchmark step, fewer filter-window warm-ups and set-ups)
constexpr int kPfbBatch = 16;      // frames per FIR / transform round (one warp each)
constexpr int kPfbThreads = 512;
constexpr int kPfbLdz = 32 * 33;   // float2 per frame row block (transpose padding)

// The radix-32 twiddles exp(S 2 pi i k / 32), k = 1, 3: cos / sin of pi/16, 3 pi/16.
#define MOFF_C32 0.98078528040323044913f
#define MOFF_S32 0.19509032201612826785f
#define MOFF_C32_3 0.83146961230254523708f
#define MOFF_S32_3 0.55557023301960222474f

// In-register 32-point DFT, natural order in and out: two 16-point DFTs of
// the even and odd elements and one radix-2 step.
template <int S>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
    }
    dft<16, S>(e);
    dft<16, S>(o);
    o[1] = rot<S>(o[1], MOFF_C32, MOFF_S32);
    o[2] = rot<S>(o[2], MOFF_C16, MOFF_S16);
    o[3] = rot<S>(o[3], MOFF_C32_3, MOFF_S32_3);
    o[4] = rot<S>(o[4], MOFF_C8, MOFF_C8);
    o[5] = rot<S>(o[5], MOFF_S32_3, MOFF_C32_3);
    o[6] = rot<S>(o[6], MOFF_S16, MOFF_C16);
    o[7] = rot<S>(o[7], MOFF_S32, MOFF_C32);
    o[8] = mul_si<S>(o[8]);
    o[9] = rot<S>(o[9], -MOFF_S32, MOFF_C32);
    o[10] = rot<S>(o[10], -MOFF_S16, MOFF_C16);
    o[11] = rot<S>(o[11], -MOFF_S32_3, MOFF_C32_3);
    o[12] = rot<S>(o[12], -MOFF_C8, MOFF_C8);
    o[13] = rot<S>(o[13], -MOFF_C32_3, MOFF_S32_3);
    o[14] = rot<S>(o[14], -MOFF_C16, MOFF_S16);
    o[15] = rot<S>(o[15], -MOFF_C32, MOFF_S32);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = cadd(e[i], o[i]);
        v[i + 16] = csub(e[i], o[i]);
    }
}

__device__ __forceinline__ uint8_t quant4(float2 X, float scale) {
    int qr = (int)rintf(X.x * scale);
    int qi = (int)rintf(X.y * scale);
    qr = qr < -7 ? -7 : (qr > 7 ? 7 : qr);
    qi = qi < -7 ? -7 : (qi > 7 ? 7 : qi);
    return (uint8_t)(((qr & 15) << 4) | (qi & 15));
}

__global__ void __launch_bounds__(kPfbThreads, 1) k_pfb1024(const PfbArgs a) {
    constexpr int CN = 1024, M = 2048, NT = 8;
    const int ap = blockIdx.y;
    const int fpc = a.frames_per_cta > 0 ? a.frames_per_cta : kPfbFrames;
    const int m0 = blockIdx.x * fpc;
    const int m_end = min(a.F, m0 + fpc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *s_z = reinterpret_cast<float2 *>(smem);                 // [kPfbBatch][kPfbLdz]
    float2 *s_tw = s_z + kPfbBatch * kPfbLdz;                        // [32 k2][32 l]
    float2 *s_twM = s_tw + 1024;                                     // exp(-2 pi i k / M)
    float4 *s_h = reinterpret_cast<float4 *>(s_twM + 1024);          // [NT][M / 4]
    for (int i = tid; i < 1024; i += kPfbThreads) {
        s_tw[i] = a.tw4[i];
        s_twM[i] = a.twM[i];
    }
    for (int i = tid; i < NT * M / 4; i += kPfbThreads) s_h[i] = reinterpret_cast<const float4 *>(a.h)[i];

    // ---- FIR window: the last 8 frames of samples 4 tid .. 4 tid + 3
    const int8_t *x = a.adc + (long long)ap * a.S + 4 * tid;
    float w[NT][4];
    auto load_frame = [&](int f, float (&dst)[4]) {
        const uint32_t b = *reinterpret_cast<const uint32_t *>(x + (long long)f * M);
        dst[0] = (float)(int8_t)(b & 0xffu);
        dst[1] = (float)(int8_t)((b >> 8) & 0xffu);
        dst[2] = (float)(int8_t)((b >> 16) & 0xffu);
        dst[3] = (float)(int8_t)(b >> 24);
    };
#pragma unroll
    for (int p = 0; p < NT - 1; ++p) load_frame(m0 + p, w[p]);
    __syncthreads();

    for (int mb = m0; mb < m_end; mb += kPfbBatch) {
        // ---- FIR of frames mb .. mb + 15 (window slot of frame m0 + i is i % 8); the
        // batch's 16 new 4-byte loads are all issued before the first is used
        uint32_t raw[kPfbBatch];
#pragma unroll
        for (int u = 0; u < kPfbBatch; ++u)
            raw[u] = mb + u < m_end ? *reinterpret_cast<const uint32_t *>(x + (long long)(mb + u + NT - 1) * M) : 0u;
#pragma unroll
        for (int u = 0; u < kPfbBatch; ++u) {
            if (mb + u < m_end) {
                {
                    float (&d)[4] = w[(u + NT - 1) % NT];
                    const uint32_t b = raw[u];
                    d[0] = (float)(int8_t)(b & 0xffu);
                    d[1] = (float)(int8_t)((b >> 8) & 0xffu);
                    d[2] = (float)(int8_t)((b >> 16) & 0xffu);
                    d[3] = (float)(int8_t)(b >> 24);
                }
                float sacc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int p = 0; p < NT; ++p) {
                    const float4 hq = s_h[p * (M / 4) + tid];
                    sacc[0] = fmaf(hq.x, w[(u + p) % NT][0], sacc[0]);
                    sacc[1] = fmaf(hq.y, w[(u + p) % NT][1], sacc[1]);
                    sacc[2] = fmaf(hq.z, w[(u + p) % NT][2], sacc[2]);
                    sacc[3] = fmaf(hq.w, w[(u + p) % NT][3], sacc[3]);
                }
                *reinterpret_cast<float4 *>(s_z + u * kPfbLdz + 2 * tid) = make_float4(sacc[0], sacc[1], sacc[2], sacc[3]);
            }
        }
        __syncthreads();
        // ---- one warp per frame: four-step 1024-point transform, split, output
        const int m = mb + warp;
        if (m < m_end) {
            float2 *zf = s_z + warp * kPfbLdz;
            float2 v[32];
#pragma unroll
            for (int n2 = 0; n2 < 32; ++n2) v[n2] = zf[lane + 32 * n2];
            dft32<-1>(v);
#pragma unroll
            for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], s_tw[k2 * 32 + lane]);
            __syncwarp();
#pragma unroll
            for (int k2 = 0; k2 < 32; ++k2) zf[k2 * 33 + lane] = v[k2];
            __syncwarp();
#pragma unroll
            for (int l = 0; l < 32; ++l) v[l] = zf[lane * 33 + l];
            dft32<-1>(v);   // v[k1] = Z[lane + 32 k1]
            const int partner = (32 - lane) & 31;
            const long long obase = ((long long)ap * a.F + m) * CN + lane;
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) {
                float2 zm;
                zm.x = __shfl_sync(0xffffffffu, v[31 - k1].x, partner);
                zm.y = __shfl_sync(0xffffffffu, v[31 - k1].y, partner);
                if (lane == 0) zm = v[(32 - k1) & 31];
                const float2 zk = v[k1];
                const float2 zc = make_float2(zm.x, -zm.y);
                const float2 ev = cscale(cadd(zk, zc), 0.5f);
                const float2 d = csub(zk, zc);
                const float2 od = make_float2(0.5f * d.y, -0.5f * d.x);   // -(i/2) d
                const float2 X = cadd(ev, cmul(s_twM[lane + 32 * k1], od));
                if (a.out_kind == 0)
                    a.codes_sm[obase + 32 * k1] = quant4(X, a.scale);
                else
                    a.spec_sm[obase + 32 * k1] = X;
            }
        }
        __syncthreads();
    }
}

size_t pfb1024_smem_bytes() { return ((size_t)kPfbBatch * kPfbLdz + 2048) * sizeof(float2) + 8 * 2048 * sizeof(float); }

// [AP][F][C] -> [F][C][AP] in 32 x 32 tiles (tile = 32 streams x 32 channels of one frame).
template <class T>
__global__ void __launch_bounds__(256) k_to_time_major(const T *__restrict__ in, T *__restrict__ out, int AP, int F,
                                                       int C) {
    __shared__ T tile[32][33];
    const int c0 = blockIdx.x * 32, ap0 = blockIdx.y * 32, f = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        const int ap = ap0 + r, c = c0 + tx;
        if (ap < AP && c < C) tile[r][tx] = in[((long long)ap * F + f) * C + c];
    }
    __syncthreads();
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        const int c = c0 + r, ap = ap0 + tx;
        if (ap < AP && c < C) out[((long long)f * C + c) * AP + ap] = tile[tx][r];
    }
}

cudaError_t launch_pfb1024(const PfbArgs &a, cudaStream_t st) {
    const size_t smem = pfb1024_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_pfb1024, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int fpc = a.frames_per_cta > 0 ? a.frames_per_cta : kPfbFrames;
    if (fpc % kPfbBatch) return cudaErrorInvalidValue;
    k_pfb1024<<<dim3((a.F + fpc - 1) / fpc, a.AP), kPfbThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// Byte reorder with 16-byte accesses: a CTA moves a 64-stream x 64-channel tile of
// one frame; each thread loads 16 channels of one stream and stores 16 streams of
// one channel.  Needs AP a multiple of 64 (C is 1024 here).
__global__ void __launch_bounds__(256) k_to_time_major_u8x16(const uint8_t *__restrict__ in, uint8_t *__restrict__ out,
                                                             int AP, int F, int C) {
    __shared__ __align__(16) uint8_t tile[64][64 + 16];
    const int c0 = blockIdx.x * 64, ap0 = blockIdx.y * 64, f = blockIdx.z;
    const int tid = threadIdx.x;
    {
        const int r = tid >> 2, q = tid & 3;      // stream ap0 + r, channels c0 + 16 q ..
        const uint4 v = *reinterpret_cast<const uint4 *>(in + ((long long)(ap0 + r) * F + f) * C + c0 + 16 * q);
        *reinterpret_cast<uint4 *>(&tile[r][16 * q]) = v;
    }
    __syncthreads();
    {
        const int cc = tid >> 2, q = tid & 3;     // channel c0 + cc, streams ap0 + 16 q ..
        uint32_t w[4];
#pragma unroll
        for (int b = 0; b < 4; ++b)
            w[b] = (uint32_t)tile[16 * q + 4 * b][cc] | ((uint32_t)tile[16 * q + 4 * b + 1][cc] << 8) |
                   ((uint32_t)tile[16 * q + 4 * b + 2][cc] << 16) | ((uint32_t)tile[16 * q + 4 * b + 3][cc] << 24);
        *reinterpret_cast<uint4 *>(out + ((long long)f * C + c0 + cc) * AP + ap0 + 16 * q) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

cudaError_t launch_pfb_reorder(const PfbArgs &a, cudaStream_t st) {
    if (a.out_kind == 0 && a.AP % 64 == 0 && ((uintptr_t)a.codes & 15) == 0 && ((uintptr_t)a.codes_sm & 15) == 0) {
        k_to_time_major_u8x16<<<dim3(1024 / 64, a.AP / 64, a.F), 256, 0, st>>>(a.codes_sm, a.codes, a.AP, a.F, 1024);
        return cudaGetLastError();
    }
    const dim3 tg((1024 + 31) / 32, (a.AP + 31) / 32, a.F);
    if (a.out_kind == 0)
        k_to_time_major<uint8_t><<<tg, 256, 0, st>>>(a.codes_sm, a.codes, a.AP, a.F, 1024);
    else
        k_to_time_major<float2><<<tg, 256, 0, st>>>(a.spec_sm, a.spec, a.AP, a.F, 1024);
    return cudaGetLastError();
}

template <int CN>
size_t pfb_smem_t() {
    using S = PfbShape<CN>;
    return (size_t)FftTw<CN>::TOTAL * 8 + (size_t)CN * 8 + 2 * (size_t)S::NB * S::LD * 8 + (size_t)CN * kPfbGroup;
}

template <int CN>
cudaError_t launch_pfb_t(const PfbArgs &a, cudaStream_t st) {
    auto k = k_pfb<CN>;
    const size_t smem = pfb_smem_t<CN>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3((a.AP + kPfbGroup - 1) / kPfbGroup, a.F), kBlock, smem, st>>>(a);
    return cudaGetLastError();
}

size_t pfb_smem_bytes(int CN) {
    switch (CN) {
        case 32: return pfb_smem_t<32>();
        case 64: return pfb_smem_t<64>();
        case 128: return pfb_smem_t<128>();
        case 256: return pfb_smem_t<256>();
        case 512: return pfb_smem_t<512>();
        case 1024: return pfb_smem_t<1024>();
        case 2048: return pfb_smem_t<2048>();
    }
    return 0;
}

cudaError_t launch_pfb(int CN, const PfbArgs &a, cudaStream_t st) {
    switch (CN) {
        case 32: return launch_pfb_t<32>(a, st);
        case 64: return launch_pfb_t<64>(a, st);
        case 128: return launch_pfb_t<128>(a, st);
        case 256: return launch_pfb_t<256>(a, st);
        case 512: return launch_pfb_t<512>(a, st);
        case 1024: return launch_pfb_t<1024>(a, st);
        case 2048: return launch_pfb_t<2048>(a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace moff
