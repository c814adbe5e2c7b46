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
