// moff_image_kernels.cuh -- the per-channel imaging hot path of the MOFF
// correlator (Morales, arXiv 0812.3669, Sec. 4, Eq. m6), FP32.
//
//   k_grid_rows : step 1 (complex weight per antenna), step 2 (scatter through
//                 each antenna's kernel, written as a deterministic gather per
//                 grid cell) and the first axis of step 3 (row transforms).
//                 One CTA = one stripe of grid rows of one channel; it keeps
//                 the stripe's kernel taps in shared memory and walks a chunk
//                 of time samples, so taps are read once per chunk.
//   k_cols_acc  : second axis of step 3 (column transforms) fused with step 4
//                 (|E|^2 and the cross-pol products summed over the chunk in
//                 registers, then added to FP64 accumulators).
// The row-transformed field goes through global memory between the two.
#pragma once
#include "moff_fft.cuh"
#include "moff_internal.h"

namespace moff {

// 4-bit two's-complement nibbles: real part high, imaginary part low.
__device__ __forceinline__ float2 decode4(uint32_t b) {
    const int hi = (int)((b >> 4) & 15u), lo = (int)(b & 15u);
    return make_float2((float)(hi - ((hi & 8) << 1)), (float)(lo - ((lo & 8) << 1)));
}

template <int N, int P, bool CSMEM, bool GRID_ONLY>
__global__ void __launch_bounds__(kBlock) k_grid_rows(const GridArgs a) {
    using FP = FftPlan<N>;
    using TW = FftTw<N>;
    constexpr int LDR = PaddedLen<N>::value;

    const int s = blockIdx.x;
    const int cl = blockIdx.y;
    const int c = a.c0 + cl;
    const int tid = threadIdx.x;
    const int rows = a.rows;
    const int nf = P * rows;
    const int ncell = nf * N;
    const int ant0 = a.st_ant_off[s];
    const int nloc = a.st_ant_off[s + 1] - ant0;
    const long long con0 = a.st_con_off[s];
    const int ncon = (int)(a.st_con_off[s + 1] - con0);
    const int *cell_off_g = a.st_cell_off + (long long)s * (ncell + 1);

    // Carve (matches grid_smem_bytes).
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *s_tw = reinterpret_cast<float2 *>(smem);
    float2 *s_buf0 = s_tw + TW::TOTAL;
    float2 *s_buf1 = s_buf0 + nf * LDR;
    float2 *s_y = s_buf1 + nf * LDR;
    float2 *s_g = s_y + a.max_nloc * P;
    float2 *s_tap = s_g + a.max_nloc * P;
    int *s_off = reinterpret_cast<int *>(s_tap + (CSMEM ? a.max_ncon : 0));
    int *s_ant = s_off + (ncell + 1);
    uint16_t *s_cy = reinterpret_cast<uint16_t *>(s_ant + a.max_nloc);

    for (int i = tid; i < TW::TOTAL; i += kBlock) s_tw[i] = a.twp[i];
    for (int i = tid; i <= ncell; i += kBlock) s_off[i] = cell_off_g[i];
    for (int i = tid; i < nloc; i += kBlock) s_ant[i] = a.st_ant[ant0 + i];
    for (int i = tid; i < nloc * P; i += kBlock) {
        const int la = i / P, q = i - la * P;
        const int ant = a.st_ant[ant0 + la];
        s_g[i] = a.gains[((long long)c * a.A + ant) * P + q];
    }
    if constexpr (CSMEM) {
        for (int i = tid; i < ncon; i += kBlock) {
            s_tap[i] = a.con_tap[con0 + i];
            s_cy[i] = a.con_y[con0 + i];
        }
    }
    __syncthreads();
    const float2 *tap = CSMEM ? s_tap : a.con_tap + con0;
    const uint16_t *cy = CSMEM ? s_cy : a.con_y + con0;

    for (int tt = 0; tt < a.nt; ++tt) {
        // Step 1: decode and weight the voltages of the antennas touching this stripe.
        const uint8_t *vrow = a.volt + (long long)(a.t0 + tt) * a.volt_tstride + (long long)c * a.A * P;
        for (int i = tid; i < nloc * P; i += kBlock) {
            const int la = i / P, q = i - la * P;
            s_y[i] = cmul(s_g[i], decode4(vrow[(long long)s_ant[la] * P + q]));
        }
        __syncthreads();
        // Step 2: each grid cell sums its kernel contributions in a fixed order.
        for (int cell = tid; cell < ncell; cell += kBlock) {
            float2 acc = make_float2(0.f, 0.f);
            const int k1 = s_off[cell + 1];
            for (int k = s_off[cell]; k < k1; ++k) {
                const float2 t = tap[k];
                const float2 y = s_y[cy[k]];
                acc.x = fmaf(t.x, y.x, fmaf(-t.y, y.y, acc.x));
                acc.y = fmaf(t.x, y.y, fmaf(t.y, y.x, acc.y));
            }
            const int f = cell / N, e = cell - f * N;
            s_buf0[f * LDR + pad16(e)] = acc;
        }
        __syncthreads();

        const int ry0 = s * rows;
        float2 *outc = a.out + (long long)(tt * a.nc + cl) * P * N * N;
        if constexpr (GRID_ONLY) {
            for (int i = tid; i < ncell; i += kBlock) {
                const int f = i / N, e = i - f * N;
                const int p = f / rows, rl = f - p * rows;
                outc[((long long)p * N + ry0 + rl) * N + e] = s_buf0[f * LDR + pad16(e)];
            }
            __syncthreads();
            continue;
        }

        // Step 3, first axis: N-point transform of every row (Stockham passes).
        {
            constexpr int R = FP::R0, NSL = N / R;
            for (int sl = tid; sl < nf * NSL; sl += kBlock) {
                const int f = sl / NSL, j = sl - f * NSL;
                const float2 *src = s_buf0 + f * LDR;
                float2 v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = src[pad16(j + r * NSL)];
                dft<R, 1>(v);
                float2 *dst = s_buf1 + f * LDR;
#pragma unroll
                for (int r = 0; r < R; ++r) dst[pad16(stockham_out<R, 1>(j, r))] = v[r];
            }
        }
        __syncthreads();
        if constexpr (FP::NP == 3) {
            constexpr int R = FP::R1, NS = FP::R0, NSL = N / R;
            for (int sl = tid; sl < nf * NSL; sl += kBlock) {
                const int f = sl / NSL, j = sl - f * NSL;
                const float2 *src = s_buf1 + f * LDR;
                float2 v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = src[pad16(j + r * NSL)];
                twiddle<R, NS, 1>(v, j, s_tw + TW::OFF1);
                dft<R, 1>(v);
                float2 *dst = s_buf0 + f * LDR;
#pragma unroll
                for (int r = 0; r < R; ++r) dst[pad16(stockham_out<R, NS>(j, r))] = v[r];
            }
            __syncthreads();
        }
        {
            constexpr int R = FP::NP == 3 ? FP::R2 : FP::R1;
            constexpr int NS = N / R;
            const float2 *srcb = FP::NP == 3 ? s_buf0 : s_buf1;
            const float2 *tw = s_tw + (FP::NP == 3 ? TW::OFF2 : TW::OFF1);
            for (int sl = tid; sl < nf * NS; sl += kBlock) {
                const int f = sl / NS, j = sl - f * NS;
                const float2 *src = srcb + f * LDR;
                float2 v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = src[pad16(j + r * NS)];
                twiddle<R, NS, 1>(v, j, tw);
                dft<R, 1>(v);
                const int p = f / rows, rl = f - p * rows;
                float2 *dst = outc + ((long long)p * N + ry0 + rl) * N;
#pragma unroll
                for (int r = 0; r < R; ++r) dst[j + r * NS] = v[r];
            }
        }
        __syncthreads();
    }
}

template <int N>
struct ColShape {
    using FP = FftPlan<N>;
    static constexpr int RL = FP::NP == 3 ? FP::R2 : FP::R1;   // radix of the last pass
    static constexpr int W = kBlock * RL / N;                  // columns per CTA
    static constexpr int NS = N / RL;                          // slots per column in the last pass
};

template <int N, int P>
__global__ void __launch_bounds__(kBlock) k_cols_acc(const ColArgs a) {
    using FP = FftPlan<N>;
    using TW = FftTw<N>;
    using CS = ColShape<N>;
    constexpr int W = CS::W;
    constexpr int RL = CS::RL;
    constexpr int NPROD = P == 1 ? 1 : 4;

    const int kx0 = blockIdx.x * W;
    const int cl = blockIdx.y;
    const int c = a.c0 + cl;
    const int tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *s_tw = reinterpret_cast<float2 *>(smem);
    float2 *s_a = s_tw + TW::TOTAL;            // [P][N][W]
    float2 *s_b = s_a + P * N * W;             // second buffer (3-pass lengths only)

    for (int i = tid; i < TW::TOTAL; i += kBlock) s_tw[i] = a.twp[i];

    float acc[NPROD][RL];
#pragma unroll
    for (int q = 0; q < NPROD; ++q)
#pragma unroll
        for (int r = 0; r < RL; ++r) acc[q][r] = 0.f;

    const int colL = tid % W, jL = tid / W;
    __syncthreads();

    for (int tt = 0; tt < a.nt; ++tt) {
        const float2 *Hc = a.H + (long long)(tt * a.nc + cl) * P * N * N + kx0;
        {   // pass 0: global -> registers -> shared
            constexpr int R = FP::R0, NSL = N / R;
            for (int sl = tid; sl < W * NSL; sl += kBlock) {
                const int col = sl % W, j = sl / W;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    float2 v[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) v[r] = Hc[((long long)p * N + j + r * NSL) * N + col];
                    dft<R, 1>(v);
#pragma unroll
                    for (int r = 0; r < R; ++r) s_a[(p * N + stockham_out<R, 1>(j, r)) * W + col] = v[r];
                }
            }
        }
        __syncthreads();
        if constexpr (FP::NP == 3) {
            constexpr int R = FP::R1, NS = FP::R0, NSL = N / R;
            for (int sl = tid; sl < W * NSL; sl += kBlock) {
                const int col = sl % W, j = sl / W;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    float2 v[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) v[r] = s_a[(p * N + j + r * NSL) * W + col];
                    twiddle<R, NS, 1>(v, j, s_tw + TW::OFF1);
                    dft<R, 1>(v);
#pragma unroll
                    for (int r = 0; r < R; ++r) s_b[(p * N + stockham_out<R, NS>(j, r)) * W + col] = v[r];
                }
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
            if constexpr (P == 1) {
#pragma unroll
                for (int r = 0; r < RL; ++r) acc[0][r] = fmaf(vx[r].x, vx[r].x, fmaf(vx[r].y, vx[r].y, acc[0][r]));
            } else {
                float2 vy[RL];
#pragma unroll
                for (int r = 0; r < RL; ++r) vy[r] = src[(N + jL + r * NS) * W + colL];
                twiddle<RL, NS, 1>(vy, jL, tw);
                dft<RL, 1>(vy);
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    acc[0][r] = fmaf(vx[r].x, vx[r].x, fmaf(vx[r].y, vx[r].y, acc[0][r]));
                    acc[1][r] = fmaf(vy[r].x, vy[r].x, fmaf(vy[r].y, vy[r].y, acc[1][r]));
                    acc[2][r] = fmaf(vx[r].x, vy[r].x, fmaf(vx[r].y, vy[r].y, acc[2][r]));
                    acc[3][r] = fmaf(vx[r].y, vy[r].x, fmaf(-vx[r].x, vy[r].y, acc[3][r]));
                }
            }
        }
        __syncthreads();
    }

    // Fold this chunk's FP32 sums into the FP64 accumulators (one owner per pixel).
    const int kx = kx0 + colL;
#pragma unroll
    for (int q = 0; q < NPROD; ++q) {
        double *d = a.acc + ((long long)c * NPROD + q) * N * N + kx;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            const int ky = jL + r * CS::NS;
            d[(long long)ky * N] += (double)acc[q][r];
        }
    }
}

template <int N>
size_t col_smem_bytes_t(int P) {
    using FP = FftPlan<N>;
    const size_t buf = (size_t)P * N * ColShape<N>::W * 8;
    return (size_t)FftTw<N>::TOTAL * 8 + buf * (FP::NP == 3 ? 2 : 1);
}

template <int N, int P, bool CSMEM, bool GO>
cudaError_t launch_grid_t(const GridArgs &a, int n_stripes, size_t smem, cudaStream_t st) {
    auto k = k_grid_rows<N, P, CSMEM, GO>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(n_stripes, a.nc), kBlock, smem, st>>>(a);
    return cudaGetLastError();
}

template <int N, int P>
cudaError_t launch_cols_t(const ColArgs &a, cudaStream_t st) {
    auto k = k_cols_acc<N, P>;
    const size_t smem = col_smem_bytes_t<N>(P);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(N / ColShape<N>::W, a.nc), kBlock, smem, st>>>(a);
    return cudaGetLastError();
}

#define MOFF_DEFINE_N(NN)                                                                            \
    cudaError_t launch_grid_n##NN(int P, bool csmem, bool go, const GridArgs &a, int n_stripes,        \
                                  size_t smem, cudaStream_t st) {                                    \
        if (P == 1) {                                                                                \
            if (go) return csmem ? launch_grid_t<NN, 1, true, true>(a, n_stripes, smem, st)          \
                                 : launch_grid_t<NN, 1, false, true>(a, n_stripes, smem, st);        \
            return csmem ? launch_grid_t<NN, 1, true, false>(a, n_stripes, smem, st)                 \
                         : launch_grid_t<NN, 1, false, false>(a, n_stripes, smem, st);               \
        }                                                                                            \
        if (go) return csmem ? launch_grid_t<NN, 2, true, true>(a, n_stripes, smem, st)              \
                             : launch_grid_t<NN, 2, false, true>(a, n_stripes, smem, st);            \
        return csmem ? launch_grid_t<NN, 2, true, false>(a, n_stripes, smem, st)                     \
                     : launch_grid_t<NN, 2, false, false>(a, n_stripes, smem, st);                   \
    }                                                                                                \
    cudaError_t launch_cols_n##NN(int P, const ColArgs &a, cudaStream_t st) {                        \
        return P == 1 ? launch_cols_t<NN, 1>(a, st) : launch_cols_t<NN, 2>(a, st);                   \
    }

}  // namespace moff
