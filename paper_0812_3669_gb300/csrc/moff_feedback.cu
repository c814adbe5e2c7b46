// moff_feedback.cu -- feedback calibration sums of Morales (arXiv 0812.3669),
// Sec. 6: correlate the electric-field image pixel towards a calibrator with
// every antenna's calibrated signal (Eq. FBeq2) and sum the pixel's power
// (Eq. FBeq1), then form the gain-error estimate.
//
// The column kernel (k_cols_acc) taps E_t,p(k_cal) for every sample of a
// chunk into etap[t][c][p]; k_fb_corr then accumulates, per (channel,
// antenna-pol),  sum_t E_t,p(k_cal) conj(y_t,a,p)  (FP32 over the chunk,
// FP64 across chunks) and the pixel power sum_t |E_t,p(k_cal)|^2.  The
// antenna's beam towards the pixel, B_a,p (its kernel placed and transformed,
// built on the host in FP64), is applied when the sums are read:
//   R_a,p = conj(B_a,p) sum_t E_t,p conj(y_t,a,p).
// The estimate uses N (the antenna count) where the paper prints 2N, and the
// conjugated ratio:  delta_g = g (1 - N conj(R) / S).
//
// Also here: the autocorrelation part of the image (the a = b terms of
// <|sum_a c_a|^2>_t), so that it can be subtracted to leave the baselines-only
// image of software holography (Sec. 3).  Since an antenna's share of pixel k
// is y_a K^_a(k) exp(+2 pi i k.anchor_a / N), its own term is
// |y_a|^2 |K^_a(k)|^2 (or y_ax conj(y_ay) K^_ax conj(K^_ay) for XY): the
// position drops out, and sum_a P_a K^_a conj(K^_a') is the transform of the
// power-weighted sum of the antennas' kernel cross-correlation patches
// ((2K-1)^2 offsets), done separably in FP64.
#include <algorithm>

#include "moff_internal.h"

namespace moff {
namespace {

__device__ __forceinline__ float2 fb_decode4(uint32_t b) {
    const int hi = (int)((b >> 4) & 15u), lo = (int)(b & 15u);
    return make_float2((float)(hi - ((hi & 8) << 1)), (float)(lo - ((lo & 8) << 1)));
}

// One thread per (antenna-pol i, channel cl) of a chunk of nt samples.
__global__ void __launch_bounds__(256) k_fb_corr(const FbArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int cl = blockIdx.y, c = a.c0 + cl;
    if (i >= a.AP) return;
    const int p = i % a.P;
    const float2 g = a.gains[(long long)c * a.AP + i];
    const uint8_t *v = a.volt + (long long)a.t0 * a.tstride + (long long)c * a.AP + i;
    float re = 0.f, im = 0.f, pw = 0.f;
    for (int t = 0; t < a.nt; ++t) {
        const float2 e = a.etap[((long long)t * a.nc + cl) * a.P + p];
        const float2 x = fb_decode4(v[(long long)t * a.tstride]);
        const float2 y = make_float2(g.x * x.x - g.y * x.y, g.x * x.y + g.y * x.x);
        re = fmaf(e.x, y.x, fmaf(e.y, y.y, re));      // e conj(y)
        im = fmaf(e.y, y.x, fmaf(-e.x, y.y, im));
        if (i < a.P) pw = fmaf(e.x, e.x, fmaf(e.y, e.y, pw));
    }
    double2 *r = a.corr + (long long)c * a.AP + i;
    r->x += (double)re;
    r->y += (double)im;
    if (i < a.P) a.power[(long long)c * a.P + p] += (double)pw;
}

// R = conj(B) * sums (FP64), written as float2; and, if delta is set, the
// gain-error estimate g (1 - N conj(R) / S) (added to the gains if apply).
__global__ void k_fb_finish(const double2 *__restrict__ corr, const double *__restrict__ power,
                            const double2 *__restrict__ beam, const int *__restrict__ chan_group, float2 *gains,
                            int C, int AP, int P, int n_ant, float2 *__restrict__ r_out, float2 *__restrict__ delta,
                            int apply) {
    const long long n = (long long)C * AP;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % AP), c = (int)(k / AP), p = i % P;
        const double2 s = corr[k], b = beam[(chan_group ? (long long)chan_group[c] * AP : 0) + i];
        const double rr = b.x * s.x + b.y * s.y, ri = b.x * s.y - b.y * s.x;   // conj(b) s
        if (r_out) r_out[k] = make_float2((float)rr, (float)ri);
        if (delta) {
            const double S = power[(long long)c * P + p];
            const float2 g = gains[k];
            // 1 - N conj(R) / S
            const double fr = S > 0.0 ? 1.0 - n_ant * rr / S : 0.0, fi = S > 0.0 ? n_ant * ri / S : 0.0;
            const float2 d = make_float2((float)(g.x * fr - g.y * fi), (float)(g.x * fi + g.y * fr));
            delta[k] = d;
            if (apply) gains[k] = make_float2(g.x + d.x, g.y + d.y);
        }
    }
}

// Autocorrelation sums of one chunk: per (channel, antenna) the products
// |y_x|^2, |y_y|^2 and y_x conj(y_y) (one pol: |y|^2) summed over the samples.
__global__ void __launch_bounds__(256) k_auto_acc(const FbArgs a) {
    const int an = blockIdx.x * blockDim.x + threadIdx.x;
    const int cl = blockIdx.y, c = a.c0 + cl;
    const int A = a.AP / a.P;
    if (an >= A) return;
    const long long gi = (long long)c * a.AP + (long long)an * a.P;
    const float2 gx = a.gains[gi], gy = a.P == 2 ? a.gains[gi + 1] : make_float2(0.f, 0.f);
    const uint8_t *v = a.volt + (long long)a.t0 * a.tstride + gi;
    float xx = 0.f, yy = 0.f, xr = 0.f, xi = 0.f;
    for (int t = 0; t < a.nt; ++t) {
        const uint8_t *vt = v + (long long)t * a.tstride;
        const float2 u = fb_decode4(vt[0]);
        const float2 y0 = make_float2(gx.x * u.x - gx.y * u.y, gx.x * u.y + gx.y * u.x);
        xx = fmaf(y0.x, y0.x, fmaf(y0.y, y0.y, xx));
        if (a.P == 2) {
            const float2 w = fb_decode4(vt[1]);
            const float2 y1 = make_float2(gy.x * w.x - gy.y * w.y, gy.x * w.y + gy.y * w.x);
            yy = fmaf(y1.x, y1.x, fmaf(y1.y, y1.y, yy));
            xr = fmaf(y0.x, y1.x, fmaf(y0.y, y1.y, xr));       // y0 conj(y1)
            xi = fmaf(y0.y, y1.x, fmaf(-y0.x, y1.y, xi));
        }
    }
    double2 *o = a.corr + ((long long)c * A + an) * 3;
    o[0].x += (double)xx;
    if (a.P == 2) {
        o[1].x += (double)yy;
        o[2].x += (double)xr;
        o[2].y += (double)xi;
    }
}

// Q[c][q][u] = sum_a pw[c][a][q] X[a][q][u]: the antennas' kernel cross-correlation
// patches weighted by their autocorrelation sums (FP64).  One thread per (q, u) of a channel.
// With channel-dependent kernels, X holds one [A][NQ][U] block per set and chan_group[c] picks it.
__global__ void k_auto_patch(const double2 *__restrict__ pw, const double2 *__restrict__ X,
                             const int *__restrict__ chan_group, int A, int NQ, int U, double2 *__restrict__ Q) {
    const int c = blockIdx.y;
    if (chan_group) X += (long long)chan_group[c] * A * NQ * U;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;    // q * U + u
    if (k >= NQ * U) return;
    const int q = k / U;
    double re = 0.0, im = 0.0;
    for (int an = 0; an < A; ++an) {
        const double2 w = pw[((long long)c * A + an) * 3 + q];
        const double2 x = X[((long long)an * NQ + q) * U + (k - q * U)];
        re += w.x * x.x - w.y * x.y;
        im += w.x * x.y + w.y * x.x;
    }
    Q[(long long)c * NQ * U + k] = make_double2(re, im);
}

// img[c][prod][ky][kx] = sum_u Q[c][q][u] exp(+2 pi i (ky uy + kx ux) / N), separably:
// a CTA per (channel, q, 64-column tile) first folds ux, then uy.  q = 0 (XX or the
// one pol) and 1 (YY) are real images; q = 2 (XY) gives Re -> product 2, Im -> 3.
__global__ void __launch_bounds__(256) k_auto_image(const double2 *__restrict__ Q, int NQ, int K, int N,
                                                    const double2 *__restrict__ wN, double *__restrict__ img,
                                                    int nprod) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = 2 * K - 1, U = L * L, h = K - 1;
    const int c = blockIdx.z, q = blockIdx.y, kx0 = blockIdx.x * 64;
    double2 *s_w = reinterpret_cast<double2 *>(smem);          // [N]
    double2 *s_q = s_w + N;                                     // [U]
    double2 *s_t = s_q + U;                                     // [L][64]
    for (int i = threadIdx.x; i < N; i += blockDim.x) s_w[i] = wN[i];
    for (int i = threadIdx.x; i < U; i += blockDim.x) s_q[i] = Q[((long long)c * NQ + q) * U + i];
    __syncthreads();
    for (int i = threadIdx.x; i < L * 64; i += blockDim.x) {
        const int uy = i / 64, kx = kx0 + (i % 64);
        double re = 0.0, im = 0.0;
        if (kx < N)
            for (int ux = 0; ux < L; ++ux) {
                const double2 v = s_q[uy * L + ux];
                const double2 w = s_w[(((long long)kx * (ux - h)) % N + N) % N];
                re += v.x * w.x - v.y * w.y;
                im += v.x * w.y + v.y * w.x;
            }
        s_t[i] = make_double2(re, im);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N * 64; i += blockDim.x) {
        const int ky = i / 64, kl = i % 64, kx = kx0 + kl;
        if (kx >= N) continue;
        double re = 0.0, im = 0.0;
        for (int uy = 0; uy < L; ++uy) {
            const double2 v = s_t[uy * 64 + kl];
            const double2 w = s_w[(((long long)ky * (uy - h)) % N + N) % N];
            re += v.x * w.x - v.y * w.y;
            im += v.x * w.y + v.y * w.x;
        }
        const long long pix = (long long)ky * N + kx;
        if (q < 2) {
            img[((long long)c * nprod + q) * N * N + pix] = re;
        } else {
            img[((long long)c * nprod + 2) * N * N + pix] = re;
            img[((long long)c * nprod + 3) * N * N + pix] = im;
        }
    }
}

__global__ void k_sub_to_f32(const double *__restrict__ acc, const double *__restrict__ sub, float *__restrict__ out,
                             long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)(acc[i] - sub[i]);
}

}  // namespace

cudaError_t launch_auto_acc(const FbArgs &a, cudaStream_t st) {
    k_auto_acc<<<dim3((a.AP / a.P + 255) / 256, a.nc), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_auto_image(const double2 *pw, const double2 *X, const int *chan_group, int C, int A, int P, int K,
                              int N, const double2 *wN, double2 *Q, double *img, cudaStream_t st) {
    const int NQ = P == 1 ? 1 : 3, L = 2 * K - 1, U = L * L;
    k_auto_patch<<<dim3((NQ * U + 255) / 256, C), 256, 0, st>>>(pw, X, chan_group, A, NQ, U, Q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = ((size_t)N + U + (size_t)L * 64) * sizeof(double2);
    e = cudaFuncSetAttribute(k_auto_image, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_auto_image<<<dim3((N + 63) / 64, NQ, C), 256, smem, st>>>(Q, NQ, K, N, wN, img, P == 1 ? 1 : 4);
    return cudaGetLastError();
}

cudaError_t launch_sub_to_f32(const double *acc, const double *sub, float *out, long long n, cudaStream_t st) {
    const int blocks = (int)std::min<long long>((n + 255) / 256, 8192);
    k_sub_to_f32<<<blocks, 256, 0, st>>>(acc, sub, out, n);
    return cudaGetLastError();
}

cudaError_t launch_fb_corr(const FbArgs &a, cudaStream_t st) {
    k_fb_corr<<<dim3((a.AP + 255) / 256, a.nc), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fb_finish(const double2 *corr, const double *power, const double2 *beam, const int *chan_group,
                             float2 *gains, int C, int AP, int P, int n_ant, float2 *r_out, float2 *delta, int apply,
                             cudaStream_t st) {
    const long long n = (long long)C * AP;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    k_fb_finish<<<blocks, 256, 0, st>>>(corr, power, beam, chan_group, gains, C, AP, P, n_ant, r_out, delta, apply);
    return cudaGetLastError();
}

}  // namespace moff
