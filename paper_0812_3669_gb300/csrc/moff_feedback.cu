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
                            const double2 *__restrict__ beam, float2 *gains, int C, int AP, int P, int n_ant,
                            float2 *__restrict__ r_out, float2 *__restrict__ delta, int apply) {
    const long long n = (long long)C * AP;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % AP), c = (int)(k / AP), p = i % P;
        const double2 s = corr[k], b = beam[i];
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

}  // namespace

cudaError_t launch_fb_corr(const FbArgs &a, cudaStream_t st) {
    k_fb_corr<<<dim3((a.AP + 255) / 256, a.nc), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fb_finish(const double2 *corr, const double *power, const double2 *beam, float2 *gains, int C,
                             int AP, int P, int n_ant, float2 *r_out, float2 *delta, int apply, cudaStream_t st) {
    const long long n = (long long)C * AP;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    k_fb_finish<<<blocks, 256, 0, st>>>(corr, power, beam, gains, C, AP, P, n_ant, r_out, delta, apply);
    return cudaGetLastError();
}

}  // namespace moff
