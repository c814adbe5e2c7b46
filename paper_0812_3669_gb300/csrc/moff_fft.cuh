// moff_fft.cuh -- register/shared-memory building blocks of the batched FFTs.
//
// Eq. m6 step 3 of Morales (arXiv 0812.3669) transforms the gridded field to
// the sky; Fig. 1 (rows d-e) draws it as a power-of-two Cooley-Tukey FFT.
// Here every 1D transform of length N is a mixed-radix Stockham autosort FFT
// (radices 2..16 held in registers, shared memory between passes), so output
// lands in natural order and no bit reversal is needed.
//
// Pass p (radix R, NS = product of the earlier radices) maps slot j in
// [0, N/R) as
//     load   v[r] = x[j + r N/R]                           r = 0..R-1
//     twiddle v[r] *= w^{(j mod NS) r / (NS R)}             (w = exp(S 2 pi i))
//     v = DFT_R(v) with exp(S 2 pi i n k / R)
//     store  y[(j / NS) NS R + (j mod NS) + r NS] = v[r]
// S = +1 is the imaging transform (Eq. m6), S = -1 the F-stage channeliser
// (Eq. FFTofE).  Twiddles come from per-pass tables built on the host in
// FP64 (table[(r-1) NS + m] = exp(+2 pi i m r / (NS R))), so lanes of a warp
// read consecutive entries.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace moff {

// Complex sums as packed FP32 pairs (add/sub.rn.f32x2: one instruction, each lane rounded as its
// scalar form, so the results equal the two scalar operations bit for bit).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// a * (S i)
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a) {
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Radix twiddles exp(S 2 pi i k / 16) as constants: cos/sin of multiples of pi/8.
#define MOFF_C8 0.70710678118654752440f   /* cos(pi/4) */
#define MOFF_C16 0.92387953251128675613f  /* cos(pi/8) */
#define MOFF_S16 0.38268343236508977173f  /* sin(pi/8) */

// a * (c + S i s)
template <int S>
__device__ __forceinline__ float2 rot(float2 a, float c, float s) {
    const float ss = S > 0 ? s : -s;
    return make_float2(a.x * c - a.y * ss, a.x * ss + a.y * c);
}

template <int S>
__device__ __forceinline__ void dft2(float2 &a, float2 &b) {
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int S>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    const float2 t2 = cadd(a1, a3), t3 = mul_si<S>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <int S>
__device__ __forceinline__ void dft8(float2 &x0, float2 &x1, float2 &x2, float2 &x3, float2 &x4,
                                     float2 &x5, float2 &x6, float2 &x7) {
    float2 e0 = x0, e1 = x2, e2 = x4, e3 = x6;
    float2 o0 = x1, o1 = x3, o2 = x5, o3 = x7;
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    o1 = rot<S>(o1, MOFF_C8, MOFF_C8);
    o2 = mul_si<S>(o2);
    o3 = rot<S>(o3, -MOFF_C8, MOFF_C8);
    x0 = cadd(e0, o0); x4 = csub(e0, o0);
    x1 = cadd(e1, o1); x5 = csub(e1, o1);
    x2 = cadd(e2, o2); x6 = csub(e2, o2);
    x3 = cadd(e3, o3); x7 = csub(e3, o3);
}

template <int R, int S>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
    if constexpr (R == 2) {
        dft2<S>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<S>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        dft8<S>(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]);
    } else if constexpr (R == 16) {
        float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], e4 = v[8], e5 = v[10], e6 = v[12], e7 = v[14];
        float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7], o4 = v[9], o5 = v[11], o6 = v[13], o7 = v[15];
        dft8<S>(e0, e1, e2, e3, e4, e5, e6, e7);
        dft8<S>(o0, o1, o2, o3, o4, o5, o6, o7);
        o1 = rot<S>(o1, MOFF_C16, MOFF_S16);
        o2 = rot<S>(o2, MOFF_C8, MOFF_C8);
        o3 = rot<S>(o3, MOFF_S16, MOFF_C16);
        o4 = mul_si<S>(o4);
        o5 = rot<S>(o5, -MOFF_S16, MOFF_C16);
        o6 = rot<S>(o6, -MOFF_C8, MOFF_C8);
        o7 = rot<S>(o7, -MOFF_C16, MOFF_S16);
        v[0] = cadd(e0, o0); v[8] = csub(e0, o0);
        v[1] = cadd(e1, o1); v[9] = csub(e1, o1);
        v[2] = cadd(e2, o2); v[10] = csub(e2, o2);
        v[3] = cadd(e3, o3); v[11] = csub(e3, o3);
        v[4] = cadd(e4, o4); v[12] = csub(e4, o4);
        v[5] = cadd(e5, o5); v[13] = csub(e5, o5);
        v[6] = cadd(e6, o6); v[14] = csub(e6, o6);
        v[7] = cadd(e7, o7); v[15] = csub(e7, o7);
    } else {
        static_assert(R == 2 || R == 4 || R == 8 || R == 16, "unsupported radix");
    }
}

// Radix plan per transform length: passes R0, R1[, R2].
template <int N> struct FftPlan;
template <> struct FftPlan<32>   { static constexpr int NP = 2, R0 = 8,  R1 = 4,  R2 = 1; };
template <> struct FftPlan<64>   { static constexpr int NP = 2, R0 = 8,  R1 = 8,  R2 = 1; };
template <> struct FftPlan<128>  { static constexpr int NP = 2, R0 = 16, R1 = 8,  R2 = 1; };
template <> struct FftPlan<256>  { static constexpr int NP = 2, R0 = 16, R1 = 16, R2 = 1; };
template <> struct FftPlan<512>  { static constexpr int NP = 3, R0 = 8,  R1 = 8,  R2 = 8; };
template <> struct FftPlan<1024> { static constexpr int NP = 3, R0 = 16, R1 = 8,  R2 = 8; };
template <> struct FftPlan<2048> { static constexpr int NP = 3, R0 = 16, R1 = 16, R2 = 8; };

template <int N>
struct FftTw {
    using P = FftPlan<N>;
    static constexpr int NS1 = P::R0;                 // NS of pass 1
    static constexpr int NS2 = P::R0 * P::R1;         // NS of pass 2
    static constexpr int OFF1 = 0;
    static constexpr int LEN1 = (P::R1 - 1) * NS1;
    static constexpr int OFF2 = LEN1;
    static constexpr int LEN2 = P::NP == 3 ? (P::R2 - 1) * NS2 : 0;
    static constexpr int TOTAL = LEN1 + LEN2;
};

// Apply the pass twiddles of slot j (pass with radix R after NS points), sign S.
template <int R, int NS, int S>
__device__ __forceinline__ void twiddle(float2 (&v)[R], int j, const float2 *__restrict__ tw) {
    if constexpr (NS > 1) {
        const int m = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = tw[(r - 1) * NS + m];
            if (S < 0) w.y = -w.y;
            v[r] = cmul(v[r], w);
        }
    }
}

// Output position of element r of slot j in a Stockham pass.
template <int R, int NS>
__device__ __forceinline__ int stockham_out(int j, int r) {
    return (j / NS) * NS * R + (j % NS) + r * NS;
}

// Padded shared-memory index (one spare float2 every 16) to spread the
// strided stores of the early passes over the banks.
__device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }
template <int N>
struct PaddedLen { static constexpr int value = N + N / 16; };

// pad16(j + r*NSL) for slot j < NSL of a pass reading at stride NSL = N/R:
// the padding term splits into a per-slot part and a compile-time part.
template <int NSL>
__device__ __forceinline__ int pad_load(int j, int r) {
    if constexpr (NSL >= 16) return pad16(j) + r * (NSL + NSL / 16);
    else return j + r * NSL + ((r * NSL) >> 4);   // j + (r*NSL mod 16) < 16
}

// pad16(stockham_out<R, NS>(j, r)) with the r-dependent part at compile time.
template <int R, int NS>
__device__ __forceinline__ int pad_store(int j, int r) {
    if constexpr (NS >= 16) {
        return pad16(stockham_out<R, NS>(j, 0)) + r * (NS + NS / 16);
    } else if constexpr (NS * R >= 16) {
        const int H = (j / NS) * NS * R, L = j % NS;   // H a multiple of 16, L + (r*NS mod 16) < 16
        return H + H / 16 + L + r * NS + ((r * NS) >> 4);
    } else {
        return pad16(stockham_out<R, NS>(j, r));
    }
}

}  // namespace moff
