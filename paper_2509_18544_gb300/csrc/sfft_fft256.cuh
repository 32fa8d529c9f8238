// 256-point complex FFT by the 16 lanes of a half-warp, FP32 with split (hi + lo) twiddles
// or FP64: the transform of the row-segment FFTs (K1) and of the FFT route of the
// convolutions.  Radix 16 x 16: a 16-point DFT in registers (radix 4 x 4), a twiddle, one
// padded shared-memory transpose, a second 16-point DFT.
#pragma once

#include "sfft_internal.cuh"

namespace sfft {
namespace {

constexpr int kP = 256;

// forward 4-point DFT in place
template <class R>
__device__ __forceinline__ void dft4(cpx<R> &a0, cpx<R> &a1, cpx<R> &a2, cpx<R> &a3) {
    cpx<R> s02 = a0 + a2, d02 = a0 - a2, s13 = a1 + a3, d13 = a1 - a3;
    a0 = s02 + s13;
    a2 = s02 - s13;
    a1 = {d02.re + d13.im, d02.im - d13.re};  // d02 - i d13
    a3 = {d02.re - d13.im, d02.im + d13.re};  // d02 + i d13
}

// v * w with the twiddle held as w = wh + wl (wl = FP32 remainder of the FP64 value).
// FP32-rounded twiddles alone have |wh| != 1, which scales the energy of every product by
// |wh|^2 -- a bias of ~-5e-8 that never averages out because the radix-16 stages reuse a
// handful of twiddles; with the remainder folded into FMAs each product is rounded once
// from (nearly) the exact value and the rounding is unbiased.
__device__ __forceinline__ cpx<float> twmul(cpx<float> v, cpx<float> wh, cpx<float> wl) {
    float tr = fmaf(v.re, wl.re, -v.im * wl.im);
    float ti = fmaf(v.re, wl.im, v.im * wl.re);
    return {fmaf(v.re, wh.re, fmaf(-v.im, wh.im, tr)), fmaf(v.re, wh.im, fmaf(v.im, wh.re, ti))};
}
__device__ __forceinline__ cpx<double> twmul(cpx<double> v, cpx<double> wh, cpx<double>) { return cmul(v, wh); }

// forward 16-point DFT of v[0..15] in natural order; tw[m] = exp(-2 pi i m / 256) (high
// part) and twl[m] its remainder, so exp(-2 pi i m / 16) = tw[16 m] + twl[16 m]
template <class R>
__device__ __forceinline__ void dft16(cpx<R> (&v)[16], const cpx<R> *tw, const cpx<R> *twl) {
    // v[j1 + 4 j2]: 4-point DFTs over j2 for each j1 -> U[j1][k1] kept at v[j1 + 4 k1]
#pragma unroll
    for (int j1 = 0; j1 < 4; j1++) dft4(v[j1], v[j1 + 4], v[j1 + 8], v[j1 + 12]);
#pragma unroll
    for (int j1 = 1; j1 < 4; j1++)
#pragma unroll
        for (int k1 = 1; k1 < 4; k1++) v[j1 + 4 * k1] = twmul(v[j1 + 4 * k1], tw[16 * j1 * k1], twl[16 * j1 * k1]);
    // 4-point DFTs over j1 for each k1 -> V[k1 + 4 k2] kept at v[4 k1 + k2]... gather first
    cpx<R> t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
        cpx<R> a0 = v[0 + 4 * k1], a1 = v[1 + 4 * k1], a2 = v[2 + 4 * k1], a3 = v[3 + 4 * k1];
        dft4(a0, a1, a2, a3);
        t[k1 + 0] = a0;
        t[k1 + 4] = a1;
        t[k1 + 8] = a2;
        t[k1 + 12] = a3;
    }
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = t[k];
}

// one 256-point complex FFT by the 16 lanes (t = lane & 15) of a half-warp: v[jj] holds
// z[t + 16 jj] on entry and X[t + 16 k2] in v[k2] on exit; e is this FFT's 16 x 17 exchange
// buffer, msk the lanes of the warp that take part.
template <class R>
__device__ __forceinline__ void fft256(cpx<R> (&v)[16], int t, cpx<R> *e, const cpx<R> *tw, const cpx<R> *twl,
                                       unsigned msk) {
    // X[k1 + 16 k2] = sum_t W16^{t k2} W256^{t k1} sum_jj x[t + 16 jj] W16^{jj k1}
    dft16(v, tw, twl);
#pragma unroll
    for (int k1 = 1; k1 < 16; k1++) v[k1] = twmul(v[k1], tw[(t * k1) & (kP - 1)], twl[(t * k1) & (kP - 1)]);
#pragma unroll
    for (int k1 = 0; k1 < 16; k1++) e[k1 * 17 + t] = v[k1];
    __syncwarp(msk);
#pragma unroll
    for (int tt = 0; tt < 16; tt++) v[tt] = e[t * 17 + tt];
    dft16(v, tw, twl);  // now over tt: X[t + 16 k2] = v[k2]
    __syncwarp(msk);
}

// ---------------------------------------------------------------- FP32 form
// The same transform with the 16-point DFTs' twiddles W16^m as split constants (no shared
// loads) and the middle twiddles from a table laid out per (k1, lane):
//   tw4[(k1 - 1) 16 + t] = (wh.re, wh.im, wl.re, wl.im) of W256^(t k1),  k1 = 1..15,
// so the 16 lanes read 16 consecutive entries (no bank conflicts) with one 16-byte load.
constexpr int kTw4 = 15 * 16;  // entries of tw4

// tw4 from the split table tw_g (tw_g[m] = high part of exp(-2 pi i m / 256), tw_g[256 + m]
// its remainder), by the threads of a CTA (the caller synchronises)
__device__ __forceinline__ void fill_tw4(float4 *tw4, const float2 *__restrict__ tw_g) {
    for (int i = threadIdx.x; i < kTw4; i += blockDim.x) {
        const int m = ((i >> 4) + 1) * (i & 15);
        const float2 h = tw_g[m], l = tw_g[kP + m];
        tw4[i] = make_float4(h.x, h.y, l.x, l.y);
    }
}

// v W16^m for a compile-time m (after unrolling), W16 = exp(-2 pi i / 16); the constants are
// cos(pi/8), sin(pi/8) and 1/sqrt(2), each as its FP32 value and remainder (to about 2^-48)
__device__ __forceinline__ cpx<float> w16f(cpx<float> v, int m) {
    const float ch = __int_as_float(0x3F6C835E), cl = __int_as_float(0x32F328D4);  // cos(pi/8)
    const float sh = __int_as_float(0x3EC3EF15), sl = __int_as_float(0x31D5D52C);  // sin(pi/8)
    const float rh = __int_as_float(0x3F3504F3), rl = __int_as_float(0x324FE77A);  // 1/sqrt(2)
    switch (m & 15) {
        case 0: return v;
        case 1: return twmul(v, {ch, -sh}, {cl, -sl});
        case 2: return twmul(v, {rh, -rh}, {rl, -rl});
        case 3: return twmul(v, {sh, -ch}, {sl, -cl});
        case 4: return {v.im, -v.re};  // -i v
        case 6: return twmul(v, {-rh, -rh}, {-rl, -rl});
        case 9: return twmul(v, {-ch, sh}, {-cl, sl});
        default: return twmul(v, {0.f, 0.f}, {0.f, 0.f});  // not reached (m = j1 k1, j1, k1 <= 3)
    }
}

__device__ __forceinline__ void dft16f(cpx<float> (&v)[16]) {
#pragma unroll
    for (int j1 = 0; j1 < 4; j1++) dft4(v[j1], v[j1 + 4], v[j1 + 8], v[j1 + 12]);
#pragma unroll
    for (int j1 = 1; j1 < 4; j1++)
#pragma unroll
        for (int k1 = 1; k1 < 4; k1++) v[j1 + 4 * k1] = w16f(v[j1 + 4 * k1], j1 * k1);
    cpx<float> t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
        cpx<float> a0 = v[0 + 4 * k1], a1 = v[1 + 4 * k1], a2 = v[2 + 4 * k1], a3 = v[3 + 4 * k1];
        dft4(a0, a1, a2, a3);
        t[k1 + 0] = a0;
        t[k1 + 4] = a1;
        t[k1 + 8] = a2;
        t[k1 + 12] = a3;
    }
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = t[k];
}

// fft256 for FP32 with the tw4 table (same input and output order)
__device__ __forceinline__ void fft256f(cpx<float> (&v)[16], int t, cpx<float> *e, const float4 *tw4,
                                        unsigned msk) {
    dft16f(v);
#pragma unroll
    for (int k1 = 1; k1 < 16; k1++) {
        const float4 w = tw4[(k1 - 1) * 16 + t];
        v[k1] = twmul(v[k1], {w.x, w.y}, {w.z, w.w});
    }
#pragma unroll
    for (int k1 = 0; k1 < 16; k1++) e[k1 * 17 + t] = v[k1];
    __syncwarp(msk);
#pragma unroll
    for (int tt = 0; tt < 16; tt++) v[tt] = e[t * 17 + tt];
    dft16f(v);
    __syncwarp(msk);
}

}  // namespace
}  // namespace sfft
