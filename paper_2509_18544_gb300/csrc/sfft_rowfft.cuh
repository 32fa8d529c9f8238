// Helpers of the row-segment FFT convolutions (cross-convolution, difference image): real
// rows packed two to a 256-point complex FFT, their half spectra in 128 slots (slot 0 holds
// the real bins 0 and 128), and the way back.
#pragma once

#include "sfft_fft256.cuh"

namespace sfft {
namespace {

constexpr int kXEx = 16 * 17 + 1;  // exchange buffer of one half-warp's FFT

// After fft256 of z = x1 + i x2 (lane t holds Z[t + 16 k2] in v[k2]), split the two real
// rows' half spectra into dst1, dst2 (128 slots each, slot 0 = (X(0), X(128)), both real),
// scaled by `scale`: X1(k) = (Z(k) + conj(Z(256 - k))) / 2, X2(k) = -i (Z(k) - conj(Z(256 - k))) / 2.
__device__ __forceinline__ void unpack_pair(const cpx<float> (&v)[16], int t, cpx<float> *e, float2 *dst1,
                                            float2 *dst2, float scale, unsigned msk) {
#pragma unroll
    for (int k2 = 0; k2 < 16; k2++) e[t + 16 * k2] = v[k2];
    __syncwarp(msk);
    const float h = 0.5f * scale;
#pragma unroll
    for (int m = 0; m < 8; m++) {
        const int k = t + 16 * m;
        if (k == 0) {
            const cpx<float> z0 = e[0], zn = e[128];
            dst1[0] = make_float2(z0.re * scale, zn.re * scale);
            if (dst2) dst2[0] = make_float2(z0.im * scale, zn.im * scale);
        } else {
            const cpx<float> a = e[k], b = e[kP - k];  // B = conj(b)
            dst1[k] = make_float2((a.re + b.re) * h, (a.im - b.im) * h);
            if (dst2) dst2[k] = make_float2((a.im + b.im) * h, (b.re - a.re) * h);
        }
    }
    __syncwarp(msk);
}

// One complex FFT of two real rows (row 2 optional): lane t loads z[t + 16 jj].
template <class In>
__device__ __forceinline__ void load_pair(const In *row1, const In *row2, int col0, int nx, int t,
                                          cpx<float> (&v)[16]) {
#pragma unroll
    for (int jj = 0; jj < 16; jj++) {
        int c = col0 + t + 16 * jj;  // col0 >= -r: c lies in [-r, nx + 255)
        if (nx >= kP) {
            c += c < 0 ? nx : 0;
            c -= c >= nx ? nx : 0;
        } else {
            c %= nx;
            c += c < 0 ? nx : 0;
        }
        v[jj].re = (float)row1[c];
        v[jj].im = row2 ? (float)row2[c] : 0.f;
    }
}

// the value at bin n of a row's full spectrum from its 128 half-spectrum slots
__device__ __forceinline__ float2 half_bin(const float2 *Y, int n) {
    if (n == 0) return make_float2(Y[0].x, 0.f);
    if (n == kP / 2) return make_float2(Y[0].y, 0.f);
    if (n < kP / 2) return Y[n];
    const float2 c = Y[kP - n];
    return make_float2(c.x, -c.y);
}

}  // namespace
}  // namespace sfft
