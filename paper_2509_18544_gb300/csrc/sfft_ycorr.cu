// K2: correlations along y at the kernel lags, per row segment and x-frequency.
//
// With A_s(y, k), B_s(y, k) the row-segment spectra from K1, the lag correlation of the
// normal matrix factorises as
//   C_AB(dx, dy) = (1/P) sum_k e^{2 pi i k (G+dx)/P} sum_s Y_s(k, dy),
//   Y_s(k, dy)  = sum_y conj(A_s(y, k)) B_s((y + dy) mod Ny, k),
// so the y direction needs no transform: this kernel evaluates Y_s(k, dy) directly for
// every (A, B) pair the normal matrix uses -- W_i x W_j (i <= j, |dy| <= L-1), W_i x Psi_r
// and W_i x S_m (|dy| <= h) -- and K3 finishes the x direction.
//
// One CTA owns one segment and `kg` consecutive frequencies; each thread owns one
// (frequency, A, B, dy-chunk of C = L lags) work item and streams over y.  Rows are staged
// in shared memory in tiles of `ytile` rows plus a halo of G = L-1 rows on each side
// (cyclic in y).  Inner step: TY rows at once, C+TY-1 B values in registers, C*TY
// complex multiply-adds.  FP32 spectra accumulate in FP32 for one tile and are then
// folded into a double-float (hi, lo) pair with an error-free two-sum, so the long sums
// over y keep ~FP64 accuracy at FP32 speed; FP64 spectra accumulate in FP64.
#include "sfft_internal.cuh"

namespace sfft {
namespace {

constexpr int kTY = 4;

// error-free transformation: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

struct Item {
    int A, B, dylo, ent0, c0, cn;  // images, first lag, first entry, valid chunk range [c0, cn)
};

__device__ __forceinline__ Item decode_item(const Geometry &g, int it) {
    Item m;
    const int L = g.L, nk = g.nk;
    const int two_pairs = 2 * g.npair;
    if (it < two_pairs) {
        int pr = it >> 1, half = it & 1;
        int i = 0, rem = pr;
        while (rem >= nk - i) {
            rem -= nk - i;
            i++;
        }
        int j = i + rem;
        m.A = i;
        m.B = nk + j;
        m.dylo = half ? 0 : -(L - 1);
        m.ent0 = pr * (2 * L - 1) + (m.dylo + L - 1);
        m.c0 = half ? 1 : 0;  // dy = 0 is produced by the lower half
        m.cn = L;
    } else {
        int qd = it - two_pairs;
        int i = qd / (g.nb + 1), r = qd % (g.nb + 1);
        m.A = i;
        m.B = 2 * nk + r;  // Psi_r for r < nb, S_m for r == nb
        m.dylo = -g.h;
        m.ent0 = g.npair * (2 * L - 1) + qd * L;
        m.c0 = 0;
        m.cn = L;
    }
    return m;
}

template <int C>
__global__ void __launch_bounds__(256) k_ycorr_f32(const cpx<float> *__restrict__ spec, Geometry g,
                                                  double *__restrict__ ypart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float> *tile = reinterpret_cast<cpx<float> *>(smem_raw);  // [ytile + 2G][kg][nimg_pad]
    const int s = blockIdx.x;
    const int k0 = blockIdx.y * g.kg;
    const int kcnt = min(g.kg, g.nkf - k0);
    const int G = g.G, ny = g.ny, YT = g.ytile, NI = g.nimg_pad;
    const int rows = YT + 2 * G;
    const int tid = threadIdx.x;
    const int kl = tid / g.items_per_k, it = tid - kl * g.items_per_k;
    const bool active = kl < kcnt;
    Item m = decode_item(g, active ? it : 0);

    float2 acc[C], hi[C], lo[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        acc[c] = make_float2(0.f, 0.f);
        hi[c] = make_float2(0.f, 0.f);
        lo[c] = make_float2(0.f, 0.f);
    }

    const size_t kstride = (size_t)ny * NI;  // elements between consecutive k for fixed s
    const cpx<float> *base = spec + ((size_t)s * g.nkf + k0) * kstride;
    const int vec_per_row = NI / 2;  // float4 = two complex values; NI is even

    for (int y0 = 0; y0 < ny; y0 += YT) {
        __syncthreads();
        // stage rows (y0 - G + r) mod ny, r in [0, rows), for the CTA's kcnt frequencies
        const int nvec = rows * kcnt * vec_per_row;
        for (int v = tid; v < nvec; v += blockDim.x) {
            int r = v / (kcnt * vec_per_row);
            int rem = v - r * (kcnt * vec_per_row);
            int kk = rem / vec_per_row, c2 = rem - kk * vec_per_row;
            int yy = ((y0 - G + r) % ny + ny) % ny;  // cyclic in y, any number of wraps
            const float4 *src = reinterpret_cast<const float4 *>(base + (size_t)kk * kstride + (size_t)yy * NI) + c2;
            reinterpret_cast<float4 *>(tile + ((size_t)r * g.kg + kk) * NI)[c2] = __ldg(src);
        }
        __syncthreads();
        if (active) {
            const int yvalid = min(YT, ny - y0);
            const cpx<float> *ta = tile + (size_t)kl * NI + m.A;
            const cpx<float> *tb = tile + (size_t)kl * NI + m.B;
            const int rs = g.kg * NI;  // row stride in the tile
            for (int yy = 0; yy < yvalid; yy += kTY) {
                float2 a[kTY];
#pragma unroll
                for (int t = 0; t < kTY; t++) {
                    cpx<float> v = ta[(size_t)(G + yy + t) * rs];
                    bool ok = yy + t < yvalid;
                    a[t] = make_float2(ok ? v.re : 0.f, ok ? v.im : 0.f);
                }
                float2 w[C + kTY - 1];
#pragma unroll
                for (int q = 0; q < C + kTY - 1; q++) {
                    cpx<float> v = tb[(size_t)(G + yy + m.dylo + q) * rs];
                    w[q] = make_float2(v.re, v.im);
                }
#pragma unroll
                for (int t = 0; t < kTY; t++)
#pragma unroll
                    for (int c = 0; c < C; c++) {
                        // conj(a) * w
                        acc[c].x = fmaf(a[t].x, w[t + c].x, acc[c].x);
                        acc[c].x = fmaf(a[t].y, w[t + c].y, acc[c].x);
                        acc[c].y = fmaf(a[t].x, w[t + c].y, acc[c].y);
                        acc[c].y = fmaf(-a[t].y, w[t + c].x, acc[c].y);
                    }
            }
            // fold this tile's FP32 partial sums into the double-float accumulators
#pragma unroll
            for (int c = 0; c < C; c++) {
                float s1, e1, s2, e2;
                two_sum(hi[c].x, acc[c].x, s1, e1);
                two_sum(hi[c].y, acc[c].y, s2, e2);
                hi[c].x = s1;
                lo[c].x += e1;
                hi[c].y = s2;
                lo[c].y += e2;
                acc[c] = make_float2(0.f, 0.f);
            }
        }
    }
    if (active) {
        double *out = ypart + (((size_t)s * g.nkf + (k0 + kl)) * g.nent) * 2;
#pragma unroll
        for (int c = 0; c < C; c++) {
            if (c >= m.c0 && c < m.cn) {
                out[2 * (m.ent0 + c)] = (double)hi[c].x + (double)lo[c].x;
                out[2 * (m.ent0 + c) + 1] = (double)hi[c].y + (double)lo[c].y;
            }
        }
    }
}

template <int C>
__global__ void __launch_bounds__(256) k_ycorr_f64(const cpx<double> *__restrict__ spec, Geometry g,
                                                  double *__restrict__ ypart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<double> *tile = reinterpret_cast<cpx<double> *>(smem_raw);
    const int s = blockIdx.x;
    const int k0 = blockIdx.y * g.kg;
    const int kcnt = min(g.kg, g.nkf - k0);
    const int G = g.G, ny = g.ny, YT = g.ytile, NI = g.nimg_pad;
    const int rows = YT + 2 * G;
    const int tid = threadIdx.x;
    const int kl = tid / g.items_per_k, it = tid - kl * g.items_per_k;
    const bool active = kl < kcnt;
    Item m = decode_item(g, active ? it : 0);
    double2 acc[C];
#pragma unroll
    for (int c = 0; c < C; c++) acc[c] = make_double2(0.0, 0.0);
    const size_t kstride = (size_t)ny * NI;
    const cpx<double> *base = spec + ((size_t)s * g.nkf + k0) * kstride;
    for (int y0 = 0; y0 < ny; y0 += YT) {
        __syncthreads();
        const int nv = rows * kcnt * NI;
        for (int v = tid; v < nv; v += blockDim.x) {
            int r = v / (kcnt * NI);
            int rem = v - r * (kcnt * NI);
            int kk = rem / NI, c2 = rem - kk * NI;
            int yy = ((y0 - G + r) % ny + ny) % ny;  // cyclic in y, any number of wraps
            tile[((size_t)r * g.kg + kk) * NI + c2] = base[(size_t)kk * kstride + (size_t)yy * NI + c2];
        }
        __syncthreads();
        if (active) {
            const int yvalid = min(YT, ny - y0);
            const cpx<double> *ta = tile + (size_t)kl * NI + m.A;
            const cpx<double> *tb = tile + (size_t)kl * NI + m.B;
            const int rs = g.kg * NI;
            for (int yy = 0; yy < yvalid; yy++) {
                cpx<double> a = ta[(size_t)(G + yy) * rs];
#pragma unroll
                for (int c = 0; c < C; c++) {
                    cpx<double> w = tb[(size_t)(G + yy + m.dylo + c) * rs];
                    acc[c].x = fma(a.re, w.re, acc[c].x);
                    acc[c].x = fma(a.im, w.im, acc[c].x);
                    acc[c].y = fma(a.re, w.im, acc[c].y);
                    acc[c].y = fma(-a.im, w.re, acc[c].y);
                }
            }
        }
    }
    if (active) {
        double *out = ypart + (((size_t)s * g.nkf + (k0 + kl)) * g.nent) * 2;
#pragma unroll
        for (int c = 0; c < C; c++)
            if (c >= m.c0 && c < m.cn) {
                out[2 * (m.ent0 + c)] = acc[c].x;
                out[2 * (m.ent0 + c) + 1] = acc[c].y;
            }
    }
}

template <int C>
cudaError_t run(const Geometry &g, int precision, const void *spec, double *ypart, cudaStream_t st) {
    dim3 grid(g.nseg, (g.nkf + g.kg - 1) / g.kg);
    int threads = ((g.kg * g.items_per_k + 31) / 32) * 32;
    size_t rows = (size_t)g.ytile + 2 * g.G;
    if (precision == SFFT_PREC_FP64) {
        size_t sm = rows * g.kg * g.nimg_pad * sizeof(cpx<double>);
        cudaError_t e = cudaFuncSetAttribute(k_ycorr_f64<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        note_launch();
        k_ycorr_f64<C><<<grid, threads, sm, st>>>((const cpx<double> *)spec, g, ypart);
    } else {
        size_t sm = rows * g.kg * g.nimg_pad * sizeof(cpx<float>);
        cudaError_t e = cudaFuncSetAttribute(k_ycorr_f32<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        note_launch();
        k_ycorr_f32<C><<<grid, threads, sm, st>>>((const cpx<float> *)spec, g, ypart);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ycorr(const Geometry &g, int precision, const void *spec, double *ypart, cudaStream_t st) {
    switch (g.C) {
        case 1: return run<1>(g, precision, spec, ypart, st);
        case 3: return run<3>(g, precision, spec, ypart, st);
        case 5: return run<5>(g, precision, spec, ypart, st);
        case 7: return run<7>(g, precision, spec, ypart, st);
        case 9: return run<9>(g, precision, spec, ypart, st);
        case 11: return run<11>(g, precision, spec, ypart, st);
        case 13: return run<13>(g, precision, spec, ypart, st);
        case 15: return run<15>(g, precision, spec, ypart, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sfft
