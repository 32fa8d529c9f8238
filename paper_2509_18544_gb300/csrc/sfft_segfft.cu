// K1: polynomial-weighted products fused into row-segment real FFTs.
//
// For every row y and segment s the kernel forms, on the fly from S, T and the mask,
//   A-images  W_i restricted to the segment's own columns [x0, x0+U) and zero-padded to P,
//   B-images  W_i, Psi_r = m w_r and S_m over the cyclic window [x0-G, x0-G+P),
// (W_i = w_i T_m, w_i = xh^p yh^q) and takes their P-point real DFTs (forward,
// exp(-2 pi i k j / P), unnormalised).  Two real images share one complex FFT; P = 256 is
// done as 16 x 16 (a 16-point DFT in registers, a twiddle, one padded shared-memory
// transpose, a second 16-point DFT).  Output: spec[s][k][y][img], k in [0, P/2].
//
// These spectra feed the lag correlations of the normal matrix of the delta-basis fit
// (SFFT subtraction step, Sec. "Pipeline steps", step 6).
#include "sfft_internal.cuh"

namespace sfft {
namespace {

constexpr int kP = 256;
constexpr int kRows = 8;  // rows per CTA

template <class R>
__device__ __forceinline__ R coord(int i, int n) {
    return n > 1 ? (R)(2 * i - (n - 1)) / (R)(n - 1) : (R)0;
}

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

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

template <class R, class In>
__global__ void __launch_bounds__(256) k_segment_fft(const In *__restrict__ sci, const In *__restrict__ tmpl,
                                                    const uint8_t *__restrict__ mask, Geometry g,
                                                    const cpx<R> *__restrict__ tw_g, const R *__restrict__ xpow_g,
                                                    const R *__restrict__ ypow_g, cpx<R> *__restrict__ spec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = g.nk, nb = g.nb, G = g.G, U = g.U, nx = g.nx, ny = g.ny;
    const int maxdeg = g.dk > g.db ? g.dk : g.db;
    const int s = blockIdx.x;
    const int x0 = s * U;
    const int tid = threadIdx.x;

    // shared layout
    cpx<R> *tw = reinterpret_cast<cpx<R> *>(smem_raw);            // [P] twiddle, high part
    cpx<R> *twl = tw + kP;                                          // [P] remainder
    cpx<R> *ex = twl + kP;                                          // [nfft][16*17]
    R *xpow = reinterpret_cast<R *>(ex + g.nfft * 16 * 17);         // [maxdeg+1][P]
    R *tv = xpow + (maxdeg + 1) * kP;                               // [P] T_m on the window
    R *sv = tv + kP;                                                // [P] S_m
    R *mv = sv + kP;                                                // [P] m
    int *ik = reinterpret_cast<int *>(mv + kP);                     // [nimg_pad] kind
    int *ip = ik + g.nimg_pad;                                      // [nimg_pad] p
    int *iq = ip + g.nimg_pad;                                      // [nimg_pad] q

    for (int i = tid; i < kP; i += blockDim.x) {
        tw[i] = tw_g[i];
        twl[i] = tw_g[kP + i];
        // coordinate powers come from FP64 tables rounded once: repeated FP32 products
        // are biased (~-3e-8 at power 4)
        int xw = wrapi(x0 - G + i, nx);
        for (int p = 0; p <= maxdeg; p++) xpow[p * kP + i] = xpow_g[(size_t)p * nx + xw];
    }
    for (int i = tid; i < g.nimg_pad; i += blockDim.x) {
        // kinds: 0 = A (W_i on own columns), 1 = B W_i, 2 = Psi_r, 3 = S_m, 4 = zero pad
        int kind, mi = 0;
        if (i < nk) { kind = 0; mi = i; }
        else if (i < 2 * nk) { kind = 1; mi = i - nk; }
        else if (i < 2 * nk + nb) { kind = 2; mi = i - 2 * nk; }
        else if (i == 2 * nk + nb) { kind = 3; }
        else { kind = 4; }
        int p = 0, q = 0;
        mono_pq(mi, p, q);
        ik[i] = kind;
        ip[i] = p;
        iq[i] = q;
    }

    const int f = tid >> 4, t = tid & 15;
    const bool fft_thread = f < g.nfft;
    // FFT lanes of this warp: all 32, or the lower 16 when the FFT count is odd
    const unsigned fmask = ((tid & ~31) + 32 <= g.nfft * 16) ? 0xffffffffu : 0x0000ffffu;
    const int y_end = min(ny, (int)(blockIdx.y + 1) * kRows);
    for (int y = blockIdx.y * kRows; y < y_end; y++) {
        __syncthreads();  // previous row's readers of ex / window are done
        const size_t rowoff = (size_t)y * g.pitch;
        for (int j = tid; j < kP; j += blockDim.x) {
            int xw = wrapi(x0 - G + j, nx);
            R good = (mask && mask[rowoff + xw]) ? (R)0 : (R)1;
            tv[j] = good * (R)tmpl[rowoff + xw];
            sv[j] = good * (R)sci[rowoff + xw];
            mv[j] = good;
        }
        __syncthreads();
        if (fft_thread) {
            cpx<R> v[16];
            int kinds[2], ps[2];
            R yq[2];
#pragma unroll
            for (int c = 0; c < 2; c++) {
                int im = 2 * f + c;
                kinds[c] = ik[im];
                ps[c] = ip[im];
                yq[c] = ypow_g[(size_t)iq[im] * ny + y];
            }
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const int n = t + 16 * jj;
                R val[2];
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    R r = (R)0;
                    switch (kinds[c]) {
                        case 0:
                            if (n < U && x0 + n < nx) r = xpow[ps[c] * kP + n + G] * yq[c] * tv[n + G];
                            break;
                        case 1: r = xpow[ps[c] * kP + n] * yq[c] * tv[n]; break;
                        case 2: r = xpow[ps[c] * kP + n] * yq[c] * mv[n]; break;
                        case 3: r = sv[n]; break;
                        default: break;
                    }
                    val[c] = r;
                }
                v[jj] = {val[0], val[1]};
            }
            // X[k1 + 16 k2] = sum_t W16^{t k2} W256^{t k1} sum_jj x[t + 16 jj] W16^{jj k1}
            dft16(v, tw, twl);
#pragma unroll
            for (int k1 = 1; k1 < 16; k1++) v[k1] = twmul(v[k1], tw[(t * k1) & (kP - 1)], twl[(t * k1) & (kP - 1)]);
            cpx<R> *e = ex + f * 16 * 17;
#pragma unroll
            for (int k1 = 0; k1 < 16; k1++) e[k1 * 17 + t] = v[k1];
            __syncwarp(fmask);
            // the 16 lanes of this FFT share one half-warp, so a warp barrier suffices
#pragma unroll
            for (int tt = 0; tt < 16; tt++) v[tt] = e[t * 17 + tt];
            dft16(v, tw, twl);  // now over tt: X[t + 16 k2] = v[k2]
            __syncwarp(fmask);
#pragma unroll
            for (int k2 = 0; k2 < 16; k2++) e[t + 16 * k2] = v[k2];  // natural order Z[k]
        }
        __syncthreads();
        // unpack the packed real pairs and write spec[s][k][y][img], k in [0, P/2]
        const int total = g.nkf * g.nimg_pad;
        for (int idx = tid; idx < total; idx += blockDim.x) {
            const int k = idx / g.nimg_pad, img = idx - k * g.nimg_pad;
            const cpx<R> *e = ex + (img >> 1) * 16 * 17;
            cpx<R> zk = e[k], zc = e[(kP - k) & (kP - 1)];
            cpx<R> out;
            if ((img & 1) == 0)
                out = {(R)0.5 * (zk.re + zc.re), (R)0.5 * (zk.im - zc.im)};
            else
                out = {(R)0.5 * (zk.im + zc.im), (R)0.5 * (zc.re - zk.re)};
            spec[(((size_t)s * g.nkf + k) * ny + y) * g.nimg_pad + img] = out;
        }
    }
}

template <class R>
size_t segfft_smem(const Geometry &g) {
    const int maxdeg = g.dk > g.db ? g.dk : g.db;
    return sizeof(cpx<R>) * (2 * kP + (size_t)g.nfft * 16 * 17) + sizeof(R) * ((size_t)(maxdeg + 1) * kP + 3 * kP) +
           sizeof(int) * 3 * g.nimg_pad;
}

template <class R, class In>
cudaError_t run(const Geometry &g, const void *sci, const void *tmpl, const uint8_t *mask, const void *tw,
                const void *xpow, const void *ypow, void *spec, cudaStream_t st) {
    size_t sm = segfft_smem<R>(g);
    auto kern = k_segment_fft<R, In>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int threads = ((g.nfft * 16 + 31) / 32) * 32;
    if (threads < 64) threads = 64;
    dim3 grid(g.nseg, (g.ny + kRows - 1) / kRows);
    note_launch();
    kern<<<grid, threads, sm, st>>>((const In *)sci, (const In *)tmpl, mask, g, (const cpx<R> *)tw,
                                    (const R *)xpow, (const R *)ypow, (cpx<R> *)spec);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_segment_fft(const Geometry &g, int dtype, int precision, const void *sci, const void *tmpl,
                               const uint8_t *mask, const void *tw_fft, const void *xpow, const void *ypow,
                               void *spec, cudaStream_t st) {
    if (g.P != kP || g.nfft > 16) return cudaErrorInvalidValue;
    if (precision == SFFT_PREC_FP64) {
        return dtype == SFFT_F64 ? run<double, double>(g, sci, tmpl, mask, tw_fft, xpow, ypow, spec, st)
                                 : run<double, float>(g, sci, tmpl, mask, tw_fft, xpow, ypow, spec, st);
    }
    return dtype == SFFT_F64 ? run<float, double>(g, sci, tmpl, mask, tw_fft, xpow, ypow, spec, st)
                             : run<float, float>(g, sci, tmpl, mask, tw_fft, xpow, ypow, spec, st);
}

}  // namespace sfft
