// Decorrelation kernel (Sec. "Pipeline steps", step 7).  The definition (noise spectrum of
// the difference image after cross-convolution, whitened at unit flux gain on an M x M
// cyclic grid) is the one sfft.h states for sfft_decorrelation_kernel.
//
// One CTA does the whole computation in FP64 shared memory (M <= 31):
//   1. the matching kernel at (x, y) from the fit's coefficients, K(d) = sum_pq a_{pq,d} w_pq;
//   2. the three real stamps (P_S, P_T, K) placed on the grid at d mod M;
//   3. their 2-D DFTs, rows then columns, skipping the rows and columns a stamp leaves empty;
//   4. Phi(k) and Q(k) = P_S(k) P_T(k) Phi(k);
//   5. inverse DFTs of Phi and Q (columns then rows, real part), written centred, FP32.
// Twiddles e^{-2 pi i m / M} are tabulated once (FP64 sincospi of m / M, exact argument);
// index products are reduced mod M in integers.  The work is O(M^3) ~ 1e6 FP64 FMAs per
// call: a one-SM kernel that runs once per pair.
#include <math.h>
#include <stdio.h>

#include "sfft_internal.cuh"

namespace sfft {

void set_global_error(const char *msg);

namespace {

constexpr int kMaxM = 31, kThreads = 512;

struct DecorrArg {
    const double *coeffs;
    const float *psf_sci, *psf_tmpl;
    float *phi, *psf_out;
    double xh, yh, var_s, var_t;
    int L, nk, K, M;
};

struct DecorrSmem {
    double g[3][kMaxM * kMaxM];            // real stamps on the grid: P_S, P_T, K
    cpx<double> r[3][kMaxM * kMaxM];       // row DFTs [row][k2]
    cpx<double> X[3][kMaxM * kMaxM];       // spectra [k1][k2]
    cpx<double> tw[kMaxM];                 // e^{-2 pi i m / M}
};

__global__ void __launch_bounds__(kThreads) k_decorr(DecorrArg a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DecorrSmem &s = *reinterpret_cast<DecorrSmem *>(smem_raw);
    const int M = a.M, MM = M * M, t = threadIdx.x;
    const int ext[3] = {a.K, a.K, a.L};  // stamp widths on the grid
    for (int e = t; e < 3 * MM; e += kThreads) (&s.g[0][0])[(e / MM) * kMaxM * kMaxM + e % MM] = 0.0;
    if (t < M) {
        double sn, cs;
        sincospi(-2.0 * t / M, &sn, &cs);
        s.tw[t] = {cs, sn};
    }
    __syncthreads();
    // 1-2: stamps onto the grid at d mod M
    const int cK = (a.K - 1) / 2, cL = (a.L - 1) / 2;
    for (int e = t; e < a.K * a.K; e += kThreads) {
        const int r = e / a.K, c = e % a.K;
        const int gi = ((r - cK + M) % M) * M + (c - cK + M) % M;
        s.g[0][gi] = (double)a.psf_sci[e];
        s.g[1][gi] = (double)a.psf_tmpl[e];
    }
    for (int e = t; e < a.L * a.L; e += kThreads) {
        double v = 0.0;
        for (int idx = 0; idx < a.nk; idx++) {
            int p, q;
            mono_pq(idx, p, q);
            double w = 1.0;
            for (int i = 0; i < p; i++) w *= a.xh;
            for (int i = 0; i < q; i++) w *= a.yh;
            v += a.coeffs[(size_t)idx * a.L * a.L + e] * w;
        }
        const int r = e / a.L, c = e % a.L;  // row = dy + h, column = dx + h
        s.g[2][((r - cL + M) % M) * M + (c - cL + M) % M] = v;
    }
    __syncthreads();
    // 3a: row DFTs of the occupied rows, over the occupied columns
    for (int e = t; e < 3 * MM; e += kThreads) {
        const int gI = e / MM, r = (e % MM) / M, k2 = e % M;
        const int w = ext[gI], c = (w - 1) / 2;
        const int rr = (r + c) % M;  // the grid row at offset rr - c; occupied when rr < w
        cpx<double> acc{0.0, 0.0};
        if (rr < w) {
            for (int j = 0; j < w; j++) {
                const int n = (j - c + M) % M;
                const double v = s.g[gI][r * M + n];
                const cpx<double> tw = s.tw[(k2 * n) % M];
                acc.re = fma(v, tw.re, acc.re);
                acc.im = fma(v, tw.im, acc.im);
            }
        }
        s.r[gI][r * M + k2] = acc;
    }
    __syncthreads();
    // 3b: column DFTs over the occupied rows
    for (int e = t; e < 3 * MM; e += kThreads) {
        const int gI = e / MM, k1 = (e % MM) / M, k2 = e % M;
        const int w = ext[gI], c = (w - 1) / 2;
        cpx<double> acc{0.0, 0.0};
        for (int j = 0; j < w; j++) {
            const int n = (j - c + M) % M;
            const cpx<double> v = s.r[gI][n * M + k2], tw = s.tw[(k1 * n) % M];
            acc.re = fma(v.re, tw.re, fma(-v.im, tw.im, acc.re));
            acc.im = fma(v.re, tw.im, fma(v.im, tw.re, acc.im));
        }
        s.X[gI][k1 * M + k2] = acc;
    }
    __syncthreads();
    // 4: Phi into X[2] (real), Q into X[0]
    const double K0 = s.X[2][0].re;
    const double num = a.var_s + K0 * K0 * a.var_t;
    for (int e = t; e < MM; e += kThreads) {
        const cpx<double> ps = s.X[0][e], pt = s.X[1][e], kk = s.X[2][e];
        const double aps = ps.re * ps.re + ps.im * ps.im, apt = pt.re * pt.re + pt.im * pt.im;
        const double akk = kk.re * kk.re + kk.im * kk.im;
        const double den = a.var_s * apt + a.var_t * akk * aps;
        const double ph = sqrt(num / fmax(den, 1e-8 * num));
        s.X[2][e] = {ph, 0.0};
        s.X[0][e] = cmul(ps, pt);
        s.X[0][e].re *= ph;
        s.X[0][e].im *= ph;
    }
    __syncthreads();
    // 5a: inverse column DFTs (conjugate twiddles) into r[2] (Phi) and r[0] (Q)
    for (int e = t; e < 2 * MM; e += kThreads) {
        const int gI = e < MM ? 2 : 0, rr = (e % MM) / M, k2 = e % M;
        cpx<double> acc{0.0, 0.0};
        for (int k1 = 0; k1 < M; k1++) {
            const cpx<double> v = s.X[gI][k1 * M + k2], tw = s.tw[(k1 * rr) % M];
            acc.re = fma(v.re, tw.re, fma(v.im, tw.im, acc.re));
            acc.im = fma(v.im, tw.re, fma(-v.re, tw.im, acc.im));
        }
        s.r[gI][rr * M + k2] = acc;
    }
    __syncthreads();
    // 5b: inverse row DFTs, real part, written centred
    const double inv = 1.0 / ((double)M * M);
    const int cM = (M - 1) / 2;
    for (int e = t; e < 2 * MM; e += kThreads) {
        const bool is_phi = e < MM;
        if (!is_phi && !a.psf_out) break;
        const int gI = is_phi ? 2 : 0, rr = (e % MM) / M, n = e % M;
        double acc = 0.0;
        for (int k2 = 0; k2 < M; k2++) {
            const cpx<double> v = s.r[gI][rr * M + k2], tw = s.tw[(k2 * n) % M];
            acc = fma(v.re, tw.re, fma(v.im, tw.im, acc));
        }
        // grid index (rr, n) holds offset (rr, n) mod M: centred output row (rr + cM) mod M
        float *dst = is_phi ? a.phi : a.psf_out;
        dst[((rr + cM) % M) * M + (n + cM) % M] = (float)(acc * inv);
    }
}

}  // namespace
}  // namespace sfft

using namespace sfft;

extern "C" sfft_status sfft_decorrelation_kernel(int32_t ny, int32_t nx, int32_t L, int32_t dk, const double *coeffs,
                                                 double x, double y, int32_t K, const float *psf_sci,
                                                 const float *psf_tmpl, double sigma_sci, double sigma_tmpl,
                                                 int32_t M, float *phi, float *psf_out, sfft_stream_t stream) {
    if (ny < 1 || nx < 1 || L < 1 || L % 2 == 0 || dk < 0 || K < 1 || K % 2 == 0 || M % 2 == 0 || M > kMaxM ||
        K > M || L > M || !coeffs || !psf_sci || !psf_tmpl || !phi || !(sigma_sci > 0.0) || !(sigma_tmpl >= 0.0)) {
        set_global_error("sfft_decorrelation_kernel: need odd L, K, M with max(K, L) <= M <= 31, dk >= 0, "
                         "device stamps and coefficients, sigma_sci > 0 and sigma_tmpl >= 0");
        return SFFT_ERR_INVALID_ARG;
    }
    DecorrArg a;
    a.coeffs = coeffs;
    a.psf_sci = psf_sci;
    a.psf_tmpl = psf_tmpl;
    a.phi = phi;
    a.psf_out = psf_out;
    a.xh = nx > 1 ? 2.0 * x / (nx - 1) - 1.0 : 0.0;
    a.yh = ny > 1 ? 2.0 * y / (ny - 1) - 1.0 : 0.0;
    a.var_s = sigma_sci * sigma_sci;
    a.var_t = sigma_tmpl * sigma_tmpl;
    a.L = L;
    a.nk = npoly(dk);
    a.K = K;
    a.M = M;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t sm = sizeof(DecorrSmem);
    cudaError_t e = cudaFuncSetAttribute(k_decorr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
        note_launch();
        k_decorr<<<1, kThreads, sm, st>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof buf, "sfft_decorrelation_kernel: %s", cudaGetErrorString(e));
        set_global_error(buf);
        return SFFT_ERR_CUDA;
    }
    return SFFT_OK;
}
