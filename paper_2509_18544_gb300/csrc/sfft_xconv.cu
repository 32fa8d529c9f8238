// Cross-convolution (Sec. "Pipeline steps", step 5): before the subtraction each image is
// convolved with the other image's point-spread function, so that both end up with the
// same, broader PSF:
//   S'(u) = sum_d P_T(d) S((u - d) mod N),   T'(u) = sum_d P_S(d) T((u - d) mod N),
// d = (dy, dx) in [-r, r]^2 over the K x K stamps (K = 2r + 1, stamp row-major, its centre
// element at d = 0), cyclic on the frame like the rest of the fit.
//
// Direct convolution, FP32 arithmetic (FP64 frames are converted on load and the result
// rounded back).  One CTA computes a 256 x 32 output tile of one job (image, stamp): the
// (256 + 2r) x (32 + 2r) input window and the stamp are staged in shared memory; each thread
// owns 8 consecutive columns of 4 rows, keeps one stamp row and one input-row window
// (8 + 2r values, 16-byte loads) in registers and does 8 K FMAs per window.  K^2 FMAs per
// pixel (625 for K = 25): the kernel is bound by the FP32 pipe, not by HBM.
// Stamps of 9 x 9 and larger take the row-segment FFT route of sfft_xconv_fft.cu instead.
#include <stdio.h>

#include "sfft_internal.cuh"

namespace sfft {
namespace {

constexpr int kTX = 256, kTY = 32;  // output tile
constexpr int kCols = 8, kRows = 4;  // outputs per thread
constexpr int kThreads = (kTX / kCols) * (kTY / kRows);  // 256

struct XJob {
    const void *src;
    const float *psf;
    void *dst;
};

template <class In, int R>
__global__ void __launch_bounds__(kThreads, 2) k_xconv(XJob j0, XJob j1, int ny, int nx, int pitch) {
    constexpr int K = 2 * R + 1;
    constexpr int KP = (K + 3) & ~3;            // stamp row padded to 16 bytes
    constexpr int W = kCols + 2 * R;            // input values one output row's 8 columns read
    constexpr int WP = (W + 3) & ~3;
    constexpr int IW = kTX + ((2 * R + 3) & ~3);  // staged window width (16-byte rows)
    constexpr int IH = kTY + 2 * R;
    extern __shared__ __align__(16) float xs[];
    float *in = xs;            // [IH][IW]: frame rows y0 - r .., columns x0 - r ..
    float *ps = in + IH * IW;  // [K][KP] stamp, zero-padded rows
    const XJob jb = blockIdx.z ? j1 : j0;
    const In *src = reinterpret_cast<const In *>(jb.src);
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    for (int e = threadIdx.x; e < K * KP; e += kThreads) {
        const int a = e / KP, b = e - a * KP;
        ps[e] = b < K ? jb.psf[a * K + b] : 0.f;
    }
    for (int e = threadIdx.x; e < IH * IW; e += kThreads) {
        const int i = e / IW, c = e - i * IW;
        int yy = (y0 - R + i) % ny, xx = (x0 - R + c) % nx;
        yy += yy < 0 ? ny : 0;
        xx += xx < 0 ? nx : 0;
        in[e] = c < kTX + 2 * R ? (float)src[(size_t)yy * pitch + xx] : 0.f;
    }
    __syncthreads();
    const int tx = threadIdx.x % (kTX / kCols), ty = threadIdx.x / (kTX / kCols);
    const int c0 = tx * kCols;  // first output column of the thread (tile-local)
    float acc[kRows][kCols];
#pragma unroll
    for (int i = 0; i < kRows; i++)
#pragma unroll
        for (int c = 0; c < kCols; c++) acc[i][c] = 0.f;
    // out(y, x) = sum_{a,b} P[a][b] in(y + 2r - a, x + 2r - b) in tile-local coordinates
    for (int a = 0; a < K; a++) {
        float p[KP];
#pragma unroll
        for (int b = 0; b < KP; b += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(ps + a * KP + b);
            p[b] = v.x, p[b + 1] = v.y, p[b + 2] = v.z, p[b + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < kRows; i++) {
            const int ly = ty * kRows + i;
            const float *row = in + (ly + 2 * R - a) * IW + c0;
            float w[WP];
#pragma unroll
            for (int q = 0; q < WP; q += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(row + q);
                w[q] = v.x, w[q + 1] = v.y, w[q + 2] = v.z, w[q + 3] = v.w;
            }
            // output column c reads input column c + 2r - b
#pragma unroll
            for (int b = 0; b < K; b++)
#pragma unroll
                for (int c = 0; c < kCols; c++) acc[i][c] = fmaf(p[b], w[c + 2 * R - b], acc[i][c]);
        }
    }
    In *dst = reinterpret_cast<In *>(jb.dst);
#pragma unroll
    for (int i = 0; i < kRows; i++) {
        const int y = y0 + ty * kRows + i;
        if (y >= ny) continue;
#pragma unroll
        for (int c = 0; c < kCols; c++) {
            const int x = x0 + c0 + c;
            if (x < nx) dst[(size_t)y * pitch + x] = (In)acc[i][c];
        }
    }
}

template <class In, int R>
cudaError_t run_r(const XJob &a, const XJob &b, int njobs, int ny, int nx, int pitch, cudaStream_t st) {
    constexpr int K = 2 * R + 1, KP = (K + 3) & ~3, IW = kTX + ((2 * R + 3) & ~3), IH = kTY + 2 * R;
    const size_t sm = sizeof(float) * ((size_t)IH * IW + (size_t)K * KP);
    cudaError_t e = cudaFuncSetAttribute(k_xconv<In, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY, njobs);
    note_launch();
    k_xconv<In, R><<<grid, kThreads, sm, st>>>(a, b, ny, nx, pitch);
    return cudaGetLastError();
}

template <class In>
cudaError_t run_in(int r, const XJob &a, const XJob &b, int njobs, int ny, int nx, int pitch, cudaStream_t st) {
    switch (r) {
        case 0: return run_r<In, 0>(a, b, njobs, ny, nx, pitch, st);
        case 1: return run_r<In, 1>(a, b, njobs, ny, nx, pitch, st);
        case 2: return run_r<In, 2>(a, b, njobs, ny, nx, pitch, st);
        case 3: return run_r<In, 3>(a, b, njobs, ny, nx, pitch, st);
        case 4: return run_r<In, 4>(a, b, njobs, ny, nx, pitch, st);
        case 5: return run_r<In, 5>(a, b, njobs, ny, nx, pitch, st);
        case 6: return run_r<In, 6>(a, b, njobs, ny, nx, pitch, st);
        case 7: return run_r<In, 7>(a, b, njobs, ny, nx, pitch, st);
        case 8: return run_r<In, 8>(a, b, njobs, ny, nx, pitch, st);
        case 9: return run_r<In, 9>(a, b, njobs, ny, nx, pitch, st);
        case 10: return run_r<In, 10>(a, b, njobs, ny, nx, pitch, st);
        case 11: return run_r<In, 11>(a, b, njobs, ny, nx, pitch, st);
        case 12: return run_r<In, 12>(a, b, njobs, ny, nx, pitch, st);
        case 13: return run_r<In, 13>(a, b, njobs, ny, nx, pitch, st);
        case 14: return run_r<In, 14>(a, b, njobs, ny, nx, pitch, st);
        case 15: return run_r<In, 15>(a, b, njobs, ny, nx, pitch, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

void set_global_error(const char *msg);
cudaError_t launch_xconv_fft(int r, int dtype, const void *src0, const float *psf0, void *dst0, const void *src1,
                             const float *psf1, void *dst1, int njobs, int ny, int nx, int pitch, cudaStream_t st);

}  // namespace sfft

using namespace sfft;

extern "C" sfft_status sfft_cross_convolve(int32_t ny, int32_t nx, int32_t pitch, int32_t dtype, int32_t K,
                                           const void *sci, const void *tmpl, const float *psf_sci,
                                           const float *psf_tmpl, void *sci_out, void *tmpl_out,
                                           sfft_stream_t stream) {
    if (ny < 1 || nx < 1 || K < 1 || K % 2 == 0 || K > 31) {
        set_global_error("sfft_cross_convolve: need ny, nx >= 1 and an odd stamp size 1 <= K <= 31");
        return SFFT_ERR_INVALID_ARG;
    }
    if (pitch == 0) pitch = nx;
    if (pitch < nx || (dtype != SFFT_F32 && dtype != SFFT_F64)) {
        set_global_error("sfft_cross_convolve: pitch < nx or unknown dtype");
        return SFFT_ERR_INVALID_ARG;
    }
    // each output needs its input and the other image's stamp; either half may be omitted
    const bool do_s = sci && psf_tmpl && sci_out, do_t = tmpl && psf_sci && tmpl_out;
    if (!do_s && !do_t) {
        set_global_error("sfft_cross_convolve: nothing to do (null images, stamps or outputs)");
        return SFFT_ERR_INVALID_ARG;
    }
    if ((do_s && (sci_out == sci || sci_out == tmpl)) || (do_t && (tmpl_out == tmpl || tmpl_out == sci))) {
        set_global_error("sfft_cross_convolve: an output may not alias an input");
        return SFFT_ERR_INVALID_ARG;
    }
    XJob a{do_s ? sci : tmpl, do_s ? psf_tmpl : psf_sci, do_s ? sci_out : tmpl_out};
    XJob b{tmpl, psf_sci, tmpl_out};
    const int njobs = do_s && do_t ? 2 : 1;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int r = (K - 1) / 2;
    // stamps of 9 x 9 and up: the row-segment FFT route (~10x fewer instructions at K = 25);
    // smaller stamps: the direct sum
    cudaError_t e = r >= 4 ? launch_xconv_fft(r, dtype, a.src, a.psf, a.dst, b.src, b.psf, b.dst, njobs, ny, nx,
                                              pitch, st)
                  : dtype == SFFT_F64 ? run_in<double>(r, a, b, njobs, ny, nx, pitch, st)
                                      : run_in<float>(r, a, b, njobs, ny, nx, pitch, st);
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof buf, "sfft_cross_convolve: %s", cudaGetErrorString(e));
        set_global_error(buf);
        return SFFT_ERR_CUDA;
    }
    return SFFT_OK;
}
