// Forced PSF photometry (Sec. "Pipeline steps", step 9: the PSF fitted to the decorrelated
// difference image at the transient's coordinates; step 8 fits it to field stars).  The
// estimator (weighted least squares of flux, and optionally a constant background, over the
// stamp's footprint, the stamp moved to the sub-pixel position by the Lanczos-3 window) is
// the one sfft.h states for sfft_forced_photometry.
//
// One CTA per job.  The sub-pixel offset is the same for every footprint pixel, so one set
// of six x and six y weights moves the whole stamp (a separable 6 x 6 filter, zeros outside
// the stamp) into shared memory; the five weighted sums of the normal equations accumulate
// in FP64 (warp shuffles, then shared memory), thread 0 solves the 1 x 1 or 2 x 2 system, and
// a second pass over the footprint forms chi^2 from the residuals.
#include <math.h>
#include <stdio.h>

#include "sfft_internal.cuh"

namespace sfft {

void set_global_error(const char *msg);

namespace {

constexpr int kMaxK = 63, kThreads = 128, kWarps = kThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sums of NS values (every thread gets the totals)
template <int NS>
__device__ __forceinline__ void block_sums(double (&v)[NS], double (*red)[NS]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; k++) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NS; k++) red[wid][k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NS; k++) {
        double s = 0.0;
        for (int w = 0; w < kWarps; w++) s += red[w][k];
        v[k] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double pixel(const sfft_phot_job &jb, size_t o) {
    return jb.dtype == SFFT_F64 ? __ldg(reinterpret_cast<const double *>(jb.image) + o)
                                : (double)__ldg(reinterpret_cast<const float *>(jb.image) + o);
}

__global__ void __launch_bounds__(kThreads) k_phot(const sfft_phot_job *__restrict__ jobs, int K, int flags,
                                                   double *__restrict__ results) {
    __shared__ float st[kMaxK * kMaxK];  // the job's stamp
    __shared__ float model[kMaxK * kMaxK];
    __shared__ float wx[6], wy[6];
    __shared__ double red[kWarps][6];
    __shared__ double sol[3];
    const sfft_phot_job jb = jobs[blockIdx.x];
    const int t = threadIdx.x, c = (K - 1) / 2, KK = K * K;
    const int pitch = jb.pitch ? jb.pitch : jb.nx;
    const double X = floor(jb.x + 0.5), Y = floor(jb.y + 0.5);
    // stamp column of model column b: c + b - fx = (c + b) + floor(-fx) + frac(-fx)
    const double gx = -(jb.x - X), gy = -(jb.y - Y);
    const double flx = floor(gx), fly = floor(gy);
    if (t == 0) lanczos3_taps((float)(gx - flx), wx);
    if (t == 32) lanczos3_taps((float)(gy - fly), wy);
    for (int e = t; e < KK; e += kThreads) st[e] = __ldg(jb.psf + e);
    __syncthreads();
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        sx += wx[k];
        sy += wy[k];
    }
    const float inv = 1.f / (sx * sy);
    const int ox = (int)flx - 2, oy = (int)fly - 2;  // stamp offset of the first tap
    for (int e = t; e < KK; e += kThreads) {
        const int a = e / K, b = e % K;  // footprint row a - c, column b - c
        float acc = 0.f;
        for (int i = 0; i < 6; i++) {
            const int r = a + oy + i;
            if (r < 0 || r >= K || wy[i] == 0.f) continue;
            float racc = 0.f;
            for (int j = 0; j < 6; j++) {
                const int s = b + ox + j;
                if (s < 0 || s >= K) continue;
                racc = fmaf(wx[j], st[r * K + s], racc);
            }
            acc = fmaf(wy[i], racc, acc);
        }
        model[e] = acc * inv;
    }
    __syncthreads();
    // normal-equation sums: w P^2, w P, w, w P D, w D, n
    double v[6] = {0, 0, 0, 0, 0, 0};
    const long long X0 = (long long)X - c, Y0 = (long long)Y - c;
    for (int e = t; e < KK; e += kThreads) {
        const long long r = Y0 + e / K, s = X0 + e % K;
        if (r < 0 || r >= jb.ny || s < 0 || s >= jb.nx) continue;
        const size_t o = (size_t)r * pitch + (size_t)s;
        if (jb.mask && __ldg(jb.mask + o)) continue;
        const double w = jb.weight ? (double)__ldg(jb.weight + o) : 1.0;
        if (!(w > 0.0)) continue;
        const double p = model[e], d = pixel(jb, o);
        v[0] += w * p * p;
        v[1] += w * p;
        v[2] += w;
        v[3] += w * p * d;
        v[4] += w * d;
        v[5] += 1.0;
    }
    block_sums<6>(v, red);
    const bool bg = flags & SFFT_PHOT_BACKGROUND;
    if (t == 0) {
        double f = 0.0, b = 0.0, var = 0.0, ok = 0.0;
        if (bg) {
            const double det = v[0] * v[2] - v[1] * v[1];
            if (v[5] >= 2.0 && det > 1e-12 * v[0] * v[2]) {
                f = (v[3] * v[2] - v[1] * v[4]) / det;
                b = (v[0] * v[4] - v[1] * v[3]) / det;
                var = v[2] / det;
                ok = 1.0;
            }
        } else if (v[5] >= 1.0 && v[0] > 0.0) {
            f = v[3] / v[0];
            var = 1.0 / v[0];
            ok = 1.0;
        }
        sol[0] = f;
        sol[1] = b;
        sol[2] = ok;
        results[(size_t)blockIdx.x * 8 + 0] = f;
        results[(size_t)blockIdx.x * 8 + 1] = sqrt(var);
        results[(size_t)blockIdx.x * 8 + 2] = b;
        results[(size_t)blockIdx.x * 8 + 4] = ok != 0.0 ? v[5] : 0.0;
        results[(size_t)blockIdx.x * 8 + 5] = ok != 0.0 ? 0.0 : 1.0;
        results[(size_t)blockIdx.x * 8 + 6] = 0.0;
        results[(size_t)blockIdx.x * 8 + 7] = 0.0;
    }
    __syncthreads();
    const double f = sol[0], b = sol[1];
    double c2[1] = {0.0};
    for (int e = t; e < KK; e += kThreads) {
        const long long r = Y0 + e / K, s = X0 + e % K;
        if (r < 0 || r >= jb.ny || s < 0 || s >= jb.nx) continue;
        const size_t o = (size_t)r * pitch + (size_t)s;
        if (jb.mask && __ldg(jb.mask + o)) continue;
        const double w = jb.weight ? (double)__ldg(jb.weight + o) : 1.0;
        if (!(w > 0.0)) continue;
        const double res = pixel(jb, o) - f * (double)model[e] - b;
        c2[0] += w * res * res;
    }
    block_sums<1>(c2, reinterpret_cast<double(*)[1]>(red));
    if (t == 0) results[(size_t)blockIdx.x * 8 + 3] = sol[2] != 0.0 ? c2[0] : 0.0;
}

}  // namespace
}  // namespace sfft

using namespace sfft;

extern "C" sfft_status sfft_forced_photometry(int32_t njobs, const sfft_phot_job *jobs, int32_t K, int32_t flags,
                                              double *results, sfft_stream_t stream) {
    if (njobs < 0 || (njobs > 0 && (!jobs || !results)) || K < 1 || K > kMaxK || K % 2 == 0 ||
        (flags & ~SFFT_PHOT_BACKGROUND)) {
        set_global_error("sfft_forced_photometry: need njobs >= 0, device jobs and results, an odd K <= 63 "
                         "and known flags");
        return SFFT_ERR_INVALID_ARG;
    }
    if (njobs == 0) return SFFT_OK;
    if (njobs > 2147483647 / 8) {
        set_global_error("sfft_forced_photometry: too many jobs for one launch");
        return SFFT_ERR_INVALID_ARG;
    }
    note_launch();
    k_phot<<<njobs, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(jobs, K, flags, results);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof buf, "sfft_forced_photometry: %s", cudaGetErrorString(e));
        set_global_error(buf);
        return SFFT_ERR_CUDA;
    }
    return SFFT_OK;
}
