// Alignment and resampling (Sec. "Pipeline steps", step 4; Sec. "GPU acceleration and
// performance"): the template image and its detection mask resampled onto the science
// grid, and the template PSF aligned to it.
//
// Coordinate model, window, bad-tap rule and flux scaling are the ones sfft.h states for
// sfft_resample.  Kernel design: one CTA per 32 x 32 output tile, four pixels per thread.
// Twenty threads first re-expand the coordinate polynomials about the tile corner
// (d_{p'q'} = sum_{p >= p', q >= q'} c_pq C(p, p') C(q, q') ax^(p - p') ay^(q - q'),
// (ax, ay) the corner's offset from the origin): the corner value d_00 in FP64, the other
// terms in FP32 (they multiply offsets below 32); each pixel then adds its FP32 Taylor part
// to the fractional part of the corner value, so the integer tap position is exact and the
// fraction carries an error below 1e-5 pixel.  The tile's tap footprint (exact, from a
// min/max over its pixels) is staged in shared memory as (value, bad) pairs -- masked and
// outside pixels as (0, 1), or (0, 0) outside with SFFT_RESAMPLE_ZERO_OUTSIDE -- so the taps
// are branch-free: sum w v and sum |w| bad.  Footprints above 56 x 56 (a scale change beyond
// ~1.5x, or a rotation with a scale above ~1.1) take a per-tap path from global memory.  A
// tap of weight exactly 0 then adds nothing either way, except that a non-finite unmasked
// pixel poisons its neighbours through 0 x inf: unmasked pixels are taken to be finite.  FP32 weights and sums (FP64
// images are converted on load).
#include <math.h>
#include <stdio.h>

#include "sfft_internal.cuh"

namespace sfft {

void set_global_error(const char *msg);

namespace {

constexpr int kTile = 32, kThreads = 256, kRowStep = kThreads / kTile, kPix = kTile / kRowStep;
constexpr int kStage = 56 * 56;  // staged footprint (value, bad) pairs: 25 KB
constexpr int kFar = -2147483647 - 1;

struct WarpArg {
    int n;  // monomials in use
    double xr, yr;
    double cu[10], cv[10];
    float xrf, yrf;          // the same rounded to FP32 (the Taylor terms)
    float cuf[10], cvf[10];
};

__device__ __forceinline__ float binom3f(int n, int k) {  // C(n, k) for 0 <= k <= n <= 3
    return (k == 0 || k == n) ? 1.f : (float)n;
}

// exponents (p, q) of the ten coordinate monomials in the order of sfft.h
__host__ __device__ constexpr int mono_p(int k) { return k == 1 || k == 4 || k == 8 ? 1 : k == 3 || k == 7 ? 2 : k == 6 ? 3 : 0; }
__host__ __device__ constexpr int mono_q(int k) { return k == 2 || k == 4 || k == 7 ? 1 : k == 5 || k == 8 ? 2 : k == 9 ? 3 : 0; }

template <class R>
__device__ __forceinline__ R powi3(R a, int e) {  // a^e for 0 <= e <= 3, without an indexed table
    return e == 0 ? R(1) : e == 1 ? a : e == 2 ? a * a : a * a * a;
}

template <int METHOD>
struct Taps;
template <>
struct Taps<SFFT_LANCZOS3> {
    static constexpr int n = 6, first = -2;
    __device__ __forceinline__ static void weights(float f, float *w) { lanczos3_taps(f, w); }
};
template <>
struct Taps<SFFT_BILINEAR> {
    static constexpr int n = 2, first = 0;
    __device__ __forceinline__ static void weights(float f, float *w) {
        w[0] = 1.f - f;
        w[1] = f;
    }
};

// Per-pixel state derived from the tile's Taylor coefficients: the first tap's column and row
// and the fractional positions (far: the map left the representable range; every tap outside).
struct PixelPos {
    int iu, iv;  // |corner| < 1e9 and the Taylor part stays small, so 32 bits hold them
    float fu, fv;
};

template <int FIRST>
__device__ __forceinline__ PixelPos pixel_pos(int n, const int *i0, const float *f0, const float (*d)[10], float fi,
                                              float fj, bool far) {
    float du = 0.f, dv = 0.f;
#pragma unroll
    for (int k = 1; k < 10; k++) {
        if (k < n) {
            const int p = mono_p(k), q = mono_q(k);
            const float m = powi3(fi, p) * powi3(fj, q);
            du = fmaf(d[0][k], m, du);
            dv = fmaf(d[1][k], m, dv);
        }
    }
    const float tu = far ? 0.f : f0[0] + du, tv = far ? 0.f : f0[1] + dv;
    const float flu = floorf(tu), flv = floorf(tv);
    PixelPos r;
    r.fu = tu - flu;
    r.fv = tv - flv;
    r.iu = far ? 0 : i0[0] + (int)flu + FIRST;
    r.iv = far ? 0 : i0[1] + (int)flv + FIRST;
    return r;
}

template <class In, int METHOD>
__global__ void __launch_bounds__(kThreads) k_resample(WarpArg wa, int flags, const In *__restrict__ in,
                                                       const uint8_t *__restrict__ in_mask, int in_ny, int in_nx,
                                                       int in_pitch, In *__restrict__ out,
                                                       uint8_t *__restrict__ out_mask, int out_ny, int out_nx,
                                                       int out_pitch) {
    using T = Taps<METHOD>;
    __shared__ int s_i0[2];    // floor of the corner's u and v
    __shared__ float s_f0[2];  // their fractions
    __shared__ float s_d[2][10];
    __shared__ int s_bb[4];  // tap footprint of the tile: u min, u max, v min, v max
    __shared__ float2 s_stage[kStage];
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile, t = threadIdx.x;
    if (t == 0) {
        s_bb[0] = s_bb[2] = 2147483647;
        s_bb[1] = s_bb[3] = -2147483647 - 1;
    }
    if (t < 20) {
        // lanes 0..9: u, lanes 10..19: v; lane k of each: Taylor coefficient k about the corner
        const int k = t % 10;
        const int pk = mono_p(k), qk = mono_q(k);
        if (k == 0) {
            // the corner value in FP64, kept as integer part + FP32 fraction (far outside: flagged)
            const double *c = t < 10 ? wa.cu : wa.cv;
            const double ax = (double)x0 - wa.xr, ay = (double)y0 - wa.yr;
            double sv = 0.0;
#pragma unroll
            for (int jm = 0; jm < 10; jm++)
                if (jm < wa.n) sv = fma(c[jm], powi3(ax, mono_p(jm)) * powi3(ay, mono_q(jm)), sv);
            const bool far = !(fabs(sv) < 1.0e9);
            const double fl = far ? 0.0 : floor(sv);
            s_i0[t < 10 ? 0 : 1] = far ? kFar : (int)fl;
            s_f0[t < 10 ? 0 : 1] = far ? 0.f : (float)(sv - fl);
        } else if (k < wa.n) {
            // d_k = sum_{p >= pk, q >= qk} c_pq C(p, pk) C(q, qk) ax^(p - pk) ay^(q - qk), FP32
            // (these terms multiply offsets below the tile size)
            const float *c = t < 10 ? wa.cuf : wa.cvf;
            const float fx = (float)x0 - wa.xrf, fy = (float)y0 - wa.yrf;
            float sv = 0.f;
#pragma unroll
            for (int jm = 1; jm < 10; jm++) {
                const int p = mono_p(jm), q = mono_q(jm);
                if (jm < wa.n && p >= pk && q >= qk)
                    sv = fmaf(c[jm] * binom3f(p, pk) * binom3f(q, qk), powi3(fx, p - pk) * powi3(fy, q - qk), sv);
            }
            s_d[t < 10 ? 0 : 1][k] = sv;
        }
    }
    __syncthreads();
    const bool far = s_i0[0] == kFar || s_i0[1] == kFar;
    const int i = t % kTile, jt = t / kTile;  // column; rows jt + kRowStep r
    const int x = x0 + i;
    // the tile's tap footprint: staged in shared memory as (value, bad) pairs when it is small
    int umin = 2147483647, umax = -2147483647 - 1, vmin = umin, vmax = umax;
    bool live_any = false;
#pragma unroll
    for (int r = 0; r < kPix; r++) {
        const int j = jt + kRowStep * r;
        if (x < out_nx && y0 + j < out_ny && !far) {
            const PixelPos pp = pixel_pos<T::first>(wa.n, s_i0, s_f0, s_d, (float)i, (float)j, far);
            umin = min(umin, (int)pp.iu);
            umax = max(umax, (int)pp.iu + T::n - 1);
            vmin = min(vmin, (int)pp.iv);
            vmax = max(vmax, (int)pp.iv + T::n - 1);
            live_any = true;
        }
    }
    umin = __reduce_min_sync(0xffffffffu, umin);
    umax = __reduce_max_sync(0xffffffffu, umax);
    vmin = __reduce_min_sync(0xffffffffu, vmin);
    vmax = __reduce_max_sync(0xffffffffu, vmax);
    const bool warp_live = __any_sync(0xffffffffu, live_any);  // every lane votes
    if ((t & 31) == 0 && warp_live) {
        atomicMin(&s_bb[0], umin);
        atomicMax(&s_bb[1], umax);
        atomicMin(&s_bb[2], vmin);
        atomicMax(&s_bb[3], vmax);
    }
    __syncthreads();
    const int bu0 = s_bb[0], bv0 = s_bb[2];
    const long long bw = (long long)s_bb[1] - bu0 + 1, bh = (long long)s_bb[3] - bv0 + 1;
    const bool staged = !far && s_bb[1] >= bu0 && bw * bh <= kStage;
    const bool zero_outside = flags & SFFT_RESAMPLE_ZERO_OUTSIDE;
    if (staged) {
        const int w = (int)bw, nst = (int)(bw * bh);
        for (int e = t; e < nst; e += kThreads) {
            const int r = bv0 + e / w, c = bu0 + e % w;
            float2 vb = make_float2(0.f, zero_outside ? 0.f : 1.f);
            if (r >= 0 && r < in_ny && c >= 0 && c < in_nx) {
                const size_t o = (size_t)r * in_pitch + (size_t)c;
                if (in_mask && __ldg(in_mask + o))
                    vb = make_float2(0.f, 1.f);
                else
                    vb = make_float2((float)__ldg(in + o), 0.f);
            }
            s_stage[e] = vb;
        }
        __syncthreads();
    }
    if (x >= out_nx) return;
#pragma unroll 1
    for (int r = 0; r < kPix; r++) {
        const int j = jt + kRowStep * r, y = y0 + j;
        if (y >= out_ny) break;
        const PixelPos pp = pixel_pos<T::first>(wa.n, s_i0, s_f0, s_d, (float)i, (float)j, far);
        float wx[T::n], wy[T::n];
        T::weights(pp.fu, wx);
        T::weights(pp.fv, wy);
        float sx = 0.f, sy = 0.f, ax = 0.f, ay = 0.f;
#pragma unroll
        for (int k = 0; k < T::n; k++) {
            sx += wx[k];
            sy += wy[k];
            ax += fabsf(wx[k]);
            ay += fabsf(wy[k]);
        }
        float acc = 0.f, bad = 0.f;
        if (staged) {
            const float2 *row = s_stage + ((int)pp.iv - bv0) * (int)bw + ((int)pp.iu - bu0);
#pragma unroll
            for (int a = 0; a < T::n; a++) {
                float rv = 0.f, rb = 0.f;
#pragma unroll
                for (int b = 0; b < T::n; b++) {
                    const float2 vb = row[b];
                    rv = fmaf(wx[b], vb.x, rv);
                    rb = fmaf(fabsf(wx[b]), vb.y, rb);
                }
                acc = fmaf(wy[a], rv, acc);
                bad = fmaf(fabsf(wy[a]), rb, bad);
                row += bw;
            }
        } else if (far) {
            bad = zero_outside ? 0.f : ax * ay;
        } else {
            for (int a = 0; a < T::n; a++) {
                if (wy[a] == 0.f) continue;
                const long long rr = pp.iv + a;
                const bool rin = rr >= 0 && rr < in_ny;
                for (int b = 0; b < T::n; b++) {
                    if (wx[b] == 0.f) continue;
                    const float w = wy[a] * wx[b];
                    const long long c = pp.iu + b;
                    if (!rin || c < 0 || c >= in_nx) {
                        if (!zero_outside) bad += fabsf(w);
                        continue;
                    }
                    const size_t o = (size_t)rr * in_pitch + (size_t)c;
                    if (in_mask && __ldg(in_mask + o)) {
                        bad += fabsf(w);
                        continue;
                    }
                    acc = fmaf(w, (float)__ldg(in + o), acc);
                }
            }
        }
        float val = acc / (sx * sy);
        if (flags & SFFT_RESAMPLE_FLUX) {
            const float fi = (float)i, fj = (float)j;
            float j00 = 0.f, j01 = 0.f, j10 = 0.f, j11 = 0.f;
#pragma unroll
            for (int k = 1; k < 10; k++) {
                if (k >= wa.n) break;
                const int p = mono_p(k), q = mono_q(k);
                // d/di and d/dj of i^p j^q
                const float ddi = p == 0 ? 0.f : (float)p * powi3(fi, p - 1) * powi3(fj, q);
                const float ddj = q == 0 ? 0.f : (float)q * powi3(fi, p) * powi3(fj, q - 1);
                j00 = fmaf(s_d[0][k], ddi, j00);
                j01 = fmaf(s_d[0][k], ddj, j01);
                j10 = fmaf(s_d[1][k], ddi, j10);
                j11 = fmaf(s_d[1][k], ddj, j11);
            }
            val *= fabsf(j00 * j11 - j01 * j10);
        }
        const size_t oo = (size_t)y * out_pitch + x;
        out[oo] = (In)val;
        if (out_mask) out_mask[oo] = bad > 0.01f * (ax * ay) ? 1 : 0;
    }
}

template <class In>
cudaError_t launch(int method, const WarpArg &wa, int flags, const void *in, const uint8_t *in_mask, int in_ny,
                   int in_nx, int in_pitch, void *out, uint8_t *out_mask, int out_ny, int out_nx, int out_pitch,
                   cudaStream_t st) {
    dim3 grid((out_nx + kTile - 1) / kTile, (out_ny + kTile - 1) / kTile);
    WarpArg w = wa;
    w.xrf = (float)wa.xr;
    w.yrf = (float)wa.yr;
    for (int k = 0; k < 10; k++) {
        w.cuf[k] = (float)wa.cu[k];
        w.cvf[k] = (float)wa.cv[k];
    }
    note_launch();
    if (method == SFFT_LANCZOS3)
        k_resample<In, SFFT_LANCZOS3><<<grid, kThreads, 0, st>>>(
            w, flags, (const In *)in, in_mask, in_ny, in_nx, in_pitch, (In *)out, out_mask, out_ny, out_nx, out_pitch);
    else
        k_resample<In, SFFT_BILINEAR><<<grid, kThreads, 0, st>>>(
            w, flags, (const In *)in, in_mask, in_ny, in_nx, in_pitch, (In *)out, out_mask, out_ny, out_nx, out_pitch);
    return cudaGetLastError();
}

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
    if (!a || !b) return false;
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + nb && pb < pa + na;
}

sfft_status run(const WarpArg &wa, int method, int flags, int in_ny, int in_nx, int in_pitch, int dtype,
                const void *in, const uint8_t *in_mask, int out_ny, int out_nx, int out_pitch, void *out,
                uint8_t *out_mask, cudaStream_t st, const char *who) {
    char buf[256];
    const size_t es = dtype == SFFT_F64 ? 8 : 4;
    const size_t in_n = (size_t)(in_ny - 1) * in_pitch + in_nx, out_n = (size_t)(out_ny - 1) * out_pitch + out_nx;
    if (ranges_overlap(out, out_n * es, in, in_n * es) || ranges_overlap(out, out_n * es, in_mask, in_n) ||
        ranges_overlap(out_mask, out_n, in, in_n * es) || ranges_overlap(out_mask, out_n, in_mask, in_n) ||
        ranges_overlap(out_mask, out_n, out, out_n * es)) {
        snprintf(buf, sizeof buf, "%s: an output overlaps an input or the other output", who);
        set_global_error(buf);
        return SFFT_ERR_INVALID_ARG;
    }
    cudaError_t e = dtype == SFFT_F64 ? launch<double>(method, wa, flags, in, in_mask, in_ny, in_nx, in_pitch, out,
                                                       out_mask, out_ny, out_nx, out_pitch, st)
                                      : launch<float>(method, wa, flags, in, in_mask, in_ny, in_nx, in_pitch, out,
                                                      out_mask, out_ny, out_nx, out_pitch, st);
    if (e != cudaSuccess) {
        snprintf(buf, sizeof buf, "%s: %s", who, cudaGetErrorString(e));
        set_global_error(buf);
        return SFFT_ERR_CUDA;
    }
    return SFFT_OK;
}

}  // namespace
}  // namespace sfft

using namespace sfft;

extern "C" sfft_status sfft_resample(const sfft_warp *warp, int32_t method, int32_t flags, int32_t in_ny,
                                     int32_t in_nx, int32_t in_pitch, int32_t dtype, const void *in,
                                     const uint8_t *in_mask, int32_t out_ny, int32_t out_nx, int32_t out_pitch,
                                     void *out, uint8_t *out_mask, sfft_stream_t stream) {
    if (!warp || !in || !out || warp->degree < 1 || warp->degree > 3 || in_ny < 1 || in_nx < 1 || out_ny < 1 ||
        out_nx < 1 || (method != SFFT_LANCZOS3 && method != SFFT_BILINEAR) ||
        (flags & ~(SFFT_RESAMPLE_FLUX | SFFT_RESAMPLE_ZERO_OUTSIDE)) || (dtype != SFFT_F32 && dtype != SFFT_F64)) {
        set_global_error("sfft_resample: need a warp of degree 1..3, non-empty frames, device images, "
                         "a known method, flags and dtype");
        return SFFT_ERR_INVALID_ARG;
    }
    if (in_pitch == 0) in_pitch = in_nx;
    if (out_pitch == 0) out_pitch = out_nx;
    if (in_pitch < in_nx || out_pitch < out_nx) {
        set_global_error("sfft_resample: pitch smaller than the row length");
        return SFFT_ERR_INVALID_ARG;
    }
    WarpArg wa;
    wa.n = npoly(warp->degree);
    wa.xr = warp->x_ref;
    wa.yr = warp->y_ref;
    for (int k = 0; k < 10; k++) {
        wa.cu[k] = k < wa.n ? warp->cu[k] : 0.0;
        wa.cv[k] = k < wa.n ? warp->cv[k] : 0.0;
    }
    return run(wa, method, flags, in_ny, in_nx, in_pitch, dtype, in, in_mask, out_ny, out_nx, out_pitch, out,
               out_mask, reinterpret_cast<cudaStream_t>(stream), "sfft_resample");
}

extern "C" sfft_status sfft_align_psf(const sfft_warp *warp, double x, double y, int32_t K, const float *psf_in,
                                      float *psf_out, sfft_stream_t stream) {
    if (!warp || !psf_in || !psf_out || warp->degree < 1 || warp->degree > 3 || K < 1 || K > 63 || K % 2 == 0) {
        set_global_error("sfft_align_psf: need a warp of degree 1..3, device stamps and an odd K <= 63");
        return SFFT_ERR_INVALID_ARG;
    }
    // Jacobian of the warp at (x, y), term by term in FP64
    const int n = npoly(warp->degree);
    const double dx = x - warp->x_ref, dy = y - warp->y_ref;
    double J[2][2] = {{0, 0}, {0, 0}};
    for (int k = 0; k < n; k++) {
        int p, q;
        mono_pq(k, p, q);
        const double ddx = p > 0 ? p * pow(dx, p - 1) * pow(dy, q) : 0.0;
        const double ddy = q > 0 ? q * pow(dx, p) * pow(dy, q - 1) : 0.0;
        J[0][0] += warp->cu[k] * ddx;
        J[0][1] += warp->cu[k] * ddy;
        J[1][0] += warp->cv[k] * ddx;
        J[1][1] += warp->cv[k] * ddy;
    }
    // output stamp pixel (r, s) reads template stamp position c + J (s - c, r - c)
    const double c = (K - 1) / 2.0;
    WarpArg wa;
    wa.n = 3;
    wa.xr = c;
    wa.yr = c;
    for (int k = 0; k < 10; k++) wa.cu[k] = wa.cv[k] = 0.0;
    wa.cu[0] = c;
    wa.cu[1] = J[0][0];
    wa.cu[2] = J[0][1];
    wa.cv[0] = c;
    wa.cv[1] = J[1][0];
    wa.cv[2] = J[1][1];
    return run(wa, SFFT_LANCZOS3, SFFT_RESAMPLE_FLUX | SFFT_RESAMPLE_ZERO_OUTSIDE, K, K, K, SFFT_F32, psf_in, nullptr,
               K, K, K, psf_out, nullptr, reinterpret_cast<cudaStream_t>(stream), "sfft_align_psf");
}
