// Difference image:  D(u) = S(u) - sum_{i,d} a_{i,d} (w_i T)((u - d) mod N) - sum_r b_r w_r(u)
// on the unmasked frames, with w_i = xh^p yh^q evaluated at the source pixel u - d.
//
// Grouping the kernel monomials by their x power p folds the y power into per-row
// coefficients:  sum_i a_{i,d} xh_s^p yh_s^q T_s = sum_p xh_s^p T_s c_p(d, y_s),
// c_p(d, y_s) = sum_{i: p_i = p} a_{i,d} yh_s^q_i, so each output pixel costs
// (DK+1) L^2 multiply-adds instead of nP(DK) L^2.
//
// The folded coefficients depend only on the source row, so k_fold tabulates them once per
// call (FP64 sums rounded once) for every row: cf[ys][dy][p][dx] and bg[y][p].
// CTA: 8 output rows x 256 columns; a warp per row, 8 consecutive pixels per thread.
// Shared memory holds the cyclic template window (rows y0-h.., columns x0-h..), the x
// powers of its columns and the folded coefficients for the CTA's rows.
#include <type_traits>

#include "sfft_internal.cuh"

namespace sfft {
namespace {

constexpr int kRowsO = 8, kRX = 8, kColsO = 32 * kRX;
// Each lane reads a window starting at column 8 * lane; a skew of one word every 8 columns
// (index c + c / 8) makes the 32 lanes' addresses 9 words apart, i.e. on 32 distinct banks.
__device__ __forceinline__ int skew(int c) { return c + (c >> 3); }

template <class R>
__device__ __forceinline__ R coordv(int i, int n) {
    return n > 1 ? (R)(2 * i - (n - 1)) / (R)(n - 1) : (R)0;
}

// cf[ys][l][p] over l = (dy+h) L + (dx+h): sum_{i: p_i = p} a_{i,l} yh(ys)^q_i, and after
// the table bg[y][p] = sum_{r: p_r = p} b_r yh(y)^q_r
template <class R>
__global__ void k_fold(const double *__restrict__ coeffs, Geometry g, R *__restrict__ cf) {
    const int L2 = g.L * g.L, np = g.dk + 1, nbp = g.db + 1;
    const size_t ncf = (size_t)g.ny * L2;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ncf) {
        const int ys = (int)(t / L2), l = (int)(t - (size_t)ys * L2);
        const double yh = g.ny > 1 ? (2.0 * ys - (g.ny - 1)) / (double)(g.ny - 1) : 0.0;
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < g.nk; i++) {
            int pi, qi;
            mono_pq(i, pi, qi);
            double w = 1.0;
            for (int q = 0; q < qi; q++) w *= yh;
            acc[pi] = fma(coeffs[(size_t)i * L2 + l], w, acc[pi]);
        }
        const int dyi = l / g.L, dxi = l - dyi * g.L;
        R *o = cf + (((size_t)ys * g.L + dyi) * np) * g.L + dxi;
        for (int p = 0; p < np; p++) o[(size_t)p * g.L] = (R)acc[p];
    } else if (t < ncf + (size_t)g.ny) {
        const int y = (int)(t - ncf);
        const double yh = g.ny > 1 ? (2.0 * y - (g.ny - 1)) / (double)(g.ny - 1) : 0.0;
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int r = 0; r < g.nb; r++) {
            int pr, qr;
            mono_pq(r, pr, qr);
            double w = 1.0;
            for (int q = 0; q < qr; q++) w *= yh;
            acc[pr] = fma(coeffs[g.nker + r], w, acc[pr]);
        }
        R *o = cf + ncf * np + (size_t)y * nbp;
        for (int p = 0; p < nbp; p++) o[p] = (R)acc[p];
    }
}

// Stages a CTA's cyclic template window (times xh^p, masked when `masked`), the folded
// coefficients of its kRows output rows and their background x-power sums in shared memory.
template <class R, class In, int LL, int kRows>
__device__ __forceinline__ void stage_window(const In *__restrict__ tmpl, const uint8_t *__restrict__ mask,
                                             bool masked, const Geometry &g, const R *__restrict__ cfold,
                                             const R *__restrict__ xpow_g, int x0, int y0, R *Tp, R *cf, R *byp) {
    constexpr int h = LL / 2;
    constexpr int WC = kColsO + 2 * h;
    constexpr int WCS = WC + WC / 8 + 1;
    constexpr int WR = kRows + 2 * h;
    const int np = g.dk + 1, nx = g.nx, ny = g.ny, tid = threadIdx.x;
    for (int e = tid; e < WR * WC; e += blockDim.x) {
        int r = e / WC, c = e - r * WC;
        int yy = ((y0 - h + r) % ny + ny) % ny;
        int xx = ((x0 - h + c) % nx + nx) % nx;
        size_t u = (size_t)yy * g.pitch + xx;
        // the residual of the fit convolves the masked template W_i = w_i T_m
        R tv = (masked && mask && mask[u]) ? (R)0 : (R)tmpl[u];
        for (int p = 0; p < np; p++) Tp[(p * WR + r) * WCS + skew(c)] = tv * xpow_g[(size_t)p * nx + xx];
    }
    // folded kernel coefficients c_p(d, y - dy) for each of the CTA's output rows
    const int ncf = kRows * LL * np * LL;
    for (int e = tid; e < ncf; e += blockDim.x) {
        int dxi = e % LL, rest = e / LL;
        int p = rest % np;
        rest /= np;
        int dyi = rest % LL, ry = rest / LL;
        int ys = (((y0 + ry) - (dyi - h)) % ny + ny) % ny;  // source row y - dy
        cf[e] = cfold[(((size_t)ys * LL + dyi) * np + p) * LL + dxi];
    }
    const R *bgf = cfold + (size_t)ny * LL * LL * np;
    for (int e = tid; e < kRows * (g.db + 1); e += blockDim.x) {
        int ry = e / (g.db + 1), p = e % (g.db + 1);
        byp[e] = bgf[(size_t)min(y0 + ry, ny - 1) * (g.db + 1) + p];
    }
}

template <class R, class In, int LL>
__global__ void __launch_bounds__(256) k_subtract(const In *__restrict__ sci, const In *__restrict__ tmpl,
                                                 const uint8_t *__restrict__ mask, bool residual, Geometry g,
                                                 const R *__restrict__ cfold, const R *__restrict__ xpow_g,
                                                 In *__restrict__ diff) {
    constexpr int h = LL / 2;
    constexpr int WC = kColsO + 2 * h;  // window columns
    constexpr int WCS = WC + WC / 8 + 1; // skewed row length
    constexpr int WR = kRowsO + 2 * h;  // window rows
    constexpr int NW = kRX + LL - 1;    // register window per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int dk = g.dk, np = dk + 1;
    R *Tp = reinterpret_cast<R *>(smem_raw);  // [np][WR][WCS] skewed: template times xh^p
    R *cf = Tp + np * WR * WCS;                // [kRowsO][LL][np][LL]
    R *byp = cf + kRowsO * LL * np * LL;       // [kRowsO][db+1]  background per x power

    const int x0 = blockIdx.x * kColsO, y0 = blockIdx.y * kRowsO;
    const int tid = threadIdx.x;
    const int nx = g.nx, ny = g.ny;

    stage_window<R, In, LL, kRowsO>(tmpl, mask, residual, g, cfold, xpow_g, x0, y0, Tp, cf, byp);
    __syncthreads();

    const int ty = tid >> 5, lane = tid & 31;
    const int y = y0 + ty;
    const int cx = lane * kRX;  // first output column of this thread within the tile
    R out[kRX];
#pragma unroll
    for (int r = 0; r < kRX; r++) out[r] = (R)0;
    for (int dyi = 0; dyi < LL; dyi++) {
        // source row y - dy sits at window row ty + h - dy = ty + (LL - 1) - dyi
        const int wr = ty + (LL - 1) - dyi;
        for (int p = 0; p < np; p++) {
            const R *trow = Tp + (p * WR + wr) * WCS;
            R wp[NW];
#pragma unroll
            for (int m = 0; m < NW; m++) wp[m] = trow[skew(cx + m)];
            const R *c = cf + ((ty * LL + dyi) * np + p) * LL;
#pragma unroll
            for (int dxi = 0; dxi < LL; dxi++) {
                R cc = c[dxi];
                // source column x - dx -> window index (r - dx + h) = r + (LL - 1) - dxi
#pragma unroll
                for (int r = 0; r < kRX; r++) out[r] += cc * wp[r + (LL - 1) - dxi];
            }
        }
    }
    if (y < ny) {
        const R *bp = byp + ty * (g.db + 1);
#pragma unroll
        for (int r = 0; r < kRX; r++) {
            int x = x0 + cx + r;
            if (x < nx) {
                R bg = (R)0;
                for (int p = 0; p <= g.db; p++) bg += bp[p] * xpow_g[(size_t)p * nx + x];
                size_t u = (size_t)y * g.pitch + x;
                if (residual) {
                    R m = (mask && mask[u]) ? (R)0 : (R)1;
                    diff[u] = (In)(m * ((R)sci[u] - bg) - out[r]);
                } else {
                    diff[u] = (In)((R)sci[u] - out[r] - bg);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Residual of the fit for the FP32 path, R = S_m - sum a (w T_m)(u - d) - m sum b w, in
// compensated arithmetic.  At a star core |S| is ~100x the residual, so plain FP32 sums
// leave rounding errors of order u |S| in R; fitted back onto the basis by the refinement
// step they bound the coefficients near 1e-6.  The terms that carry |S| are those near the
// kernel centre, where both the kernel and the star's profile peak: for |dx|, |dy| <= kCore
// every product is split exactly (p + e = c w, e from an FMA) and the running sum is a
// hi + lo pair updated by an error-free two-sum (Knuth).  The outer lags, whose terms are
// the product of two wings, accumulate in plain FP32 in a separate sum.  R then carries
// about the rounding of its operands (the folded coefficients and xh^p T_m, each rounded
// once to FP32).  Each thread holds two output rows (ty, ty + kRowsC / 2) as the two lanes
// of packed FP32x2 operations.
constexpr int kRowsC = 8;
constexpr int kCore = 2;

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// s + e = a + b exactly (round-to-nearest adds, no reassociation: the _rn intrinsics are
// never contracted or reordered by the compiler)
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    float2 bb = __fadd2_rn(s, neg2(a));
    e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
}

template <class In>
__device__ __forceinline__ void split_input(In v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)((double)v - (double)hi);
}
template <>
__device__ __forceinline__ void split_input<float>(float v, float &hi, float &lo) {
    hi = v;
    lo = 0.f;
}

template <class In, int LL>
__global__ void __launch_bounds__(128, 2) k_residual_comp(const In *__restrict__ sci, const In *__restrict__ tmpl,
                                                      const uint8_t *__restrict__ mask, Geometry g,
                                                      const float *__restrict__ cfold,
                                                      const float *__restrict__ xpow_g, In *__restrict__ resid) {
    constexpr int h = LL / 2;
    constexpr int WC = kColsO + 2 * h;
    constexpr int WCS = WC + WC / 8 + 1;
    constexpr int WR = kRowsC + 2 * h;
    constexpr int NW = kRX + LL - 1;
    constexpr int kHalf = kRowsC / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int np = g.dk + 1, nx = g.nx, ny = g.ny;
    float *Tp = reinterpret_cast<float *>(smem_raw);  // [np][WR][WCS]
    float *cf = Tp + np * WR * WCS;                    // [kRowsC][LL][np][LL]
    float *byp = cf + kRowsC * LL * np * LL;           // [kRowsC][db+1]

    const int x0 = blockIdx.x * kColsO, y0 = blockIdx.y * kRowsC;
    stage_window<float, In, LL, kRowsC>(tmpl, mask, true, g, cfold, xpow_g, x0, y0, Tp, cf, byp);
    __syncthreads();

    const int ty = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cx = lane * kRX;
    const int ya = y0 + ty, yb = ya + kHalf;
    float2 hi[kRX], lo[kRX];
    // start from m (S - bg): S split exactly into hi + lo, the background subtracted by two-sum
#pragma unroll
    for (int r = 0; r < kRX; r++) {
        const int x = x0 + cx + r;
        float sh[2] = {0.f, 0.f}, sl[2] = {0.f, 0.f}, bg[2] = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int y = k ? yb : ya;
            if (y < ny && x < nx) {
                const size_t u = (size_t)y * g.pitch + x;
                if (!(mask && mask[u])) {
                    split_input<In>(sci[u], sh[k], sl[k]);
                    const float *bp = byp + (k ? ty + kHalf : ty) * (g.db + 1);
                    float b = 0.f;
                    for (int p = 0; p <= g.db; p++) b = fmaf(bp[p], xpow_g[(size_t)p * nx + x], b);
                    bg[k] = b;
                }
            }
        }
        float2 s, e;
        two_sum2(make_float2(sh[0], sh[1]), make_float2(-bg[0], -bg[1]), s, e);
        hi[r] = s;
        lo[r] = __fadd2_rn(e, make_float2(sl[0], sl[1]));
    }
    float2 wing[kRX];
#pragma unroll
    for (int r = 0; r < kRX; r++) wing[r] = make_float2(0.f, 0.f);
    for (int dyi = 0; dyi < LL; dyi++) {
        const int wra = ty + (LL - 1) - dyi, wrb = wra + kHalf;
        const bool core_row = dyi >= h - kCore && dyi <= h + kCore;
        for (int p = 0; p < np; p++) {
            const float *ta = Tp + (p * WR + wra) * WCS, *tb = Tp + (p * WR + wrb) * WCS;
            float2 wp[NW];
#pragma unroll
            for (int m = 0; m < NW; m++) wp[m] = make_float2(ta[skew(cx + m)], tb[skew(cx + m)]);
            const float *ca = cf + ((ty * LL + dyi) * np + p) * LL;
            const float *cb = cf + (((ty + kHalf) * LL + dyi) * np + p) * LL;
            if (core_row) {
#pragma unroll
                for (int dxi = 0; dxi < LL; dxi++) {
                    const float2 cc = make_float2(ca[dxi], cb[dxi]);
                    if (dxi >= h - kCore && dxi <= h + kCore) {
#pragma unroll
                        for (int r = 0; r < kRX; r++) {
                            const float2 w = wp[r + (LL - 1) - dxi];
                            const float2 pr = __fmul2_rn(cc, w);
                            const float2 pe = __ffma2_rn(cc, w, neg2(pr));  // cc w - pr, exact
                            float2 s, e;
                            two_sum2(hi[r], neg2(pr), s, e);
                            hi[r] = s;
                            lo[r] = __fadd2_rn(lo[r], __fadd2_rn(e, neg2(pe)));
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < kRX; r++) wing[r] = __ffma2_rn(cc, wp[r + (LL - 1) - dxi], wing[r]);
                    }
                }
            } else {
#pragma unroll
                for (int dxi = 0; dxi < LL; dxi++) {
                    const float2 cc = make_float2(ca[dxi], cb[dxi]);
#pragma unroll
                    for (int r = 0; r < kRX; r++) wing[r] = __ffma2_rn(cc, wp[r + (LL - 1) - dxi], wing[r]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kRX; r++) {
        const int x = x0 + cx + r;
        if (x >= nx) continue;
        if (ya < ny) resid[(size_t)ya * g.pitch + x] = (In)((double)hi[r].x + ((double)lo[r].x - (double)wing[r].x));
        if (yb < ny) resid[(size_t)yb * g.pitch + x] = (In)((double)hi[r].y + ((double)lo[r].y - (double)wing[r].y));
    }
}

template <class R, class In, int LL>
cudaError_t run(const Geometry &g, const void *sci, const void *tmpl, const uint8_t *mask, bool residual,
                const double *coeffs, const void *xpow, void *cfold, void *diff, cudaStream_t st) {
    {
        size_t nt = (size_t)g.ny * LL * LL + g.ny;
        note_launch();
        k_fold<R><<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(coeffs, g, (R *)cfold);
    }
    constexpr int h = LL / 2;
    const int np = g.dk + 1;
    constexpr int WCS = (kColsO + 2 * h) + (kColsO + 2 * h) / 8 + 1;
    size_t sm = sizeof(R) * ((size_t)np * (kRowsO + 2 * h) * WCS +
                             (size_t)kRowsO * LL * np * LL + (size_t)kRowsO * (g.db + 1));
    if constexpr (std::is_same<R, float>::value) {
        if (residual) {
            const size_t smc = sizeof(float) * ((size_t)np * (kRowsC + 2 * h) * WCS +
                                                (size_t)kRowsC * LL * np * LL + (size_t)kRowsC * (g.db + 1));
            auto kc = k_residual_comp<In, LL>;
            cudaError_t e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(kc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
            if (e != cudaSuccess) return e;
            dim3 gridc((g.nx + kColsO - 1) / kColsO, (g.ny + kRowsC - 1) / kRowsC);
            note_launch();
            kc<<<gridc, 128, smc, st>>>((const In *)sci, (const In *)tmpl, mask, g, (const float *)cfold,
                                        (const float *)xpow, (In *)diff);
            return cudaGetLastError();
        }
    }
    auto kern = k_subtract<R, In, LL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + kColsO - 1) / kColsO, (g.ny + kRowsO - 1) / kRowsO);
    note_launch();
    kern<<<grid, 256, sm, st>>>((const In *)sci, (const In *)tmpl, mask, residual, g, (const R *)cfold,
                                (const R *)xpow, (In *)diff);
    return cudaGetLastError();
}

template <class R, class In>
cudaError_t dispatch_L(const Geometry &g, const void *sci, const void *tmpl, const uint8_t *mask, bool residual,
                       const double *coeffs, const void *xpow, void *cfold, void *diff, cudaStream_t st) {
    switch (g.L) {
        case 1: return run<R, In, 1>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
        case 3: return run<R, In, 3>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
        case 5: return run<R, In, 5>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
        case 7: return run<R, In, 7>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
        case 9: return run<R, In, 9>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
        case 11: return run<R, In, 11>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
        case 13: return run<R, In, 13>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
        case 15: return run<R, In, 15>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_subtract(const Geometry &g, int dtype, int precision, const void *sci, const void *tmpl,
                            const uint8_t *mask, bool residual, const double *coeffs, const void *xpow,
                            const void *ypow, void *cfold, void *diff, cudaStream_t st) {
    (void)ypow;
    if (g.dk > 7 || g.db > 7) return cudaErrorInvalidValue;
    if (precision == SFFT_PREC_FP64)
        return dtype == SFFT_F64 ? dispatch_L<double, double>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st)
                                 : dispatch_L<double, float>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
    return dtype == SFFT_F64 ? dispatch_L<float, double>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st)
                             : dispatch_L<float, float>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, st);
}

}  // namespace sfft

// ---------------------------------------------------------------------------------------
// Difference image without any allocation: the same fold and subtract kernels, with their
// scratch (coordinate powers and folded coefficients) in a fixed device array that the
// library holds for the life of the process.
#include <stdio.h>

#include <mutex>

namespace sfft {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB, on every device that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// xh^p for p < np, FP64 powers rounded once (the table the planned path uploads)
template <class R>
__global__ void k_xpow_table(int nx, int np, R *__restrict__ out) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    double c = nx > 1 ? (2.0 * x - (nx - 1)) / (double)(nx - 1) : 0.0, v = 1.0;
    for (int p = 0; p < np; p++) {
        out[(size_t)p * nx + x] = (R)v;
        v *= c;
    }
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

void set_global_error(const char *msg);

}  // namespace sfft

using namespace sfft;

extern "C" sfft_status sfft_subtract_noalloc(const sfft_desc *desc, const void *sci, const void *tmpl,
                                             const double *coeffs, void *diff, sfft_stream_t stream) {
    char err[256];
    if (!desc || !sci || !tmpl || !coeffs || !diff) {
        set_global_error("sfft_subtract_noalloc: null argument");
        return SFFT_ERR_INVALID_ARG;
    }
    Geometry g;
    if (!make_geometry(*desc, g, err, sizeof err)) {
        set_global_error(err);
        return SFFT_ERR_INVALID_ARG;
    }
    if (diff == sci || diff == tmpl || (reinterpret_cast<uintptr_t>(sci) & 15) || (reinterpret_cast<uintptr_t>(tmpl) & 15)) {
        set_global_error("sfft_subtract_noalloc: diff aliases an input, or an input is not 16-byte aligned");
        return SFFT_ERR_INVALID_ARG;
    }
    if (g.dk > 7 || g.db > 7) {
        set_global_error("sfft_subtract_noalloc: dk and db must be <= 7");
        return SFFT_ERR_INVALID_ARG;
    }
    const size_t rsz = desc->precision == SFFT_PREC_FP64 ? 8 : 4;
    const int npx = (g.dk > g.db ? g.dk : g.db) + 1;
    const size_t xpow_bytes = align256((size_t)npx * g.nx * rsz);
    const size_t fold_bytes = align256(((size_t)g.ny * g.L * g.L * (g.dk + 1) + (size_t)g.ny * (g.db + 1)) * rsz);
    if (xpow_bytes + fold_bytes > kNoAllocScratchBytes) {
        snprintf(err, sizeof err,
                 "sfft_subtract_noalloc: this frame needs %zu bytes of scratch, the fixed device array holds %zu",
                 xpow_bytes + fold_bytes, kNoAllocScratchBytes);
        set_global_error(err);
        return SFFT_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_global_error("sfft_subtract_noalloc: no current CUDA device");
        return SFFT_ERR_CUDA;
    }
    void *scratch = nullptr;
    {
        // once per device, with that device current: the device address of the array
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) {
                snprintf(err, sizeof err, "sfft_subtract_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                set_global_error(err);
                return SFFT_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = ptr;
        }
        scratch = g_noalloc_ptr[dev];
    }
    // every value of both tables is written below before any kernel reads it, so the
    // previous call's contents never leak into this one
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void *xpow = scratch;
    void *cfold = static_cast<unsigned char *>(scratch) + xpow_bytes;
    note_launch();
    if (rsz == 8)
        k_xpow_table<double><<<(g.nx + 255) / 256, 256, 0, st>>>(g.nx, npx, (double *)xpow);
    else
        k_xpow_table<float><<<(g.nx + 255) / 256, 256, 0, st>>>(g.nx, npx, (float *)xpow);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        if (desc->precision == SFFT_PREC_FP64)
            e = desc->dtype == SFFT_F64 ? dispatch_L<double, double>(g, sci, tmpl, nullptr, false, coeffs, xpow, cfold, diff, st)
                                        : dispatch_L<double, float>(g, sci, tmpl, nullptr, false, coeffs, xpow, cfold, diff, st);
        else
            e = desc->dtype == SFFT_F64 ? dispatch_L<float, double>(g, sci, tmpl, nullptr, false, coeffs, xpow, cfold, diff, st)
                                        : dispatch_L<float, float>(g, sci, tmpl, nullptr, false, coeffs, xpow, cfold, diff, st);
    }
    if (e != cudaSuccess) {
        snprintf(err, sizeof err, "sfft_subtract_noalloc: %s", cudaGetErrorString(e));
        set_global_error(err);
        return SFFT_ERR_CUDA;
    }
    return SFFT_OK;
}
