// K2 in y-block FFT form, and the y-direction inverse of its cross-spectra.
//
// The normal matrix of the delta-basis fit (SFFT subtraction, Sec. "Pipeline steps",
// step 6) needs, per row segment s and x-frequency k of the segment spectra from K1, the
// y-direction lag correlations
//   Y(k, dy) = sum_s sum_y conj(A_s(y, k)) B_s((y + dy) mod Ny, k),   |dy| <= G = L - 1,
// for every (A, B) image pair the matrix uses: W_i x W_j (i <= j, |dy| <= L - 1) and
// W_i x Psi_r, W_i x S_m (|dy| <= h).  They are computed blockwise in y, the way K1 works
// in x: block t of a segment covers rows [t Uy, t Uy + Uy), Uy = Py - 2G.  Its A column is
// A_s(t Uy + j, k) for j < Uy, zero up to Py; its B column is B_s((t Uy - G + j) mod Ny, k)
// for j < Py.  With Ahat, Bhat the Py-point DFTs of the columns (e^{-2 pi i ky j / Py}),
//   Y(k, dy) = (1/Py) sum_ky e^{+2 pi i ky (G + dy) / Py} sum_{s,t} conj(Ahat_st(ky)) Bhat_st(ky)
// holds exactly: a lag |dy| <= G never carries a row of A's block past the end of B's.
//
// k_ycorr_fft: one CTA per (frequency k, share of the (segment, block) units, pair group).
// Per unit it stages the base spectra of the block's Py rows (cp.async, double-buffered),
// forms each image's column (the row factor yh^q applied here: W_pq = yh^q xh^p T_m has the
// spectrum yh^q times that of its x-weighted base image), takes the Py = 128-point DFT of
// every column (16 lanes per column, radix 8 x 16 with one padded shared-memory exchange,
// split twiddles), and adds conj(Ahat) Bhat for its pairs at every ky.  FP32 products are
// summed in FP32 registers over 8 units and then folded into a (hi, lo) float pair in
// shared memory by an error-free two-sum; FP64 products are summed in FP64.
// k_yinv: one warp per (frequency, pair): adds the CTAs' shares (double-float) and
// evaluates the inverse DFT at the pair's lags in double-float arithmetic, writing the
// per-frequency table that the x-direction inverse (k_lagx) turns into lag tables.
#include "sfft_internal.cuh"

namespace sfft {
namespace {

constexpr int kPy = 128;     // y-block FFT length
constexpr int kCS = 136;     // shared-memory stride of a column (8 x 17 exchange layout fits)
constexpr int kSP = kPy + 4;  // stride of a staged base column
constexpr int kFold = 8;     // FP32: units summed in registers before each two-sum fold

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <class R>
__device__ __forceinline__ cpx<R> twmul(cpx<R> v, cpx<R> wh, cpx<R> wl);
template <>
__device__ __forceinline__ cpx<float> twmul(cpx<float> v, cpx<float> wh, cpx<float> wl) {
    // v (wh + wl): the FP32 twiddle wh plus its remainder wl, so that every product is rounded
    // once from (nearly) the exact value (FP32-rounded twiddles alone have |wh| != 1)
    float tr = fmaf(v.re, wl.re, -v.im * wl.im);
    float ti = fmaf(v.re, wl.im, v.im * wl.re);
    return {fmaf(v.re, wh.re, fmaf(-v.im, wh.im, tr)), fmaf(v.re, wh.im, fmaf(v.im, wh.re, ti))};
}
template <>
__device__ __forceinline__ cpx<double> twmul(cpx<double> v, cpx<double> wh, cpx<double>) {
    return cmul(v, wh);
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

// forward 8-point DFT, natural order in and out: two 4-point DFTs of the even and odd
// samples, the odd ones turned by W8^k (W8^1 = tw[16], W8^3 = tw[48] of the 128-point table)
template <class R>
__device__ __forceinline__ void dft8(cpx<R> (&v)[8], const cpx<R> *tw, const cpx<R> *twl) {
    cpx<R> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    cpx<R> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    o1 = twmul(o1, tw[16], twl[16]);
    o2 = cpx<R>{o2.im, -o2.re};  // W8^2 = -i
    o3 = twmul(o3, tw[48], twl[48]);
    v[0] = e0 + o0;
    v[4] = e0 - o0;
    v[1] = e1 + o1;
    v[5] = e1 - o1;
    v[2] = e2 + o2;
    v[6] = e2 - o2;
    v[3] = e3 + o3;
    v[7] = e3 - o3;
}

// One 128-point forward DFT by the 16 lanes (t = lane & 15) of a half-warp.  On entry
// v[jj] = z[t + 16 jj]; on exit v[m] = Z[t + 16 m].  e is the FFT's exchange buffer
// (8 x 17 complex values), msk the lanes of the warp that take part.
//   Z[k1 + 8 k2] = sum_t W16^{t k2} W128^{t k1} sum_jj z[t + 16 jj] W8^{jj k1}
// Stage 1 is the 8-point DFT over jj and the W128^{t k1} turn.  Stage 2 is, for each k1, a
// 16-point DFT over t, split into its even outputs (k2 = 2m: an 8-point DFT of u_t + u_{t+8})
// and odd outputs (k2 = 2m + 1: an 8-point DFT of (u_t - u_{t+8}) W16^t); lane t takes
// k1 = t & 7 and the half t >> 3, so it produces Z[t + 16 m].
template <class R>
__device__ __forceinline__ void fft128(cpx<R> (&v)[8], int t, cpx<R> *e, const cpx<R> *tw, const cpx<R> *twl,
                                       unsigned msk) {
    dft8(v, tw, twl);
#pragma unroll
    for (int k1 = 1; k1 < 8; k1++) v[k1] = twmul(v[k1], tw[t * k1], twl[t * k1]);
#pragma unroll
    for (int k1 = 0; k1 < 8; k1++) e[k1 * 17 + t] = v[k1];
    __syncwarp(msk);
    const int k1 = t & 7, half = t >> 3;
    const R sgn = half ? (R)-1 : (R)1;
#pragma unroll
    for (int tt = 0; tt < 8; tt++) {
        const cpx<R> a = e[k1 * 17 + tt], b = e[k1 * 17 + tt + 8];
        const cpx<R> d = {a.re + sgn * b.re, a.im + sgn * b.im};
        const int wi = half ? 8 * tt : 0;  // W16^tt = W128^{8 tt}; index 0 is exactly 1
        v[tt] = twmul(d, tw[wi], twl[wi]);
    }
    __syncwarp(msk);
    dft8(v, tw, twl);
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
template <int B>
__device__ __forceinline__ void cp_async_n(void *smem, const void *gmem) {
    if constexpr (B == 16) cp_async16(smem, gmem);
    else if constexpr (B == 8) cp_async8(smem, gmem);
    else cp_async4(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The columns of a unit: A-side W_i (i < nk), then in the main pass the B-side W_j, Psi_r
// and S_m, in the refinement pass the residual R.  Pairs: W_i x W_j (i <= j, row-major upper
// triangle), then W_i x Psi_r and W_i x S_m (i major); in the refinement W_i x R.
struct YArgs {
    int nsplit;   // CTAs per frequency sharing the units
    int npairs;   // pairs per CTA group (grid.z enumerates the groups)
    int ncol;     // columns per unit
    int nstage;   // staged base columns per row
};

template <class R>
struct YSmem {
    // tw + twl, two staging buffers, the columns, the running sums (16 bytes each), yh^q for
    // two units, the pair and column tables
    static size_t bytes(int nstage, int qmax, int ncol, int npairs) {
        return sizeof(cpx<R>) * (2 * (size_t)kPy + 2 * (size_t)nstage * kSP + (size_t)ncol * kCS) +
               16 * (size_t)npairs * kPy + sizeof(R) * 2 * (size_t)(qmax > 0 ? qmax : 1) * kPy +
               sizeof(int) * (2 * (size_t)npairs + 3 * (size_t)ncol);
    }
};

template <class R, int NT, int NACC, bool WS>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : 2) k_ycorr_fft(const cpx<R> *__restrict__ spec, const cpx<R> *__restrict__ rspec,
                                                      const R *__restrict__ ypow, const cpx<R> *__restrict__ tw_g,
                                                      Geometry g, YArgs ya, void *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NGRP = NT / kPy;  // threads per ky
    const int qmax = g.dk > g.db ? g.dk : g.db;
    const int nq = qmax > 0 ? qmax : 1;
    const int nstage = ya.nstage, ncol = ya.ncol, npairs = ya.npairs;
    const int k = blockIdx.x, split = blockIdx.y;
    const int pair0 = WS ? 0 : blockIdx.z * npairs;                  // first pair of this CTA
    const int npg = WS ? g.nk : min(npairs, g.npair_all - pair0);    // its pairs
    const int pstride = WS ? g.nk : g.npair_all;                     // pairs per (split, k) in `out`
    const int tid = threadIdx.x;
    const int G = g.G, ny = g.ny, nkf = g.nkf, nrec = g.nrec, Uy = g.Uy, nyb = g.nyb;

    cpx<R> *tw = reinterpret_cast<cpx<R> *>(smem_raw);  // [Py] W128^m, high part
    cpx<R> *twl = tw + kPy;                             // [Py] remainder
    cpx<R> *stg = twl + kPy;                            // [2][nstage][kSP] staged base columns
    cpx<R> *cols = stg + 2 * (size_t)nstage * kSP;      // [ncol][kCS] column spectra
    // [npairs][Py] running sums, 16 bytes each: (hi, lo) float pairs, or FP64 values
    float4 *hl = reinterpret_cast<float4 *>(cols + (size_t)ncol * kCS);
    double2 *hd = reinterpret_cast<double2 *>(hl);
    R *yq = reinterpret_cast<R *>(hl + (size_t)npairs * kPy);  // [2][nq][Py] yh^q, q = 1..qmax
    int *pa = reinterpret_cast<int *>(yq + 2 * (size_t)nq * kPy);  // [npairs] A column of each pair
    int *pb = pa + npairs;                                          // [npairs] B column
    int *cst = pb + npairs;                                         // [ncol] staged base column
    int *cq = cst + ncol;                                           // [ncol] yh power
    int *ca = cq + ncol;                                            // [ncol] 1: A side

    for (int i = tid; i < kPy; i += NT) {
        tw[i] = tw_g[i];
        twl[i] = tw_g[kPy + i];
    }
    // base images of K1 per record: A_p (p <= dk), B_p (p <= dk), m_p (p <= db), S_m; the
    // refinement stages A_0..A_dk and then the residual
    const int na = g.dk + 1;
    for (int c = tid; c < ncol; c += NT) {
        int st = 0, q = 0, a = 0, p = 0;
        if (c < g.nk) {
            mono_pq(c, p, q);
            st = p;
            a = 1;
        } else if (WS) {
            st = na;  // the residual column
        } else if (c < 2 * g.nk) {
            mono_pq(c - g.nk, p, q);
            st = na + p;
        } else if (c < 2 * g.nk + g.nb) {
            mono_pq(c - 2 * g.nk, p, q);
            st = 2 * na + p;
        } else {
            st = g.nbase - 1;
        }
        cst[c] = st;
        cq[c] = q;
        ca[c] = a;
    }
    for (int i = tid; i < npg; i += NT) {
        const int pi = pair0 + i;
        int A, B;
        if (WS) {
            A = pi;
            B = g.nk;
        } else if (pi < g.npair) {
            int a = 0, rem = pi;
            while (rem >= g.nk - a) {
                rem -= g.nk - a;
                a++;
            }
            A = a;
            B = g.nk + a + rem;
        } else {
            const int qd = pi - g.npair;
            A = qd / (g.nb + 1);
            B = 2 * g.nk + qd % (g.nb + 1);
        }
        pa[i] = A;
        pb[i] = B;
    }
    for (int i = tid; i < npairs * kPy; i += NT) hl[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    // this CTA's share of the (segment, block) units, segment-major
    const int nunits = g.nseg * nyb;
    const int u0 = (int)((long)nunits * split / ya.nsplit), u1 = (int)((long)nunits * (split + 1) / ya.nsplit);

    auto stage = [&](int u, int buf) {
        const int s = u / nyb, t = u - s * nyb;
        const int yb = t * Uy - G;
        cpx<R> *dst = stg + (size_t)buf * nstage * kSP;
        for (int v = tid; v < kPy * nstage; v += NT) {
            const int jr = v / nstage, c = v - jr * nstage;
            int yy = (yb + jr) % ny;
            yy += yy < 0 ? ny : 0;
            const cpx<R> *src = (WS && c == nstage - 1) ? rspec + ((size_t)s * ny + yy) * nkf + k
                                                        : spec + (((size_t)s * ny + yy) * nkf + k) * nrec + c;
            cp_async_n<sizeof(cpx<R>)>(dst + (size_t)c * kSP + jr, src);
        }
        R *yqd = yq + (size_t)buf * nq * kPy;
        for (int v = tid; v < qmax * kPy; v += NT) {
            const int q = v / kPy, jr = v - q * kPy;
            int yy = (yb + jr) % ny;
            yy += yy < 0 ? ny : 0;
            cp_async_n<sizeof(R)>(yqd + v, ypow + (size_t)(q + 1) * ny + yy);
        }
        cp_async_commit();
    };

    float2 acc[NACC];  // FP32 path: products of up to kFold units before a fold
#pragma unroll
    for (int m = 0; m < NACC; m++) acc[m] = make_float2(0.f, 0.f);
    const int ky = tid % kPy, grp = tid / kPy;

    auto fold = [&]() {
#pragma unroll
        for (int m = 0; m < NACC; m++) {
            const int i = grp + NGRP * m;
            if (i < npg) {
                float4 hv = hl[(size_t)i * kPy + ky];
                float s1, e1, s2, e2;
                two_sum(hv.x, acc[m].x, s1, e1);
                two_sum(hv.y, acc[m].y, s2, e2);
                hl[(size_t)i * kPy + ky] = make_float4(s1, s2, hv.z + e1, hv.w + e2);
            }
            acc[m] = make_float2(0.f, 0.f);
        }
    };

    __syncthreads();
    if (u0 < u1) stage(u0, 0);
    int buf = 0;
    const int hw = tid >> 4, lt = tid & 15;
    const int wbase = (tid & ~31) >> 4;  // half-warp index of this warp's lane 0
    for (int u = u0; u < u1; u++) {
        cp_async_wait_all();
        __syncthreads();  // unit u staged; the previous unit's products are done with cols
        if (u + 1 < u1) stage(u + 1, buf ^ 1);
        const int t = u % nyb;
        const int avalid = min(Uy, ny - t * Uy);  // rows of the A column (the last block is short)
        const cpx<R> *sb = stg + (size_t)buf * nstage * kSP;
        const R *yqb = yq + (size_t)buf * nq * kPy;
        // every column's DFT: half-warp hw takes columns hw, hw + NT/16, ...
        for (int c0 = 0; c0 < ncol; c0 += NT / 16) {
            const int c = c0 + hw;
            const unsigned msk = (c0 + wbase < ncol ? 0x0000ffffu : 0u) | (c0 + wbase + 1 < ncol ? 0xffff0000u : 0u);
            if (c < ncol) {
                const cpx<R> *src = sb + (size_t)cst[c] * kSP;
                const int q = cq[c];
                const bool aside = ca[c] != 0;
                const R *yr = q > 0 ? yqb + (size_t)(q - 1) * kPy : nullptr;
                cpx<R> v[8];
#pragma unroll
                for (int jj = 0; jj < 8; jj++) {
                    const int j = lt + 16 * jj;
                    // A column: frame row t Uy + j is staged row j + G (zero past the block's
                    // own rows); B columns: staged row j
                    const bool ok = aside ? j < avalid : true;
                    const int jr = aside ? (ok ? j + G : 0) : j;
                    cpx<R> x = src[jr];
                    R w = yr ? yr[jr] : (R)1;
                    w = ok ? w : (R)0;
                    v[jj] = cpx<R>{x.re * w, x.im * w};
                }
                cpx<R> *e = cols + (size_t)c * kCS;
                fft128(v, lt, e, tw, twl, msk);
#pragma unroll
                for (int m = 0; m < 8; m++) e[lt + 16 * m] = v[m];
            }
        }
        __syncthreads();
        // cross-spectra of this unit: thread (ky, grp) takes pairs grp, grp + NGRP, ...
#pragma unroll
        for (int m = 0; m < NACC; m++) {
            const int i = grp + NGRP * m;
            if (i < npg) {
                const cpx<R> a = cols[(size_t)pa[i] * kCS + ky], b = cols[(size_t)pb[i] * kCS + ky];
                if constexpr (sizeof(R) == 4) {
                    acc[m].x = fmaf(a.re, b.re, fmaf(a.im, b.im, acc[m].x));
                    acc[m].y = fmaf(a.re, b.im, fmaf(-a.im, b.re, acc[m].y));
                } else {
                    double2 hv = hd[(size_t)i * kPy + ky];
                    hv.x = fma(a.re, b.re, fma(a.im, b.im, hv.x));
                    hv.y = fma(a.re, b.im, fma(-a.im, b.re, hv.y));
                    hd[(size_t)i * kPy + ky] = hv;
                }
            }
        }
        if constexpr (sizeof(R) == 4) {
            if ((u - u0) % kFold == kFold - 1) fold();
        }
        buf ^= 1;
    }
    if constexpr (sizeof(R) == 4) fold();
    __syncthreads();  // every thread's sums are in shared memory
    // this CTA's share: [split][k][pair][ky], 16 bytes per value
    float4 *o = reinterpret_cast<float4 *>(out) + (((size_t)split * nkf + k) * pstride + pair0) * kPy;
    for (int i = tid; i < npg * kPy; i += NT) o[i] = hl[i];
}

// ---------------------------------------------------------------- FP32, compile-time basis
// The same computation for FP32 spectra with the basis sizes as template parameters, laid
// out for few instructions per unit:
//  * staging: each thread owns fixed 16-byte chunks of the block's row records (cp.async),
//    so a unit only recomputes the rows' addresses;
//  * transforms: each half-warp transforms two columns at once, their values packed as
//    float2 (column c, column c + 1) so that every add and every twiddle product is one
//    packed FP32x2 instruction for both columns (the twiddles are shared);
//  * products: thread group g owns A images g and nk-1-g (equal pair counts) and every
//    B column of theirs; conj(a) b is accumulated as P += a.re b and Q += a.im b in packed
//    FFMA2 (re = P.x + Q.y, im = P.y - Q.x at the fold), folded every kFold2 units.
constexpr int kFold2 = 16;

struct C2 {  // the same element of two columns
    float2 re, im;
};

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ C2 c2add(C2 a, C2 b) { return {f2add(a.re, b.re), f2add(a.im, b.im)}; }
__device__ __forceinline__ C2 c2sub(C2 a, C2 b) { return {f2sub(a.re, b.re), f2sub(a.im, b.im)}; }

// v (wh + wl) for both columns; T = three float4 of the twiddle: (whr, whr, -whi, -whi),
// (whi, whi, wlr, wlr), (-wli, -wli, wli, wli); the small terms are added first
__device__ __forceinline__ C2 c2tw(C2 v, const float4 *T) {
    const float4 t0 = T[0], t1 = T[1], t2 = T[2];
    const float2 whr = make_float2(t0.x, t0.y), nwhi = make_float2(t0.z, t0.w);
    const float2 whi = make_float2(t1.x, t1.y), wlr = make_float2(t1.z, t1.w);
    const float2 nwli = make_float2(t2.x, t2.y), wli = make_float2(t2.z, t2.w);
    float2 re = __fmul2_rn(v.im, nwli);
    re = __ffma2_rn(v.re, wlr, re);
    re = __ffma2_rn(v.im, nwhi, re);
    re = __ffma2_rn(v.re, whr, re);
    float2 im = __fmul2_rn(v.im, wlr);
    im = __ffma2_rn(v.re, wli, im);
    im = __ffma2_rn(v.im, whr, im);
    im = __ffma2_rn(v.re, whi, im);
    return {re, im};
}

__device__ __forceinline__ void c2dft4(C2 &a0, C2 &a1, C2 &a2, C2 &a3) {
    const C2 s02 = c2add(a0, a2), d02 = c2sub(a0, a2), s13 = c2add(a1, a3), d13 = c2sub(a1, a3);
    a0 = c2add(s02, s13);
    a2 = c2sub(s02, s13);
    a1 = {f2add(d02.re, d13.im), f2sub(d02.im, d13.re)};  // d02 - i d13
    a3 = {f2sub(d02.re, d13.im), f2add(d02.im, d13.re)};  // d02 + i d13
}

// x / sqrt(2) with the constant split into its FP32 value and remainder (0x3F3504F3 and
// 0x324FE77A: 1/sqrt(2) to about 2^-48), so the product is rounded once from (nearly) the
// exact value
__device__ __forceinline__ float2 f2rs2(float2 x) {
    const float h = __int_as_float(0x3F3504F3), l = __int_as_float(0x324FE77A);
    const float2 ch = make_float2(h, h), cl = make_float2(l, l);
    return __ffma2_rn(x, ch, __fmul2_rn(x, cl));
}

// forward 8-point DFT (natural order); W8^1 = (1 - i)/sqrt(2), W8^3 = -(1 + i)/sqrt(2), W8^2 = -i
__device__ __forceinline__ void c2dft8(C2 (&v)[8], const float4 *tw3) {
    (void)tw3;
    C2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    c2dft4(e0, e1, e2, e3);
    c2dft4(o0, o1, o2, o3);
    {
        // o1 W8 = ((re + im) + i (im - re)) / sqrt(2); o3 W8^3 = ((im - re) - i (re + im)) / sqrt(2)
        const float2 s1 = f2add(o1.re, o1.im), d1 = f2sub(o1.im, o1.re);
        const float2 s3 = f2add(o3.re, o3.im), d3 = f2sub(o3.im, o3.re);
        o1 = {f2rs2(s1), f2rs2(d1)};
        o3 = {f2rs2(d3), f2rs2(make_float2(-s3.x, -s3.y))};
    }
    v[0] = c2add(e0, o0);
    v[4] = c2sub(e0, o0);
    v[1] = c2add(e1, o1);
    v[5] = c2sub(e1, o1);
    v[2] = {f2add(e2.re, o2.im), f2sub(e2.im, o2.re)};  // e2 - i o2
    v[6] = {f2sub(e2.re, o2.im), f2add(e2.im, o2.re)};  // e2 + i o2
    v[3] = c2add(e3, o3);
    v[7] = c2sub(e3, o3);
}

// v (wr + i wi) with wr = rh + rl and wi = ih + il given as FP32 splits (compile-time
// constants), in the operation order of c2tw (small terms first)
__device__ __forceinline__ C2 c2mulk(C2 v, float rh, float rl, float ih, float il) {
    const float2 whr = make_float2(rh, rh), nwhi = make_float2(-ih, -ih), whi = make_float2(ih, ih);
    const float2 wlr = make_float2(rl, rl), nwli = make_float2(-il, -il), wli = make_float2(il, il);
    float2 re = __fmul2_rn(v.im, nwli);
    re = __ffma2_rn(v.re, wlr, re);
    re = __ffma2_rn(v.im, nwhi, re);
    re = __ffma2_rn(v.re, whr, re);
    float2 im = __fmul2_rn(v.im, wlr);
    im = __ffma2_rn(v.re, wli, im);
    im = __ffma2_rn(v.im, whr, im);
    im = __ffma2_rn(v.re, whi, im);
    return {re, im};
}

// v W16^TT, W16 = exp(-2 pi i / 16), from the split constants cos(pi/8), sin(pi/8) and
// 1/sqrt(2) (each the FP32 value and its remainder, to about 2^-48)
template <int TT>
__device__ __forceinline__ C2 c2w16(C2 v) {
    const float ch = __int_as_float(0x3F6C835E), cl = __int_as_float(0x32F328D4);  // cos(pi/8)
    const float sh = __int_as_float(0x3EC3EF15), sl = __int_as_float(0x31D5D52C);  // sin(pi/8)
    const float rh = __int_as_float(0x3F3504F3), rl = __int_as_float(0x324FE77A);  // 1/sqrt(2)
    if constexpr (TT == 0) return v;
    else if constexpr (TT == 1) return c2mulk(v, ch, cl, -sh, -sl);
    else if constexpr (TT == 2) return c2mulk(v, rh, rl, -rh, -rl);
    else if constexpr (TT == 3) return c2mulk(v, sh, sl, -ch, -cl);
    else if constexpr (TT == 4) return {v.im, make_float2(-v.re.x, -v.re.y)};  // -i v
    else if constexpr (TT == 5) return c2mulk(v, -sh, -sl, -ch, -cl);
    else if constexpr (TT == 6) return c2mulk(v, -rh, -rl, -rh, -rl);
    else return c2mulk(v, -ch, -cl, -sh, -sl);
}

template <int TT>
__device__ __forceinline__ void c2stage2(C2 (&v)[8], const float4 *e, int k1, bool half, float2 sg) {
    const float4 a = e[k1 * 17 + TT], b = e[k1 * 17 + TT + 8];
    const C2 d = {__ffma2_rn(make_float2(b.x, b.y), sg, make_float2(a.x, a.y)),
                  __ffma2_rn(make_float2(b.z, b.w), sg, make_float2(a.z, a.w))};
    if constexpr (TT == 0) {
        v[0] = d;
    } else {
        const C2 w = c2w16<TT>(d);
        v[TT] = {half ? w.re : d.re, half ? w.im : d.im};
    }
}

// 128-point forward DFT of two columns by the 16 lanes of a half-warp (the decomposition of
// fft128); e: 8 x 17 float4 exchange slots (re pair, im pair).  tw3: the first stage's
// twiddles W128^(t k1) as [k1 - 1][t] entries of three float4 (consecutive lanes read
// consecutive entries: no bank conflicts); the second stage's W16^tt are constants.
__device__ __forceinline__ void c2fft128(C2 (&v)[8], int t, float4 *e, const float4 *tw3, unsigned msk) {
    c2dft8(v, tw3);
#pragma unroll
    for (int k1 = 1; k1 < 8; k1++) v[k1] = c2tw(v[k1], tw3 + 3 * ((k1 - 1) * 16 + t));
#pragma unroll
    for (int k1 = 0; k1 < 8; k1++) e[k1 * 17 + t] = make_float4(v[k1].re.x, v[k1].re.y, v[k1].im.x, v[k1].im.y);
    __syncwarp(msk);
    const int k1 = t & 7;
    const bool half = t >> 3;
    const float2 sg = half ? make_float2(-1.f, -1.f) : make_float2(1.f, 1.f);
    c2stage2<0>(v, e, k1, half, sg);
    c2stage2<1>(v, e, k1, half, sg);
    c2stage2<2>(v, e, k1, half, sg);
    c2stage2<3>(v, e, k1, half, sg);
    c2stage2<4>(v, e, k1, half, sg);
    c2stage2<5>(v, e, k1, half, sg);
    c2stage2<6>(v, e, k1, half, sg);
    c2stage2<7>(v, e, k1, half, sg);
    __syncwarp(msk);
    c2dft8(v, tw3);
}

template <int DK, int DB>
struct Basis {
    static constexpr int nk = (DK + 1) * (DK + 2) / 2, nb = (DB + 1) * (DB + 2) / 2;
    static constexpr int ncol = 2 * nk + nb + 1;                 // columns per unit
    static constexpr int ncp = (ncol + 1) / 2;                   // column pairs
    static constexpr int nbase = 2 * (DK + 1) + (DB + 1) + 1;
    static constexpr int nrec = (nbase + 1) & ~1;                // complex values per record
    // consumer groups of 128 threads, each owning whole A images (about equal pair counts):
    // nk = 1, 3: one group; nk = 6: {0, 3, 4} and {1, 2, 5}
    static constexpr int ngrp = nk == 6 ? 2 : 1;
    static constexpr int NC = ngrp * kPy;                        // consumer threads (products)
    static constexpr int NP = ((ncp * 16 + 31) / 32) * 32;       // producer threads (16 per pair)
    static constexpr int NT = NP + NC;
    static constexpr int qmax = DK > DB ? DK : DB;
    static constexpr int npair = nk * (nk + 1) / 2, npair_all = npair + nk * (nb + 1);
    static constexpr int chunks = kPy * nrec / 2;                // 16-byte staging chunks per unit
    static constexpr int nst = (chunks + NP - 1) / NP;           // per producer thread
};

// thread roles of the warp-specialised kernel: NPS producer sets of B::NP threads (set s
// transforms the units u0 + s, u0 + s + NPS, ...), then the B::NC consumers; 2 NPS column
// buffers, so that every set double-buffers its own units
template <int DK, int DB, int NPS>
struct Roles {
    using B = Basis<DK, DB>;
    static constexpr int NP = B::NP, NPT = NPS * B::NP, NC = B::NC, NT = NPT + NC, NBUF = 2 * NPS;
};

template <int DK, int DB, int NPS>
struct Smem32 {
    using B = Basis<DK, DB>;
    static constexpr int ncolp = (B::ncol + 1) & ~1;  // columns rounded to whole pairs
    static constexpr int nbuf = 2 * NPS;
    // tw3 [7][16][3] float4 (room for [Py][3]), stg [NPS][2][Py][nrec] float2, yq [NPS][2][qmax][Py],
    // cols [nbuf][ncolp][Py] float4 (re, re, im, im), column tables [ncol][3] int
    static constexpr size_t tw3 = 0;
    static constexpr size_t stg = tw3 + 16 * 3 * kPy;
    static constexpr size_t yq = stg + 8 * 2 * NPS * (size_t)kPy * B::nrec;
    static constexpr size_t cols = yq + 4 * 2 * NPS * (size_t)(B::qmax > 0 ? B::qmax : 1) * kPy;
    static constexpr size_t tab = cols + 16 * nbuf * (size_t)ncolp * kPy;
    static constexpr size_t bytes = tab + 4 * 3 * (size_t)B::ncol;
};

// pair index of (A image i, B column c): W_i x W_j (c = nk + j, i <= j) or W_i x Psi_r / S_m
__host__ __device__ constexpr int pair_of(int nk, int nb, int i, int c) {
    return c < 2 * nk ? i * nk - i * (i - 1) / 2 + (c - nk - i) : nk * (nk + 1) / 2 + i * (nb + 1) + (c - 2 * nk);
}

// named CTA barriers (id 0 is __syncthreads): count threads, whole warps
__device__ __forceinline__ void nb_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void nb_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

// adds (hi, lo) of P (complex FP32 partial) into the double-float value at h
__device__ __forceinline__ void fold_into(float4 *h, float2 P) {
    const float4 hv = *h;
    float s1, e1, s2, e2;
    two_sum(hv.x, P.x, s1, e1);
    two_sum(hv.y, P.y, s2, e2);
    *h = make_float4(s1, s2, hv.z + e1, hv.w + e2);
}

// One consumer thread's share of one A image I (I < 0: none): its products with every B
// column c = nk + I .. ncol - 1 at frequency ky, in acc.  cols[b][c][ky] = (re, re, im, im),
// so conj(a) b = (b.re, b.re)(a.re, -a.im) + (b.im, b.im)(a.im, a.re): two packed FMAs on
// one accumulator.
template <int DK, int DB, int I>
struct ImageAcc {
    using B = Basis<DK, DB>;
    static constexpr int n = I < 0 ? 0 : B::ncol - B::nk - I;
    float2 acc[n > 0 ? n : 1];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int m = 0; m < n; m++) acc[m] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void add(const float4 *cb) {
        if constexpr (n > 0) {
            const float4 a = cb[(size_t)I * kPy];
            const float2 p1 = make_float2(a.x, -a.z), p2 = make_float2(a.z, a.x);
#pragma unroll
            for (int m = 0; m < n; m++) {
                const float4 v = cb[(size_t)(B::nk + I + m) * kPy];
                acc[m] = __ffma2_rn(make_float2(v.x, v.y), p1, acc[m]);
                acc[m] = __ffma2_rn(make_float2(v.z, v.w), p2, acc[m]);
            }
        }
    }
    __device__ __forceinline__ void fold(float4 *share, int ky) {
#pragma unroll
        for (int m = 0; m < n; m++) {
            fold_into(share + (size_t)pair_of(B::nk, B::nb, I, B::nk + I + m) * kPy + ky, acc[m]);
            acc[m] = make_float2(0.f, 0.f);
        }
    }
};

// a consumer group: A images I0, I1, I2 (-1: none), summed over the units in FP32 and
// folded into the CTA's share in global memory every kFold2 units.  Unit u sits in column
// buffer (u - u0) mod NBUF: barrier 1 + b says it is full, 5 + b that it has been read.
template <int DK, int DB, int NPS, int I0, int I1, int I2>
__device__ __forceinline__ void consume(const float4 *cols, int ky, int u0, int u1, float4 *share) {
    using R = Roles<DK, DB, NPS>;
    constexpr int ncolp = Smem32<DK, DB, NPS>::ncolp, NB = R::NC + R::NP;
    ImageAcc<DK, DB, I0> a0;
    ImageAcc<DK, DB, I1> a1;
    ImageAcc<DK, DB, I2> a2;
    a0.zero();
    a1.zero();
    a2.zero();
    for (int u = u0; u < u1; u++) {
        const int b = (u - u0) % R::NBUF;
        nb_sync(1 + b, NB);  // cols[b] holds unit u
        const float4 *cb = cols + (size_t)b * ncolp * kPy + ky;
        a0.add(cb);
        a1.add(cb);
        a2.add(cb);
        nb_arrive(5 + b, NB);  // done reading cols[b]
        if ((u - u0) % kFold2 == kFold2 - 1) {
            a0.fold(share, ky);
            a1.fold(share, ky);
            a2.fold(share, ky);
        }
    }
    a0.fold(share, ky);
    a1.fold(share, ky);
    a2.fold(share, ky);
}

// Warp-specialised: the first NPS x NP threads are producers in NPS sets (a set stages its
// units' rows, forms and transforms their columns into cols[b], b = (u - u0) mod 2 NPS), the
// other NC threads consumers (the products of cols[b], units in order).  Barriers 1 + b
// ("cols[b] full") and 5 + b ("cols[b] read") hand each buffer over between one set and the
// consumers; barrier 9 + s orders set s's staging.  A set transforms its next unit while the
// consumers multiply earlier ones, and with two sets two units are transformed at once.  The
// CTA's share of the sums, [pair][ky] (hi, lo) float pairs, lives in its slice of `out`
// (zeroed here, folded into by the consumers).
template <int DK, int DB, int NPS>
__global__ void __launch_bounds__(Roles<DK, DB, NPS>::NT, 1)
    k_ycorr_fft32(const float2 *__restrict__ spec, const float *__restrict__ ypow, const float2 *__restrict__ tw_g,
                  Geometry g, int nsplit, float4 *__restrict__ out) {
    using B = Basis<DK, DB>;
    using R = Roles<DK, DB, NPS>;
    using SM = Smem32<DK, DB, NPS>;
    constexpr int NT = R::NT, NP = R::NP, NQ = B::qmax > 0 ? B::qmax : 1, ncolp = SM::ncolp, NB = R::NC + R::NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *tw3 = reinterpret_cast<float4 *>(smem_raw + SM::tw3);
    float2 *stg = reinterpret_cast<float2 *>(smem_raw + SM::stg);
    float *yq = reinterpret_cast<float *>(smem_raw + SM::yq);
    float4 *cols = reinterpret_cast<float4 *>(smem_raw + SM::cols);
    int *cst = reinterpret_cast<int *>(smem_raw + SM::tab), *cq = cst + B::ncol, *ca = cq + B::ncol;
    const int k = blockIdx.x, split = blockIdx.y, tid = threadIdx.x;
    const int G = g.G, ny = g.ny, nkf = g.nkf, Uy = g.Uy, nyb = g.nyb;
    float4 *share = out + ((size_t)split * nkf + k) * B::npair_all * kPy;

    for (int i = tid; i < 7 * 16; i += NT) {
        const int m = (i >> 4) * (i & 15) + (i & 15);  // (k1 - 1, t) -> t k1
        const float2 h = tw_g[m], l = tw_g[kPy + m];   // exp(-2 pi i m / Py): high part, remainder
        tw3[3 * i] = make_float4(h.x, h.x, -h.y, -h.y);
        tw3[3 * i + 1] = make_float4(h.y, h.y, l.x, l.x);
        tw3[3 * i + 2] = make_float4(-l.y, -l.y, l.y, l.y);
    }
    for (int c = tid; c < B::ncol; c += NT) {
        int st = 0, q = 0, a = 0, p = 0;
        if (c < B::nk) {
            mono_pq(c, p, q);
            st = p;
            a = 1;
        } else if (c < 2 * B::nk) {
            mono_pq(c - B::nk, p, q);
            st = DK + 1 + p;
        } else if (c < 2 * B::nk + B::nb) {
            mono_pq(c - 2 * B::nk, p, q);
            st = 2 * (DK + 1) + p;
        } else {
            st = B::nbase - 1;
        }
        cst[c] = st;
        cq[c] = q;
        ca[c] = a;
    }
    for (int i = tid; i < B::npair_all * kPy; i += NT) share[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int nunits = g.nseg * nyb;
    const int u0 = (int)((long)nunits * split / nsplit), u1 = (int)((long)nunits * (split + 1) / nsplit);
    __syncthreads();  // tables built, the share zeroed (each consumer later touches its own entries)

    if (tid < R::NPT) {
        // ------------------------------------------------------------ producers, set ps
        const int ps = tid / NP, ptid = tid - ps * NP;
        const bool tiny = ny < kPy + 2 * G;  // rows may wrap more than once
        auto wrap = [&](int y) {
            if (tiny) {
                y %= ny;
                return y < 0 ? y + ny : y;
            }
            y += y < 0 ? ny : 0;
            return y >= ny ? y - ny : y;
        };
        float2 *stg_s = stg + (size_t)ps * 2 * kPy * B::nrec;
        float *yq_s = yq + (size_t)ps * 2 * NQ * kPy;
        auto stage = [&](int u, int buf) {
            const int s = u / nyb, t = u - s * nyb;
            const int yb = t * Uy - G;
            float2 *dst = stg_s + (size_t)buf * kPy * B::nrec;
#pragma unroll
            for (int i = 0; i < B::nst; i++) {
                // chunk `item`: row jr of the block, 16-byte piece `off / 2` of its record
                const int item = ptid + i * NP;
                if (item >= B::chunks) continue;
                const int jr = item / (B::nrec / 2), off = 2 * (item - jr * (B::nrec / 2));
                const int yy = wrap(yb + jr);
                const float2 *src = spec + (((size_t)s * ny + yy) * nkf + k) * B::nrec + off;
                cp_async16(dst + jr * B::nrec + off, src);
            }
            for (int v = ptid; v < B::qmax * kPy; v += NP) {
                const int q = v / kPy, jr = v - q * kPy;
                cp_async4(yq_s + (size_t)buf * NQ * kPy + v, ypow + (size_t)(q + 1) * ny + wrap(yb + jr));
            }
            cp_async_commit();
        };
        const int hw = ptid >> 4, lt = ptid & 15;
        const int wbase = (ptid & ~31) >> 4;
        if (u0 + ps < u1) stage(u0 + ps, 0);
        int sbuf = 0;
        for (int u = u0 + ps; u < u1; u += NPS) {
            const int b = (u - u0) % R::NBUF;
            cp_async_wait_all();
            nb_sync(9 + ps, NP);  // unit u staged for every thread of the set; its previous transforms done
            if (u + NPS < u1) stage(u + NPS, sbuf ^ 1);
            if (u - u0 >= R::NBUF) nb_sync(5 + b, NB);  // consumers have read cols[b] (unit u - NBUF)
            const int t = u % nyb;
            const int avalid = min(Uy, ny - t * Uy);
            const float2 *sb = stg_s + (size_t)sbuf * kPy * B::nrec;
            const float *yqb = yq_s + (size_t)sbuf * NQ * kPy;
            float4 *cb = cols + (size_t)b * ncolp * kPy;
            if (hw < B::ncp) {
                const unsigned msk = (wbase < B::ncp ? 0x0000ffffu : 0u) | (wbase + 1 < B::ncp ? 0xffff0000u : 0u);
                const int c0 = 2 * hw, c1 = c0 + 1 < B::ncol ? c0 + 1 : c0;  // an odd count repeats its last column
                const int s0 = cst[c0], s1 = cst[c1], q0 = cq[c0], q1 = cq[c1], a0 = ca[c0], a1 = ca[c1];
                C2 v[8];
#pragma unroll
                for (int jj = 0; jj < 8; jj++) {
                    const int j = lt + 16 * jj;
                    // A column: frame row t Uy + j is staged row j + G (zero past the block's own
                    // rows); B columns: staged row j
                    const bool ok0 = !a0 || j < avalid, ok1 = !a1 || j < avalid;
                    const int r0 = a0 ? (ok0 ? j + G : 0) : j, r1 = a1 ? (ok1 ? j + G : 0) : j;
                    const float2 x0 = sb[r0 * B::nrec + s0], x1 = sb[r1 * B::nrec + s1];
                    float w0 = q0 ? yqb[(q0 - 1) * kPy + r0] : 1.f, w1 = q1 ? yqb[(q1 - 1) * kPy + r1] : 1.f;
                    w0 = ok0 ? w0 : 0.f;
                    w1 = ok1 ? w1 : 0.f;
                    v[jj] = {make_float2(x0.x * w0, x1.x * w1), make_float2(x0.y * w0, x1.y * w1)};
                }
                // the pair's two column slots (2 x 128 float4) hold its 8 x 17 exchange first
                float4 *pc = cb + (size_t)c0 * kPy;
                c2fft128(v, lt, pc, tw3, msk);
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    pc[lt + 16 * m] = make_float4(v[m].re.x, v[m].re.x, v[m].im.x, v[m].im.x);
                    if (c1 != c0) pc[kPy + lt + 16 * m] = make_float4(v[m].re.y, v[m].re.y, v[m].im.y, v[m].im.y);
                }
            }
            nb_arrive(1 + b, NB);  // cols[b] holds unit u
            sbuf ^= 1;
        }
        // take the consumers' last "read" arrivals on this set's buffers, so that every
        // barrier generation completes
        for (int u = u0 + ps; u < u1; u += NPS)
            if (u + R::NBUF >= u1) nb_sync(5 + (u - u0) % R::NBUF, NB);
        return;
    }
    // ---------------------------------------------------------------- consumers
    const int ct = tid - R::NPT, ky = ct % kPy, grp = ct / kPy;
    if constexpr (B::nk == 6) {
        if (grp == 0) consume<DK, DB, NPS, 0, 3, 4>(cols, ky, u0, u1, share);
        else consume<DK, DB, NPS, 1, 2, 5>(cols, ky, u0, u1, share);
    } else if constexpr (B::nk == 3) {
        consume<DK, DB, NPS, 0, 1, 2>(cols, ky, u0, u1, share);
    } else {
        consume<DK, DB, NPS, 0, -1, -1>(cols, ky, u0, u1, share);
    }
}

template <int DK, int DB, int NPS>
cudaError_t run_fft32(const Geometry &g, const void *spec, const void *ypow, const void *tw_y, double *part,
                      cudaStream_t st) {
    using SM = Smem32<DK, DB, NPS>;
    auto kern = k_ycorr_fft32<DK, DB, NPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    dim3 grid(g.nkf, g.y2split, 1);
    note_launch();
    kern<<<grid, Roles<DK, DB, NPS>::NT, SM::bytes, st>>>((const float2 *)spec, (const float *)ypow, (const float2 *)tw_y,
                                                     g, g.y2split, reinterpret_cast<float4 *>(part));
    return cudaGetLastError();
}

// the bases with a compile-time FP32 kernel (shared memory within the budget, one pair
// group); others run the generic kernel
bool fft32_specialised(int dk, int db) {
    return (dk == 2 && (db == 2 || db == 1 || db == 0)) || (dk == 1 && db <= 2) || (dk == 0 && db <= 2);
}
static_assert(Smem32<2, 2, 2>::bytes <= 227 * 1024, "the DK = DB = 2 kernel's shared memory, two producer sets");

cudaError_t dispatch_fft32(const Geometry &g, const void *spec, const void *ypow, const void *tw_y, double *part,
                           cudaStream_t st) {
#define SFFT_Y32(a, b)                                                                           \
    if (g.dk == a && g.db == b)                                                                  \
        return g.ysets == 1 ? run_fft32<a, b, 1>(g, spec, ypow, tw_y, part, st)                  \
                            : run_fft32<a, b, 2>(g, spec, ypow, tw_y, part, st);
    SFFT_Y32(2, 2) SFFT_Y32(2, 1) SFFT_Y32(2, 0) SFFT_Y32(1, 2) SFFT_Y32(1, 1) SFFT_Y32(1, 0) SFFT_Y32(0, 2)
    SFFT_Y32(0, 1) SFFT_Y32(0, 0)
#undef SFFT_Y32
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- y-direction inverse
// double-float helpers: exact product error by FMA, error-free sum
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

// (sh, sl) += (ah + al)(bh + bl) for real operands, to about u^2
__device__ __forceinline__ void df_mac(float &sh, float &sl, float ah, float al, float bh, float bl) {
    float p, e, s, e2;
    two_prod(ah, bh, p, e);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    two_sum(sh, p, s, e2);
    sh = s;
    sl += e2 + e;
}

// ysum[k][ent(pair, dy)] = (1/Py) sum_ky e^{+2 pi i ky (G + dy)/Py} sum_c part[c][k][pair][ky]
// one warp per (k, pair); lane l takes ky = l + 32 j.  ws: the refinement's W_i x R pairs,
// written to the W_i x S_m entries.
template <class R>
__global__ void __launch_bounds__(256) k_yinv(const void *__restrict__ part, const void *__restrict__ twi, Geometry g,
                                             int nsplit, int npairs, bool ws, double2 *__restrict__ ysum) {
    const int warp = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= g.nkf * npairs) return;  // whole warps leave together
    const int k = warp / npairs, pi = warp - k * npairs;
    const int L = g.L, h = g.h, G = g.G, Lw = 2 * L - 1;
    int m0, m1, ent0;  // lag range m = G + dy in [m0, m1]; entry of m0
    if (!ws && pi < g.npair) {
        m0 = 0;
        m1 = 2 * G;
        ent0 = pi * Lw;
    } else {
        const int qd = ws ? pi * (g.nb + 1) + g.nb : pi - g.npair;
        m0 = G - h;
        m1 = G + h;
        ent0 = g.npair * Lw + qd * L;
    }
    constexpr int J = kPy / 32;
    const int pstride = ws ? g.nk : g.npair_all;                  // pairs per (split, k)
    const size_t stride = (size_t)g.nkf * pstride * kPy;          // between the CTAs' shares
    const size_t base = ((size_t)k * pstride + pi) * kPy;
    if constexpr (sizeof(R) == 4) {
        const float4 *p4 = reinterpret_cast<const float4 *>(part);
        const float4 *w4 = reinterpret_cast<const float4 *>(twi);  // (cos hi, sin hi, cos lo, sin lo)
        float crh[J], crl[J], cih[J], cil[J];
#pragma unroll
        for (int j = 0; j < J; j++) {
            float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
            for (int c = 0; c < nsplit; c++) {
                const float4 v = p4[c * stride + base + lane + 32 * j];
                float s, e;
                two_sum(rh, v.x, s, e);
                rh = s;
                rl += e + v.z;
                two_sum(ih, v.y, s, e);
                ih = s;
                il += e + v.w;
            }
            crh[j] = rh;
            crl[j] = rl;
            cih[j] = ih;
            cil[j] = il;
        }
        for (int m = m0; m <= m1; m++) {
            float yrh = 0.f, yrl = 0.f, yih = 0.f, yil = 0.f;
#pragma unroll
            for (int j = 0; j < J; j++) {
                const int kyv = lane + 32 * j;
                const float4 w = w4[(kyv * m) & (kPy - 1)];
                // (cr + i ci)(wr + i wi): re = cr wr - ci wi, im = cr wi + ci wr
                df_mac(yrh, yrl, crh[j], crl[j], w.x, w.z);
                df_mac(yrh, yrl, -cih[j], -cil[j], w.y, w.w);
                df_mac(yih, yil, crh[j], crl[j], w.y, w.w);
                df_mac(yih, yil, cih[j], cil[j], w.x, w.z);
            }
            // fixed shuffle tree over the lanes, double-float adds
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float orh = __shfl_xor_sync(0xffffffffu, yrh, o), orl = __shfl_xor_sync(0xffffffffu, yrl, o);
                const float oih = __shfl_xor_sync(0xffffffffu, yih, o), oil = __shfl_xor_sync(0xffffffffu, yil, o);
                float s, e;
                two_sum(yrh, orh, s, e);
                yrh = s;
                yrl += e + orl;
                two_sum(yih, oih, s, e);
                yih = s;
                yil += e + oil;
            }
            if (lane == 0)
                ysum[(size_t)k * g.nent + ent0 + (m - m0)] =
                    make_double2(((double)yrh + (double)yrl) * (1.0 / kPy), ((double)yih + (double)yil) * (1.0 / kPy));
        }
    } else {
        const double2 *p2 = reinterpret_cast<const double2 *>(part);
        const double2 *w2 = reinterpret_cast<const double2 *>(twi);
        double cr[J], ci[J];
#pragma unroll
        for (int j = 0; j < J; j++) {
            double sr = 0.0, si = 0.0;
            for (int c = 0; c < nsplit; c++) {
                const double2 v = p2[c * stride + base + lane + 32 * j];
                sr += v.x;
                si += v.y;
            }
            cr[j] = sr;
            ci[j] = si;
        }
        for (int m = m0; m <= m1; m++) {
            double yr = 0.0, yi = 0.0;
#pragma unroll
            for (int j = 0; j < J; j++) {
                const double2 w = w2[((lane + 32 * j) * m) & (kPy - 1)];
                yr = fma(cr[j], w.x, fma(-ci[j], w.y, yr));
                yi = fma(cr[j], w.y, fma(ci[j], w.x, yi));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                yr += __shfl_xor_sync(0xffffffffu, yr, o);
                yi += __shfl_xor_sync(0xffffffffu, yi, o);
            }
            if (lane == 0) ysum[(size_t)k * g.nent + ent0 + (m - m0)] = make_double2(yr / kPy, yi / kPy);
        }
    }
}

template <class R, int NT, int NACC, bool WS>
cudaError_t run_fft(const Geometry &g, const void *spec, const void *rspec, const void *ypow, const void *tw_y,
                    double *part, cudaStream_t st) {
    YArgs ya;
    ya.nsplit = WS ? g.y2split_ws : g.y2split;
    ya.npairs = WS ? g.nk : g.ypg;
    ya.ncol = WS ? g.nk + 1 : 2 * g.nk + g.nb + 1;
    ya.nstage = WS ? g.dk + 2 : g.nbase;
    const int qmax = g.dk > g.db ? g.dk : g.db;
    if (ya.npairs > NACC * (NT / kPy) || ya.ncol > 64) return cudaErrorInvalidValue;
    const size_t sm = YSmem<R>::bytes(ya.nstage, qmax, ya.ncol, ya.npairs);
    auto kern = k_ycorr_fft<R, NT, NACC, WS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    dim3 grid(g.nkf, ya.nsplit, WS ? 1 : g.npg);
    note_launch();
    kern<<<grid, NT, sm, st>>>((const cpx<R> *)spec, (const cpx<R> *)rspec, (const R *)ypow, (const cpx<R> *)tw_y,
                               g, ya, part);
    return cudaGetLastError();
}

}  // namespace

size_t yfft_smem_bytes(const Geometry &g, int precision, bool ws) {
    const int qmax = g.dk > g.db ? g.dk : g.db;
    const int nstage = ws ? g.dk + 2 : g.nbase, ncol = ws ? g.nk + 1 : 2 * g.nk + g.nb + 1;
    const int np = ws ? g.nk : g.ypg;
    return precision == SFFT_PREC_FP64 ? YSmem<double>::bytes(nstage, qmax, ncol, np)
                                       : YSmem<float>::bytes(nstage, qmax, ncol, np);
}

cudaError_t launch_ycorr_fft(const Geometry &g, int precision, const void *spec, const void *rspec, const void *ypow,
                             const void *tw_y, double *part, bool ws, cudaStream_t st) {
    if (g.Py != kPy) return cudaErrorInvalidValue;
    if (precision == SFFT_PREC_FP64)
        return ws ? run_fft<double, 256, 8, true>(g, spec, rspec, ypow, tw_y, part, st)
                  : run_fft<double, 512, 16, false>(g, spec, rspec, ypow, tw_y, part, st);
    if (!ws && g.npg == 1 && fft32_specialised(g.dk, g.db)) return dispatch_fft32(g, spec, ypow, tw_y, part, st);
    return ws ? run_fft<float, 256, 8, true>(g, spec, rspec, ypow, tw_y, part, st)
              : run_fft<float, 512, 16, false>(g, spec, rspec, ypow, tw_y, part, st);
}

cudaError_t launch_yinv(const Geometry &g, int precision, const double *part, const void *twi, double *ysum, bool ws,
                        cudaStream_t st) {
    const int npairs = ws ? g.nk : g.npair_all;
    const int nsplit = ws ? g.y2split_ws : g.y2split;
    const size_t threads = (size_t)g.nkf * npairs * 32;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    note_launch();
    if (precision == SFFT_PREC_FP64)
        k_yinv<double><<<blocks, 256, 0, st>>>(part, twi, g, nsplit, npairs, ws, (double2 *)ysum);
    else
        k_yinv<float><<<blocks, 256, 0, st>>>(part, twi, g, nsplit, npairs, ws, (double2 *)ysum);
    return cudaGetLastError();
}

}  // namespace sfft
