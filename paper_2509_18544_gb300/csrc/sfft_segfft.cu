// K1: polynomial-weighted products fused into row-segment real FFTs.
//
// For every row y and segment s the kernel forms, on the fly from S, T and the mask,
//   A-images  W_i restricted to the segment's own columns [x0, x0+U) and zero-padded to P,
//   B-images  W_i, Psi_r = m w_r and S_m over the cyclic window [x0-G, x0-G+P),
// (W_i = w_i T_m, w_i = xh^p yh^q) and takes their P-point real DFTs (forward,
// exp(-2 pi i k j / P), unnormalised).  Two real images share one complex FFT; P = 256 is
// done as 16 x 16 (a 16-point DFT in registers, a twiddle, one padded shared-memory
// transpose, a second 16-point DFT).  Output: spec[s][y][k][img], k in [0, P/2].
//
// These spectra feed the lag correlations of the normal matrix of the delta-basis fit
// (SFFT subtraction step, Sec. "Pipeline steps", step 6).
#include <algorithm>

#include <type_traits>

#include "sfft_fft256.cuh"

namespace sfft {
namespace {

template <class R>
__device__ __forceinline__ R coord(int i, int n) {
    return n > 1 ? (R)(2 * i - (n - 1)) / (R)(n - 1) : (R)0;
}

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

constexpr int kRowsPerCta = 32;
constexpr int kMaxRowsPP = 4;  // rows transformed per pass
// exchange buffer per FFT: 16 x 17 (padded transpose) + 1, so that buffers of consecutive
// FFTs start two banks apart instead of on the same bank
constexpr int kEx = 16 * 17 + 1;

// The weights factor: w_i = xh^p yh^q with yh constant along a row, so the row-segment
// spectrum of any image is yh^q times the spectrum of its x-weighted base image.  The
// kernel transforms only the base images
//   b = p            A side: xh^p T_m on the segment's own columns (p <= DK)
//   b = DK+1+p       B side: xh^p T_m on the window
//   b = 2(DK+1)+p    xh^p m on the window (p <= DB)
//   b = nbase-1      S_m on the window
// two to a complex FFT, and writes every output image from its base spectrum times yh^q.
// Two real images packed into one complex FFT share its rounding, which is relative to the
// larger of them: the star images (T, S) are up to ~1e5 times the mask images (m xh^p), so
// the FFT slots keep the two families apart -- T-side and S images in slots 0 .. 2(DK+1)
// (a zero pad after S), then the mask images (a zero pad if their count is odd).
__host__ __device__ __forceinline__ int n_base(int dk, int db) { return 2 * (dk + 1) + (db + 1) + 1; }
__host__ __device__ __forceinline__ int n_fft_slots(int dk, int db) { return 2 * (dk + 1) + 2 + 2 * ((db + 2) / 2); }
// FFT slot of base image b
__host__ __device__ __forceinline__ int slot_of_base(int b, int dk, int db) {
    const int na = dk + 1;
    if (b < 2 * na) return b;                  // A_p, B_p
    if (b == n_base(dk, db) - 1) return 2 * na;  // S_m
    return 2 * na + 2 + (b - 2 * na);          // m xh^p
}

// Spectra of every image of a row segment, rows_pp rows per pass.  Layout of the output:
// spec[s][y][k][img] (a contiguous block of nkf * nrec values per row segment).  On the
// y-FFT route the records hold the base images themselves (img = b, no yh^q factor: the
// y correlation applies it); on the direct route every image W_i, Psi_r, S_m of the normal
// matrix, each its base spectrum times yh^q.
template <class R, class In, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_segment_fft(const In *__restrict__ sci, const In *__restrict__ tmpl,
                                                    const uint8_t *__restrict__ mask, Geometry g, int rows_pp,
                                                    const cpx<R> *__restrict__ tw_g, const R *__restrict__ xpow_g,
                                                    const R *__restrict__ ypow_g, cpx<R> *__restrict__ spec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = g.nk, nb = g.nb, G = g.G, U = g.U, nx = g.nx, ny = g.ny, NI = g.nrec, nkf = g.nkf;
    const int maxdeg = g.dk > g.db ? g.dk : g.db;
    const int nbase = n_base(g.dk, g.db), nbfft = n_fft_slots(g.dk, g.db) / 2;
    const int s = blockIdx.x;
    const int x0 = s * U;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int per_row = nbfft * 16;

    cpx<R> *tw = reinterpret_cast<cpx<R> *>(smem_raw);  // [P] twiddle, high part
    cpx<R> *twl = tw + kP;                              // [P] remainder
    cpx<R> *ex = twl + kP;                              // [rows_pp][nbfft][kEx]
    R *xpow = reinterpret_cast<R *>(ex + (size_t)rows_pp * nbfft * kEx);  // [maxdeg+1][P]
    R *ones = xpow + (maxdeg + 1) * kP;                 // [P] ones (S_m has no coordinate weight)
    R *tv = ones + kP;                                  // [rows_pp][P] T_m on the window
    R *sv = tv + rows_pp * kP;                          // [rows_pp][P] S_m
    R *mv = sv + rows_pp * kP;                          // [rows_pp][P] m
    int *bk = reinterpret_cast<int *>(mv + rows_pp * kP);  // [2 nbfft] base kind
    int *bp = bk + 2 * nbfft;                           // [2 nbfft] base x power
    int *ob = bp + 2 * nbfft;                           // [nrec] base of each output image (-1: zero)
    int *oq = ob + NI;                                  // [nrec] y power of each output image
    int *wcol = oq + NI;                                // [P] frame column of each window column

    constexpr bool kF32 = std::is_same<R, float>::value;
    if constexpr (kF32) fill_tw4(reinterpret_cast<float4 *>(tw), reinterpret_cast<const float2 *>(tw_g));
    for (int i = tid; i < kP; i += nthr) {
        if constexpr (!kF32) {
            tw[i] = tw_g[i];
            twl[i] = tw_g[kP + i];
        }
        // coordinate powers come from FP64 tables rounded once: repeated FP32 products
        // are biased (~-3e-8 at power 4)
        int xw = wrapi(x0 - G + i, nx);
        for (int p = 0; p <= maxdeg; p++) xpow[p * kP + i] = xpow_g[(size_t)p * nx + xw];
        ones[i] = (R)1;
        wcol[i] = xw;
    }
    for (int b = tid; b < 2 * nbfft; b += nthr) {
        // kinds per FFT slot: 0 = A (own columns), 1 = B (window), 2 = m (window), 3 = S_m,
        // 4 = zero pad
        const int na = g.dk + 1;
        int kind, p = 0;
        if (b < na) { kind = 0; p = b; }
        else if (b < 2 * na) { kind = 1; p = b - na; }
        else if (b == 2 * na) { kind = 3; }
        else if (b >= 2 * na + 2 && b < 2 * na + 2 + g.db + 1) { kind = 2; p = b - 2 * na - 2; }
        else { kind = 4; }
        bk[b] = kind;
        bp[b] = p;
    }
    for (int i = tid; i < NI; i += nthr) {
        const int na = g.dk + 1;
        int base = -1, p = 0, q = 0;
        if (g.yfft) { base = i < nbase ? i : -1; }  // y-FFT route: the base images themselves
        else if (i < nk) { mono_pq(i, p, q); base = p; }
        else if (i < 2 * nk) { mono_pq(i - nk, p, q); base = na + p; }
        else if (i < 2 * nk + nb) { mono_pq(i - 2 * nk, p, q); base = 2 * na + p; }
        else if (i == 2 * nk + nb) { base = nbase - 1; q = 0; }
        ob[i] = base < 0 ? -1 : slot_of_base(base, g.dk, g.db);  // the FFT slot it is unpacked from
        oq[i] = q;
    }

    const int ybeg = blockIdx.y * kRowsPerCta, yend = min(ny, ybeg + kRowsPerCta);
    // window positions loaded per thread per pass (rows_pp rows x P positions): position
    // q = tid + c nthr is row q / P, window column q % P; its wrapped frame column is fixed
    // for the whole kernel, so it is computed once
    constexpr int kMaxPf = 4;
    const int npos = rows_pp * kP;
    auto load_pos = [&](int c, int ybase, R &t_out, R &s_out, R &m_out) {
        const int q = tid + c * nthr;
        const int y = ybase + (q >> 8);
        if (y < yend) {
            const size_t u = (size_t)y * g.pitch + wcol[q & (kP - 1)];
            // all three loads issue together (none waits for the mask byte); then selects,
            // not products: a masked pixel never enters, whatever value it holds
            const In tr = tmpl[u], sr = sci[u];
            const bool bad = mask ? mask[u] != 0 : false;
            t_out = bad ? (R)0 : (R)tr;
            s_out = bad ? (R)0 : (R)sr;
            m_out = bad ? (R)0 : (R)1;
        } else {
            t_out = s_out = m_out = (R)0;
        }
    };
    __syncthreads();  // wcol
    // prologue: window of the first pass straight to shared memory (the host gives every
    // launch at least npos / kMaxPf threads)
#pragma unroll
    for (int c = 0; c < kMaxPf; c++) {
        const int q = tid + c * nthr;
        if (q < npos) load_pos(c, ybeg, tv[q], sv[q], mv[q]);
    }
    __syncthreads();

    const int r_fft = tid / per_row, rem = tid - r_fft * per_row;
    const int f = rem >> 4, t = rem & 15;
    for (int y0 = ybeg; y0 < yend; y0 += rows_pp) {
        // prefetch the next pass's window into registers
        R pft[kMaxPf], pfs[kMaxPf], pfm[kMaxPf];
        const bool more = y0 + rows_pp < yend;
#pragma unroll
        for (int c = 0; c < kMaxPf; c++) {
            int q = tid + c * nthr;
            if (more && q < npos) load_pos(c, y0 + rows_pp, pft[c], pfs[c], pfm[c]);
        }
        // yh^q of this thread's unpacked image for the pass's rows, loaded before the FFTs
        R yqv[kMaxRowsPP];
        {
            const int img = tid % NI, b = ob[img], q = oq[img];
#pragma unroll
            for (int rr = 0; rr < kMaxRowsPP; rr++) {
                const int y = y0 + rr;
                yqv[rr] = (b < 0 || rr >= rows_pp || y >= yend) ? (R)0
                                                              : (q == 0 ? (R)1 : ypow_g[(size_t)q * ny + y]);
            }
        }
        // FFT lanes of this warp: each half-warp is one FFT of a row that exists
        auto half_active = [&](int base) {
            int rr = base / per_row;
            return base < rows_pp * per_row && y0 + rr < yend;
        };
        const int wbase = tid & ~31;
        const unsigned msk = (half_active(wbase) ? 0x0000ffffu : 0u) | (half_active(wbase + 16) ? 0xffff0000u : 0u);
        if (r_fft < rows_pp && y0 + r_fft < yend) {
            const R *tvr = tv + r_fft * kP, *svr = sv + r_fft * kP, *mvr = mv + r_fft * kP;
            // per base image of this lane's pair: source row, coordinate-power row, offset of
            // the pixel inside the window and the number of valid positions (branch-free
            // construction of z = x_{2f} + i x_{2f+1} below)
            const R *src[2], *xpr[2];
            int off[2], lim[2];
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const int b = 2 * f + c, kind = bk[b];
                src[c] = kind == 2 ? mvr : (kind == 3 ? svr : tvr);
                xpr[c] = kind == 3 ? ones : xpow + bp[b] * kP;
                off[c] = kind == 0 ? G : 0;
                lim[c] = kind == 0 ? min(U, nx - x0) : (kind == 4 ? 0 : kP);
            }
            cpx<R> v[16];
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const int n = t + 16 * jj;
                R val[2];
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const int q = n < lim[c] ? n + off[c] : 0;
                    R r = xpr[c][q] * src[c][q];
                    val[c] = n < lim[c] ? r : (R)0;
                }
                v[jj] = {val[0], val[1]};
            }
            cpx<R> *e = ex + (r_fft * nbfft + f) * kEx;
            if constexpr (kF32) fft256f(v, t, e, reinterpret_cast<const float4 *>(tw), msk);
            else fft256(v, t, e, tw, twl, msk);
#pragma unroll
            for (int k2 = 0; k2 < 16; k2++) e[t + 16 * k2] = v[k2];  // natural order Z[k]
        }
        __syncthreads();
        // unpack the packed real pairs, scale by yh^q; each row segment is one contiguous block
        const int per_out = nkf * NI;
        const int nrow = min(rows_pp, yend - y0);
        const int nun = (nthr / NI) * NI;  // threads that unpack: whole sets of NI
        if (nun > 0) {
            // every thread keeps one image and walks the bins (consecutive threads write
            // consecutive values), so no index is divided per value
            const int img = tid % NI, kstep = nun / NI;
            const int b = ob[img];
            const bool odd = b & 1;
#pragma unroll
            for (int rr = 0; rr < kMaxRowsPP; rr++) {
                if (rr >= nrow || tid >= nun) break;
                const int y = y0 + rr;
                const cpx<R> *e = ex + (rr * nbfft + (b < 0 ? 0 : b >> 1)) * kEx;
                cpx<R> *o = spec + ((size_t)s * ny + y) * per_out + img;
                const R hy = (R)0.5 * yqv[rr];
                for (int k = tid / NI; k < nkf; k += kstep) {
                    const cpx<R> zk = e[k], zc = e[(kP - k) & (kP - 1)];
                    o[(size_t)k * NI] = odd ? cpx<R>{hy * (zk.im + zc.im), hy * (zc.re - zk.re)}
                                            : cpx<R>{hy * (zk.re + zc.re), hy * (zk.im - zc.im)};
                }
            }
        } else {
            for (int idx = tid; idx < nrow * per_out; idx += nthr) {
                const int rr = idx / per_out, r2 = idx - rr * per_out;
                const int k = r2 / NI, img = r2 - k * NI;
                const int b = ob[img], q = oq[img], y = y0 + rr;
                const R yq = b < 0 ? (R)0 : (q == 0 ? (R)1 : ypow_g[(size_t)q * ny + y]);
                const R hy = (R)0.5 * yq;
                const cpx<R> *e = ex + (rr * nbfft + (b < 0 ? 0 : b >> 1)) * kEx;
                cpx<R> zk = e[k], zc = e[(kP - k) & (kP - 1)];
                cpx<R> out;
                if ((b & 1) == 0)
                    out = {hy * (zk.re + zc.re), hy * (zk.im - zc.im)};
                else
                    out = {hy * (zk.im + zc.im), hy * (zc.re - zk.re)};
                spec[((size_t)s * ny + y) * per_out + r2] = out;
            }
        }
        // the next pass's window (its FFT readers are past the barrier above)
#pragma unroll
        for (int c = 0; c < kMaxPf; c++) {
            int q = tid + c * nthr;
            if (more && q < npos) {
                tv[q] = pft[c];
                sv[q] = pfs[c];
                mv[q] = pfm[c];
            }
        }
        __syncthreads();
    }
}

// Spectrum of one image (the refinement residual) over every row segment, written into the
// S_m slot of spec.  Two rows share one complex FFT (z = X_y + i X_{y+1}).
template <class R, class In>
__global__ void __launch_bounds__(128) k_segment_fft_single(const In *__restrict__ img, Geometry g,
                                                           const cpx<R> *__restrict__ tw_g, int slot,
                                                           cpx<R> *__restrict__ spec, cpx<R> *__restrict__ rspec) {
    // split twiddles: tw, twl (FP64), or the FP32 form's tw4 table in the same bytes
    __shared__ __align__(16) unsigned char twraw[2 * kP * sizeof(cpx<R>)];
    cpx<R> *tw = reinterpret_cast<cpx<R> *>(twraw), *twl = tw + kP;
    constexpr bool kF32 = std::is_same<R, float>::value;
    static_assert(!kF32 || kTw4 * sizeof(float4) <= sizeof(twraw), "tw4 fits the twiddle bytes");
    __shared__ cpx<R> ex[8][kEx];
    const int G = g.G, nx = g.nx, ny = g.ny, NI = g.nrec, nkf = g.nkf;
    const int s = blockIdx.x, x0 = s * g.U;
    if constexpr (kF32) {
        fill_tw4(reinterpret_cast<float4 *>(twraw), reinterpret_cast<const float2 *>(tw_g));
    } else {
        for (int i = threadIdx.x; i < kP; i += blockDim.x) {
            tw[i] = tw_g[i];
            twl[i] = tw_g[kP + i];
        }
    }
    __syncthreads();
    const int f = threadIdx.x >> 4, t = threadIdx.x & 15;  // 8 FFTs of row pairs
    const int y = (blockIdx.y * 8 + f) * 2;
    const bool act = y < ny;
    const unsigned msk = 0xffffffffu;  // both half-warps always run the FFT (zeros past the end)
    cpx<R> v[16];
#pragma unroll
    for (int jj = 0; jj < 16; jj++) {
        int xw = wrapi(x0 - G + t + 16 * jj, nx);
        R a = act ? (R)img[(size_t)y * g.pitch + xw] : (R)0;
        R b = (act && y + 1 < ny) ? (R)img[(size_t)(y + 1) * g.pitch + xw] : (R)0;
        v[jj] = {a, b};
    }
    cpx<R> *e = ex[f];
    if constexpr (kF32) fft256f(v, t, e, reinterpret_cast<const float4 *>(twraw), msk);
    else fft256(v, t, e, tw, twl, msk);
#pragma unroll
    for (int k2 = 0; k2 < 16; k2++) e[t + 16 * k2] = v[k2];
    __syncwarp(msk);
    if (act) {
        // compact [segment][row][bin] buffer when given (coalesced), else the image slot
        const size_t stride = rspec ? 1 : NI;
        cpx<R> *o = rspec ? rspec : spec + slot;
        for (int k = t; k < nkf; k += 16) {
            cpx<R> zk = e[k], zc = e[(kP - k) & (kP - 1)];
            o[(((size_t)s * ny + y) * nkf + k) * stride] = {(R)0.5 * (zk.re + zc.re), (R)0.5 * (zk.im - zc.im)};
            if (y + 1 < ny)
                o[(((size_t)s * ny + y + 1) * nkf + k) * stride] = {(R)0.5 * (zk.im + zc.im), (R)0.5 * (zc.re - zk.re)};
        }
    }
}

// rows per pass and threads: every base FFT of rows_pp rows (16 lanes each), at least
// 256 threads so that kMaxPf positions per thread cover the rows_pp x P window
struct SegLaunch {
    int rows_pp, threads;
};
SegLaunch seg_launch(const Geometry &g) {
    const int nbfft = n_fft_slots(g.dk, g.db) / 2;
    SegLaunch l;
    l.rows_pp = std::max(1, std::min(kMaxRowsPP, 384 / (nbfft * 16)));
    l.threads = std::max(256, (l.rows_pp * nbfft * 16 + 31) / 32 * 32);
    return l;
}

template <class R>
size_t segfft_smem(const Geometry &g, int rows_pp) {
    const int maxdeg = g.dk > g.db ? g.dk : g.db;
    const int nbfft = n_fft_slots(g.dk, g.db) / 2;
    return sizeof(cpx<R>) * (2 * kP + (size_t)rows_pp * nbfft * kEx) +
           sizeof(R) * ((size_t)(maxdeg + 2) * kP + 3 * (size_t)rows_pp * kP) +
           sizeof(int) * (4 * nbfft + 2 * g.nrec + kP);
}

template <class R, class In>
cudaError_t run(const Geometry &g, const void *sci, const void *tmpl, const uint8_t *mask, const void *tw,
                const void *xpow, const void *ypow, void *spec, cudaStream_t st) {
    const SegLaunch l = seg_launch(g);
    size_t sm = segfft_smem<R>(g, l.rows_pp);
    auto kern = k_segment_fft<R, In, 384, 2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    dim3 grid(g.nseg, (g.ny + kRowsPerCta - 1) / kRowsPerCta);
    note_launch();
    kern<<<grid, l.threads, sm, st>>>((const In *)sci, (const In *)tmpl, mask, g, l.rows_pp, (const cpx<R> *)tw,
                                      (const R *)xpow, (const R *)ypow, (cpx<R> *)spec);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_segment_fft_single(const Geometry &g, int dtype, int precision, const void *img, const void *tw_fft,
                                      int slot, void *spec, void *rspec, cudaStream_t st) {
    if (g.P != kP) return cudaErrorInvalidValue;
    dim3 grid(g.nseg, (g.ny + 15) / 16);
    note_launch();
    if (precision == SFFT_PREC_FP64) {
        if (dtype == SFFT_F64)
            k_segment_fft_single<double, double><<<grid, 128, 0, st>>>((const double *)img, g, (const cpx<double> *)tw_fft, slot, (cpx<double> *)spec, (cpx<double> *)rspec);
        else
            k_segment_fft_single<double, float><<<grid, 128, 0, st>>>((const float *)img, g, (const cpx<double> *)tw_fft, slot, (cpx<double> *)spec, (cpx<double> *)rspec);
    } else {
        if (dtype == SFFT_F64)
            k_segment_fft_single<float, double><<<grid, 128, 0, st>>>((const double *)img, g, (const cpx<float> *)tw_fft, slot, (cpx<float> *)spec, (cpx<float> *)rspec);
        else
            k_segment_fft_single<float, float><<<grid, 128, 0, st>>>((const float *)img, g, (const cpx<float> *)tw_fft, slot, (cpx<float> *)spec, (cpx<float> *)rspec);
    }
    return cudaGetLastError();
}

cudaError_t launch_segment_fft(const Geometry &g, int dtype, int precision, const void *sci, const void *tmpl,
                               const uint8_t *mask, const void *tw_fft, const void *xpow, const void *ypow,
                               void *spec, cudaStream_t st) {
    if (g.P != kP || n_fft_slots(g.dk, g.db) > 48) return cudaErrorInvalidValue;
    if (precision == SFFT_PREC_FP64) {
        return dtype == SFFT_F64 ? run<double, double>(g, sci, tmpl, mask, tw_fft, xpow, ypow, spec, st)
                                 : run<double, float>(g, sci, tmpl, mask, tw_fft, xpow, ypow, spec, st);
    }
    return dtype == SFFT_F64 ? run<float, double>(g, sci, tmpl, mask, tw_fft, xpow, ypow, spec, st)
                             : run<float, float>(g, sci, tmpl, mask, tw_fft, xpow, ypow, spec, st);
}

}  // namespace sfft
