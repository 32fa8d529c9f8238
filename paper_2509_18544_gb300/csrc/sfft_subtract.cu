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
#include <algorithm>
#include <type_traits>

#include "sfft_internal.cuh"

namespace sfft {
namespace {

template <class R>
__device__ __forceinline__ R coordv(int i, int n) {
    return n > 1 ? (R)(2 * i - (n - 1)) / (R)(n - 1) : (R)0;
}

// cf[ys][l][p] over l = (dy+h) L + (dx+h): sum_{i: p_i = p} a_{i,l} yh(ys)^q_i, and after
// the table bg[y][p] = sum_{r: p_r = p} b_r yh(y)^q_r.  iny = 1 / (ny - 1) (0 when ny = 1),
// from the host: yh = (2 y - (ny - 1)) iny (no FP64 division per thread).  The monomial
// loops are unrolled over degree <= 7 so that the sums stay in registers.
template <class R>
__global__ void k_fold(const double *__restrict__ coeffs, Geometry g, double iny, R *__restrict__ cf) {
    const int L2 = g.L * g.L, np = g.dk + 1, nbp = g.db + 1;
    const size_t ncf = (size_t)g.ny * L2;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ncf) {
        const int ys = (int)(t / L2), l = (int)(t - (size_t)ys * L2);
        const double yh = (2.0 * ys - (g.ny - 1)) * iny;
        double pw[8], acc[8];
        pw[0] = 1.0;
#pragma unroll
        for (int q = 1; q < 8; q++) pw[q] = q <= g.dk ? pw[q - 1] * yh : 0.0;
#pragma unroll
        for (int p = 0; p < 8; p++) acc[p] = 0.0;
        int i = 0;  // monomial index: total degree first, then q ascending
#pragma unroll
        for (int d = 0; d < 8; d++) {
            if (d > g.dk) break;
#pragma unroll
            for (int q = 0; q <= d; q++, i++) acc[d - q] = fma(coeffs[(size_t)i * L2 + l], pw[q], acc[d - q]);
        }
        const int dyi = l / g.L, dxi = l - dyi * g.L;
        R *o = cf + (((size_t)ys * g.L + dyi) * np) * g.L + dxi;
#pragma unroll
        for (int p = 0; p < 8; p++)
            if (p < np) o[(size_t)p * g.L] = (R)acc[p];
    } else if (t < ncf + (size_t)g.ny) {
        const int y = (int)(t - ncf);
        const double yh = (2.0 * y - (g.ny - 1)) * iny;
        double pw[8], acc[8];
        pw[0] = 1.0;
#pragma unroll
        for (int q = 1; q < 8; q++) pw[q] = q <= g.db ? pw[q - 1] * yh : 0.0;
#pragma unroll
        for (int p = 0; p < 8; p++) acc[p] = 0.0;
        int r = 0;
#pragma unroll
        for (int d = 0; d < 8; d++) {
            if (d > g.db) break;
#pragma unroll
            for (int q = 0; q <= d; q++, r++) acc[d - q] = fma(coeffs[g.nker + r], pw[q], acc[d - q]);
        }
        R *o = cf + ncf * np + (size_t)y * nbp;
#pragma unroll
        for (int p = 0; p < 8; p++)
            if (p < nbp) o[p] = (R)acc[p];
    }
}

// Streaming layout: a CTA owns a strip of kCols<R> output columns and a chunk of rows, which
// it walks in bands of kBand rows.  Shared memory keeps a ring of kBand + 2h template rows
// (each as np planes xh^p T, for the strip's columns plus the h-column halo on each side),
// so every source row is staged once per chunk; after a band the kBand rows no longer
// needed are overwritten by the next band's new rows.  The folded coefficients of a band's
// rows are staged beside it.
constexpr int kBand = 8;
template <class R> struct Tile {
    static constexpr int kRX = 32 / (int)sizeof(R);   // consecutive pixels per lane
    static constexpr int kCols = 32 * kRX;            // strip width
};
// Lanes read register windows starting kRX columns apart.  FP32: the window is read as
// 16-byte vectors, and a 4-word pad after every 32 words puts the 8 lanes of a quarter-warp
// (starting 8 words apart) on distinct banks.  FP64: one pad word every 4 doubles puts the
// 16 lanes of a half-warp on distinct bank pairs.
template <class R>
__host__ __device__ constexpr int skew(int c) {
    return sizeof(R) == 4 ? c + 4 * (c >> 5) : c + (c >> 2);
}
template <class R, int LL> struct Win {
    static constexpr int h = LL / 2;
    static constexpr int WC = Tile<R>::kCols + 2 * h;                                           // window columns
    static constexpr int WCS = sizeof(R) == 4 ? (WC + 4 * ((WC + 31) / 32) + 3) / 4 * 4
                                              : WC + WC / 4 + 1;                                 // padded row
    static constexpr int RING = kBand + 2 * h;                                                   // ring rows
    static constexpr int NW = Tile<R>::kRX + LL - 1;                                             // register window
    static constexpr int NW4 = (NW + 3) / 4;                                                     // 16-byte loads of it
    static constexpr int LLP = (LL + 3) / 4 * 4;                                                 // coefficient row stride
    static_assert(NW4 * 4 >= NW && LLP >= LL, "window and coefficient rows cover their values");
    // floats of the np template planes, rounded up to 16 bytes so that the coefficient rows
    // after them can be read as 16-byte vectors
    __host__ __device__ static constexpr int planes(int np) { return (np * RING * WCS + 3) & ~3; }
};

__device__ __forceinline__ int wrapi(int v, int n) {
    if (v >= 0 && v < n) return v;
    v %= n;
    return v < 0 ? v + n : v;
}

// Shared memory of the streaming kernels (byte offsets, each region on 16 bytes):
//   Tp   [np][RING][WCS] R      the template ring, as np planes xh^p T
//   cf   [kBand][LL][np][LLP] R the band's folded coefficients
//   xo   [db+1][OC] R           xh^p of the strip's output columns
//   ss   [kBand][OC] In         science values of the band's output rows
//   sk   [RING][kCols] bytes    per ring row: 1 where the output column's pixel is masked
//   byp  [kBand][db+1] R        the band's background x-power sums
//   xps  [npx][WC] R            xh^p of the window columns
// Output-side rows use the kernel's skewed column index, so that a lane's run of kRX
// consecutive columns is read without bank conflicts.
template <class R, class In, int LL> struct Layout {
    using W = Win<R, LL>;
    static constexpr int kC = Tile<R>::kCols;
    static constexpr int OC = (skew<R>(kC - 1) + 4) & ~3;
    __host__ __device__ static constexpr size_t al(size_t b) { return (b + 15) & ~(size_t)15; }
    __host__ __device__ static constexpr size_t cf(int np) { return al(sizeof(R) * (size_t)W::planes(np)); }
    __host__ __device__ static constexpr size_t xo(int np) {
        return al(cf(np) + sizeof(R) * (size_t)kBand * LL * np * W::LLP);
    }
    __host__ __device__ static constexpr size_t ss(int np, int db) { return al(xo(np) + sizeof(R) * (size_t)(db + 1) * OC); }
    __host__ __device__ static constexpr size_t sk(int np, int db) { return al(ss(np, db) + sizeof(In) * (size_t)kBand * OC); }
    __host__ __device__ static constexpr size_t byp(int np, int db) { return al(sk(np, db) + (size_t)W::RING * kC); }
    __host__ __device__ static constexpr size_t xps(int np, int db) {
        return al(byp(np, db) + sizeof(R) * (size_t)kBand * (db + 1));
    }
    static size_t bytes(int np, int db) {
        const int npx = np > db + 1 ? np : db + 1;
        return xps(np, db) + sizeof(R) * (size_t)npx * W::WC;
    }
};

// one 4- or 8-byte element, global to shared, asynchronously (completed by cp_async_wait)
template <class T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// xh^p of the strip's window columns (x0 - h ..), p < npx: xps[p][c]
template <class R, int LL>
__device__ __forceinline__ void fill_xps(const Geometry &g, const R *__restrict__ xpow_g, int x0, int npx, R *xps) {
    using W = Win<R, LL>;
    for (int e = threadIdx.x; e < npx * W::WC; e += blockDim.x) {
        const int p = e / W::WC, c = e - p * W::WC;
        xps[e] = xpow_g[(size_t)p * g.nx + wrapi(x0 - W::h + c, g.nx)];
    }
}

// v = hi + lo exactly (FP64 inputs), or hi = v (FP32)
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

// xh^p of the strip's output columns, p <= db: xo[p][skew(c)]
template <class R, int LL>
__device__ __forceinline__ void fill_xo(const Geometry &g, const R *__restrict__ xpow_g, int x0, R *xo) {
    using Ly = Layout<R, R, LL>;
    for (int e = threadIdx.x; e < (g.db + 1) * Ly::kC; e += blockDim.x) {
        const int p = e / Ly::kC, c = e % Ly::kC;
        xo[p * Ly::OC + skew<R>(c)] = xpow_g[(size_t)p * g.nx + min(x0 + c, g.nx - 1)];
    }
}

// Science values of output rows yb .. yb + kBand - 1 (rows before yc1, columns inside the
// frame), copied asynchronously: ss[r][skew(c)].
template <class R, class In, int LL>
__device__ __forceinline__ void async_sci(const In *__restrict__ sci, const Geometry &g, int x0, int yb, int yc1,
                                          In *ss) {
    using Ly = Layout<R, In, LL>;
    constexpr int total = kBand * Ly::kC;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int r = e / Ly::kC, c = e % Ly::kC, y = yb + r, x = x0 + c;
        if (y < yc1 && x < g.nx) cp_async_elem(ss + r * Ly::OC + skew<R>(c), sci + (size_t)y * g.pitch + x);
    }
}

// n consecutive values starting at p (with VEC and FP32 values, 16-byte loads: the caller
// guarantees that p is on 16 bytes)
template <class R, int N, bool VEC>
__device__ __forceinline__ void load_run(const R *p, R (&v)[N]) {
    if constexpr (sizeof(R) == 4 && VEC && N % 4 == 0) {
#pragma unroll
        for (int k = 0; k < N / 4; k++) {
            const float4 q = *reinterpret_cast<const float4 *>(p + 4 * k);
            v[4 * k] = q.x;
            v[4 * k + 1] = q.y;
            v[4 * k + 2] = q.z;
            v[4 * k + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; k++) v[k] = p[k];
    }
}

// the skip flags of a lane's kRX consecutive pixels, one byte each
template <int N>
__device__ __forceinline__ unsigned long long load_flags(const unsigned char *p) {
    static_assert(N == 4 || N == 8, "runs of 4 or 8 pixels");
    if constexpr (N == 8) return *reinterpret_cast<const unsigned long long *>(p);
    else return *reinterpret_cast<const unsigned *>(p);
}

// Stages `count` consecutive source rows starting at (unwrapped) row ys0 into their ring
// slots, as np planes xh^p T (T_m when `masked`).  Each thread first issues the loads of
// kBatch elements, then forms and stores their planes, so a band costs a few load
// latencies rather than one per element.
template <class R, class In, int LL, int kBatch>
__device__ __forceinline__ void stage_rows(const In *__restrict__ tmpl, const uint8_t *__restrict__ mask, bool masked,
                                           const Geometry &g, const R *xps, int x0, int ys0, int count,
                                           int ring_origin, R *Tp, unsigned char *sk) {
    using W = Win<R, LL>;
    constexpr int kC = Tile<R>::kCols;
    const int np = g.dk + 1, nx = g.nx, total = count * W::WC;
    for (int base = 0; base < total; base += kBatch * (int)blockDim.x) {
        In tv[kBatch];
        unsigned char bad[kBatch];
        int col[kBatch], slot[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; i++) {
            const int e = base + i * (int)blockDim.x + (int)threadIdx.x;
            col[i] = -1;
            tv[i] = (In)0;
            bad[i] = 0;
            if (e < total) {
                const int r = e / W::WC, c = e - r * W::WC;
                const int ys = ys0 + r;
                const size_t u = (size_t)wrapi(ys, g.ny) * g.pitch + wrapi(x0 - W::h + c, nx);
                tv[i] = tmpl[u];
                bad[i] = masked && mask ? mask[u] : 0;
                col[i] = c;
                slot[i] = (ys - ring_origin) % W::RING;
            }
        }
#pragma unroll
        for (int i = 0; i < kBatch; i++) {
            if (col[i] < 0) continue;
            const R t = bad[i] ? (R)0 : (R)tv[i];
            R *dst = Tp + (size_t)slot[i] * W::WCS + skew<R>(col[i]);
            dst[0] = t;
            for (int p = 1; p < np; p++) dst[(size_t)p * W::RING * W::WCS] = t * xps[p * W::WC + col[i]];
            // the row's mask flags at the strip's output columns
            const int oc = col[i] - W::h;
            if (oc >= 0 && oc < kC) sk[slot[i] * kC + oc] = bad[i] ? 1 : 0;
        }
    }
}

// Folded coefficients c_p(d, y - dy) of output rows yb .. yb + kBand - 1 and their
// background x-power sums, copied asynchronously: cf[(ry LL + dyi) np + p][LLP].
template <class R, int LL>
__device__ __forceinline__ void async_coeffs(const Geometry &g, const R *__restrict__ cfold, int yb, R *cf, R *byp) {
    using W = Win<R, LL>;
    constexpr int h = LL / 2;
    const int np = g.dk + 1, ny = g.ny;
    // a warp per (row, dy): the np LL values of one source row and dy are contiguous
    const int nq = np * LL, lane = threadIdx.x & 31;
    for (int rd = threadIdx.x >> 5; rd < kBand * LL; rd += blockDim.x >> 5) {
        const int ry = rd / LL, dyi = rd - ry * LL;
        const int ys = wrapi(yb + ry - (dyi - h), ny);  // source row y - dy
        const R *src = cfold + ((size_t)ys * LL + dyi) * nq;
        for (int q = lane; q < nq; q += 32) {
            const int p = q / LL, dxi = q - p * LL;
            cp_async_elem(cf + ((ry * LL + dyi) * np + p) * W::LLP + dxi, src + q);
        }
    }
    const R *bgf = cfold + (size_t)ny * LL * LL * np;
    for (int e = threadIdx.x; e < kBand * (g.db + 1); e += blockDim.x) {
        int ry = e / (g.db + 1), p = e % (g.db + 1);
        cp_async_elem(byp + e, bgf + (size_t)min(yb + ry, ny - 1) * (g.db + 1) + p);
    }
}

// window of one lane: wp[m] = row[c0 + m], m < NW (FP32: 16-byte loads; FP64: scalar)
template <class R, int LL>
__device__ __forceinline__ void load_window(const R *row, int c0, R (&wp)[Win<R, LL>::NW4 * 4]) {
    using W = Win<R, LL>;
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int k = 0; k < W::NW4; k++) {
            const float4 v = *reinterpret_cast<const float4 *>(row + skew<R>(c0 + 4 * k));
            wp[4 * k] = v.x;
            wp[4 * k + 1] = v.y;
            wp[4 * k + 2] = v.z;
            wp[4 * k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int m = 0; m < W::NW; m++) wp[m] = row[skew<R>(c0 + m)];
    }
}

// coefficients c[0 .. LL) of one (row, dy, p) triple (FP32: 16-byte loads of the padded row)
template <class R, int LL>
__device__ __forceinline__ void load_coeffs(const R *c, R (&cc)[Win<R, LL>::LLP]) {
    using W = Win<R, LL>;
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int k = 0; k < W::LLP / 4; k++) {
            const float4 v = *reinterpret_cast<const float4 *>(c + 4 * k);
            cc[4 * k] = v.x;
            cc[4 * k + 1] = v.y;
            cc[4 * k + 2] = v.z;
            cc[4 * k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < LL; k++) cc[k] = c[k];
    }
}

// Difference image (residual = false) or the fit residual m (S - bg) - conv(T_m)
// (residual = true), one warp per output row of a band.
template <class R, class In, int LL>
__global__ void __launch_bounds__(32 * kBand, 2) k_subtract(const In *__restrict__ sci, const In *__restrict__ tmpl,
                                                        const uint8_t *__restrict__ mask, bool residual, Geometry g,
                                                        int rows_per_chunk, const R *__restrict__ cfold,
                                                        const R *__restrict__ xpow_g, In *__restrict__ diff) {
    using W = Win<R, LL>;
    using Ly = Layout<R, In, LL>;
    constexpr int h = W::h, kRX = Tile<R>::kRX;
    constexpr int kRowBatch = (kBand * W::WC + 32 * kBand - 1) / (32 * kBand);  // a band's new rows in one batch
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int np = g.dk + 1, nx = g.nx, ny = g.ny;
    R *Tp = reinterpret_cast<R *>(smem_raw);
    R *cf = reinterpret_cast<R *>(smem_raw + Ly::cf(np));
    R *xo = reinterpret_cast<R *>(smem_raw + Ly::xo(np));
    In *ss = reinterpret_cast<In *>(smem_raw + Ly::ss(np, g.db));
    unsigned char *sk = smem_raw + Ly::sk(np, g.db);
    R *byp = reinterpret_cast<R *>(smem_raw + Ly::byp(np, g.db));
    R *xps = reinterpret_cast<R *>(smem_raw + Ly::xps(np, g.db));
    const int npx = np > g.db + 1 ? np : g.db + 1;

    const int x0 = blockIdx.x * Tile<R>::kCols;
    const int yc0 = blockIdx.y * rows_per_chunk, yc1 = min(ny, yc0 + rows_per_chunk);
    if (yc0 >= ny) return;
    const int ring_origin = yc0 - h;
    const int ty = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cx = lane * kRX, ob = skew<R>(cx);  // skew(cx + r) = ob + r for r < kRX

    fill_xps<R, LL>(g, xpow_g, x0, npx, xps);
    fill_xo<R, LL>(g, xpow_g, x0, xo);
    __syncthreads();
    // every global load of a band happens in the staging phase before it: the coefficients
    // and science values as asynchronous copies that complete while the template rows load
    async_coeffs<R, LL>(g, cfold, yc0, cf, byp);
    async_sci<R, In, LL>(sci, g, x0, yc0, yc1, ss);
    stage_rows<R, In, LL, 8>(tmpl, mask, residual, g, xps, x0, yc0 - h, W::RING, ring_origin, Tp, sk);
    cp_async_wait();
    for (int yb = yc0; yb < yc1; yb += kBand) {
        __syncthreads();
        const int y = yb + ty;
        R out[kRX];
#pragma unroll
        for (int r = 0; r < kRX; r++) out[r] = (R)0;
        for (int dyi = 0; dyi < LL; dyi++) {
            // source row y - dy = y + h - dyi
            const int slot = (y + h - dyi - ring_origin) % W::RING;
            for (int p = 0; p < np; p++) {
                const R *trow = Tp + (p * W::RING + slot) * W::WCS;
                R wp[W::NW4 * 4];
                load_window<R, LL>(trow, cx, wp);
                R ccs[W::LLP];
                load_coeffs<R, LL>(cf + ((ty * LL + dyi) * np + p) * W::LLP, ccs);
#pragma unroll
                for (int dxi = 0; dxi < LL; dxi++) {
                    const R cc = ccs[dxi];
                    // source column x - dx -> window index r - dx + h = r + (LL - 1) - dxi
#pragma unroll
                    for (int r = 0; r < kRX; r++) out[r] += cc * wp[r + (LL - 1) - dxi];
                }
            }
        }
        if (y < yc1) {
            const R *bp = byp + ty * (g.db + 1);
            In svi[kRX];
            R sv[kRX], bg[kRX];
            // 16-byte loads only where the skew is the FP32 one (runs start on 4 elements)
            load_run<In, kRX, sizeof(R) == 4>(ss + ty * Ly::OC + ob, svi);
#pragma unroll
            for (int r = 0; r < kRX; r++) sv[r] = (R)svi[r];
            const unsigned long long mv =
                residual ? load_flags<kRX>(sk + ((y - ring_origin) % W::RING) * Ly::kC + cx) : 0ull;
#pragma unroll
            for (int r = 0; r < kRX; r++) bg[r] = (R)0;
            for (int p = 0; p <= g.db; p++) {
                R xv[kRX];
                load_run<R, kRX, sizeof(R) == 4>(xo + p * Ly::OC + ob, xv);
#pragma unroll
                for (int r = 0; r < kRX; r++) bg[r] += bp[p] * xv[r];
            }
#pragma unroll
            for (int r = 0; r < kRX; r++) {
                const int x = x0 + cx + r;
                if (x < nx) {
                    const size_t u = (size_t)y * g.pitch + x;
                    if (residual) {
                        diff[u] = (In)((((mv >> (8 * r)) & 0xff) ? (R)0 : sv[r] - bg[r]) - out[r]);
                    } else {
                        diff[u] = (In)(sv[r] - out[r] - bg[r]);
                    }
                }
            }
        }
        __syncthreads();
        // the next band reads source rows up to yb + 2 kBand + h - 1; the kBand new ones
        // replace rows yb - h .. yb - h + kBand - 1, which no later band reads
        if (yb + kBand < yc1) {
            async_coeffs<R, LL>(g, cfold, yb + kBand, cf, byp);
            async_sci<R, In, LL>(sci, g, x0, yb + kBand, yc1, ss);
            stage_rows<R, In, LL, kRowBatch>(tmpl, mask, residual, g, xps, x0, yb + kBand + h, kBand,
                                                   ring_origin, Tp, sk);
            cp_async_wait();
        }
    }
}

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            sms = v;
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// rows per chunk: a multiple of kBand that gives about `per_sm` CTAs per SM
int rows_per_chunk(const Geometry &g, int strips, int per_sm) {
    const int want = std::max(1, (per_sm * sm_count() + strips - 1) / strips);
    int rpc = (g.ny + want - 1) / want;
    rpc = (rpc + kBand - 1) / kBand * kBand;
    return std::max(rpc, kBand);
}

template <class R, class In, int LL>
cudaError_t run(const Geometry &g, const void *sci, const void *tmpl, const uint8_t *mask, bool residual,
                const double *coeffs, const void *xpow, void *cfold, void *diff, double *mom_part, double *mom,
                cudaStream_t st) {
    {
        size_t nt = (size_t)g.ny * LL * LL + g.ny;
        note_launch();
        k_fold<R><<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(coeffs, g, g.ny > 1 ? 1.0 / (g.ny - 1) : 0.0,
                                                                 (R *)cfold);
    }
    const int np = g.dk + 1;
    const size_t sm = Layout<R, In, LL>::bytes(np, g.db);
    const int strips = (g.nx + Tile<R>::kCols - 1) / Tile<R>::kCols;
    auto kern = k_subtract<R, In, LL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const int rpc = rows_per_chunk(g, strips, sizeof(R) == 4 ? (g.sub_per_sm > 0 ? g.sub_per_sm : 2) : 1);
    dim3 grid(strips, (g.ny + rpc - 1) / rpc);
    note_launch();
    kern<<<grid, 32 * kBand, sm, st>>>((const In *)sci, (const In *)tmpl, mask, residual, g, rpc, (const R *)cfold,
                                        (const R *)xpow, (In *)diff);
    return cudaGetLastError();
}

template <class R, class In>
cudaError_t dispatch_L(const Geometry &g, const void *sci, const void *tmpl, const uint8_t *mask, bool residual,
                       const double *coeffs, const void *xpow, void *cfold, void *diff, double *mom_part, double *mom,
                       cudaStream_t st) {
    switch (g.L) {
        case 1: return run<R, In, 1>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
        case 3: return run<R, In, 3>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
        case 5: return run<R, In, 5>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
        case 7: return run<R, In, 7>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
        case 9: return run<R, In, 9>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
        case 11: return run<R, In, 11>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
        case 13: return run<R, In, 13>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
        case 15: return run<R, In, 15>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_subtract(const Geometry &g, int dtype, int precision, const void *sci, const void *tmpl,
                            const uint8_t *mask, bool residual, const double *coeffs, const void *xpow,
                            const void *ypow, void *cfold, void *diff, double *mom_part, double *mom,
                            cudaStream_t st) {
    (void)ypow;
    if (g.dk > 7 || g.db > 7) return cudaErrorInvalidValue;
    // the FP32 paths' residual: compensated kernel of sfft_residual.cu
    if (residual && precision != SFFT_PREC_FP64)
        return launch_residual_comp(g, dtype, sci, tmpl, mask, coeffs, xpow, cfold, diff, mom_part, mom, st);
    if (precision == SFFT_PREC_FP64)
        return dtype == SFFT_F64 ? dispatch_L<double, double>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st)
                                 : dispatch_L<double, float>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
    return dtype == SFFT_F64 ? dispatch_L<float, double>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st)
                             : dispatch_L<float, float>(g, sci, tmpl, mask, residual, coeffs, xpow, cfold, diff, mom_part, mom, st);
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
            e = desc->dtype == SFFT_F64 ? dispatch_L<double, double>(g, sci, tmpl, nullptr, false, coeffs, xpow, cfold, diff, nullptr, nullptr, st)
                                        : dispatch_L<double, float>(g, sci, tmpl, nullptr, false, coeffs, xpow, cfold, diff, nullptr, nullptr, st);
        else
            e = desc->dtype == SFFT_F64 ? dispatch_L<float, double>(g, sci, tmpl, nullptr, false, coeffs, xpow, cfold, diff, nullptr, nullptr, st)
                                        : dispatch_L<float, float>(g, sci, tmpl, nullptr, false, coeffs, xpow, cfold, diff, nullptr, nullptr, st);
    }
    if (e != cudaSuccess) {
        snprintf(err, sizeof err, "sfft_subtract_noalloc: %s", cudaGetErrorString(e));
        set_global_error(err);
        return SFFT_ERR_CUDA;
    }
    return SFFT_OK;
}
