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
// Work unit (one CTA): one segment, `kg` consecutive frequencies, one of `ysplit` chunks of
// rows.  Each thread owns one (frequency, A, B, dy-chunk of C = L lags) item and streams
// over the chunk's rows.  Rows are staged in shared memory by cp.async in tiles of
// `ytile` rows plus a halo of G = L-1 rows on each side (cyclic in y), double-buffered so
// the next tile loads while this one is consumed.  Inner step: TY rows, C+TY-1 B values in
// registers, C*TY complex multiply-adds.  FP32 spectra accumulate in FP32 for one tile and
// are then folded into a double-float (hi, lo) pair with an error-free two-sum; FP64
// spectra accumulate in FP64.  Items can be restricted to the W x S_m pairs (the
// refinement pass correlates the basis with a residual image stored in the S_m slot).
#include <stdlib.h>

#include "sfft_internal.cuh"

namespace sfft {
namespace {

constexpr int kTY = 8;

// error-free transformation: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// compact staging for the W x S_m pass: W_0..W_{nk-1} padded to an even count, then the
// 16-byte pair of images that holds the S_m slot
__host__ __device__ __forceinline__ int ws_nka(const Geometry &g) { return (g.nk + 1) & ~1; }
__host__ __device__ __forceinline__ int ws_slot(const Geometry &g) { return 2 * g.nk + g.nb; }

struct Item {
    int A, B, dylo, ent0, c0, cn;  // images, first lag, first entry, valid chunk range [c0, cn)
};

// item numbering: 2*npair W-W half items, then nk*(nb+1) W-(Psi|S) items.  With
// ws_only, item it is the W_it x S_m item.
__device__ __forceinline__ Item decode_item(const Geometry &g, int it, bool ws_only) {
    Item m;
    const int L = g.L, nk = g.nk;
    const int two_pairs = 2 * g.npair;
    if (ws_only) {
        // W_it x S_m with the compact staging: B sits after the padded W block
        m.A = it;
        m.B = ws_nka(g) + (ws_slot(g) & 1);
        m.dylo = -g.h;
        m.ent0 = g.npair * (2 * L - 1) + (it * (g.nb + 1) + g.nb) * L;
        m.c0 = 0;
        m.cn = L;
        return m;
    }
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

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct Launch {
    int items;     // items per frequency in this launch
    int kg;        // frequencies per CTA
    int ngroups;   // frequency groups
    int ysplit;    // row chunks
    bool ws_only;  // W x S_m items only
    int cw;        // staged images per frequency (all nimg_pad, or the compact W_i + S_m set)
};

// stage rows [y0 - G, y0 - G + rows) (cyclic) of the CTA's frequencies into buf via 16-byte
// cp.async; layout buf[r][kl][img]
template <class CT>
__device__ __forceinline__ void stage_tile(const CT *__restrict__ spec, const Geometry &g, int s, int k0, int kcnt,
                                           int kg, int y0, int rows, bool ws, int cw, CT *buf) {
    const int NI = g.nimg_pad, ny = g.ny;
    constexpr int per16 = 16 / (int)sizeof(CT);  // complex values per 16-byte chunk
    const int chunks_k = cw / per16;              // chunks per frequency in the staged layout
    const int per_row = kcnt * chunks_k;
    const int total = rows * per_row;
    const int nka = ws_nka(g), slot_pair = ws_slot(g) & ~1;
    for (int v = threadIdx.x; v < total; v += blockDim.x) {
        int r = v / per_row, c = v - r * per_row;
        int kk = c / chunks_k, cc = c - kk * chunks_k;
        int yy = ((y0 - g.G + r) % ny + ny) % ny;
        // source image index of this chunk's first value
        int img = ws ? (cc * per16 < nka ? cc * per16 : slot_pair + (cc * per16 - nka)) : cc * per16;
        const CT *src = spec + (((size_t)s * ny + yy) * g.nkf + k0 + kk) * NI + img;
        CT *dst = buf + ((size_t)r * kg + kk) * cw + cc * per16;
        cp_async16(dst, src);
    }
    cp_async_commit();
}

template <int C>
__global__ void __launch_bounds__(256, 2) k_ycorr_f32(const cpx<float> *__restrict__ spec, Geometry g, Launch ln,
                                                     double *__restrict__ ypart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int YT = g.ytile, G = g.G, ny = g.ny;
    const int rows = YT + 2 * G;
    cpx<float> *buf0 = reinterpret_cast<cpx<float> *>(smem_raw);
    cpx<float> *buf1 = buf0 + (size_t)rows * ln.kg * ln.cw;
    const int s = blockIdx.x / ln.ysplit, ych = blockIdx.x % ln.ysplit;
    const int k0 = blockIdx.y * ln.kg;
    const int kcnt = min(ln.kg, g.nkf - k0);
    const int chunk = (ny + ln.ysplit - 1) / ln.ysplit;
    const int ya = ych * chunk, yb = min(ny, ya + chunk);
    const int tid = threadIdx.x;
    const int kl = tid / ln.items, it = tid - kl * ln.items;
    const bool active = kl < kcnt;
    Item m = decode_item(g, active ? it : 0, ln.ws_only);

    float2 acc[C], hi[C], lo[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        acc[c] = make_float2(0.f, 0.f);
        hi[c] = make_float2(0.f, 0.f);
        lo[c] = make_float2(0.f, 0.f);
    }
    const int rs = ln.kg * ln.cw;  // row stride inside a staged tile
    if (ya < yb) stage_tile(spec, g, s, k0, kcnt, ln.kg, ya, rows, ln.ws_only, ln.cw, buf0);
    int cur = 0;
    for (int y0 = ya; y0 < yb; y0 += YT) {
        cp_async_wait_all();
        __syncthreads();
        cpx<float> *tile = cur ? buf1 : buf0;
        if (y0 + YT < yb) stage_tile(spec, g, s, k0, kcnt, ln.kg, y0 + YT, rows, ln.ws_only, ln.cw, cur ? buf0 : buf1);
        if (active) {
            const int yvalid = min(YT, yb - y0);
            const cpx<float> *ta = tile + (size_t)kl * ln.cw + m.A;
            const cpx<float> *tb = tile + (size_t)kl * ln.cw + m.B;
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
        cur ^= 1;
    }
    cp_async_wait_all();
    if (active) {
        // (hi, lo) float pairs; K3 adds them in FP64 (keeps FP64 work off this kernel's tail)
        float4 *out = reinterpret_cast<float4 *>(ypart) + (((size_t)s * ln.ysplit + ych) * g.nkf + (k0 + kl)) * g.nent;
#pragma unroll
        for (int c = 0; c < C; c++) {
            if (c >= m.c0 && c < m.cn) out[m.ent0 + c] = make_float4(hi[c].x, hi[c].y, lo[c].x, lo[c].y);
        }
    }
}

// Same work as k_ycorr_f32 with Blackwell's packed FP32x2 FMA: the complex multiply-add
// conj(a) w is split into two packed accumulators P += {a.re, a.re} * w and
// Q += {a.im, a.im} * w (re = P.x + Q.y, im = P.y - Q.x at the fold), which halves the FMA
// instruction count without any operand shuffles.
//
// Its tile is stored [frequency][image][row] (row stride RP complex values), so a thread's
// A and B rows are contiguous and every row offset in the inner loop is an immediate; RP is
// even and 2 mod 4, which keeps the 16-byte A loads aligned and spreads the eight images a
// quarter-warp reads over distinct banks.  Each staging thread owns one (frequency, image)
// column of the tile and a fixed set of rows, so no index is divided per element; A rows
// past the end of the row chunk are staged as zeros instead of being masked per row.
__host__ __device__ __forceinline__ int tile_rp(int rows) { return ((rows + 3) & ~3) + 2; }

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}

// stages rows [0, rows) = frame rows y0 - G .. of frequencies k0 .. k0 + kcnt - 1 into the
// [kk][img][row] tile; A images (img < nk) read zero at rows >= G + a_valid
__device__ __forceinline__ void stage_tile_t(const cpx<float> *__restrict__ spec, const Geometry &g, int s, int k0,
                                             int kcnt, int kg, int cw, int y0, int rows, int RP, int a_valid,
                                             cpx<float> *buf) {
    const int NPT = kg * cw, ny = g.ny, NI = g.nimg_pad;
    int p0, pstep, r0, rstep;
    if ((int)blockDim.x >= NPT) {
        p0 = threadIdx.x % NPT;
        pstep = NPT;
        r0 = threadIdx.x / NPT;
        rstep = blockDim.x / NPT;
        if (r0 >= rstep) r0 = rows;  // leftover threads stage nothing
    } else {
        p0 = threadIdx.x;
        pstep = blockDim.x;
        r0 = 0;
        rstep = 1;
    }
    const size_t row_stride = (size_t)g.nkf * NI;
    for (int p = p0; p < NPT; p += pstep) {
        const int kk = p / cw, img = p - kk * cw;
        if (kk >= kcnt) continue;  // frequency past the spectrum: no thread reads it
        const cpx<float> *src = spec + ((size_t)s * ny * g.nkf + k0 + kk) * NI + img;
        cpx<float> *dst = buf + (size_t)p * RP;
        const int zfrom = img < g.nk ? g.G + a_valid : rows;
        int yy = y0 - g.G + r0;
        yy = yy >= 0 && yy < ny ? yy : ((yy % ny) + ny) % ny;
        for (int r = r0; r < rows; r += rstep) {
            if (r >= zfrom)
                dst[r] = cpx<float>{0.f, 0.f};
            else
                cp_async8(dst + r, src + (size_t)yy * row_stride);
            yy += rstep;
            if (yy >= ny) yy = rstep < ny ? yy - ny : yy % ny;
        }
    }
    cp_async_commit();
}

template <int C, int TYP>
__global__ void __launch_bounds__(256, (C <= 11 ? 2 : 1)) k_ycorr_f32x2(const cpx<float> *__restrict__ spec, Geometry g, Launch ln,
                                                       double *__restrict__ ypart) {
    static_assert(TYP % 2 == 0, "A rows are loaded in pairs");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int YT = g.ytile, G = g.G, ny = g.ny;
    const int rows = YT + 2 * G, RP = tile_rp(rows);
    const int cw = ln.cw;
    cpx<float> *buf0 = reinterpret_cast<cpx<float> *>(smem_raw);
    cpx<float> *buf1 = buf0 + (size_t)ln.kg * cw * RP;
    const int s = blockIdx.x / ln.ysplit, ych = blockIdx.x % ln.ysplit;
    const int k0 = blockIdx.y * ln.kg;
    const int kcnt = min(ln.kg, g.nkf - k0);
    const int chunk = (ny + ln.ysplit - 1) / ln.ysplit;
    const int ya = ych * chunk, yb = min(ny, ya + chunk);
    const int tid = threadIdx.x;
    const int kl = tid / ln.items, it = tid - kl * ln.items;
    const bool active = kl < kcnt;
    Item m = decode_item(g, active ? it : 0, false);
    float2 P[C], Q[C], hi[C], lo[C];
#pragma unroll
    for (int c = 0; c < C; c++) P[c] = Q[c] = hi[c] = lo[c] = make_float2(0.f, 0.f);
    if (ya < yb) stage_tile_t(spec, g, s, k0, kcnt, ln.kg, cw, ya, rows, RP, min(YT, yb - ya), buf0);
    int cur = 0;
    for (int y0 = ya; y0 < yb; y0 += YT) {
        cp_async_wait_all();
        __syncthreads();
        const cpx<float> *tile = cur ? buf1 : buf0;
        if (y0 + YT < yb)
            stage_tile_t(spec, g, s, k0, kcnt, ln.kg, cw, y0 + YT, rows, RP, min(YT, yb - y0 - YT), cur ? buf0 : buf1);
        if (active) {
            const int yvalid = min(YT, yb - y0);
            const float4 *ta = reinterpret_cast<const float4 *>(tile + (size_t)(kl * cw + m.A) * RP + G);
            const float2 *tb = reinterpret_cast<const float2 *>(tile + (size_t)(kl * cw + m.B) * RP + G + m.dylo);
            for (int yy = 0; yy < yvalid; yy += TYP) {
                float2 ar[TYP], ai[TYP];
#pragma unroll
                for (int t = 0; t < TYP; t += 2) {
                    const float4 v = ta[(yy + t) >> 1];  // rows yy + t, yy + t + 1 (zero past the chunk)
                    ar[t] = make_float2(v.x, v.x);
                    ai[t] = make_float2(v.y, v.y);
                    ar[t + 1] = make_float2(v.z, v.z);
                    ai[t + 1] = make_float2(v.w, v.w);
                }
                float2 w[C + TYP - 1];
#pragma unroll
                for (int q = 0; q < C + TYP - 1; q++) w[q] = tb[yy + q];
#pragma unroll
                for (int t = 0; t < TYP; t++)
#pragma unroll
                    for (int c = 0; c < C; c++) {
                        P[c] = __ffma2_rn(ar[t], w[t + c], P[c]);
                        Q[c] = __ffma2_rn(ai[t], w[t + c], Q[c]);
                    }
            }
#pragma unroll
            for (int c = 0; c < C; c++) {
                float s1, e1, s2, e2;
                two_sum(hi[c].x, P[c].x + Q[c].y, s1, e1);
                two_sum(hi[c].y, P[c].y - Q[c].x, s2, e2);
                hi[c].x = s1;
                lo[c].x += e1;
                hi[c].y = s2;
                lo[c].y += e2;
                P[c] = Q[c] = make_float2(0.f, 0.f);
            }
        }
        cur ^= 1;
    }
    cp_async_wait_all();
    if (active) {
        float4 *out = reinterpret_cast<float4 *>(ypart) + (((size_t)s * ln.ysplit + ych) * g.nkf + (k0 + kl)) * g.nent;
#pragma unroll
        for (int c = 0; c < C; c++)
            if (c >= m.c0 && c < m.cn) out[m.ent0 + c] = make_float4(hi[c].x, hi[c].y, lo[c].x, lo[c].y);
    }
}

template <int C>
__global__ void __launch_bounds__(256) k_ycorr_f64(const cpx<double> *__restrict__ spec, Geometry g, Launch ln,
                                                  double *__restrict__ ypart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int YT = g.ytile, G = g.G, ny = g.ny;
    const int rows = YT + 2 * G;
    cpx<double> *buf0 = reinterpret_cast<cpx<double> *>(smem_raw);
    cpx<double> *buf1 = buf0 + (size_t)rows * ln.kg * ln.cw;
    const int s = blockIdx.x / ln.ysplit, ych = blockIdx.x % ln.ysplit;
    const int k0 = blockIdx.y * ln.kg;
    const int kcnt = min(ln.kg, g.nkf - k0);
    const int chunk = (ny + ln.ysplit - 1) / ln.ysplit;
    const int ya = ych * chunk, yb = min(ny, ya + chunk);
    const int tid = threadIdx.x;
    const int kl = tid / ln.items, it = tid - kl * ln.items;
    const bool active = kl < kcnt;
    Item m = decode_item(g, active ? it : 0, ln.ws_only);
    double2 acc[C];
#pragma unroll
    for (int c = 0; c < C; c++) acc[c] = make_double2(0.0, 0.0);
    const int rs = ln.kg * ln.cw;
    if (ya < yb) stage_tile(spec, g, s, k0, kcnt, ln.kg, ya, rows, ln.ws_only, ln.cw, buf0);
    int cur = 0;
    for (int y0 = ya; y0 < yb; y0 += YT) {
        cp_async_wait_all();
        __syncthreads();
        cpx<double> *tile = cur ? buf1 : buf0;
        if (y0 + YT < yb) stage_tile(spec, g, s, k0, kcnt, ln.kg, y0 + YT, rows, ln.ws_only, ln.cw, cur ? buf0 : buf1);
        if (active) {
            const int yvalid = min(YT, yb - y0);
            const cpx<double> *ta = tile + (size_t)kl * ln.cw + m.A;
            const cpx<double> *tb = tile + (size_t)kl * ln.cw + m.B;
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
        cur ^= 1;
    }
    cp_async_wait_all();
    if (active) {
        double *out = ypart + ((((size_t)s * ln.ysplit + ych) * g.nkf + (k0 + kl)) * g.nent) * 2;
#pragma unroll
        for (int c = 0; c < C; c++)
            if (c >= m.c0 && c < m.cn) {
                out[2 * (m.ent0 + c)] = acc[c].x;
                out[2 * (m.ent0 + c) + 1] = acc[c].y;
            }
    }
}

// W_i x S_m correlations of the refinement pass (the S_m slot holds the residual image):
// one thread per (segment, row chunk, frequency, W_i), streaming the chunk's rows straight
// from global memory with the L residual values of the lag window in a rotating register
// window (the loop is unrolled by C so the rotation is free).  Output: (hi, lo) float pairs
// per (segment, chunk, frequency, i, dy) -> wspart.
// On the y-FFT route the spectrum records hold the x-weighted base images: W_i = yh^q xh^p
// T_m is then yh(y)^q times the A-side base p, applied per row here (ypow: the FP32 table).
template <int C, bool BASE>
__global__ void __launch_bounds__(256) k_ycorr_ws(const cpx<float> *__restrict__ spec, const cpx<float> *__restrict__ rspec,
                                                 Geometry g, int ychunks, float4 *__restrict__ wspart,
                                                 const float *__restrict__ ypow) {
    const int nk = g.nk, nkf = g.nkf, ny = g.ny, NI = g.nrec, h = g.h;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long total = (long)g.nseg * ychunks * nkf * nk;
    if (t >= total) return;
    const int i = (int)(t % nk);
    const int k = (int)((t / nk) % nkf);
    const int sy = (int)(t / ((long)nk * nkf));
    const int s = sy / ychunks, ych = sy % ychunks;
    const int chunk = (ny + ychunks - 1) / ychunks;
    const int ya = ych * chunk, yb = min(ny, ya + chunk);
    const size_t rowstride = (size_t)nkf * NI;  // complex values between consecutive rows
    int slot = i, qy = 0;                       // record slot of W_i and its row power
    if (BASE) mono_pq(i, slot, qy);
    const float *yqr = ypow + (size_t)qy * ny;  // row 0 of the table is all ones
    const cpx<float> *base = spec + ((size_t)s * ny * nkf + k) * NI;
    const cpx<float> *rbase = rspec + (size_t)s * ny * nkf + k;  // the residual, compact: row stride nkf
    float2 acc[C], hi[C], lo[C], w[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        acc[c] = hi[c] = lo[c] = make_float2(0.f, 0.f);
    }
    // window: w[c] = R(y - h + c) for the current row y (cyclic in y)
#pragma unroll
    for (int c = 0; c < C - 1; c++) {
        int yy = ((ya - h + c) % ny + ny) % ny;
        cpx<float> v = rbase[(size_t)yy * nkf];
        w[c] = make_float2(v.re, v.im);
    }
    int y = ya;
    while (y < yb) {
        // the block's loads first (C entering values of R and C values of W_i), so that they
        // are all in flight together; rows past the chunk read as zero
        float2 rin[C], av[C];
#pragma unroll
        for (int u = 0; u < C; u++) {
            const bool ok = y + u < yb;
            int yy = y + u + h;
            yy = yy >= ny ? yy - ny : yy;
            const cpx<float> v = ok ? rbase[(size_t)yy * nkf] : cpx<float>{0.f, 0.f};
            const cpx<float> a = ok ? base[(size_t)(y + u) * rowstride + slot] : cpx<float>{0.f, 0.f};
            rin[u] = make_float2(v.re, v.im);
            if (BASE) {
                const float w = ok ? yqr[y + u] : 0.f;
                av[u] = make_float2(a.re * w, a.im * w);
            } else {
                av[u] = make_float2(a.re, a.im);
            }
        }
#pragma unroll
        for (int u = 0; u < C; u++) {
            // entering value R(y + h) goes to slot (C - 1 + u) % C; lag dy = c - h sits in slot (c + u) % C
            w[(C - 1 + u) % C] = rin[u];
#pragma unroll
            for (int c = 0; c < C; c++) {
                const float2 b = w[(c + u) % C];
                acc[c].x = fmaf(av[u].x, b.x, acc[c].x);
                acc[c].x = fmaf(av[u].y, b.y, acc[c].x);
                acc[c].y = fmaf(av[u].x, b.y, acc[c].y);
                acc[c].y = fmaf(-av[u].y, b.x, acc[c].y);
            }
        }
        // rotate so that slot 0 again holds R(y_next - h): the unrolled block advanced C rows,
        // which maps every slot back onto itself
        y += C;
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
    float4 *out = wspart + (((size_t)sy * nkf + k) * nk + i) * C;
#pragma unroll
    for (int c = 0; c < C; c++) out[c] = make_float4(hi[c].x, hi[c].y, lo[c].x, lo[c].y);
}

template <int C>
cudaError_t run_ws(const Geometry &g, const void *spec, const void *rspec, float4 *wspart, const void *ypow,
                   cudaStream_t st) {
    const long total = (long)g.nseg * g.ychunks_ws * g.nkf * g.nk;
    note_launch();
    if (g.yfft)
        k_ycorr_ws<C, true><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            (const cpx<float> *)spec, (const cpx<float> *)rspec, g, g.ychunks_ws, wspart, (const float *)ypow);
    else
        k_ycorr_ws<C, false><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            (const cpx<float> *)spec, (const cpx<float> *)rspec, g, g.ychunks_ws, wspart, (const float *)ypow);
    return cudaGetLastError();
}

template <int C>
cudaError_t run(const Geometry &g, int precision, const void *spec, double *ypart, bool ws_only, const void *rspec,
                const void *ypow, cudaStream_t st) {
    if (ws_only && precision != SFFT_PREC_FP64)
        return run_ws<C>(g, spec, rspec, reinterpret_cast<float4 *>(ypart), ypow, st);
    Launch ln;
    ln.ws_only = ws_only;
    ln.items = ws_only ? g.nk : g.items_per_k;
    ln.kg = ws_only ? g.kg_ws : g.kg;
    ln.ngroups = (g.nkf + ln.kg - 1) / ln.kg;
    ln.ysplit = g.ysplit;
    ln.cw = ws_only ? ws_nka(g) + 2 : g.nimg_pad;
    dim3 grid(g.nseg * ln.ysplit, ln.ngroups);
    int threads = ((ln.kg * ln.items + 31) / 32) * 32;
    size_t rows = (size_t)g.ytile + 2 * g.G;
    if (precision == SFFT_PREC_FP64) {
        size_t sm = 2 * rows * ln.kg * ln.cw * sizeof(cpx<double>);
        cudaError_t e = cudaFuncSetAttribute(k_ycorr_f64<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        note_launch();
        k_ycorr_f64<C><<<grid, threads, sm, st>>>((const cpx<double> *)spec, g, ln, ypart);
    } else {
        // packed FP32x2 variant (transposed tile) unless the tuning picked the scalar one
        size_t sm = g.ycorr_scalar ? 2 * rows * ln.kg * ln.cw * sizeof(cpx<float>)
                                   : 2 * (size_t)tile_rp((int)rows) * ln.kg * ln.cw * sizeof(cpx<float>);
        auto kern = g.ycorr_scalar ? k_ycorr_f32<C> : k_ycorr_f32x2<C, 8>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        note_launch();
        kern<<<grid, threads, sm, st>>>((const cpx<float> *)spec, g, ln, ypart);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ycorr(const Geometry &g, int precision, const void *spec, double *ypart, bool ws_only,
                         const void *rspec, const void *ypow, cudaStream_t st) {
    // the direct kernels of the main pass read the per-image records only; the refinement's
    // W x R kernel reads either layout
    if (g.yfft && !(ws_only && precision != SFFT_PREC_FP64)) return cudaErrorInvalidValue;
    switch (g.C) {
        case 1: return run<1>(g, precision, spec, ypart, ws_only, rspec, ypow, st);
        case 3: return run<3>(g, precision, spec, ypart, ws_only, rspec, ypow, st);
        case 5: return run<5>(g, precision, spec, ypart, ws_only, rspec, ypow, st);
        case 7: return run<7>(g, precision, spec, ypart, ws_only, rspec, ypow, st);
        case 9: return run<9>(g, precision, spec, ypart, ws_only, rspec, ypow, st);
        case 11: return run<11>(g, precision, spec, ypart, ws_only, rspec, ypow, st);
        case 13: return run<13>(g, precision, spec, ypart, ws_only, rspec, ypow, st);
        case 15: return run<15>(g, precision, spec, ypart, ws_only, rspec, ypow, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sfft
