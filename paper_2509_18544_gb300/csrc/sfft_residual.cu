// Residual of the fit on the FP32 paths (the refinement step of the solve, Sec. "SFFT"):
//   R(u) = S_m(u) - sum_{i,d} a_{i,d} (w_i T_m)(u - d) - m(u) sum_r b_r w_r(u)
// in compensated arithmetic, with the residual's background moments sum_u m(u) w_r(u) R(u).
//
// Per-tap weights.  Grouping the kernel monomials by their x power p folds the y powers
// into per-source-row coefficients c_p(d, y_s) (as for the difference image), so the
// kernel term of output pixel (x, y) is
//   sum_d W(d, x - dx, y - dy) T_m(x - dx, y - dy),  W = sum_p c_p(d, y_s) xh(x_s)^p.
// With the integer source coordinate Z_s = 2 x_s - (nx - 1) = (nx - 1) xh(x_s), exact in
// FP32, W = sum_p ct_p Z_s^p with ct_p = c_p / (nx - 1)^p, evaluated by Horner's rule per
// tap and pixel from a lane's register window of Z_s (the wrapped columns' own
// coordinates, so the cyclic boundary needs nothing more).  Shared memory then holds T_m
// alone (not the np planes xh^p T_m), and one staged window feeds every power; the weight
// costs np - 1 FMAs per tap and pixel, as many as the products of the plane form.
//
// Compensation.  At a star core |S| is ~100x the residual, so plain FP32 sums would leave
// rounding errors of order u |S| in R; fitted back onto the basis by the refinement they
// bound the coefficients near 1e-6.  The terms that carry |S| are the weights' constant
// parts ct_0 near the kernel centre (|dx|, |dy| <= kCoreR), where the kernel and the star's
// profile peak: each of their products is split exactly (p + e = c w, e from an FMA) and the
// running sum is a hi + lo pair updated by an error-free two-sum (Knuth).  The other lags
// and the weights' coordinate parts (the kernel's spatial variation) accumulate in plain
// FP32.
//
// Work split: a CTA of 4 warps owns a strip of 128 output columns and a chunk of rows,
// walked in bands of 8 rows; a thread holds 4 consecutive pixels of two rows (ty and
// ty + 4) as the two lanes of packed FP32x2 operations.  The template ring stores each
// pair of rows (s, s + 4) interleaved, two columns to a 16-byte chunk, so one 16-byte
// shared load gives two window columns of both rows; chunks are XOR-swizzled so that the
// 8 lanes of each quarter-warp read distinct banks.
#include "sfft_internal.cuh"

namespace sfft {

int device_sm_count();

namespace {

constexpr int kBandR = 8;              // output rows per band
constexpr int kHalfR = kBandR / 2;     // a thread's second row is kHalfR below its first
constexpr int kThreadsR = 16 * kBandR;  // 4 warps, two rows each
constexpr int kRR = 4;                 // consecutive pixels per lane
constexpr int kColsR = 32 * kRR;       // strip width
constexpr int kCoreR = 2;              // compensated lags of ct_0: |dx|, |dy| <= kCoreR
constexpr int kMaxDBR = 4;             // background degree the fused moments support
constexpr int kMaxMomR = (kMaxDBR + 1) * (kMaxDBR + 2) / 2;

template <int LL> struct RWin {
    static constexpr int h = LL / 2;
    static constexpr int WC = kColsR + 2 * h;     // window columns of a strip
    static constexpr int NCH = (WC + 1) / 2;      // 16-byte chunks of a ring row (2 columns x 2 rows)
    static constexpr int NCHP = (NCH + 1) & ~1;   // even, so that swizzled chunks stay in the row
    static constexpr int RING = kBandR + 2 * h;   // ring rows
    static constexpr int NW = kRR + LL - 1;       // window columns of a lane
    static constexpr int NWC = (NW + 1) / 2;      // chunks of it
};

// chunk j of a ring row sits at j ^ ((j >> 3) & 1): lane l of a quarter-warp reads chunk
// 2 l + q, and for every q the 8 lanes then fall on 8 distinct 16-byte bank groups
__device__ __forceinline__ int swz(int j) { return j ^ ((j >> 3) & 1); }

// Shared memory (byte offsets, each region on 16 bytes):
//   tp  [RING][NCHP] float4          pair slot s: (T[s][2j], T[s+4][2j], T[s][2j+1], T[s+4][2j+1])
//   cf  [kHalf][LL][LL][NPM] float2  the band's ct_p per (row, dy, dx, p): (row ry, row ry + kHalf)
//   xo  [db+1][kColsR] float         xh^p of the strip's output columns
//   ss  [kBand][kColsR] float2       science values of the band's rows, split hi + lo
//   sk  [RING][kColsR] bytes         per ring row: 1 where the output column's pixel is masked
//   byp [kBand][db+1] float          the band's background x-power sums
template <int LL, int NPM> struct RLayout {
    using W = RWin<LL>;
    __host__ __device__ static constexpr size_t al(size_t b) { return (b + 15) & ~(size_t)15; }
    static constexpr size_t cf = al((size_t)W::RING * W::NCHP * 16);
    static constexpr size_t xo = al(cf + 8 * (size_t)kHalfR * LL * LL * NPM);
    __host__ __device__ static constexpr size_t ss(int db) { return al(xo + 4 * (size_t)(db + 1) * kColsR); }
    __host__ __device__ static constexpr size_t sk(int db) { return al(ss(db) + 8 * (size_t)kBandR * kColsR); }
    __host__ __device__ static constexpr size_t byp(int db) { return al(sk(db) + (size_t)W::RING * kColsR); }
    __host__ __device__ static constexpr size_t bytes(int db) { return al(byp(db) + 4 * (size_t)kBandR * (db + 1)); }
};

__device__ __forceinline__ int wrapr(int v, int n) {
    if (v >= 0 && v < n) return v;
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// s + e = a + b exactly (round-to-nearest adds; the _rn intrinsics are never contracted or
// reordered by the compiler)
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    float2 bb = __fadd2_rn(s, neg2(a));
    e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
}

// The coefficient table, FP64 sums rounded once:
//   ct[ys][dy][p][dx] = c_p(d, ys) / (nx - 1)^p,  c_p(d, ys) = sum_{i: p_i = p} a_{i,d} yh(ys)^q_i
// (ct_p = 0 for p >= 1 when nx = 1, where xh = 0), then the background table
// bg[y][p] = sum_{r: p_r = p} b_r yh(y)^q_r (as for the difference image).  iny = 1 / (ny - 1)
// and sx = 1 / (nx - 1) (0 for a single row or column) come from the host: no FP64 division
// per thread; the monomial loops are unrolled over degree <= 7 so the sums stay in registers.
__global__ void k_fold_x(const double *__restrict__ coeffs, Geometry g, double iny, double sx,
                         float *__restrict__ cf) {
    const int L2 = g.L * g.L, np = g.dk + 1, nbp = g.db + 1;
    const size_t ncf = (size_t)g.ny * L2;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncf + (size_t)g.ny) return;
    const bool bgrow = t >= ncf;
    const int ys = bgrow ? (int)(t - ncf) : (int)(t / L2), l = bgrow ? 0 : (int)(t - (size_t)ys * L2);
    const double yh = (2.0 * ys - (g.ny - 1)) * iny;
    double pw[8], c[8];
    pw[0] = 1.0;
#pragma unroll
    const int deg = bgrow ? g.db : g.dk;
#pragma unroll
    for (int q = 1; q < 8; q++) pw[q] = q <= deg ? pw[q - 1] * yh : 0.0;
#pragma unroll
    for (int p = 0; p < 8; p++) c[p] = 0.0;
    int i = 0;  // monomial index: total degree first, then q ascending
#pragma unroll
    for (int d = 0; d < 8; d++) {
        if (d > deg) break;
#pragma unroll
        for (int q = 0; q <= d; q++, i++) {
            const double a = bgrow ? coeffs[g.nker + i] : coeffs[(size_t)i * L2 + l];
            c[d - q] = fma(a, pw[q], c[d - q]);
        }
    }
    if (!bgrow) {
        const int dyi = l / g.L, dxi = l - dyi * g.L;
        float *o = cf + (((size_t)ys * g.L + dyi) * np) * g.L + dxi;
        double sp = 1.0;
#pragma unroll
        for (int p = 0; p < 8; p++, sp *= sx)
            if (p < np) o[(size_t)p * g.L] = (float)(c[p] * sp);
    } else {
        float *o = cf + ncf * np + (size_t)ys * nbp;
#pragma unroll
        for (int p = 0; p < 8; p++)
            if (p < nbp) o[p] = (float)c[p];
    }
}

// ct_p of output rows yb .. yb + kBand - 1 (source rows y - dy) and their background sums,
// copied asynchronously into the paired layout: element 2 p + (ry >= kHalf) of
// cf[((ry mod kHalf) LL + dyi) LL + dxi][2 NPM].
template <int LL, int NPM>
__device__ __forceinline__ void stage_coeffs(const Geometry &g, const float *__restrict__ cexp, int yb, float *cf,
                                             float *byp) {
    constexpr int h = LL / 2;
    const int np = g.dk + 1, ny = g.ny, nq = np * LL, lane = threadIdx.x & 31;
    // a warp per (row, dy): the np LL values of one source row and dy are contiguous
    for (int rd = threadIdx.x >> 5; rd < kBandR * LL; rd += kThreadsR / 32) {
        const int ry = rd / LL, dyi = rd - ry * LL;
        const int ys = wrapr(yb + ry - (dyi - h), ny);
        const float *src = cexp + ((size_t)ys * LL + dyi) * nq;
        float *dst = cf + ((ry % kHalfR) * LL + dyi) * LL * 2 * NPM + ry / kHalfR;
        for (int q = lane; q < nq; q += 32) {
            const int k = q / LL, dxi = q - k * LL;
            cp_async4(dst + (dxi * NPM + k) * 2, src + q);
        }
    }
    const float *bgf = cexp + (size_t)ny * LL * LL * np;
    for (int e = threadIdx.x; e < kBandR * (g.db + 1); e += kThreadsR) {
        const int ry = e / (g.db + 1), p = e % (g.db + 1);
        cp_async4(byp + e, bgf + (size_t)min(yb + ry, ny - 1) * (g.db + 1) + p);
    }
}

// Science values of rows yb .. yb + kBand - 1 (rows before yc1, columns inside the frame),
// split into hi + lo (lo = 0 for FP32 frames): loads issued here, stores by store_sci.
struct SciRun {
    float2 v[kBandR * kColsR / kThreadsR];
};
__device__ __forceinline__ void load_sci(const void *__restrict__ sci, bool f64, const Geometry &g, int x0, int yb,
                                         int yc1, SciRun &s) {
    constexpr int N = kBandR * kColsR / kThreadsR;
#pragma unroll
    for (int i = 0; i < N; i++) {
        const int e = i * kThreadsR + (int)threadIdx.x, r = e / kColsR, c = e % kColsR, y = yb + r, x = x0 + c;
        s.v[i] = make_float2(0.f, 0.f);
        if (y < yc1 && x < g.nx) {
            const size_t u = (size_t)y * g.pitch + x;
            if (f64) {
                const double d = static_cast<const double *>(sci)[u];
                const float hi = (float)d;
                s.v[i] = make_float2(hi, (float)(d - (double)hi));
            } else {
                s.v[i].x = static_cast<const float *>(sci)[u];
            }
        }
    }
}
__device__ __forceinline__ void store_sci(const SciRun &s, float2 *ss) {
    constexpr int N = kBandR * kColsR / kThreadsR;
#pragma unroll
    for (int i = 0; i < N; i++) ss[i * kThreadsR + threadIdx.x] = s.v[i];
}

// Stages `count` consecutive source rows from (unwrapped) row ys0 into the ring, T_m as
// FP32: row ys is the first row of pair slot slot(ys) and the second row of pair slot
// slot(ys - kHalf).  Each thread issues the loads of kBatch elements, then stores them.
template <int LL, int kBatch>
__device__ __forceinline__ void stage_ring(const void *__restrict__ tmpl, bool f64, const uint8_t *__restrict__ mask,
                                           const Geometry &g, int x0, int ys0, int count, int ring_origin, float *tpf,
                                           unsigned char *sk) {
    using W = RWin<LL>;
    const int nx = g.nx, total = count * W::WC;
    for (int base = 0; base < total; base += kBatch * kThreadsR) {
        float tv[kBatch];
        unsigned char bad[kBatch];
        size_t uu[kBatch];
        bool ok[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; i++) {
            const int e = base + i * kThreadsR + (int)threadIdx.x;
            ok[i] = e < total;
            const int r = e / W::WC, c = e - r * W::WC;
            uu[i] = ok[i] ? (size_t)wrapr(ys0 + r, g.ny) * g.pitch + wrapr(x0 - W::h + c, nx) : 0;
        }
        if (f64) {
#pragma unroll
            for (int i = 0; i < kBatch; i++) tv[i] = ok[i] ? (float)static_cast<const double *>(tmpl)[uu[i]] : 0.f;
        } else {
#pragma unroll
            for (int i = 0; i < kBatch; i++) tv[i] = ok[i] ? static_cast<const float *>(tmpl)[uu[i]] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < kBatch; i++) bad[i] = (ok[i] && mask) ? mask[uu[i]] : 0;
#pragma unroll
        for (int i = 0; i < kBatch; i++) {
            if (!ok[i]) continue;
            const int e = base + i * kThreadsR + (int)threadIdx.x;
            const int r = e / W::WC, c = e - r * W::WC, ys = ys0 + r;
            const float t = bad[i] ? 0.f : tv[i];
            const int s1 = (ys - ring_origin) % W::RING;
            int s2 = (ys - kHalfR - ring_origin) % W::RING;
            s2 += s2 < 0 ? W::RING : 0;
            const int o = swz(c >> 1) * 4 + (c & 1) * 2;
            tpf[s1 * W::NCHP * 4 + o] = t;
            tpf[s2 * W::NCHP * 4 + o + 1] = t;
            const int oc = c - W::h;
            if (oc >= 0 && oc < kColsR) sk[s1 * kColsR + oc] = bad[i] ? 1 : 0;
        }
    }
}

// With mom_part, the kernel also writes this CTA's part of the residual's background
// moments sum_u m(u) w_r(u) R(u) (r < nP(DB), in the monomial order): FP32 sums over a
// thread's pixels of a row, FP64 across rows and warps; mom_part[cta nP(DB) + r].
// NPM = DK + 1: the x powers of each tap's weight.
template <int LL, int NPM>
__global__ void __launch_bounds__(kThreadsR, 4)
    k_residual_x(const void *__restrict__ sci, const void *__restrict__ tmpl, bool f64, const uint8_t *__restrict__ mask,
                 Geometry g, int rows_per_chunk, const float *__restrict__ cexp, const float *__restrict__ xpow_g,
                 void *__restrict__ resid, double *__restrict__ mom_part) {
    using W = RWin<LL>;
    using Ly = RLayout<LL, NPM>;
    constexpr int h = W::h;
    constexpr int kRowBatch = (kBandR * W::WC + kThreadsR - 1) / kThreadsR;  // a band's new rows in one batch
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int np = NPM, nx = g.nx, ny = g.ny, db = g.db;
    float *tpf = reinterpret_cast<float *>(smem_raw);
    const float4 *tp4 = reinterpret_cast<const float4 *>(smem_raw);
    float *cf = reinterpret_cast<float *>(smem_raw + Ly::cf);
    float *xo = reinterpret_cast<float *>(smem_raw + Ly::xo);
    float2 *ss = reinterpret_cast<float2 *>(smem_raw + Ly::ss(db));
    unsigned char *sk = smem_raw + Ly::sk(db);
    float *byp = reinterpret_cast<float *>(smem_raw + Ly::byp(db));
    __shared__ double macc[kHalfR][kMaxMomR];  // per warp: moment sums of its rows (written at the end)

    const int x0 = blockIdx.x * kColsR;
    const int yc0 = blockIdx.y * rows_per_chunk, yc1 = min(ny, yc0 + rows_per_chunk);
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    if (yc0 >= ny) {
        if (mom_part)
            for (int j = threadIdx.x; j < g.nb; j += blockDim.x) mom_part[(size_t)cta * g.nb + j] = 0.0;
        return;
    }
    const int ring_origin = yc0 - h;
    const int ty = threadIdx.x >> 5, lane = threadIdx.x & 31, cx = lane * kRR;
    const float yscale = ny > 1 ? 1.f / (float)(ny - 1) : 0.f;
    // lane j < nP(DB) of each warp sums moment j of the warp's rows as an FP32 hi + lo pair
    // (two-sum), converted to FP64 once at the end: the band loop runs no FP64 instruction
    int mpr = 0, mqs = 0;
    if (lane < g.nb) mono_pq(lane, mpr, mqs);
    float mh = 0.f, ml = 0.f;
    float zya = (float)(2 * (yc0 + ty) - (ny - 1));  // 2 ya - (ny - 1) of the band's first row, exact
    for (int e = threadIdx.x; e < (db + 1) * kColsR; e += blockDim.x) {
        const int p = e / kColsR, c = e - p * kColsR;
        xo[e] = xpow_g[(size_t)p * nx + min(x0 + c, nx - 1)];
    }
    // Z_s = 2 x_s - (nx - 1) of this lane's window columns (wrapped, exact), as pairs
    float2 Zw[W::NW];
#pragma unroll
    for (int j = 0; j < W::NW; j++) {
        const float z = (float)(2 * wrapr(x0 + cx - h + j, nx) - (nx - 1));
        Zw[j] = make_float2(z, z);
    }

    // every global load of a band happens in the staging phase before it
    {
        stage_coeffs<LL, NPM>(g, cexp, yc0, cf, byp);
        SciRun sv;
        load_sci(sci, f64, g, x0, yc0, yc1, sv);
        stage_ring<LL, 8>(tmpl, f64, mask, g, x0, yc0 - h, W::RING, ring_origin, tpf, sk);
        store_sci(sv, ss);
        cp_async_wait_all();
    }
    for (int yb = yc0; yb < yc1; yb += kBandR) {
        __syncthreads();
        const int ya = yb + ty, yb2 = ya + kHalfR;
        const bool in_a = ya < yc1, in_b = yb2 < yc1;
        const int sla = (ya - ring_origin) % W::RING, slb = (sla + kHalfR) % W::RING;
        const unsigned skip[2] = {in_a ? *reinterpret_cast<const unsigned *>(sk + sla * kColsR + cx) : 0x01010101u,
                                  in_b ? *reinterpret_cast<const unsigned *>(sk + slb * kColsR + cx) : 0x01010101u};
        float2 hi[kRR], lo[kRR], wing[kRR];
        unsigned good = 0;  // bit 2 r + k: pixel r of row k exists and is not masked
        // start from m (S - bg): S as hi + lo, the background subtracted by two-sum
        {
            float xv[kMaxDBR + 1][kRR];
#pragma unroll
            for (int p = 0; p <= kMaxDBR; p++) {
                if (p > db) break;
                const float4 q = *reinterpret_cast<const float4 *>(xo + p * kColsR + cx);
                xv[p][0] = q.x, xv[p][1] = q.y, xv[p][2] = q.z, xv[p][3] = q.w;
            }
#pragma unroll
            for (int r = 0; r < kRR; r++) {
                float sh[2] = {0.f, 0.f}, sl[2] = {0.f, 0.f}, bg[2] = {0.f, 0.f};
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    if (x0 + cx + r < nx && !((skip[k] >> (8 * r)) & 0xff)) {
                        const int row = k ? ty + kHalfR : ty;
                        good |= 1u << (2 * r + k);
                        const float2 sv = ss[row * kColsR + cx + r];
                        sh[k] = sv.x;
                        sl[k] = sv.y;
                        const float *bp = byp + row * (db + 1);
                        float b = 0.f;
#pragma unroll
                        for (int p = 0; p <= kMaxDBR; p++) {
                            if (p > db) break;
                            b = fmaf(bp[p], xv[p][r], b);
                        }
                        bg[k] = b;
                    }
                }
                float2 sm, e;
                two_sum2(make_float2(sh[0], sh[1]), make_float2(-bg[0], -bg[1]), sm, e);
                hi[r] = sm;
                lo[r] = __fadd2_rn(e, make_float2(sl[0], sl[1]));
                wing[r] = make_float2(0.f, 0.f);
            }
        }
        for (int dyi = 0; dyi < LL; dyi++) {
            // pair slot of source rows (ya + h - dyi, yb2 + h - dyi)
            const int ps = (ya + h - dyi - ring_origin) % W::RING;
            const float4 *row = tp4 + ps * W::NCHP;
            float2 wv[2 * W::NWC];
#pragma unroll
            for (int q = 0; q < W::NWC; q++) {
                const float4 v = row[swz(2 * lane + q)];
                wv[2 * q] = make_float2(v.x, v.y);
                wv[2 * q + 1] = make_float2(v.z, v.w);
            }
            const bool core_row = dyi >= h - kCoreR && dyi <= h + kCoreR;
            const float2 *cb = reinterpret_cast<const float2 *>(cf) + (ty * LL + dyi) * LL * NPM;
#pragma unroll
            for (int dxi = 0; dxi < LL; dxi++) {
                float2 e[NPM];
#pragma unroll
                for (int k = 0; k < NPM; k++) e[k] = cb[dxi * NPM + k];
                const bool core_col = dxi >= h - kCoreR && dxi <= h + kCoreR;
#pragma unroll
                for (int r = 0; r < kRR; r++) {
                    const int j = r + (LL - 1) - dxi;  // window column of the tap's source
                    const float2 w = wv[j];
                    // m = sum_{p >= 1} ct_p Z_s^(p-1) by Horner (zero when np = 1)
                    float2 m = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = NPM - 1; k >= 1; k--) {
                        m = k == NPM - 1 ? e[k] : __ffma2_rn(m, Zw[j], e[k]);
                    }
                    if (core_col && core_row) {
                        // the Z^0 term exactly: product split by FMA, sum by two-sum
                        const float2 pr = __fmul2_rn(e[0], w);
                        const float2 pe = __ffma2_rn(e[0], w, neg2(pr));  // e0 w - pr, exact
                        float2 sm, er;
                        two_sum2(hi[r], neg2(pr), sm, er);
                        hi[r] = sm;
                        lo[r] = __fadd2_rn(lo[r], __fadd2_rn(er, neg2(pe)));
                        if (NPM > 1) wing[r] = __ffma2_rn(__fmul2_rn(m, Zw[j]), w, wing[r]);
                    } else {
                        const float2 E = NPM > 1 ? __ffma2_rn(m, Zw[j], e[0]) : e[0];
                        wing[r] = __ffma2_rn(E, w, wing[r]);
                    }
                }
            }
        }
        float ma[kMaxDBR + 1], mb[kMaxDBR + 1];  // sum over this thread's pixels of m R xh^p, rows a, b
#pragma unroll
        for (int p = 0; p <= kMaxDBR; p++) ma[p] = mb[p] = 0.f;
#pragma unroll
        for (int r = 0; r < kRR; r++) {
            const int x = x0 + cx + r;
            if (x >= nx) continue;
            // R = hi + lo - wing.  FP32 output: (hi - wing) is within a few rounding units of R
            // (lo is of the order u |hi|), so the two FP32 adds cost about one extra rounding
            // of R; on this part an FP64 add runs at 1/64 of the FP32 rate.
            float fa, fb;
            if (!f64) {
                const float2 t = __fadd2_rn(__fadd2_rn(hi[r], neg2(wing[r])), lo[r]);
                fa = t.x;
                fb = t.y;
                float *ro = static_cast<float *>(resid);
                if (in_a) ro[(size_t)ya * g.pitch + x] = fa;
                if (in_b) ro[(size_t)yb2 * g.pitch + x] = fb;
            } else {
                const double ra = (double)hi[r].x + ((double)lo[r].x - (double)wing[r].x);
                const double rb = (double)hi[r].y + ((double)lo[r].y - (double)wing[r].y);
                double *ro = static_cast<double *>(resid);
                if (in_a) ro[(size_t)ya * g.pitch + x] = ra;
                if (in_b) ro[(size_t)yb2 * g.pitch + x] = rb;
                fa = (float)ra;
                fb = (float)rb;
            }
            if (mom_part) {
                fa = (good >> (2 * r)) & 1u ? fa : 0.f;
                fb = (good >> (2 * r + 1)) & 1u ? fb : 0.f;
#pragma unroll
                for (int p = 0; p <= kMaxDBR; p++) {
                    if (p > db) break;
                    const float xv = xo[p * kColsR + cx + r];
                    ma[p] = fmaf(fa, xv, ma[p]);
                    mb[p] = fmaf(fb, xv, mb[p]);
                }
            }
        }
        if (mom_part) {
#pragma unroll
            for (int p = 0; p <= kMaxDBR; p++) {
                if (p > db) break;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ma[p] += __shfl_xor_sync(0xffffffffu, ma[p], o);
                    mb[p] += __shfl_xor_sync(0xffffffffu, mb[p], o);
                }
            }
            // lane j < nP(DB) adds moment j of the two rows (FP32 weights yh^q) to its sum
            if (lane < g.nb) {
                const float yha = zya * yscale, yhb = (zya + (float)(2 * kHalfR)) * yscale;
                float wa = 1.f, wb = 1.f;
                for (int q = 0; q < mqs; q++) wa *= yha, wb *= yhb;
                float va = 0.f, vb = 0.f;
#pragma unroll
                for (int p = 0; p <= kMaxDBR; p++)
                    if (p == mpr) va = ma[p], vb = mb[p];
                const float v = fmaf(wa, va, wb * vb);
                const float sm = __fadd_rn(mh, v), bb = __fadd_rn(sm, -mh);
                ml = __fadd_rn(ml, __fadd_rn(__fadd_rn(mh, -__fadd_rn(sm, -bb)), __fadd_rn(v, -bb)));
                mh = sm;
            }
        }
        zya += (float)(2 * kBandR);
        __syncthreads();
        // the next band reads source rows up to yb + 2 kBand + h - 1; the kBand new ones
        // replace rows yb - h .. yb - h + kBand - 1, which no later band reads
        if (yb + kBandR < yc1) {
            stage_coeffs<LL, NPM>(g, cexp, yb + kBandR, cf, byp);
            SciRun sv;
            load_sci(sci, f64, g, x0, yb + kBandR, yc1, sv);
            stage_ring<LL, kRowBatch>(tmpl, f64, mask, g, x0, yb + kBandR + h, kBandR, ring_origin, tpf, sk);
            store_sci(sv, ss);
            cp_async_wait_all();
        }
    }
    if (mom_part) {
        if (lane < g.nb) macc[ty][lane] = (double)mh + (double)ml;
        __syncthreads();
        for (int j = threadIdx.x; j < g.nb; j += blockDim.x) {
            double v = 0.0;
            for (int w = 0; w < kHalfR; w++) v += macc[w][j];
            mom_part[(size_t)cta * g.nb + j] = v;
        }
    }
}

template <int LL, int NPM>
cudaError_t run_res(const Geometry &g, bool f64, const void *sci, const void *tmpl, const uint8_t *mask,
                    const float *cexp, const float *xpow, void *resid, double *mom_part, double *mom, cudaStream_t st) {
    auto kern = k_residual_x<LL, NPM>;
    const size_t smem = RLayout<LL, NPM>::bytes(g.db);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreadsR, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // rows per chunk: a multiple of kBand that gives one wave of per_sm CTAs per SM
    const int strips = (g.nx + kColsR - 1) / kColsR;
    int want = (per_sm * device_sm_count() + strips - 1) / strips;
    want = want < 1 ? 1 : want;
    int rpc = (g.ny + want - 1) / want;
    rpc = (rpc + kBandR - 1) / kBandR * kBandR;
    rpc = rpc < kBandR ? kBandR : rpc;
    const dim3 grid(strips, (g.ny + rpc - 1) / rpc);
    note_launch();
    kern<<<grid, kThreadsR, smem, st>>>(sci, tmpl, f64, mask, g, rpc, cexp, xpow, resid, mom ? mom_part : nullptr);
    e = cudaGetLastError();
    // the residual's background moments go after the npoly(2 DB) mask moments
    if (e == cudaSuccess && mom)
        e = launch_mom_reduce(mom_part, (int)(grid.x * grid.y), g.nb, mom + npoly(2 * g.db), st);
    return e;
}

template <int LL>
cudaError_t run_res_np(const Geometry &g, bool f64, const void *sci, const void *tmpl, const uint8_t *mask,
                       const float *cexp, const float *xpow, void *resid, double *mom_part, double *mom,
                       cudaStream_t st) {
    switch (g.dk) {
        case 0: return run_res<LL, 1>(g, f64, sci, tmpl, mask, cexp, xpow, resid, mom_part, mom, st);
        case 1: return run_res<LL, 2>(g, f64, sci, tmpl, mask, cexp, xpow, resid, mom_part, mom, st);
        case 2: return run_res<LL, 3>(g, f64, sci, tmpl, mask, cexp, xpow, resid, mom_part, mom, st);
        case 3: return run_res<LL, 4>(g, f64, sci, tmpl, mask, cexp, xpow, resid, mom_part, mom, st);
        default: return cudaErrorInvalidValue;  // plans take DK <= 3 (at most 256 work items per frequency)
    }
}

}  // namespace

// largest number of CTAs the FP32 residual kernel can have (sizes its moment partials)
int residual_ctas_max(const Geometry &g) {
    return ((g.nx + kColsR - 1) / kColsR) * ((g.ny + kBandR - 1) / kBandR);
}

cudaError_t launch_residual_comp(const Geometry &g, int dtype, const void *sci, const void *tmpl,
                                 const uint8_t *mask, const double *coeffs, const void *xpow, void *cfold,
                                 void *resid, double *mom_part, double *mom, cudaStream_t st) {
    if (g.dk > 3 || g.db > kMaxDBR) return cudaErrorInvalidValue;
    {
        const size_t nt = (size_t)g.ny * g.L * g.L + g.ny;
        note_launch();
        k_fold_x<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(
            coeffs, g, g.ny > 1 ? 1.0 / (g.ny - 1) : 0.0, g.nx > 1 ? 1.0 / (g.nx - 1) : 0.0, (float *)cfold);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const bool f64 = dtype == SFFT_F64;
    const float *ce = (const float *)cfold, *xp = (const float *)xpow;
    switch (g.L) {
        case 1: return run_res_np<1>(g, f64, sci, tmpl, mask, ce, xp, resid, mom_part, mom, st);
        case 3: return run_res_np<3>(g, f64, sci, tmpl, mask, ce, xp, resid, mom_part, mom, st);
        case 5: return run_res_np<5>(g, f64, sci, tmpl, mask, ce, xp, resid, mom_part, mom, st);
        case 7: return run_res_np<7>(g, f64, sci, tmpl, mask, ce, xp, resid, mom_part, mom, st);
        case 9: return run_res_np<9>(g, f64, sci, tmpl, mask, ce, xp, resid, mom_part, mom, st);
        case 11: return run_res_np<11>(g, f64, sci, tmpl, mask, ce, xp, resid, mom_part, mom, st);
        case 13: return run_res_np<13>(g, f64, sci, tmpl, mask, ce, xp, resid, mom_part, mom, st);
        case 15: return run_res_np<15>(g, f64, sci, tmpl, mask, ce, xp, resid, mom_part, mom, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sfft
