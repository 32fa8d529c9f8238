// K3 / K4: lag tables and normal-equation assembly (FP64).
//
//   ysum[k][e]        = sum_s ypart[s][k][e]                         (segments)
//   C(e, dx)          = sum_k Re(ysum[k][e] * tw_x[k][G + dx])       (x-direction inverse DFT
//                       restricted to the kernel lags, tw_x = w_k e^{2 pi i k m / P} / P)
//   background block  = mask moments  sum_u m xh^a yh^b  (a + b <= 2 DB)
//   background rhs    = science moments sum_u m S xh^a yh^b (a + b <= DB)
// and the assembly of the normal equations of the delta-basis least-squares fit:
//   N[(i,d),(j,d')] = C_{W_i,W_j}(d - d'),  N[(i,d), r] = C_{W_i,Psi_r}(d),
//   N[r, r'] = <Psi_r, Psi_r'>,  b[(i,d)] = C_{W_i,S_m}(d),  b[r] = <Psi_r, S_m>.
#include "sfft_internal.cuh"

namespace sfft {
namespace {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (ah + al)(bh + bl) as an unevaluated float pair (ph + pl), to about u^2: ah bh split
// exactly by FMA, the cross terms added to its error, then a fast two-sum (|p| >= |e|)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    ph = p + e;
    pl = e - (ph - p);
}

// (sh, sl) += (ah + al)
__device__ __forceinline__ void df_add(float &sh, float &sl, float ah, float al) {
    float s, e;
    two_sum(sh, ah, s, e);
    sh = s;
    sl += e + al;
}

template <class R>
__device__ __forceinline__ R coordv(int i, int n) {
    return n > 1 ? (R)(2 * i - (n - 1)) / (R)(n - 1) : (R)0;
}

constexpr int kMaxDB = 4;
constexpr int kMaxMomRows = 128;  // rows of one moments CTA (the plan's mom_rows is at most this)

// Column sums over a band of rows, multiplied by x powers and reduced per CTA (FP64 on the
// FP64 path; double-float FP32 pairs on the FP32 path, converted to FP64 per warp).  Each
// thread sums kMomCols adjacent columns; DB is a template parameter so that every loop over
// the powers unrolls without guards.
constexpr int kMomCols = 2;
constexpr int kMomRowBatch = 8;
template <class R, class In, int DB>
__global__ void __launch_bounds__(256, 2) k_moments(const In *__restrict__ sci, const uint8_t *__restrict__ mask,
                                                const R *__restrict__ ypow, Geometry g, double inx,
                                                double *__restrict__ part) {
    constexpr int NB2 = 2 * DB + 1, NB1 = DB + 1;
    __shared__ double red[8][64];
    // yh^b of the chunk's rows, b <= 2 DB (FP64 powers rounded once: the shared table)
    __shared__ R yw[NB2][kMaxMomRows];
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * kMomCols;
    const int ya = blockIdx.y * g.mom_rows, yb = min(g.ny, ya + g.mom_rows);
    for (int e = threadIdx.x; e < NB2 * kMaxMomRows; e += blockDim.x) {
        const int b = e / kMaxMomRows, r = e % kMaxMomRows;
        yw[b][r] = ya + r < yb ? ypow[(size_t)b * g.ny + ya + r] : (R)0;
    }
    __syncthreads();
    // hi/lo column sums: cm[b] = sum m yh^b (b <= 2 DB), cs[b] = sum m S yh^b (b <= DB)
    R cmh[kMomCols][NB2], cml[kMomCols][NB2], csh[kMomCols][NB1], csl[kMomCols][NB1];
#pragma unroll
    for (int c = 0; c < kMomCols; c++) {
#pragma unroll
        for (int b = 0; b < NB2; b++) cmh[c][b] = cml[c][b] = (R)0;
#pragma unroll
        for (int b = 0; b < NB1; b++) csh[c][b] = csl[c][b] = (R)0;
    }
    bool colok[kMomCols];
#pragma unroll
    for (int c = 0; c < kMomCols; c++) colok[c] = x0 + c < g.nx;
    if (colok[0]) {
        // kMomRowBatch rows at a time: every load of the batch issues before the first is used
        // (no load waits for a mask byte), then the sums run in row order and fold into hi + lo
        for (int y0 = ya; y0 < yb; y0 += kMomRowBatch) {
            const int nr = min(kMomRowBatch, yb - y0);
            R mv[kMomRowBatch][kMomCols], sv[kMomRowBatch][kMomCols];
#pragma unroll
            for (int i = 0; i < kMomRowBatch; i++) {
#pragma unroll
                for (int c = 0; c < kMomCols; c++) {
                    mv[i][c] = sv[i][c] = (R)0;
                    if (i < nr && colok[c]) {
                        const size_t u = (size_t)(y0 + i) * g.pitch + x0 + c;
                        const In sr = sci[u];
                        const bool bad = mask ? mask[u] != 0 : false;
                        mv[i][c] = bad ? (R)0 : (R)1;
                        sv[i][c] = bad ? (R)0 : (R)sr;  // a masked pixel never enters, whatever it holds
                    }
                }
            }
            R cma[kMomCols][NB2], csa[kMomCols][NB1];
#pragma unroll
            for (int c = 0; c < kMomCols; c++) {
#pragma unroll
                for (int b = 0; b < NB2; b++) cma[c][b] = (R)0;
#pragma unroll
                for (int b = 0; b < NB1; b++) csa[c][b] = (R)0;
            }
#pragma unroll
            for (int i = 0; i < kMomRowBatch; i++) {
                // rows past the chunk hold m = S = 0 and weight 0: they add exact zeros
#pragma unroll
                for (int b = 0; b < NB2; b++) {
                    const R w = yw[b][y0 - ya + i < kMaxMomRows ? y0 - ya + i : 0];
#pragma unroll
                    for (int c = 0; c < kMomCols; c++) {
                        cma[c][b] += mv[i][c] * w;
                        if (b < NB1) csa[c][b] += sv[i][c] * w;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < kMomCols; c++) {
#pragma unroll
                for (int b = 0; b < NB2; b++) {
                    if constexpr (sizeof(R) == 4) {
                        float s, e;
                        two_sum(cmh[c][b], cma[c][b], s, e);
                        cmh[c][b] = s;
                        cml[c][b] += e;
                    } else {
                        cmh[c][b] += cma[c][b];
                    }
                }
#pragma unroll
                for (int b = 0; b < NB1; b++) {
                    if constexpr (sizeof(R) == 4) {
                        float s, e;
                        two_sum(csh[c][b], csa[c][b], s, e);
                        csh[c][b] = s;
                        csl[c][b] += e;
                    } else {
                        csh[c][b] += csa[c][b];
                    }
                }
            }
        }
    }
    // x powers of this thread's columns, xh = (2 x - (nx - 1)) inx (inx = 1 / (nx - 1) from the
    // host): FP64 on the FP64 path; on the FP32 path as double-float pairs, so that the
    // epilogue runs on the FP32 pipe (GB300 issues FP64 at 1/64 of the FP32 rate) and
    // converts to FP64 once per warp and moment
    double xh[kMomCols];
    float pah[kMomCols][NB2], pal[kMomCols][NB2];
#pragma unroll
    for (int c = 0; c < kMomCols; c++) {
        const double xd = colok[c] ? (2.0 * (x0 + c) - (g.nx - 1)) * inx : 0.0;
        xh[c] = xd;
        if constexpr (sizeof(R) == 4) {
            const float h = (float)xd, l = (float)(xd - (double)h);
            pah[c][0] = 1.f;
            pal[c][0] = 0.f;
#pragma unroll
            for (int a = 1; a < NB2; a++) df_mul(pah[c][a - 1], pal[c][a - 1], h, l, pah[c][a], pal[c][a]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nmask = (2 * DB + 1) * (2 * DB + 2) / 2;
    constexpr int nmom = nmask + (DB + 1) * (DB + 2) / 2;
#pragma unroll
    for (int j = 0; j < nmom; j++) {
        int a, b;
        double v = 0.0;
        if (j < nmask) mono_pq(j, a, b);
        else mono_pq(j - nmask, a, b);
        if constexpr (sizeof(R) == 4) {
            float vh = 0.f, vl = 0.f;
#pragma unroll
            for (int c = 0; c < kMomCols; c++) {
                if (!colok[c]) continue;
                float ch = 0.f, cl = 0.f, th = 1.f, tl = 0.f;
                if (j < nmask) {
#pragma unroll
                    for (int bb = 0; bb < NB2; bb++)
                        if (bb == b) ch = cmh[c][bb], cl = cml[c][bb];
                } else {
#pragma unroll
                    for (int bb = 0; bb < NB1; bb++)
                        if (bb == b) ch = csh[c][bb], cl = csl[c][bb];
                }
#pragma unroll
                for (int aa = 0; aa < NB2; aa++)
                    if (aa == a) th = pah[c][aa], tl = pal[c][aa];
                float ph, pl;
                df_mul(th, tl, ch, cl, ph, pl);
                df_add(vh, vl, ph, pl);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, vh, o), ol = __shfl_xor_sync(0xffffffffu, vl, o);
                df_add(vh, vl, oh, ol);
            }
            v = (double)vh + (double)vl;
        } else {
#pragma unroll
            for (int c = 0; c < kMomCols; c++) {
                if (!colok[c]) continue;
                double cs = 0.0;
                if (j < nmask) {
#pragma unroll
                    for (int bb = 0; bb < NB2; bb++)
                        if (bb == b) cs = (double)cmh[c][bb] + (double)cml[c][bb];
                } else {
#pragma unroll
                    for (int bb = 0; bb < NB1; bb++)
                        if (bb == b) cs = (double)csh[c][bb] + (double)csl[c][bb];
                }
                double xa = 1.0;
                for (int e = 0; e < a; e++) xa *= xh[c];
                v += xa * cs;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        }
        if (lane == 0) red[warp][j & 63] = v;
        if ((j & 63) == 63 || j == nmom - 1) {
            __syncthreads();
            int jbase = j & ~63;
            for (int jj = threadIdx.x; jj <= (j & 63); jj += blockDim.x) {
                double s = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w][jj];
                part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * nmom + jbase + jj] = s;
            }
            __syncthreads();
        }
    }
}

// one CTA per moment: strided partial sums, then a fixed-order tree (deterministic)
__global__ void __launch_bounds__(256) k_mom_reduce(const double *__restrict__ part, int nparts, int nmom,
                                                   double *__restrict__ mom) {
    __shared__ double red[256];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x) s += part[(size_t)p * nmom + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mom[j] = red[0];
}

// partial sums of the segments and row chunks: FP64 values (FP64 spectra) or (hi, lo)
// float pairs (FP32 spectra), both 16 bytes per complex entry
__global__ void k_ysum(const double2 *__restrict__ ypart, Geometry g, bool pairs, double2 *__restrict__ ysum) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)g.nkf * g.nent;
    if (idx >= total) return;
    double2 s = make_double2(0.0, 0.0);
    const int nsg = g.nseg * g.ysplit;
    if (pairs) {
        // (hi, lo) FP32 partials summed as a double-float: the high parts by error-free
        // two-sums, the low parts and the errors in FP32 (their rounding is ~u^2 of the sum);
        // one conversion to FP64 at the end (FP64 adds run at 1/64 of the FP32 rate)
        float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
        for (int sg = 0; sg < nsg; sg++) {
            const float4 v = reinterpret_cast<const float4 *>(ypart)[(size_t)sg * total + idx];
            float t, e;
            two_sum(hx, v.x, t, e);
            hx = t;
            lx += e + v.z;
            two_sum(hy, v.y, t, e);
            hy = t;
            ly += e + v.w;
        }
        s = make_double2((double)hx + (double)lx, (double)hy + (double)ly);
    } else {
        for (int sg = 0; sg < nsg; sg++) {
            double2 v = ypart[(size_t)sg * total + idx];
            s.x += v.x;
            s.y += v.y;
        }
    }
    ysum[idx] = s;
}

// refinement pass: sum the W_i x S_m partials of every segment and row chunk into ysum;
// one warp per output, the lanes take interleaved partials and a fixed shuffle tree adds
// them (the same order on every run)
__global__ void __launch_bounds__(256) k_ysum_ws(const float4 *__restrict__ wspart, Geometry g,
                                                 double2 *__restrict__ ysum) {
    const int L = g.L;
    const size_t idx = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // (k, i, c)
    const int lane = threadIdx.x & 31;
    const size_t per = (size_t)g.nkf * g.nk * L;
    if (idx >= per) return;  // whole warps leave together
    const int nsy = g.nseg * g.ychunks_ws;
    // each lane sums its partials as a double-float (see k_ysum), then one FP64 value per lane
    float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
    for (int sy = lane; sy < nsy; sy += 32) {
        const float4 v = wspart[(size_t)sy * per + idx];
        float t, e;
        two_sum(hx, v.x, t, e);
        hx = t;
        lx += e + v.z;
        two_sum(hy, v.y, t, e);
        hy = t;
        ly += e + v.w;
    }
    double sx = (double)hx + (double)lx, syv = (double)hy + (double)ly;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        syv += __shfl_xor_sync(0xffffffffu, syv, o);
    }
    if (lane == 0) {
        const int c = (int)(idx % L), i = (int)((idx / L) % g.nk), k = (int)(idx / ((size_t)L * g.nk));
        const int ent = g.npair * (2 * L - 1) + (i * (g.nb + 1) + g.nb) * L + c;
        ysum[(size_t)k * g.nent + ent] = make_double2(sx, syv);
    }
}

__global__ void k_lagx(const double2 *__restrict__ ysum, const double2 *__restrict__ tw_x, Geometry g, bool ws_only,
                       double *__restrict__ lagww, double *__restrict__ lagwg, double *__restrict__ lagws) {
    const int L = g.L, h = g.h, Lw = 2 * L - 1, G = g.G;
    const int nww = g.npair * Lw * Lw;
    const int nrest = g.nk * (g.nb + 1) * L * L;
    // one warp per output: the lanes take interleaved bins, a fixed shuffle tree adds them
    int t = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (ws_only) {
        // warp -> (i, dyi, dxi) of the W_i x S_m table, mapped into the full numbering
        if (t >= g.nk * L * L) return;  // whole warps leave together
        int i = t / (L * L), l = t - i * L * L;
        t = nww + ((i * (g.nb + 1) + g.nb) * L * L) + l;
    }
    if (t >= nww + nrest) return;
    int ent, dx;
    double *out;
    if (t < nww) {
        ent = t / Lw;  // = pr * Lw + dyi
        int dxi = t - ent * Lw;
        dx = dxi - (L - 1);
        out = lagww + t;  // [pr][dyi][dxi]
    } else {
        int u = t - nww;
        int e2 = u / L, dxi = u - e2 * L;  // e2 = qd * L + dyi
        ent = g.npair * Lw + e2;
        dx = dxi - h;
        int qd = e2 / L, dyi = e2 - qd * L;
        int i = qd / (g.nb + 1), r = qd - i * (g.nb + 1);
        if (r < g.nb)
            out = lagwg + (((size_t)i * g.nb + r) * L + dyi) * L + dxi;
        else
            out = lagws + ((size_t)i * L + dyi) * L + dxi;
    }
    const int m = G + dx;
    const int W = 2 * G + 1;
    double acc = 0.0;
    for (int k = lane; k < g.nkf; k += 32) {
        double2 y = ysum[(size_t)k * g.nent + ent];
        double2 w = tw_x[(size_t)k * W + m];
        acc = fma(y.x, w.x, acc);
        acc = fma(-y.y, w.y, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) *out = acc;
}

__global__ void k_assemble(const double *__restrict__ lagww, const double *__restrict__ lagwg,
                           const double *__restrict__ lagws, const double *__restrict__ mom, Geometry g,
                           double *__restrict__ N, double *__restrict__ b) {
    const int n = g.n, L = g.L, h = g.h, Lw = 2 * L - 1, ns = L * L, nker = g.nker, nk = g.nk;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)n * n;
    if (idx < total) {
        int row = (int)(idx / n), col = (int)(idx - (size_t)row * n);
        double v;
        if (row < nker && col < nker) {
            int i = row / ns, l = row - i * ns, j = col / ns, l2 = col - j * ns;
            int dy = l / L - h, dx = l % L - h, dy2 = l2 / L - h, dx2 = l2 % L - h;
            // an autocorrelation has C(D) = C(-D): read one canonical lag so N is exactly symmetric
            if (i == j && (dy - dy2 < 0 || (dy == dy2 && dx - dx2 < 0))) {
                int t1 = dy; dy = dy2; dy2 = t1;
                int t2 = dx; dx = dx2; dx2 = t2;
            }
            if (i <= j) {
                int pr = i * nk - i * (i - 1) / 2 + (j - i);
                v = lagww[((size_t)pr * Lw + (dy - dy2 + L - 1)) * Lw + (dx - dx2 + L - 1)];
            } else {
                int pr = j * nk - j * (j - 1) / 2 + (i - j);
                v = lagww[((size_t)pr * Lw + (dy2 - dy + L - 1)) * Lw + (dx2 - dx + L - 1)];
            }
        } else if (row < nker) {
            int i = row / ns, l = row - i * ns, r = col - nker;
            v = lagwg[((size_t)i * g.nb + r) * ns + l];
        } else if (col < nker) {
            int j = col / ns, l2 = col - j * ns, r = row - nker;
            v = lagwg[((size_t)j * g.nb + r) * ns + l2];
        } else {
            int r = row - nker, r2 = col - nker, p1, q1, p2, q2;
            mono_pq(r, p1, q1);
            mono_pq(r2, p2, q2);
            int q = q1 + q2, d = p1 + p2 + q;
            v = mom[d * (d + 1) / 2 + q];
        }
        N[idx] = v;
    }
    if (idx < (size_t)n) {
        int row = (int)idx;
        b[row] = row < nker ? lagws[row] : mom[npoly(2 * g.db) + (row - nker)];
    }
}

}  // namespace

int moments_ctas(const Geometry &g) {
    return ((g.nx + 256 * kMomCols - 1) / (256 * kMomCols)) * ((g.ny + g.mom_rows - 1) / g.mom_rows);
}

namespace {

template <class R, class In>
cudaError_t launch_moments_t(const Geometry &g, const void *sci, const uint8_t *mask, const void *ypow,
                             double *mom_part, cudaStream_t st) {
    dim3 grid((g.nx + 256 * kMomCols - 1) / (256 * kMomCols), (g.ny + g.mom_rows - 1) / g.mom_rows);
    const In *s = (const In *)sci;
    const R *yp = (const R *)ypow;
    const double inx = g.nx > 1 ? 1.0 / (double)(g.nx - 1) : 0.0;
    note_launch();
    switch (g.db) {
        case 0: k_moments<R, In, 0><<<grid, 256, 0, st>>>(s, mask, yp, g, inx, mom_part); break;
        case 1: k_moments<R, In, 1><<<grid, 256, 0, st>>>(s, mask, yp, g, inx, mom_part); break;
        case 2: k_moments<R, In, 2><<<grid, 256, 0, st>>>(s, mask, yp, g, inx, mom_part); break;
        case 3: k_moments<R, In, 3><<<grid, 256, 0, st>>>(s, mask, yp, g, inx, mom_part); break;
        case 4: k_moments<R, In, 4><<<grid, 256, 0, st>>>(s, mask, yp, g, inx, mom_part); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_moments(const Geometry &g, int dtype, int precision, const void *sci, const uint8_t *mask,
                           const void *ypow, double *mom_part, cudaStream_t st) {
    if (g.db > kMaxDB || g.mom_rows > kMaxMomRows) return cudaErrorInvalidValue;
    if (precision == SFFT_PREC_FP64)
        return dtype == SFFT_F64 ? launch_moments_t<double, double>(g, sci, mask, ypow, mom_part, st)
                                 : launch_moments_t<double, float>(g, sci, mask, ypow, mom_part, st);
    return dtype == SFFT_F64 ? launch_moments_t<float, double>(g, sci, mask, ypow, mom_part, st)
                             : launch_moments_t<float, float>(g, sci, mask, ypow, mom_part, st);
}

cudaError_t launch_lag_tables(const Geometry &g, const double *ypart, double *ysum, const double *tw_x,
                              double *lagww, double *lagwg, double *lagws, const double *mom_part, double *mom,
                              bool ws_only, bool pairs, bool have_ysum, cudaStream_t st) {
    size_t total = (size_t)g.nkf * g.nent;
    if (!have_ysum) note_launch();
    if (have_ysum) {
        // the y-FFT route's inverse already wrote ysum
    } else if (ws_only && pairs) {
        size_t per = (size_t)g.nkf * g.nk * g.L;  // one warp each
        k_ysum_ws<<<(unsigned)((per * 32 + 255) / 256), 256, 0, st>>>((const float4 *)ypart, g, (double2 *)ysum);
    } else {
        k_ysum<<<(unsigned)((total + 255) / 256), 256, 0, st>>>((const double2 *)ypart, g, pairs, (double2 *)ysum);
    }
    int nout = ws_only ? g.nk * g.L * g.L : g.npair * (2 * g.L - 1) * (2 * g.L - 1) + g.nk * (g.nb + 1) * g.L * g.L;
    note_launch();
    k_lagx<<<(unsigned)(((size_t)nout * 32 + 255) / 256), 256, 0, st>>>((const double2 *)ysum, (const double2 *)tw_x, g, ws_only, lagww,
                                               lagwg, lagws);
    if (mom_part) {  // the refinement of the FP32 path reduces its moments elsewhere
        note_launch();
        k_mom_reduce<<<g.nmom, 256, 0, st>>>(mom_part, g.mom_ctas, g.nmom, mom);
    }
    return cudaGetLastError();
}

cudaError_t launch_mom_reduce(const double *part, int nparts, int nmom, double *mom, cudaStream_t st) {
    note_launch();
    k_mom_reduce<<<nmom, 256, 0, st>>>(part, nparts, nmom, mom);
    return cudaGetLastError();
}

__global__ void k_refine_rhs(const double *__restrict__ lagws, const double *__restrict__ mom, Geometry g,
                             double *__restrict__ c) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row < g.n) c[row] = row < g.nker ? lagws[row] : mom[npoly(2 * g.db) + (row - g.nker)];
}

cudaError_t launch_refine_rhs(const Geometry &g, const double *lagws, const double *mom, double *c, cudaStream_t st) {
    note_launch();
    k_refine_rhs<<<(g.n + 255) / 256, 256, 0, st>>>(lagws, mom, g, c);
    return cudaGetLastError();
}

cudaError_t launch_assemble(const Geometry &g, const double *lagww, const double *lagwg, const double *lagws,
                            const double *mom, double *N, double *b, cudaStream_t st) {
    size_t total = (size_t)g.n * g.n;
    note_launch();
    k_assemble<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(lagww, lagwg, lagws, mom, g, N, b);
    return cudaGetLastError();
}

}  // namespace sfft
