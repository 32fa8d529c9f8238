// Difference image by row-segment FFTs (the subtraction, Sec. "Pipeline steps", step 6):
//   D(y, x) = S(y, x) - sum_pq sum_d a_{pq,d} (w_pq T)((y, x) - d) - sum_rs b_rs w_rs(y, x),
// the same value as the direct kernel of sfft_subtract.cu, for the FP32 paths.  With the
// source-pixel polynomial w_pq = xh^p yh^q, the kernel term is, per (p, q), a cyclic
// convolution of the image yh^q xh^p T with the L x L stamp K_pq[a][b] = a_{pq,(b-h, a-h)}.
// Per 256-column segment (output columns [x0, x0 + U), U = 256 - 2h, input window
// Z_{p,y}(j) = xh^p T at column x0 - h + j) and as in the cross-convolution:
//   conv(y, x0 + i) = IDFT_256( sum_pq sum_a Khat_{pq,a}(k) yh(y - a + h)^q
//                               Zhat_{p, y - a + h}(k) )(i + 2h),
// so only the DK + 1 x-weighted base images are transformed, the row factor yh^q multiplies
// their spectra in the correlation over rows, and the stamp spectra Khat (scaled by 1/256)
// come from a prologue kernel into the plan's workspace.  FP32 arithmetic with split
// twiddles: the FFT rounding is ~1e-7 of a row's scale, well inside the 1e-5 max|T| the
// difference image is held to.
#include <math.h>

#include "sfft_rowfft.cuh"

namespace sfft {

int device_sm_count();

namespace {

constexpr int kSThreads = 256;
constexpr int kSChunk = 32;
constexpr int kMaxDBF = 4;  // background degree of the FFT route

// Khat[(pq L + a) 128 + slot]: the 256-point DFTs of the stamp rows, 1/256 included
__global__ void __launch_bounds__(256) k_kspec(const double *__restrict__ theta, const float2 *__restrict__ tw_g,
                                               int L, int nk, float2 *__restrict__ kspec) {
    __shared__ float4 tw4[kTw4];
    __shared__ cpx<float> ex[16][kXEx];
    const int t = threadIdx.x, hw = t >> 4, lt = t & 15;
    const unsigned msk = (hw & 1) ? 0xffff0000u : 0x0000ffffu;
    fill_tw4(tw4, tw_g);
    __syncthreads();
    const int rows = nk * L;  // stamp rows, pq-major
    for (int pr = blockIdx.x * 16 + hw; 2 * pr < rows; pr += gridDim.x * 16) {
        const int r1 = 2 * pr, r2 = 2 * pr + 1;
        cpx<float> v[16];
#pragma unroll
        for (int jj = 0; jj < 16; jj++) {
            const int m = lt + 16 * jj;
            v[jj].re = m < L ? (float)theta[(size_t)r1 * L + m] : 0.f;
            v[jj].im = (m < L && r2 < rows) ? (float)theta[(size_t)r2 * L + m] : 0.f;
        }
        fft256f(v, lt, ex[hw], tw4, msk);
        unpack_pair(v, lt, ex[hw], kspec + (size_t)r1 * 128, r2 < rows ? kspec + (size_t)r2 * 128 : nullptr,
                    1.f / kP, msk);
    }
}

template <int H, int NP>
struct SF {
    static constexpr int L = 2 * H + 1, U = kP - 2 * H, NIN = kSChunk + 2 * H;
    static constexpr int NK = NP * (NP + 1) / 2;  // kernel monomials (DK = NP - 1)
    // shared memory: split twiddles, 16 exchange buffers, the chunk's base-image spectra
    // [NP][NIN][128], the input rows' yh^q [NIN][NP], the background coefficients
    static constexpr size_t tw = 0;
    static constexpr size_t ex = tw + 2 * kP * sizeof(cpx<float>);
    static constexpr size_t spec = ex + 16 * (size_t)kXEx * sizeof(cpx<float>);
    static constexpr size_t yq = spec + (size_t)NP * NIN * 128 * sizeof(float2);
    static constexpr size_t bgc = yq + (size_t)NIN * NP * sizeof(float);
    static constexpr size_t crow = bgc + 16 * sizeof(float);  // [kSChunk][kMaxDBF + 1]
    static constexpr size_t bytes = crow + (size_t)kSChunk * (kMaxDBF + 1) * sizeof(float);
};

// the kernel term of every (p, q), p + q < NP, in the monomial order (total degree, then q
// ascending): one loop over the monomials (a single copy of the unrolled row loop, small
// enough for the instruction cache), the next monomial's stamp spectra loaded while the
// current one is summed.  Complex products as two packed FMAs (see sfft_xconv_fft.cu);
// slot 0 packs the real bins 0 and 128, whose products are elementwise.
template <int H, int NP>
__device__ __forceinline__ void mac_all(const float2 *spec, const float *yq, const float2 *__restrict__ kspec,
                                        int slot, int j0, bool packed, float2 (&acc)[16]) {
    constexpr int L = 2 * H + 1, NIN = SF<H, NP>::NIN, NK = SF<H, NP>::NK;
    float2 kn[L];
#pragma unroll
    for (int a = 0; a < L; a++) kn[a] = kspec[(size_t)a * 128 + slot];
#pragma unroll 1
    for (int idx = 0; idx < NK; idx++) {
        float2 kp[L], kpn[L];
#pragma unroll
        for (int a = 0; a < L; a++) {
            kp[a] = kn[a];
            kpn[a] = packed ? make_float2(0.f, 0.f) : make_float2(-kn[a].y, kn[a].x);
        }
        if (idx + 1 < NK) {
#pragma unroll
            for (int a = 0; a < L; a++) kn[a] = kspec[((size_t)(idx + 1) * L + a) * 128 + slot];
        }
        int p, q;
        mono_pq(idx, p, q);
        const float2 *sp = spec + (size_t)p * NIN * 128;
#pragma unroll
        for (int d = -(L - 1); d <= 15; d++) {
            const int i = j0 + 2 * H + d;  // input row of the chunk
            const float2 zr = sp[i * 128 + slot];
            const float w = yq[i * NP + q];  // yh^q of that row (1 for q = 0)
            const float2 z = make_float2(zr.x * w, zr.y * w);
            const float2 za = make_float2(z.x, packed ? z.y : z.x), zb = make_float2(z.y, z.y);
#pragma unroll
            for (int a = 0; a < L; a++) {
                const int jj = d + a;
                if (jj >= 0 && jj < 16) {
                    acc[jj] = __ffma2_rn(za, kp[a], acc[jj]);
                    acc[jj] = __ffma2_rn(zb, kpn[a], acc[jj]);
                }
            }
        }
    }
}

template <class In, int H, int NP>
__global__ void __launch_bounds__(kSThreads, 1)
    k_subtract_fft(const In *__restrict__ sci, const In *__restrict__ tmpl, Geometry g, const double *__restrict__ theta,
                   const float2 *__restrict__ kspec, const float2 *__restrict__ tw_g, const float *__restrict__ xpow,
                   const float *__restrict__ ypow, In *__restrict__ diff) {
    using F = SF<H, NP>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float> *tw = reinterpret_cast<cpx<float> *>(smem_raw + F::tw);
    float2 *spec = reinterpret_cast<float2 *>(smem_raw + F::spec);
    float *yq = reinterpret_cast<float *>(smem_raw + F::yq);
    float *bgc = reinterpret_cast<float *>(smem_raw + F::bgc);
    float *crow = reinterpret_cast<float *>(smem_raw + F::crow);
    const int ny = g.ny, nx = g.nx, pitch = g.pitch, nb = g.nb, db = g.db;
    const int x0 = blockIdx.x * F::U, t = threadIdx.x, hw = t >> 4, lt = t & 15;
    const unsigned msk = (hw & 1) ? 0xffff0000u : 0x0000ffffu;
    cpx<float> *e = reinterpret_cast<cpx<float> *>(smem_raw + F::ex) + hw * kXEx;
    float4 *tw4 = reinterpret_cast<float4 *>(tw);  // the FP32 FFT's table, in the tw / twl bytes
    fill_tw4(tw4, tw_g);
    if (t < nb) bgc[t] = (float)theta[(size_t)F::NK * F::L * F::L + t];
    const int slot = t >> 1, jh = 16 * (t & 1);
    const bool packed = slot == 0;
    const int nchunks = (ny + kSChunk - 1) / kSChunk;
    for (int c = blockIdx.y; c < nchunks; c += gridDim.y) {
        const int y0 = c * kSChunk;
        __syncthreads();  // twiddles ready; the previous chunk's spectra consumed
        for (int i = t; i < F::NIN * NP; i += kSThreads) {
            const int r = i / NP, q = i - r * NP;
            int yy = (y0 - H + r) % ny;
            yy += yy < 0 ? ny : 0;
            yq[i] = ypow[(size_t)q * ny + yy];
        }
        // background per output row: c_r(y) = sum_s b_rs yh(y)^s, r + s <= DB
        for (int i = t; i < kSChunk * (db + 1); i += kSThreads) {
            const int row = i / (db + 1), r = i - row * (db + 1), y = y0 + row;
            float c = 0.f;
            if (y < ny)
                for (int sd = 0; sd + r <= db; sd++) {
                    const int deg = r + sd, idx = deg * (deg + 1) / 2 + sd;  // monomial (r, sd)
                    c = fmaf(bgc[idx], ypow[(size_t)sd * ny + y], c);
                }
            crow[row * (kMaxDBF + 1) + r] = c;
        }
        // 1. the base images' spectra of the chunk's input rows, two rows to a complex FFT
        // (the next item's rows are loaded while the current one is transformed)
        constexpr int NITEMS = NP * (F::NIN / 2);
        auto load_item = [&](int pr, cpx<float>(&v)[16]) {
            const int p = pr / (F::NIN / 2), r1 = 2 * (pr - p * (F::NIN / 2)), r2 = r1 + 1;
            int yy1 = (y0 - H + r1) % ny, yy2 = (y0 - H + r2) % ny;
            yy1 += yy1 < 0 ? ny : 0;
            yy2 += yy2 < 0 ? ny : 0;
            const In *row1 = tmpl + (size_t)yy1 * pitch, *row2 = tmpl + (size_t)yy2 * pitch;
            const float *xp = xpow + (size_t)p * nx;
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                int col = x0 - H + lt + 16 * jj;
                if (nx >= kP) {
                    col += col < 0 ? nx : 0;
                    col -= col >= nx ? nx : 0;
                } else {
                    col %= nx;
                    col += col < 0 ? nx : 0;
                }
                const float w = p ? xp[col] : 1.f;
                v[jj] = {w * (float)row1[col], w * (float)row2[col]};
            }
        };
        cpx<float> vn[16];
        if (hw < NITEMS) load_item(hw, vn);
        for (int pr = hw; pr < NITEMS; pr += 16) {
            cpx<float> v[16];
#pragma unroll
            for (int jj = 0; jj < 16; jj++) v[jj] = vn[jj];
            if (pr + 16 < NITEMS) load_item(pr + 16, vn);
            fft256f(v, lt, e, tw4, msk);
            const int p = pr / (F::NIN / 2), r1 = 2 * (pr - p * (F::NIN / 2));
            float2 *sp = spec + (size_t)p * F::NIN * 128;
            unpack_pair(v, lt, e, sp + r1 * 128, sp + (r1 + 1) * 128, 1.f, msk);
        }
        __syncthreads();
        // 2. the correlation over rows for this thread's slot and 16 output rows
        float2 acc[16];
#pragma unroll
        for (int jj = 0; jj < 16; jj++) acc[jj] = make_float2(0.f, 0.f);
        mac_all<H, NP>(spec, yq, kspec, slot, jh, packed, acc);
        __syncthreads();  // every input slot read
#pragma unroll
        for (int jj = 0; jj < 16; jj++) spec[(jh + jj) * 128 + slot] = acc[jj];
        __syncthreads();
        // 3. output rows 2 hw, 2 hw + 1: conv = conj(FFT(conj(Y1 + i Y2))), D = S - conv - bg
        {
            const int o1 = 2 * hw, o2 = o1 + 1;
            const float2 *Y1 = spec + o1 * 128, *Y2 = spec + o2 * 128;
            cpx<float> v[16];
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const int n = lt + 16 * jj;
                const float2 a = half_bin(Y1, n), b = half_bin(Y2, n);
                v[jj] = {a.x - b.y, -(a.y + b.x)};
            }
            fft256f(v, lt, e, tw4, msk);
#pragma unroll
            for (int k2 = 0; k2 < 16; k2++) {
                const int i = lt + 16 * k2 - 2 * H, x = x0 + i;
                if (i < 0 || i >= F::U || x >= nx) continue;
                const float xh = db > 0 ? xpow[(size_t)nx + x] : 0.f;  // xh (table row 1; present when DB >= 1)
#pragma unroll
                for (int o = 0; o < 2; o++) {
                    const int y = y0 + o1 + o;
                    if (y >= ny) continue;
                    // bg = sum_r xh^r c_r(y), Horner in xh
                    const float *cr = crow + (o1 + o) * (kMaxDBF + 1);
                    float bg = cr[db];
                    for (int r = db - 1; r >= 0; r--) bg = fmaf(bg, xh, cr[r]);
                    const size_t u = (size_t)y * pitch + x;
                    const float conv = o ? -v[k2].im : v[k2].re;
                    diff[u] = (In)((float)sci[u] - conv - bg);
                }
            }
        }
    }
}

template <class In, int H, int NP>
cudaError_t run_sub_fft(const Geometry &g, const In *sci, const In *tmpl, const double *coeffs, const float2 *tw,
                        const float *xpow, const float *ypow, const float2 *kspec, In *diff, cudaStream_t st) {
    using F = SF<H, NP>;
    auto kern = k_subtract_fft<In, H, NP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::bytes);
    if (e != cudaSuccess) return e;
    // segments x chunk groups: one wave of one CTA per SM, each CTA a run of 32-row chunks
    const int nseg = (g.nx + F::U - 1) / F::U, nchunks = (g.ny + kSChunk - 1) / kSChunk;
    int groups = device_sm_count() / nseg;
    groups = groups < 1 ? 1 : (groups > nchunks ? nchunks : groups);
    note_launch();
    kern<<<dim3(nseg, groups), kSThreads, F::bytes, st>>>(sci, tmpl, g, coeffs, kspec, tw, xpow, ypow, diff);
    return cudaGetLastError();
}

template <class In, int NP>
cudaError_t run_sub_h(const Geometry &g, const In *sci, const In *tmpl, const double *coeffs, const float2 *tw,
                      const float *xpow, const float *ypow, const float2 *kspec, In *diff, cudaStream_t st) {
    switch (g.h) {
        case 1: return run_sub_fft<In, 1, NP>(g, sci, tmpl, coeffs, tw, xpow, ypow, kspec, diff, st);
        case 2: return run_sub_fft<In, 2, NP>(g, sci, tmpl, coeffs, tw, xpow, ypow, kspec, diff, st);
        case 3: return run_sub_fft<In, 3, NP>(g, sci, tmpl, coeffs, tw, xpow, ypow, kspec, diff, st);
        case 4: return run_sub_fft<In, 4, NP>(g, sci, tmpl, coeffs, tw, xpow, ypow, kspec, diff, st);
        case 5: return run_sub_fft<In, 5, NP>(g, sci, tmpl, coeffs, tw, xpow, ypow, kspec, diff, st);
        case 6: return run_sub_fft<In, 6, NP>(g, sci, tmpl, coeffs, tw, xpow, ypow, kspec, diff, st);
        case 7: return run_sub_fft<In, 7, NP>(g, sci, tmpl, coeffs, tw, xpow, ypow, kspec, diff, st);
        default: return cudaErrorNotSupported;
    }
}

template <class In>
cudaError_t run_sub_in(const Geometry &g, const void *sci, const void *tmpl, const double *coeffs, const float2 *tw,
                       const float *xpow, const float *ypow, const float2 *kspec, void *diff, cudaStream_t st) {
    const In *s = (const In *)sci, *t = (const In *)tmpl;
    In *d = (In *)diff;
    switch (g.dk) {
        case 0: return run_sub_h<In, 1>(g, s, t, coeffs, tw, xpow, ypow, kspec, d, st);
        case 1: return run_sub_h<In, 2>(g, s, t, coeffs, tw, xpow, ypow, kspec, d, st);
        case 2: return run_sub_h<In, 3>(g, s, t, coeffs, tw, xpow, ypow, kspec, d, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace

cudaError_t launch_subtract_fft(const Geometry &g, int dtype, const void *sci, const void *tmpl, const double *coeffs,
                                const void *tw_fft, const void *xpow, const void *ypow, float2 *kspec, void *diff,
                                cudaStream_t st) {
    if (g.dk > 2 || g.h < 1 || g.h > 7 || g.db > 4) return cudaErrorNotSupported;
    const float2 *tw = (const float2 *)tw_fft;
    const int rows = g.nk * g.L;
    note_launch();
    k_kspec<<<(rows / 2 + 16) / 16, 256, 0, st>>>(coeffs, tw, g.L, g.nk, kspec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return dtype == SFFT_F64
               ? run_sub_in<double>(g, sci, tmpl, coeffs, tw, (const float *)xpow, (const float *)ypow, kspec, diff, st)
               : run_sub_in<float>(g, sci, tmpl, coeffs, tw, (const float *)xpow, (const float *)ypow, kspec, diff, st);
}

}  // namespace sfft
